// Host-side tensor-map encoding through the CUDA driver entry point (no
// link-time dependency on libcuda: the runtime hands out the driver function).
#include <cudaTypedefs.h>

#include <mutex>

#include "tma.cuh"

namespace sil {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

bool encode_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType type, int esz,
                    uint64_t inner, uint64_t outer, uint64_t row_stride_bytes, uint32_t box_inner,
                    uint32_t box_outer, CUtensorMapSwizzle swizzle) {
  auto fn = encode_fn();
  if (!fn || inner == 0 || outer == 0) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || row_stride_bytes % 16 != 0) return false;
  if ((uint64_t(box_inner) * esz) % 16 != 0 || box_inner > 256 || box_outer > 256) return false;
  if (inner >= (uint64_t(1) << 32) || outer >= (uint64_t(1) << 32)) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {row_stride_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, type, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tmap_1d(CUtensorMap* map, const void* base, CUtensorMapDataType type, uint64_t n,
                    uint32_t box) {
  auto fn = encode_fn();
  if (!fn || n == 0 || n >= (uint64_t(1) << 32) || box > 256) return false;
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0 || (box * 4) % 16 != 0) return false;
  cuuint64_t dims[1] = {n};
  cuuint64_t strides[1] = {0};
  cuuint32_t boxd[1] = {box};
  cuuint32_t estr[1] = {1};
  return fn(map, type, 1, const_cast<void*>(base), dims, strides, boxd, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace sil
