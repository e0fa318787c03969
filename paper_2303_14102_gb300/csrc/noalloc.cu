// sil_score_noalloc: pass 2 (finalisation, scoring, mean) without a caller
// workspace.
//
// Who needs this: some callers cannot hand the library device memory at the
// point where they want a score.  Examples are code running inside a host
// framework that owns all device memory through its own pool (a raw
// cudaMalloc there can fail even though the pool has room, or fragment it),
// and plugins whose host application forbids allocation on its hot path.  For
// them this entry point keeps its scratch -- the centred centroids, the
// per-cluster constants, the global centre, the per-CTA partial sums and the
// status word -- in one fixed, file-scope device array.  The entry point
// itself calls no cudaMalloc, cudaFree or allocating library routine.
//
// When the memory is reserved: the CUDA driver reserves the array when it
// loads this file's module on a device.  With lazy module loading (the
// default of current CUDA drivers) that is the first sil_score_noalloc call
// on the device, whose address lookup loads the module; with
// CUDA_MODULE_LOADING=EAGER it is when the library is loaded.  A caller whose
// memory budget is fixed later should therefore make one call at start-up;
// after it, calls on that device reserve nothing more, and the array stays
// until the process exits.
//
// Limits and rules:
//   - k <= SIL_NOALLOC_MAX_K (1024) and d <= SIL_NOALLOC_MAX_D (256); larger
//     sizes return SIL_EUNSUPPORTED before anything is enqueued.  The array is
//     sized for exactly that: about 1.1 MB.
//   - The first call on a device (and the first after the device's context
//     was destroyed and re-created, e.g. by cudaDeviceReset, which gives the
//     array a new address) looks the array's device address up with that
//     device current and caches it per context; make that first call before
//     any stream capture begins.
//   - Every call on a device uses the same array.  Two calls whose work
//     overlaps on the GPU (different streams, or different host threads
//     without ordering) race on it and give wrong results; order them.
//   - The array keeps the previous call's contents.  The only part that must
//     start at zero, the status word, is cleared by each call; everything
//     else is fully rewritten before it is read.
#include <cuda.h>

#include <mutex>

#include "sil_internal.cuh"

namespace {

constexpr int kMaxK = SIL_NOALLOC_MAX_K;
constexpr int kMaxD = SIL_NOALLOC_MAX_D;  // a multiple of 4
constexpr size_t kAlign = 256;
constexpr size_t al(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// byte offsets inside the scratch array
constexpr size_t kOffStatus = 0;
constexpr size_t kOffG = kOffStatus + al(4);
constexpr size_t kOffGf = kOffG + al(size_t(kMaxD) * 8);
constexpr size_t kOffZf = kOffGf + al(size_t(kMaxD) * 4);
constexpr size_t kOffCl = kOffZf + al(size_t(kMaxK) * kMaxD * 4);
constexpr size_t kOffPartials = kOffCl + al(size_t(kMaxK) * 16);
constexpr size_t kScratchBytes = kOffPartials + al(size_t(sil::kMaxPartials) * 8);

// The scratch itself.  In host code this name is only a stand-in for the
// symbol, never a usable address: host code passes the address obtained from
// cudaGetSymbolAddress instead.
static __device__ __align__(256) unsigned char g_sil_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};
CUcontext g_dev_ctx[kMaxDevices] = {};

// The current CUDA context, through the driver entry point the runtime hands
// out (no link-time dependency on the driver library); nullptr if unknown.
CUcontext current_context() {
  using Fn = CUresult (*)(CUcontext*);
  static Fn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<Fn>(p);
  });
  CUcontext c = nullptr;
  if (fn == nullptr || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Device address of the scratch on the current device, looked up once per
// device and context (a re-created context gets the array at a new address).
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SIL_ECUDA;
  // nullptr before the runtime has made a context current: the lookup below
  // then creates the primary context and the next call looks up once more
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_dev_ptr[dev] == nullptr || ctx == nullptr || ctx != g_dev_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sil_noalloc_scratch) != cudaSuccess || p == nullptr)
      return SIL_ECUDA;
    g_dev_ptr[dev] = p;
    g_dev_ctx[dev] = ctx;
  }
  *out = static_cast<unsigned char*>(g_dev_ptr[dev]);
  return SIL_OK;
}

inline int cu(cudaError_t e) { return e == cudaSuccess ? SIL_OK : SIL_ECUDA; }

}  // namespace

extern "C" int sil_score_noalloc(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                                 const float* col_scale, const int32_t* labels, int32_t k,
                                 int32_t dist, const int64_t* count, const double* s1,
                                 const double* s2, float* s_out, double* S_out, void* saved,
                                 uint32_t* dev_status, void* stream) {
  using namespace sil;
  if (n < 0 || d <= 0 || k <= 0 || ldx < d) return SIL_EINVAL;
  if (dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return SIL_EINVAL;
  if (dist != SIL_SQEUCLIDEAN && dist != SIL_COSINE && dist != SIL_EUCLIDEAN_RMS) return SIL_EINVAL;
  if (n > 0 && (X == nullptr || labels == nullptr)) return SIL_EINVAL;
  if (dtype == SIL_FP8_E4M3 && col_scale == nullptr) return SIL_EINVAL;
  if (!count || !s1 || !s2) return SIL_EINVAL;
  if (k > kMaxK || d > kMaxD) return SIL_EUNSUPPORTED;

  unsigned char* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != SIL_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = reinterpret_cast<uint32_t*>(base + kOffStatus);
  if ((rc = cu(cudaMemsetAsync(wst, 0, 4, st))) != SIL_OK) return rc;

  FinLaunch f{};
  f.count = reinterpret_cast<const unsigned long long*>(count);
  f.s1 = s1;
  f.s2 = s2;
  f.k = k;
  f.d = d;
  f.dist = dist;
  f.g = reinterpret_cast<double*>(base + kOffG);
  f.gf = reinterpret_cast<float*>(base + kOffGf);
  f.zf = reinterpret_cast<float*>(base + kOffZf);
  f.cl = reinterpret_cast<float4*>(base + kOffCl);
  f.status = wst;
  f.stream = st;
  if ((rc = cu(launch_finalize(f))) != SIL_OK) return rc;

  ScoreLaunch s{};
  s.X = X;
  s.dtype = dtype;
  s.n = n;
  s.d = d;
  s.ldx = ldx;
  s.cs = col_scale;
  s.labels = labels;
  s.k = k;
  s.dist = dist;
  s.zf = f.zf;
  s.cl = f.cl;
  s.gf = f.gf;
  s.s_out = s_out;
  if (saved) {
    s.sa = static_cast<float*>(saved);
    s.sb = s.sa + n;
    s.skstar = reinterpret_cast<int32_t*>(s.sb + n);
  }
  s.partials = reinterpret_cast<double*>(base + kOffPartials);
  int32_t np = 0;
  s.n_partials = &np;
  s.status = wst;
  s.stream = st;
  if ((rc = cu(launch_score_simt(s))) != SIL_OK) return rc;
  return cu(launch_reduce_S(s.partials, np, n, wst, dev_status, S_out, st));
}
