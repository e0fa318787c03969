// Pass 2 on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// The K dot products of every point with the centred centroids (the
// x_i . Y_k term of Eq. 10/11, and x_hat_i . Omega_k of Eq. 17/18) form the
// GEMM  X (n x d) . Z^T (d x K).  This kernel runs it in BF16 with FP32
// accumulation in tensor memory, at FP32-level accuracy:
//   * Z = mu' is split into hi + lo BF16 parts (mu' - hi rounded again), so
//     B carries ~16 significant bits;
//   * FP32 X (MODE 0) is split the same way by converter warps inside the
//     kernel and the GEMM is hi.Zhi + hi.Zlo + lo.Zhi (the lo.lo term is
//     below FP32 rounding of the result);
//   * BF16 X (MODE 1) is exact in BF16 and TMA writes it straight into the
//     operand layout: x.Zhi + x.Zlo;
//   * FP8-E4M3 X (MODE 2) with per-column scales s: the codes q are exact in
//     BF16 (converter warps widen them) and the scales are folded into the
//     centroids, x.mu' = q.(s * mu'): q.Zhi + q.Zlo.
// The epilogue reads each point's accumulators from TMEM, forms
// d_k = ||x'||^2 + cb_k - 2 inv x.mu'_k (cb_k = bias_k + 2 g.mu'_k folds the
// centring on the global mean g back in; inv = 1/||x|| for cosine) and ranks
// the clusters k != own cluster by it.  b_i itself is then the nearest
// cluster's distance in the difference form ||x' - mu'_k||^2 + W_k/n_k,
// from the point's operand row, which stays in shared memory until the
// epilogue has read it; the own-cluster term a_i uses the same form on the
// converter warps.  The n x K matrix never leaves TMEM.
//
// Clusters are processed in blocks of at most 256 (the MMA N).  With one
// block the epilogue finishes s_i and the per-CTA sums itself.  With G > 1
// blocks the grid is (point ranges) x (G blocks): each CTA keeps its block's
// split centroids resident in shared memory and streams the X tiles of its
// point range -- the G CTAs of a range read the same tiles at about the same
// time, so the repeats are served by L2 -- and writes, per point, the
// distance to the nearest cluster of its block (and its index when the
// backward record is wanted).  The CTA whose block holds the point's own
// cluster also writes a_i.  k_tc_combine then takes the minimum over the
// blocks and finishes s_i.
//
// One persistent CTA per SM, warp-specialised:
//   warp 0       TMA producer (X tiles, labels; the split centroids once)
//   warp 1       TMEM allocation + single-thread tcgen05.mma issue
//   converters   one or two groups of 8 warps, two threads per tile row (one
//                per half) -- FP32 -> BF16 hi/lo or FP8 -> BF16 in the
//                swizzled K-major layout, ||x'||^2 and the exact a_i, with the
//                block's centroids, the global centre and the cluster
//                constants staged in shared memory
//   epilogue     one or two groups of 4 warps: tcgen05.ld, masked running
//                minimum, b_i in the difference form where needed, s_i, sums
// With two groups of a role, group g takes tiles g, g + 2, ... (see
// tc_epi_groups / tc_conv_groups).  Ring buffers: raw X stages (MODE 0 and
// 2), A buffers, a ring of row-term slots and two TMEM accumulators, each
// guarded by mbarriers.  Every wait is bounded (SIL_ETIMEOUT); on a timeout
// all roles stop, in-flight copies and MMAs are waited for (bounded) and TMEM
// is freed before the CTA exits.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "sil_internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace sil {

namespace {

constexpr int kTM = 128;                   // points per tile = TMEM lanes
constexpr int kTcThreads = 448;            // 14 warps (one epilogue warpgroup)
constexpr int kConvWarps = 8;              // warps per converter group
constexpr int kEpiWarp0 = 2 + kConvWarps;  // warps 10..13 of the one-group layout

enum TcMode { kModeF32 = 0, kModeBF16 = 1, kModeFP8 = 2 };

// Warpgroups of the narrow kernel.  For rows of up to 64 columns two epilogue
// groups of 4 warps, each taking every other tile (and owning one of the two
// TMEM accumulators), so that the latency-bound epilogue of two tiles
// overlaps; one otherwise (the converters of 128-column rows need the
// registers).  FP32 rows of up to 64 columns whose cluster block is at most
// twice as wide as the row -- conversion (the hi/lo split) outweighs the
// epilogue there -- also get two converter groups of 8 warps that alternate
// tiles (26 warps, 72 registers each); with wider blocks the epilogue
// needs the registers more.
__host__ __device__ constexpr int tc_epi_groups(int dp) { return dp <= 64 ? 2 : 1; }
__host__ __device__ constexpr int tc_conv_groups(int mode, int dp, int kp) {
  return mode == kModeF32 && dp <= 64 && kp <= 2 * dp ? 2 : 1;
}
__host__ __device__ constexpr int tc_threads(int dp, int cg) {
  return 32 * (2 + kConvWarps * cg + 4 * tc_epi_groups(dp));
}
constexpr int kAtomBytes = kTM * 128;      // one 128-row x 128-byte swizzle column
constexpr int kMaxBlockN = 256;            // clusters per block (MMA N)
constexpr int kSmemMax = 227 * 1024;
constexpr int kSideSlots = 4;  // row-term ring of the modes whose converters write it


// Per-row code handed from the converters to the epilogue: the own cluster's
// index within this CTA's block (>= 0), -2 - index for a singleton own
// cluster, kOwnElsewhere when the own cluster is in another block, and
// kRowInvalid for rows past n, bad labels and zero-norm rows (cosine).
constexpr int kOwnElsewhere = -1;
constexpr int kRowInvalid = -0x7fffffff - 1;


__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  // element with the lower column index goes to the low half
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Two E4M3 codes (low byte first) widened exactly to FP32.
__device__ __forceinline__ float2 fp8x2_to_float2(uint32_t two_codes) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t(two_codes & 0xFFFFu), __NV_E4M3);
  return __half22float2(__half2(h));
}

// Squared distance ||x inv - g - z||^2 of tile row r, read back from its
// operand row in the A buffer (FP32: hi + lo, ~17 bits; BF16: exact; FP8:
// the code times its column scale), to the centroid z (dz columns, from
// shared memory when zsm is set, else global memory).  The difference form
// has no cancellation, unlike ||x'||^2 + bias - 2 x'.mu'.
template <int MODE, int DP>
__device__ __forceinline__ float tc_row_dist(const unsigned char* ab, int lo_off, int r, float inv,
                                             const float* gsm, const float* csm, const float* zsm,
                                             const float* zg, int dz) {
  float2 acc = make_float2(0.f, 0.f);
  const float2 inv2 = make_float2(inv, inv);
#pragma unroll
  for (int c8 = 0; c8 < DP / 8; ++c8) {
    const int col = 8 * c8;
    const int off = DP == 32 ? sw64(r, c8) : (col / 64) * kAtomBytes + sw128(r, (col % 64) / 8);
    const uint4 hv = *reinterpret_cast<const uint4*>(ab + off);
    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
    float x[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[e]));
      x[2 * e] = f.x;
      x[2 * e + 1] = f.y;
    }
    if (MODE == kModeF32) {
      const uint4 lv = *reinterpret_cast<const uint4*>(ab + lo_off + off);
      const uint32_t lw[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&lw[e]));
        x[2 * e] += f.x;
        x[2 * e + 1] += f.y;
      }
    }
#pragma unroll
    for (int h4 = 0; h4 < 2; ++h4) {
      const int c4 = col + 4 * h4;
      float2 xa = make_float2(x[4 * h4], x[4 * h4 + 1]), xb = make_float2(x[4 * h4 + 2], x[4 * h4 + 3]);
      if (MODE == kModeFP8) {
        const float4 s4 = *reinterpret_cast<const float4*>(csm + c4);
        xa = __fmul2_rn(xa, make_float2(s4.x, s4.y));
        xb = __fmul2_rn(xb, make_float2(s4.z, s4.w));
      }
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c4 < dz) z = zsm ? *reinterpret_cast<const float4*>(zsm + c4) : __ldg(reinterpret_cast<const float4*>(zg + c4));
      const float4 g = *reinterpret_cast<const float4*>(gsm + c4);
      const float2 ca = __ffma2_rn(xa, inv2, make_float2(-g.x, -g.y));
      const float2 cb = __ffma2_rn(xb, inv2, make_float2(-g.z, -g.w));
      const float2 da = __fadd2_rn(ca, make_float2(-z.x, -z.y));
      const float2 db = __fadd2_rn(cb, make_float2(-z.z, -z.w));
      acc = __ffma2_rn(da, da, acc);
      acc = __ffma2_rn(db, db, acc);
    }
  }
  return acc.x + acc.y;
}

// The same distance with the row read from global memory (FP32, d columns);
// z may point to shared or global memory.  SPLIT rounds each element to the
// hi + lo BF16 pair the A buffer would hold, so that both sources give the
// same bits.
template <bool SPLIT>
__device__ __forceinline__ float tc_row_dist_global(const float* xr, int d, float inv, const float* gsm,
                                                    const float* zg) {
  auto rd = [](float v) {
    if (!SPLIT) return v;
    const float hi = __bfloat162float(__float2bfloat16_rn(v));
    return hi + __bfloat162float(__float2bfloat16_rn(v - hi));
  };
  float2 acc = make_float2(0.f, 0.f);
  const float2 inv2 = make_float2(inv, inv);
  int c = 0;
  for (; c + 4 <= d; c += 4) {
    const float4 x = __ldg(reinterpret_cast<const float4*>(xr + c));
    const float4 z = *reinterpret_cast<const float4*>(zg + c);
    const float4 g = *reinterpret_cast<const float4*>(gsm + c);
    const float2 ca = __ffma2_rn(make_float2(rd(x.x), rd(x.y)), inv2, make_float2(-g.x, -g.y));
    const float2 cb = __ffma2_rn(make_float2(rd(x.z), rd(x.w)), inv2, make_float2(-g.z, -g.w));
    const float2 da = __fadd2_rn(ca, make_float2(-z.x, -z.y));
    const float2 db = __fadd2_rn(cb, make_float2(-z.z, -z.w));
    acc = __ffma2_rn(da, da, acc);
    acc = __ffma2_rn(db, db, acc);
  }
  float t = acc.x + acc.y;
  for (; c < d; ++c) {
    const float e = fmaf(rd(__ldg(xr + c)), inv, -gsm[c]) - zg[c];
    t = fmaf(e, e, t);
  }
  return t;
}

// The same distance with a BF16 or FP8 row (d columns) read from global
// memory: the values its A-buffer row holds (FP8: the code times its column
// scale), in tc_row_dist's order of operations, so that both sources give the
// same bits.  Rows start on 16-byte boundaries (a TMA requirement of X).
template <int MODE, int DP>
__device__ __forceinline__ float tc_row_dist_lp_global(const unsigned char* xr, int d, float inv, const float* gsm,
                                                       const float* csm, const float* zg, int dz) {
  float2 acc = make_float2(0.f, 0.f);
  const float2 inv2 = make_float2(inv, inv);
#pragma unroll 1
  for (int c8 = 0; c8 < DP / 8; ++c8) {  // a rare path: few live registers
    const int col = 8 * c8;
    float x[8];
    if (col + 8 <= d) {
      if (MODE == kModeBF16) {
        const uint4 hv = __ldg(reinterpret_cast<const uint4*>(xr + 2 * col));
        const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&hw[e]));
          x[2 * e] = f.x;
          x[2 * e + 1] = f.y;
        }
      } else {
        const uint2 cv = __ldg(reinterpret_cast<const uint2*>(xr + col));
        const uint32_t cw[2] = {cv.x, cv.y};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 f0 = fp8x2_to_float2(cw[e]), f1 = fp8x2_to_float2(cw[e] >> 16);
          x[4 * e] = f0.x;
          x[4 * e + 1] = f0.y;
          x[4 * e + 2] = f1.x;
          x[4 * e + 3] = f1.y;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float v = 0.f;
        if (col + e < d) {
          if (MODE == kModeBF16) {
            v = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(xr)[col + e]);
          } else {
            v = fp8x2_to_float2(uint32_t(xr[col + e])).x;
          }
        }
        x[e] = v;
      }
    }
#pragma unroll
    for (int h4 = 0; h4 < 2; ++h4) {
      const int c4 = col + 4 * h4;
      float2 xa = make_float2(x[4 * h4], x[4 * h4 + 1]), xb = make_float2(x[4 * h4 + 2], x[4 * h4 + 3]);
      if (MODE == kModeFP8) {
        const float4 s4 = *reinterpret_cast<const float4*>(csm + c4);
        xa = __fmul2_rn(xa, make_float2(s4.x, s4.y));
        xb = __fmul2_rn(xb, make_float2(s4.z, s4.w));
      }
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c4 < dz) z = *reinterpret_cast<const float4*>(zg + c4);
      const float4 g = *reinterpret_cast<const float4*>(gsm + c4);
      const float2 ca = __ffma2_rn(xa, inv2, make_float2(-g.x, -g.y));
      const float2 cb = __ffma2_rn(xb, inv2, make_float2(-g.z, -g.w));
      const float2 da = __fadd2_rn(ca, make_float2(-z.x, -z.y));
      const float2 db = __fadd2_rn(cb, make_float2(-z.z, -z.w));
      acc = __ffma2_rn(da, da, acc);
      acc = __ffma2_rn(db, db, acc);
    }
  }
  return acc.x + acc.y;
}

// The expanded form d_k = ||x'||^2 + v_k, v_k = cb_k - 2 inv x.mu'_k, loses
// about log2(kappa) bits to cancellation, kappa = (||x inv|| + ||mu'_k||)^2 / d_k,
// and the tensor-core sums round towards zero, so that loss is a bias that
// survives the mean S.  Rows with kappa above kCondExact take the difference
// form instead (the bias left on the others is ~1e-7 relative or less).
// rb = ||g|| + sqrt(max_k bias_k) bounds ||x inv|| - ||x'|| + ||mu'_k||.
constexpr float kCondExact = 6.f;
__device__ __forceinline__ bool tc_ill_conditioned(float xn2, float best, float rb) {
  const float m = sqrtf(xn2) + rb;
  return !(m * m <= kCondExact * (xn2 + best));
}

// rb of tc_ill_conditioned over all k clusters (so that the choice of form
// for a row does not depend on how the clusters are split into blocks) and
// the centre g (dp columns, zero padded); warp-collective.
__device__ __forceinline__ float tc_cond_radius(const float4* cl, int k, const float* g, int dp, int lane) {
  float mb = 0.f, g2 = 0.f;
  for (int i = lane; i < k; i += 32) {
    const float v = __ldg(&cl[i]).x;
    if (v < INFINITY) mb = fmaxf(mb, v);
  }
  for (int c = lane; c < dp; c += 32) g2 = fmaf(g[c], g[c], g2);
  for (int o = 16; o > 0; o >>= 1) {
    mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    g2 += __shfl_xor_sync(0xffffffffu, g2, o);
  }
  return sqrtf(g2) + sqrtf(mb);
}

// Minimum over the columns k != own of v_k = cb_k + sc acc_k of this warp's
// 32 TMEM lanes (acc at tbase), with its index in kb when ARG; 16 NLD columns
// per round trip to TMEM (NLD loads in flight, one wait).  Warp-collective.
template <bool ARG, int NLD>
__device__ __forceinline__ float tc_lane_min(uint32_t tbase, int kp, const float* cbs, float sc, int own, int& kb) {
  float best = INFINITY;
  const float2 sc2 = make_float2(sc, sc);
  for (int c0 = 0; c0 < kp; c0 += 16 * NLD) {
    uint32_t rv[NLD][16];
#pragma unroll
    for (int j = 0; j < NLD; ++j)
      if (c0 + 16 * j < kp) tmem_ld16_async(tbase + uint32_t(c0 + 16 * j), rv[j]);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      if (c0 + 16 * j >= kp) break;
      reg_fence16(rv[j]);
      const float4* cb4 = reinterpret_cast<const float4*>(cbs + c0 + 16 * j);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 cq = cb4[q4];
        const float2 va = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[j][4 * q4]), __uint_as_float(rv[j][4 * q4 + 1])),
                                     make_float2(cq.x, cq.y));
        const float2 vb = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[j][4 * q4 + 2]), __uint_as_float(rv[j][4 * q4 + 3])),
                                     make_float2(cq.z, cq.w));
        const float vals[4] = {va.x, va.y, vb.x, vb.y};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int kk = c0 + 16 * j + 4 * q4 + e;
          if (ARG) {
            if (kk != own && vals[e] < best) {
              best = vals[e];
              kb = kk;
            }
          } else if (kk != own) {
            best = fminf(best, vals[e]);
          }
        }
      }
    }
  }
  return best;
}

// Index of the first column k != own whose v_k, recomputed exactly as
// tc_lane_min computes it, equals best; -1 if none or !want.  Warp-collective.
__device__ __forceinline__ int tc_lane_find(uint32_t tbase, int kp, const float* cbs, float sc, int own, float best,
                                            bool want) {
  int kb = -1;
  const float2 sc2 = make_float2(sc, sc);
  for (int c0 = 0; c0 < kp; c0 += 16) {  // one load in flight: few live registers
    uint32_t rv[16];
    tmem_ld16_async(tbase + uint32_t(c0), rv);
    tmem_wait_ld();
    reg_fence16(rv);
    const float4* cb4 = reinterpret_cast<const float4*>(cbs + c0);
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const float4 cq = cb4[q4];
      const float2 va = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[4 * q4]), __uint_as_float(rv[4 * q4 + 1])),
                                   make_float2(cq.x, cq.y));
      const float2 vb = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[4 * q4 + 2]), __uint_as_float(rv[4 * q4 + 3])),
                                   make_float2(cq.z, cq.w));
      const float vals[4] = {va.x, va.y, vb.x, vb.y};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int kk = c0 + 4 * q4 + e;
        if (kb < 0 && kk != own && vals[e] == best) kb = kk;  // the first, as the argmin pass
      }
    }
  }
  return want ? kb : -1;
}

// ------------------------------------------------------------ parameters
__host__ __device__ inline int tc_pow2(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

struct TcK {
  int64_t n;
  int32_t d;
  int32_t k;
  int32_t kp;        // MMA N = clusters per block (multiple of 16)
  int32_t nblk;      // cluster blocks G (= gridDim.y)
  int32_t acc_cols;  // TMEM columns per accumulator (power of two >= kp)
  int32_t dz;
  int32_t cosine;
  int32_t rms;  // Eq. 2 on the square roots of a and b (approximate Euclidean)
  float scale;
  int32_t nxs;  // raw X stages (MODE 0, 2)
  int32_t nab;  // A buffers
  int32_t zst;  // stride of the staged centroids (0: not staged)
  int32_t own_rows;  // 1: the converters take the own-cluster term a warp per row (tc_own_term_by_warp; one group)
  const void* xg;  // the rows, for the difference form of ill-conditioned rows
  int64_t ldx;
  const float* zf;
  const float4* cl;
  const float* gf;
  const float* cb;  // [nblk * kp]
  const float* cs;  // FP8 column scales
  float* s_out;
  float* sa;
  float* sb;
  int32_t* skstar;
  double* partials;
  float* pmin;    // [nblk][n] distance to the block's nearest cluster, NaN for an invalid row
  int32_t* parg;  // [nblk][n] its index (backward record)
  float* pown;    // [n]       a_i before scaling, from the own cluster's block
  uint32_t* status;
  int32_t zbox_rows;   // rows of Z per TMA box (the block width, or 16 when widths vary)
  const TcItem* items; // several labelings in one launch: item blockIdx.y (else nullptr)
};

struct TcMaps {
  CUtensorMap x, lab, zh, zl;
};

// Shared-memory plan (byte offsets from a 1024-aligned base).
struct TcSmem {
  int zh, zl, abuf, abuf_stride, lo_off, alab, xs, xs_stride, side, side_stride, cb, gsm, csm, clsm, zsm,
      zst, bars, total;
};

__host__ __device__ constexpr int raw_tile_bytes(int mode, int dp) {
  return mode == kModeF32 ? (dp / 32) * kAtomBytes : mode == kModeFP8 ? (dp / 128) * kAtomBytes : 0;
}

// zst: row stride (floats) of the staged centroids, 0 = read them from global memory.
// FP32 rows wider than 128 columns (dp = 256) use the K-chunked layout: the A
// buffers and raw X stages hold one 64-column chunk of a tile, and the row
// terms live in a ring of two tile slots of their own.
__host__ __device__ inline TcSmem tc_smem(int mode, int dp, int kp, int nxs, int nab, int zst) {
  // operand atoms: 64 BF16 columns (128-byte rows), or one atom of 32
  // columns (64-byte rows) when dp = 32
  const int natom = dp >= 64 ? dp / 64 : 1;
  const int rowb = dp >= 64 ? 128 : dp * 2;
  const bool wide = dp > 128;
  const int natom_a = wide ? 1 : natom;  // atoms of one A buffer
  const bool staged = mode != kModeBF16;
  TcSmem s;
  int o = 0;
  s.zh = o; o += natom * kp * rowb;
  o = (o + 1023) & ~1023;
  s.zl = o; o += natom * kp * rowb;
  o = (o + 1023) & ~1023;
  s.abuf = o;
  s.lo_off = natom_a * kTM * rowb;
  s.abuf_stride = natom_a * kTM * rowb * (mode == kModeF32 ? 2 : 1);
  o += nab * s.abuf_stride;
  s.alab = o;  // BF16: the labels of the tile in A buffer i (TMA, with the tile)
  o += staged ? 0 : nab * kTM * 4;
  o = (o + 1023) & ~1023;
  s.xs = o;
  s.xs_stride = staged ? raw_tile_bytes(mode, wide ? 64 : dp) + 1024 : 0;  // + labels (512 B), keeps 1024 alignment
  o += staged ? nxs * s.xs_stride : 0;
  s.side = o;
  s.side_stride = kTM * 16 + 512;  // xn2, aown, inv, code (+ scratch of the wide kernel)
  // a ring of its own, so that an A buffer is free once its MMAs (and, BF16,
  // the converters' reads) are done
  o += kSideSlots * s.side_stride;
  s.cb = o; o += kp * 4 + 32;  // + 8 floats of block-reduction scratch
  o = (o + 15) & ~15;
  s.gsm = o; o += dp * 4;
  s.csm = o; o += mode == kModeFP8 ? dp * 4 : 0;
  s.clsm = o; o += kp * 16;
  s.zst = zst;
  s.zsm = o; o += kp * zst * 4;
  o = (o + 15) & ~15;
  s.bars = o; o += 8 * (2 * nxs + 4 * nab + 4 + 1 + 2 * kSideSlots) + 16;  // + TMEM base, abort flag
  s.total = o + 1024;  // slack for aligning the dynamic base to 1024
  return s;
}

struct TcBars {
  uint64_t *xfull, *xempty, *afull, *aempty, *accfull, *accempty, *zfull, *sfull, *sempty;
  uint32_t* tmem_base;
  int* abort_flag;
};

__device__ inline TcBars tc_bars(unsigned char* base, const TcSmem& L, int nxs, int nab) {
  TcBars b;
  uint64_t* p = reinterpret_cast<uint64_t*>(base + L.bars);
  b.xfull = p; p += nxs;
  b.xempty = p; p += nxs;
  b.afull = p; p += nab;
  b.aempty = p; p += nab;
  b.accfull = p; p += 2;
  b.accempty = p; p += 2;
  b.zfull = p; p += 1;
  b.sfull = p; p += kSideSlots;
  b.sempty = p; p += kSideSlots;
  b.tmem_base = reinterpret_cast<uint32_t*>(p);
  b.abort_flag = reinterpret_cast<int*>(p) + 1;
  return b;
}


// Self-test of failure detection without a fault: one CTA waits on mbarriers
// that nothing completes, through the production waits.  Warp 0 runs tc_wait
// (the pass-2 roles' wait), which must give up after kWaitTimeoutNs with
// SIL_ETIMEOUT and raise the shared abort flag; warp 1 runs mbar_wait (the
// pass-1 row gather's wait), which must return false; warp 2 starts its
// tc_wait half a limit later and must leave on warp 0's abort, before its own
// limit.  out[3]: the bits of warps 0 and 1, and 1 from warp 2 if it left on
// the abort.  Shared memory and `out` only; every loop ends on the global
// timer, the sleep loop also after a fixed number of rounds.
__global__ void k_selftest_wait(uint32_t* out) {
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    abort_flag = 0;
  }
  fence_mbar_init();
  __syncthreads();
  if (lane == 0 && warp == 0) {
    tc_wait(&bars[0], 0, &abort_flag, out);
  } else if (lane == 0 && warp == 1) {
    if (!mbar_wait(&bars[1], 0)) set_status(out + 1, SIL_ETIMEOUT);
  } else if (lane == 0 && warp == 2) {
    const uint64_t t0 = globaltimer_ns();
    // half a limit (a sleep may end early: the time bound ends the loop; the
    // round count only guards against a timer that does not advance)
    for (int i = 0; i < 1000000 && globaltimer_ns() - t0 < kWaitTimeoutNs / 2; ++i) __nanosleep(100000);
    const uint64_t t1 = globaltimer_ns();
    const bool done = tc_wait(&bars[0], 0, &abort_flag, out + 2);
    if (!done && globaltimer_ns() - t1 < kWaitTimeoutNs) atomicOr(out + 2, 1u);
  }
  __syncthreads();
}

// The exact own-cluster term ||x' - mu'_c||^2 (x' = x inv - g) of the rows of
// one converter warp whose cluster c is in this block, a row at a time with
// every lane on DP/32 consecutive columns, so that the centroid row and the
// point row are read coalesced: for plans of several cluster blocks whose
// centroids stay in global memory, where a thread per half row would gather a
// centroid row 16 bytes at a time.  The point row comes from the tile's A
// buffer (BF16: as stored; FP8: the code times its column scale), or, FP32,
// from global memory (the A buffer holds its hi/lo split); the arithmetic per
// element is the converters'.  want: this lane is the first half of a row
// that needs the term (lanes 0-15 hold rows wr0 + lane); returns the term for
// those lanes and keep for the others.  Warp-collective.
template <int MODE, int DP>
__device__ __forceinline__ float tc_own_term_by_warp(const TcK& a, const unsigned char* ab, const unsigned char* gsm_b,
                                                     const unsigned char* csm_b, const float* zfp, int kb0,
                                                     int64_t row0, int wr0, int lane, bool want, int ol, float inv,
                                                     float keep) {
  constexpr int CPL = DP / 32;  // columns per lane
  constexpr int NB = 4;         // rows with their loads in flight
  const float* gsm = reinterpret_cast<const float*>(gsm_b);
  const float* csm = reinterpret_cast<const float*>(csm_b);
  const int c0 = CPL * lane;
  float gl[CPL], sc[CPL];
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
    gl[e] = gsm[c0 + e];
    sc[e] = MODE == kModeFP8 ? csm[c0 + e] : 1.f;
  }
  __syncwarp();  // FP8: the warp's own A rows, written by its lanes
  unsigned m = __ballot_sync(0xffffffffu, want);
  float out = keep;
  while (m) {
    int rr[NB];
    float xv[NB][CPL], zv[NB][CPL];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      rr[j] = m ? __ffs(m) - 1 : -1;  // warp-uniform
      m &= m - 1;
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
#pragma unroll
      for (int e = 0; e < CPL; ++e) xv[j][e] = zv[j][e] = 0.f;
      if (rr[j] < 0) continue;
      const int olj = __shfl_sync(0xffffffffu, ol, rr[j]);
      const float* zr = zfp + int64_t(kb0 + olj) * a.dz;
#pragma unroll
      for (int e = 0; e < CPL; ++e) zv[j][e] = c0 + e < a.dz ? __ldg(zr + c0 + e) : 0.f;
      const int R = wr0 + rr[j];  // tile row
      if (MODE == kModeF32) {
        const float* xr = static_cast<const float*>(a.xg) + (row0 + R) * a.ldx;
#pragma unroll
        for (int e = 0; e < CPL; ++e) xv[j][e] = c0 + e < a.d ? __ldg(xr + c0 + e) : 0.f;
      } else {
        // BF16 operand row R (128-byte swizzle in atoms of 64 columns): the
        // lane's CPL columns lie in one 16-byte chunk
        const unsigned char* p = ab + (c0 / 64) * kAtomBytes + sw128(R, (c0 % 64) / 8) + (c0 % 8) * 2;
        uint32_t w[(CPL + 1) / 2];
        if constexpr (CPL == 4) {
          const uint2 u = *reinterpret_cast<const uint2*>(p);
          w[0] = u.x;
          w[1] = u.y;
        } else if constexpr (CPL == 2) {
          w[0] = *reinterpret_cast<const uint32_t*>(p);
        } else {
          w[0] = *reinterpret_cast<const unsigned short*>(p);
        }
#pragma unroll
        for (int e = 0; e < CPL; ++e) {
          const float v = __uint_as_float((e & 1 ? w[e / 2] >> 16 : w[e / 2]) << 16);
          xv[j][e] = MODE == kModeFP8 ? v * sc[e] : v;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (rr[j] < 0) continue;
      const float invj = __shfl_sync(0xffffffffu, inv, rr[j]);
      float p = 0.f;
#pragma unroll
      for (int e = 0; e < CPL; ++e) {
        const float dd = fmaf(xv[j][e], invj, -gl[e]) - zv[j][e];
        p = fmaf(dd, dd, p);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      if (lane == rr[j]) out = p;
    }
  }
  return out;
}

template <int MODE, int DP, bool TRACK, int CG, bool BATCH = false>
__global__ void __launch_bounds__(tc_threads(DP, CG), 1) k_score_tc(TcK a, const __grid_constant__ TcMaps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles, by offsetting the shared array
  // itself so that every access below stays a shared-space access
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr bool NARROW = DP == 32;           // one 64-byte-swizzled atom of 32 columns
  constexpr int natom = NARROW ? 1 : DP / 64;
  constexpr int ROWB = NARROW ? 64 : 128;     // bytes of one operand row in an atom
  constexpr bool STAGED = MODE != kModeBF16;  // converters build the A operand
  constexpr int EG = tc_epi_groups(DP);
  constexpr int EPI0 = 2 + kConvWarps * CG;  // first epilogue warp
  // the plans never pass odd rings to two converter groups (see
  // tc_rings_ok); refuse them here too rather than alias mbarrier phases
  if (CG == 2 && ((a.nab & 1) || (STAGED && (a.nxs & 1)))) {
    if (threadIdx.x == 0) set_status(a.status + (BATCH ? a.items[blockIdx.y].b : 0), SIL_EUNSUPPORTED);
    return;
  }
  // where the epilogue reads an ill-conditioned row back: plans without the
  // argmin pass (few such rows) from global memory, so that an A buffer is
  // free once its MMAs (and, BF16, the converters' reads) are done; the others
  // from the A buffer, held until then
  constexpr bool ROWS_GLOBAL = !TRACK;
  const TcSmem L = tc_smem(MODE, DP, a.kp, a.nxs, a.nab, a.zst);
  const TcBars B = tc_bars(base, L, a.nxs, a.nab);
  volatile int* abort_flag = B.abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = cdiv(a.n, kTM);
  // tiles of this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...; cluster block blockIdx.y
  const int my_tiles = blockIdx.x < ntiles ? int(cdiv(ntiles - blockIdx.x, gridDim.x)) : 0;
  // This CTA's clusters: block blockIdx.y (of a.kp clusters) of one
  // labeling, or -- several labelings scored in one launch -- all the
  // clusters (at most 512) of labeling a.items[blockIdx.y], with its own
  // constants, labels row, status word and partial-sum slot.
  int kall = a.k, kb0 = int(blockIdx.y) * a.kp, kpc = a.kp, zrow = kb0, lab_b = -1;
  const float* cbp = a.cb;
  const float4* clp = a.cl;
  const float* zfp = a.zf;
  const float* gfp = a.gf;
  bool fused = a.nblk == 1;
  int64_t pidx = blockIdx.x;
  uint32_t* sts = a.status;
  int64_t plane = blockIdx.y, own_plane = 0;
  if constexpr (BATCH) {
    const TcItem it = a.items[blockIdx.y];
    kall = it.k;
    kb0 = it.kb0;
    kpc = it.kp;
    zrow = it.zrow;
    lab_b = it.b;
    cbp = a.cb + it.zrow - it.kb0;  // cbp[kb0 + i] is the block's row i
    clp = a.cl + it.cl_off;
    zfp = a.zf + it.zf_off;
    gfp = a.gf + it.g_off;
    fused = it.nblk == 1;
    pidx = int64_t(it.b) * gridDim.x + blockIdx.x;
    sts = a.status + it.b;
    plane = it.plane;
    own_plane = it.own_plane;
  }
  const int kblk = min(kpc, kall - kb0);  // clusters of this block (>= 1)
  // TMEM: two accumulators (double-buffered tiles) when a block fits in 256
  // columns, one of up to 512 otherwise
  const int acc_cols = BATCH ? tc_pow2(kpc) : a.acc_cols;
  const int nslot = !BATCH || acc_cols <= 256 ? 2 : 1;
  const int sl_shift = nslot == 2 ? 1 : 0;  // tile t uses accumulator t & sl_mask, phase (t >> sl_shift) & 1
  const int sl_mask = nslot - 1;
  float* cbs = reinterpret_cast<float*>(base + L.cb);

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nxs; ++i) {
      mbar_init(&B.xfull[i], 1);
      mbar_init(&B.xempty[i], kConvWarps);
    }
    for (int i = 0; i < a.nab; ++i) {
      mbar_init(&B.afull[i], STAGED ? kConvWarps : 1);  // converters, or the TMA transaction
      // MMA commit (+ BF16: the converter warps; + the 4 epilogue warps where
      // they read the operand rows back)
      mbar_init(&B.aempty[i], 1 + (STAGED ? 0 : kConvWarps) + (ROWS_GLOBAL ? 0 : 4));
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&B.accfull[i], 1);
      mbar_init(&B.accempty[i], 4);
    }
    for (int i = 0; i < kSideSlots; ++i) {
      mbar_init(&B.sfull[i], kConvWarps);
      mbar_init(&B.sempty[i], 4);
    }
    mbar_init(B.zfull, 1);
    *B.abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < kpc; i += blockDim.x) cbs[i] = cbp[kb0 + i];
  float* gsm = reinterpret_cast<float*>(base + L.gsm);
  float* csm = reinterpret_cast<float*>(base + L.csm);
  float4* clsm = reinterpret_cast<float4*>(base + L.clsm);
  float* zsm = reinterpret_cast<float*>(base + L.zsm);
  for (int i = threadIdx.x; i < DP; i += blockDim.x) gsm[i] = i < a.dz ? gfp[i] : 0.f;
  if (MODE == kModeFP8)
    for (int i = threadIdx.x; i < DP; i += blockDim.x) csm[i] = i < a.d ? a.cs[i] : 0.f;
  for (int i = threadIdx.x; i < kblk; i += blockDim.x) clsm[i] = clp[kb0 + i];
  if (a.zst)
    for (int i = threadIdx.x; i < kblk * a.zst; i += blockDim.x) {
      const int kk = i / a.zst, c = i - kk * a.zst;
      zsm[i] = c < a.dz ? zfp[int64_t(kb0 + kk) * a.dz + c] : 0.f;
    }
  if (warp == 1) {  // TMEM: nslot accumulators of acc_cols columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(B.tmem_base)),
                 "r"(nslot * acc_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *B.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------- TMA producer
    if (lane == 0) {
      // the block's split centroids: kpc rows of Z in boxes of a.zbox_rows
      // rows (atoms laid out for a.kp rows)
      mbar_arrive_expect_tx(B.zfull, uint32_t(2 * natom * kpc * ROWB));
      for (int at = 0; at < natom; ++at) {
        for (int r0 = 0; r0 < kpc; r0 += a.zbox_rows) {
          tma_load_2d(base + L.zh + at * a.kp * ROWB + r0 * ROWB, &maps.zh, at * 64, zrow + r0, B.zfull);
          tma_load_2d(base + L.zl + at * a.kp * ROWB + r0 * ROWB, &maps.zl, at * 64, zrow + r0, B.zfull);
        }
      }
      int t = 0;
      for (; t < my_tiles; ++t) {
        const int32_t row0 = int32_t((blockIdx.x + int64_t(t) * gridDim.x) * kTM);
        if (STAGED) {
          const int j = t % a.nxs;
          if (!tc_wait(&B.xempty[j], ((t / a.nxs) & 1) ^ 1, abort_flag, sts)) break;
          unsigned char* xs = base + L.xs + j * L.xs_stride;
          constexpr int raw = raw_tile_bytes(MODE, DP);
          mbar_arrive_expect_tx(&B.xfull[j], uint32_t(raw + kTM * 4));
          if (MODE == kModeF32) {
            for (int s32 = 0; s32 < DP / 32; ++s32)
              tma_load_2d(xs + s32 * kAtomBytes, &maps.x, s32 * 32, row0, &B.xfull[j]);
          } else {
            for (int s128 = 0; s128 < DP / 128; ++s128)
              tma_load_2d(xs + s128 * kAtomBytes, &maps.x, s128 * 128, row0, &B.xfull[j]);
          }
          if constexpr (!BATCH) tma_load_1d(xs + raw, &maps.lab, row0, &B.xfull[j]);
          else tma_load_2d(xs + raw, &maps.lab, row0, lab_b, &B.xfull[j]);
        } else {
          const int i = t % a.nab;
          if (!tc_wait(&B.aempty[i], ((t / a.nab) & 1) ^ 1, abort_flag, sts)) break;
          unsigned char* ab = base + L.abuf + i * L.abuf_stride;
          mbar_arrive_expect_tx(&B.afull[i], uint32_t(natom * kAtomBytes + kTM * 4));
          for (int at = 0; at < natom; ++at)
            tma_load_2d(ab + at * kAtomBytes, &maps.x, at * 64, row0, &B.afull[i]);
          if constexpr (!BATCH) tma_load_1d(base + L.alab + i * kTM * 4, &maps.lab, row0, &B.afull[i]);
          else tma_load_2d(base + L.alab + i * kTM * 4, &maps.lab, row0, lab_b, &B.afull[i]);
        }
      }
      if (*abort_flag) {
        // wait (bounded) for every copy this thread issued and nobody consumed
        const int ring = STAGED ? a.nxs : a.nab;
        uint64_t* full = STAGED ? B.xfull : B.afull;
        const int first = t - ring > 0 ? t - ring : 0;
        for (int u = first; u < t; ++u) mbar_wait(&full[u % ring], uint32_t((u / ring) & 1));
        mbar_wait(B.zfull, 0);
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------- MMA issuer
    if (lane == 0) {
      // blocks wider than 256 clusters (one labeling of a batched launch) run
      // as two MMAs of N <= 256 into adjacent TMEM columns
      const int nh = BATCH && kpc > 256 ? 2 : 1;
      int t = 0;
      bool ok = tc_wait(B.zfull, 0, abort_flag, sts);
      for (; ok && t < my_tiles; ++t) {
        const int i = t % a.nab, bsel = t & sl_mask;
        if (!tc_wait(&B.afull[i], (t / a.nab) & 1, abort_flag, sts)) break;
        if (!tc_wait(&B.accempty[bsel], ((t >> sl_shift) & 1) ^ 1, abort_flag, sts)) break;
        tc_fence_after();
        const uint32_t ahi = smem_u32(base + L.abuf + i * L.abuf_stride);
        const uint32_t alo = ahi + uint32_t(L.lo_off);
        for (int hh = 0; hh < nh; ++hh) {
          const uint32_t idesc = umma_idesc_bf16(kTM, hh == 0 ? (kpc < 256 ? kpc : 256) : kpc - 256);
          const uint32_t d_tmem = tmem + uint32_t(bsel * acc_cols + hh * 256);
          const uint32_t zh = smem_u32(base + L.zh) + uint32_t(hh * 256 * ROWB);
          const uint32_t zl = smem_u32(base + L.zl) + uint32_t(hh * 256 * ROWB);
          // The small correction products (x.Z_lo, x_lo.Z_hi) go into the fresh
          // accumulator first and the large x_hi.Z_hi products last: each
          // tensor-core accumulation rounds relative to the running magnitude,
          // so this order adds the fewest steps at the final, largest magnitude
          // (a measured bias of ~1e-6 in b_i when the order was interleaved).
          if constexpr (NARROW) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t o = uint32_t(ks * 32);
              umma_bf16(d_tmem, umma_desc_sw64(ahi + o), umma_desc_sw64(zl + o), idesc, ks != 0);
              umma_bf16(d_tmem, umma_desc_sw64(alo + o), umma_desc_sw64(zh + o), idesc, 1);
            }
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t o = uint32_t(ks * 32);
              umma_bf16(d_tmem, umma_desc_sw64(ahi + o), umma_desc_sw64(zh + o), idesc, 1);
            }
          } else {
#pragma unroll
            for (int at = 0; at < natom; ++at) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t ao = uint32_t(at * kAtomBytes + ks * 32);
                const uint32_t bo = uint32_t(at * a.kp * 128 + ks * 32);
                umma_bf16(d_tmem, umma_desc_sw128(ahi + ao), umma_desc_sw128(zl + bo), idesc, (at | ks) != 0);
                if (MODE == kModeF32)
                  umma_bf16(d_tmem, umma_desc_sw128(alo + ao), umma_desc_sw128(zh + bo), idesc, 1);
              }
            }
#pragma unroll
            for (int at = 0; at < natom; ++at) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint32_t ao = uint32_t(at * kAtomBytes + ks * 32);
                const uint32_t bo = uint32_t(at * a.kp * 128 + ks * 32);
                umma_bf16(d_tmem, umma_desc_sw128(ahi + ao), umma_desc_sw128(zh + bo), idesc, 1);
              }
            }
          }
        }
        umma_commit(&B.accfull[bsel]);
        umma_commit(&B.aempty[i]);
      }
      if (*abort_flag && t > 0) {
        // the last committed accumulator must be complete before TMEM is freed
        const int u = t - 1;
        mbar_wait(&B.accfull[u & sl_mask], uint32_t((u >> sl_shift) & 1));
      }
    }
  } else if (warp < EPI0) {
    // ------------------------------------------------ converter warps 2..EPI0-1
    // lanes 0-15 and 16-31 of a warp hold the two halves of the same 16 rows;
    // group cg takes tiles cg, cg + CG, ...
    constexpr int HP = DP / 2;  // columns per half
    const int h = lane >> 4;
    const int cg = (warp - 2) / kConvWarps;
    const int r = ((warp - 2) % kConvWarps) * 16 + (lane & 15);  // tile row of this thread
    for (int t = cg; t < my_tiles; t += CG) {
      const int i = t % a.nab;
      const int64_t row = (blockIdx.x + int64_t(t) * gridDim.x) * kTM + r;
      unsigned char* ab = base + L.abuf + i * L.abuf_stride;
      const int sl = t % kSideSlots;  // row-term slot
      float* side = reinterpret_cast<float*>(base + L.side + sl * L.side_stride);
      float x[HP];
      int own;
      if (STAGED) {
        const int j = t % a.nxs;
        if (!tc_wait(&B.xfull[j], (t / a.nxs) & 1, abort_flag, sts)) break;
        // FP8 writes the A operand while it reads the stage; FP32 waits for its
        // A buffer only after the row terms (the MMA of the previous tile in
        // that buffer overlaps them)
        if (MODE == kModeFP8 && !tc_wait(&B.aempty[i], ((t / a.nab) & 1) ^ 1, abort_flag, sts)) break;
        const unsigned char* xs = base + L.xs + j * L.xs_stride;
        if (MODE == kModeF32) {
#pragma unroll
          for (int c4 = 0; c4 < HP / 4; ++c4) {
            const int col = h * HP + 4 * c4;
            const float4 v =
                *reinterpret_cast<const float4*>(xs + (col / 32) * kAtomBytes + sw128(r, (col % 32) / 4));
            x[4 * c4 + 0] = v.x;
            x[4 * c4 + 1] = v.y;
            x[4 * c4 + 2] = v.z;
            x[4 * c4 + 3] = v.w;
          }
        } else {
          // FP8 codes, 16 per 16-byte chunk; the A operand takes the codes
          // themselves (exact in BF16), the per-point terms below the scaled values
#pragma unroll
          for (int c16 = 0; c16 < HP / 16; ++c16) {
            const int col = h * HP + 16 * c16;
            const uint4 u =
                *reinterpret_cast<const uint4*>(xs + (col / 128) * kAtomBytes + sw128(r, (col % 128) / 16));
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
            uint32_t hw[8];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float2 f0 = fp8x2_to_float2(w[e]);
              const float2 f1 = fp8x2_to_float2(w[e] >> 16);
              x[16 * c16 + 4 * e + 0] = f0.x;
              x[16 * c16 + 4 * e + 1] = f0.y;
              x[16 * c16 + 4 * e + 2] = f1.x;
              x[16 * c16 + 4 * e + 3] = f1.y;
              hw[2 * e] = pack_bf16x2(f0.x, f0.y);
              hw[2 * e + 1] = pack_bf16x2(f1.x, f1.y);
            }
            // 16 columns = two 16-byte chunks of the BF16 operand
            *reinterpret_cast<uint4*>(ab + (col / 64) * kAtomBytes + sw128(r, (col % 64) / 8)) =
                make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(ab + ((col + 8) / 64) * kAtomBytes + sw128(r, ((col + 8) % 64) / 8)) =
                make_uint4(hw[4], hw[5], hw[6], hw[7]);
          }
          fence_proxy_async_smem();
#pragma unroll
          for (int c4 = 0; c4 < HP / 4; ++c4) {
            const float4 s4 = *reinterpret_cast<const float4*>(csm + h * HP + 4 * c4);
            const float2 xa = __fmul2_rn(make_float2(x[4 * c4], x[4 * c4 + 1]), make_float2(s4.x, s4.y));
            const float2 xb = __fmul2_rn(make_float2(x[4 * c4 + 2], x[4 * c4 + 3]), make_float2(s4.z, s4.w));
            x[4 * c4 + 0] = xa.x;
            x[4 * c4 + 1] = xa.y;
            x[4 * c4 + 2] = xb.x;
            x[4 * c4 + 3] = xb.y;
          }
        }
        own = reinterpret_cast<const int32_t*>(xs + raw_tile_bytes(MODE, DP))[r];
        // the stage is in registers now: let the producer refill it.  The
        // refill is an async-proxy (TMA) write after these generic-proxy
        // reads, so the reads are fenced against it before the release.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.xempty[j]);
      } else {
        if (!tc_wait(&B.afull[i], (t / a.nab) & 1, abort_flag, sts)) break;
#pragma unroll
        for (int c8 = 0; c8 < HP / 8; ++c8) {
          const int col = h * HP + 8 * c8;
          const uint4 u = *reinterpret_cast<const uint4*>(ab + (col / 64) * kAtomBytes + sw128(r, (col % 64) / 8));
          const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[e]));
            x[8 * c8 + 2 * e] = f.x;
            x[8 * c8 + 2 * e + 1] = f.y;
          }
        }
        own = reinterpret_cast<const int32_t*>(base + L.alab + i * kTM * 4)[r];
      }
      bool valid = row < a.n;
      if (valid && (own < 0 || own >= kall)) {
        if (h == 0) set_status(sts, SIL_ELABEL);
        valid = false;
      }
      float inv = 1.f;
      if (a.cosine) {
        float2 ss2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < HP; c += 2) {
          const float2 xv = make_float2(x[c], x[c + 1]);
          ss2 = __ffma2_rn(xv, xv, ss2);
        }
        float ss = ss2.x + ss2.y;
        ss += __shfl_xor_sync(0xffffffffu, ss, 16);
        if (valid && !(ss > 0.f)) {
          if (h == 0) set_status(sts, SIL_EZERONORM);
          valid = false;
        }
        inv = ss > 0.f ? rsqrtf(ss) : 0.f;
      }
      // is the point's own cluster in this block?
      const int ol = own - kb0;
      const bool in_blk = valid && ol >= 0 && ol < kblk;
      const int olc = in_blk ? ol : 0;
      // ||x'||^2 and the exact own-cluster term (x' = x inv - g), half a row
      // each, two columns per packed FP32x2 instruction
      float2 xn2 = make_float2(0.f, 0.f), ae = xn2;
      const float2 inv2 = make_float2(inv, inv);
      if (!(CG == 1 && a.own_rows)) {  // uniform branch
#pragma unroll
        for (int c4 = 0; c4 < HP / 4; ++c4) {
          const int col = h * HP + 4 * c4;
          const float4 g = *reinterpret_cast<const float4*>(gsm + col);
          float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (col < a.dz) {
            if (a.zst)  // staged centroids (uniform branch)
              z = *reinterpret_cast<const float4*>(zsm + olc * a.zst + col);
            else
              z = __ldg(reinterpret_cast<const float4*>(zfp + int64_t(kb0 + olc) * a.dz + col));
          }
          const float2 xa = make_float2(x[4 * c4], x[4 * c4 + 1]), xb = make_float2(x[4 * c4 + 2], x[4 * c4 + 3]);
          const float2 ca = __ffma2_rn(xa, inv2, make_float2(-g.x, -g.y));
          const float2 cb = __ffma2_rn(xb, inv2, make_float2(-g.z, -g.w));
          xn2 = __ffma2_rn(ca, ca, xn2);
          xn2 = __ffma2_rn(cb, cb, xn2);
          const float2 da = __fadd2_rn(ca, make_float2(-z.x, -z.y));
          const float2 db = __fadd2_rn(cb, make_float2(-z.z, -z.w));
          ae = __ffma2_rn(da, da, ae);
          ae = __ffma2_rn(db, db, ae);
        }
      } else {  // the own-cluster term comes from tc_own_term_by_warp
#pragma unroll
        for (int c4 = 0; c4 < HP / 4; ++c4) {
          const float4 g = *reinterpret_cast<const float4*>(gsm + h * HP + 4 * c4);
          const float2 xa = make_float2(x[4 * c4], x[4 * c4 + 1]), xb = make_float2(x[4 * c4 + 2], x[4 * c4 + 3]);
          const float2 ca = __ffma2_rn(xa, inv2, make_float2(-g.x, -g.y));
          const float2 cb = __ffma2_rn(xb, inv2, make_float2(-g.z, -g.w));
          xn2 = __ffma2_rn(ca, ca, xn2);
          xn2 = __ffma2_rn(cb, cb, xn2);
        }
      }
      float xn2s = xn2.x + xn2.y, aes = ae.x + ae.y;
      xn2s += __shfl_xor_sync(0xffffffffu, xn2s, 16);
      aes += __shfl_xor_sync(0xffffffffu, aes, 16);
      if (MODE == kModeF32) {
        if (!tc_wait(&B.aempty[i], ((t / a.nab) & 1) ^ 1, abort_flag, sts)) break;
        // hi/lo BF16 split of this half row into the swizzled A buffer
#pragma unroll
        for (int c8 = 0; c8 < HP / 8; ++c8) {
          const int col = h * HP + 8 * c8;
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 xv = make_float2(x[8 * c8 + 2 * e], x[8 * c8 + 2 * e + 1]);
            const __nv_bfloat162 hv = __floats2bfloat162_rn(xv.x, xv.y);
            const float2 hf = __bfloat1622float2(hv);
            const float2 rem = __fadd2_rn(xv, make_float2(-hf.x, -hf.y));
            hw[e] = *reinterpret_cast<const uint32_t*>(&hv);
            lw[e] = pack_bf16x2(rem.x, rem.y);
          }
          const int off = NARROW ? sw64(r, col / 8) : (col / 64) * kAtomBytes + sw128(r, (col % 64) / 8);
          *reinterpret_cast<uint4*>(ab + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(ab + L.lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_proxy_async_smem();
      }
      if (STAGED) {
        // the A buffer is complete: the MMA may start while the row terms wait
        // for their slot
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.afull[i]);
      }
      if (CG == 1 && a.own_rows) aes = tc_own_term_by_warp<MODE, DP>(a, ab, base + L.gsm, base + L.csm, zfp, kb0,
                                                          (blockIdx.x + int64_t(t) * gridDim.x) * kTM,
                                                          r - (lane & 15), lane, in_blk && h == 0, ol, inv, aes);
      if (!STAGED) {
        // the operand rows and labels are read: TMA (async proxy) may refill
        // the buffer once the MMAs are done too
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.aempty[i]);
      }
      if (!tc_wait(&B.sempty[sl], ((t / kSideSlots) & 1) ^ 1, abort_flag, sts)) break;
      if (h == 0) {
        float aown = 0.f;
        int code = valid ? kOwnElsewhere : kRowInvalid;
        if (in_blk) {
          const float4 co = clsm[ol];
          aown = fmaf(co.y, aes, co.z);
          code = co.w < 1.5f ? -2 - ol : ol;  // singleton: s_i = 0, b_i still reported
        }
        side[r] = xn2s;
        side[kTM + r] = aown;
        side[2 * kTM + r] = inv;
        reinterpret_cast<int*>(side)[3 * kTM + r] = code;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.sfull[sl]);
    }
  } else {
    // ---------------------------------------------- epilogue warps EPI0..
    const int q = warp & 3;       // TMEM lane quarter this warp may access
    const int r = q * 32 + lane;  // tile row = TMEM lane
    // this warp's group takes tiles eg, eg + EG, ... and owns accumulator eg;
    // with a single (wide) accumulator group 0 takes every tile, so that no
    // group waits on a barrier phase the other group's tile also completes
    const int eg = (warp - EPI0) >> 2;
    const int egs = nslot == 2 ? EG : 1;
    const float rb = tc_cond_radius(clp, kall, gsm, DP, lane);
    float tsum = 0.f;
    for (int t = eg; eg < egs && t < my_tiles; t += egs) {
      const int i = t % a.nab, bsel = t & sl_mask, sl = t % kSideSlots;
      if (!tc_wait(&B.accfull[bsel], (t >> sl_shift) & 1, abort_flag, sts)) break;
      if (!tc_wait(&B.sfull[sl], (t / kSideSlots) & 1, abort_flag, sts)) break;
      tc_fence_after();
      const float* side = reinterpret_cast<const float*>(base + L.side + sl * L.side_stride);
      const int code = reinterpret_cast<const int*>(side)[3 * kTM + r];
      const bool row_ok = code != kRowInvalid;
      const int own = code >= 0 ? code : (row_ok && code <= -2 ? -2 - code : -1);  // in-block index
      const float sc = -2.f * side[2 * kTM + r];
      const float xn2 = side[r];
      const uint32_t tbase = tmem + uint32_t(bsel * acc_cols) + (uint32_t(q * 32) << 16);
      int kb = -1;
      // two warpgroups keep half the registers each: two loads in flight
      const float best = tc_lane_min<TRACK, EG == 2 ? 2 : 4>(tbase, kpc, cbs, sc, own, kb);
      // The GEMM ranks the clusters; for ill-conditioned rows b_i is then the
      // nearest cluster's distance in the difference form, like a_i, from the
      // point's operand row: its A buffer (held until this has been read), or,
      // for FP32 plans without the argmin pass, the row read back from global
      // memory and rounded to the same hi + lo bits.
      const bool exact = row_ok && best < INFINITY && tc_ill_conditioned(xn2, best, rb);
      if (!TRACK && __any_sync(0xffffffffu, exact)) kb = tc_lane_find(tbase, kpc, cbs, sc, own, best, exact);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.accempty[bsel]);
      float dk = best < INFINITY ? xn2 + best : INFINITY;
      const int64_t row = (blockIdx.x + int64_t(t) * gridDim.x) * kTM + r;
      if (exact && kb >= 0) {
        const float4 co = clsm[kb];
        const float wn = co.y > 0.f ? co.z / co.y : 0.f;  // W_k / n_k
        if (ROWS_GLOBAL) {
          const float* zk = a.zst ? zsm + kb * a.zst : zfp + int64_t(kb0 + kb) * a.dz;
          if (MODE == kModeF32)
            dk = wn + tc_row_dist_global<true>(static_cast<const float*>(a.xg) + row * a.ldx, a.d, side[2 * kTM + r],
                                               gsm, zk);
          else
            dk = wn + tc_row_dist_lp_global<MODE, DP>(
                          static_cast<const unsigned char*>(a.xg) + row * a.ldx * (MODE == kModeBF16 ? 2 : 1), a.d,
                          side[2 * kTM + r], gsm, csm, zk, a.dz);
        } else {
          if (!STAGED) tc_wait(&B.afull[i], (t / a.nab) & 1, abort_flag, sts);  // TMA-written rows
          dk = wn + tc_row_dist<MODE, DP>(base + L.abuf + i * L.abuf_stride, L.lo_off, r, side[2 * kTM + r], gsm,
                                          csm, a.zst ? zsm + kb * a.zst : nullptr, zfp + int64_t(kb0 + kb) * a.dz,
                                          a.dz);
        }
      }
      if (!ROWS_GLOBAL) {
        // the operand rows are read: the converters (or, BF16, TMA) may
        // rebuild the buffer
        if (!STAGED) fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.aempty[i]);
      }
      if (row < a.n) {
        if (fused) {
          float av = 0.f, bv = INFINITY, sv = 0.f;
          if (row_ok) {
            const bool has_b = dk < INFINITY;
            av = fmaxf(0.f, a.scale * side[kTM + r]);
            bv = has_b ? fmaxf(0.f, a.scale * dk) : INFINITY;
            if (code >= 0 && has_b) {
              sv = sil_eq2(av, bv, a.rms != 0);
            }
            if (!has_b) kb = -1;
          } else {
            kb = -1;
          }
          if (a.s_out) a.s_out[row] = sv;
          if (TRACK && a.sa) {
            a.sa[row] = av;
            a.sb[row] = bv;
            a.skstar[row] = kb;
          }
          tsum += sv;
        } else {
          const int64_t o = plane * a.n + row;
          a.pmin[o] = row_ok ? dk : __int_as_float(0x7fc00000);
          if (TRACK && a.parg) a.parg[o] = (row_ok && dk < INFINITY) ? kb0 + kb : -1;
          if (own >= 0) a.pown[own_plane * a.n + row] = side[kTM + r];
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.sempty[sl]);
    }
    if (fused) {
      // block partial over the epilogue threads
      for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
      float* red = cbs + a.kp;  // 8 floats of scratch right after cb (within the plan's padding)
      if (lane == 0) red[warp - EPI0] = tsum;
      asm volatile("bar.sync 1, %0;" ::"n"(128 * EG) : "memory");
      if (warp == EPI0 && lane == 0) {
        double p = 0.0;
        for (int w = 0; w < 4 * EG; ++w) p += double(red[w]);
        a.partials[pidx] = p;
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(nslot * acc_cols)
                 : "memory");
  }
}

// FP32 rows of 129..256 columns.  The same roles and epilogue as k_score_tc,
// but the GEMM runs over K-chunks of 64 columns: the producer loads one chunk
// of a tile per raw stage (labels with chunk 0), converter threads split one
// chunk at a time into an A buffer while they accumulate their row terms over
// the chunks, and the MMA warp accumulates the four chunks of a tile into one
// TMEM accumulator.  The split centroids of all 256 columns stay resident.
// Row terms: squared Euclidean uses the exact difference forms chunk by
// chunk; cosine needs 1/||x|| before x' exists, so it accumulates x.x, x.g,
// x.(g + mu'_c), g.g and ||g + mu'_c||^2 and forms ||x' ||^2 and
// ||x' - mu'_c||^2 from them at the end (all terms are O(1) for unit vectors).
template <bool TRACK>
__global__ void __launch_bounds__(kTcThreads, 1) k_score_tc_wide(TcK a, const __grid_constant__ TcMaps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr int DP = 256, NCH = 4, natom = 4;
  const TcSmem L = tc_smem(kModeF32, DP, a.kp, a.nxs, a.nab, a.zst);
  const TcBars B = tc_bars(base, L, a.nxs, a.nab);
  volatile int* abort_flag = B.abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = cdiv(a.n, kTM);
  const int my_tiles = blockIdx.x < ntiles ? int(cdiv(ntiles - blockIdx.x, gridDim.x)) : 0;
  const int kb0 = int(blockIdx.y) * a.kp;
  const int kblk = min(a.kp, a.k - kb0);
  const bool fused = a.nblk == 1;
  float* cbs = reinterpret_cast<float*>(base + L.cb);

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.nxs; ++i) {
      mbar_init(&B.xfull[i], 1);
      mbar_init(&B.xempty[i], kConvWarps);
    }
    for (int i = 0; i < a.nab; ++i) {
      mbar_init(&B.afull[i], kConvWarps);
      mbar_init(&B.aempty[i], 1);  // MMA commit
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&B.accfull[i], 1);
      mbar_init(&B.accempty[i], 4);
    }
    for (int i = 0; i < kSideSlots; ++i) {
      mbar_init(&B.sfull[i], kConvWarps);
      mbar_init(&B.sempty[i], 4);
    }
    mbar_init(B.zfull, 1);
    *B.abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < a.kp; i += blockDim.x) cbs[i] = a.cb[kb0 + i];
  float* gsm = reinterpret_cast<float*>(base + L.gsm);
  float4* clsm = reinterpret_cast<float4*>(base + L.clsm);
  float* zsm = reinterpret_cast<float*>(base + L.zsm);
  for (int i = threadIdx.x; i < DP; i += blockDim.x) gsm[i] = i < a.dz ? a.gf[i] : 0.f;
  for (int i = threadIdx.x; i < kblk; i += blockDim.x) clsm[i] = a.cl[kb0 + i];
  if (a.zst)
    for (int i = threadIdx.x; i < kblk * a.zst; i += blockDim.x) {
      const int kk = i / a.zst, c = i - kk * a.zst;
      zsm[i] = c < a.dz ? a.zf[int64_t(kb0 + kk) * a.dz + c] : 0.f;
    }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(B.tmem_base)),
                 "r"(2 * a.acc_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *B.tmem_base;
  constexpr int raw = 2 * kAtomBytes;  // two 32-column FP32 boxes per chunk

  if (warp == 0) {
    // ------------------------------------------------------- TMA producer
    if (lane == 0) {
      mbar_arrive_expect_tx(B.zfull, uint32_t(2 * natom * a.kp * 128));
      for (int at = 0; at < natom; ++at) {
        tma_load_2d(base + L.zh + at * a.kp * 128, &maps.zh, at * 64, kb0, B.zfull);
        tma_load_2d(base + L.zl + at * a.kp * 128, &maps.zl, at * 64, kb0, B.zfull);
      }
      int u = 0;
      for (int t = 0; t < my_tiles && !*abort_flag; ++t) {
        const int32_t row0 = int32_t((blockIdx.x + int64_t(t) * gridDim.x) * kTM);
        for (int c = 0; c < NCH; ++c, ++u) {
          const int j = u % a.nxs;
          if (!tc_wait(&B.xempty[j], ((u / a.nxs) & 1) ^ 1, abort_flag, a.status)) break;
          unsigned char* xs = base + L.xs + j * L.xs_stride;
          mbar_arrive_expect_tx(&B.xfull[j], uint32_t(raw + (c == 0 ? kTM * 4 : 0)));
          tma_load_2d(xs, &maps.x, c * 64, row0, &B.xfull[j]);
          tma_load_2d(xs + kAtomBytes, &maps.x, c * 64 + 32, row0, &B.xfull[j]);
          if (c == 0) tma_load_1d(xs + raw, &maps.lab, row0, &B.xfull[j]);
        }
      }
      if (*abort_flag) {
        const int first = u - a.nxs > 0 ? u - a.nxs : 0;
        for (int v = first; v < u; ++v) mbar_wait(&B.xfull[v % a.nxs], uint32_t((v / a.nxs) & 1));
        mbar_wait(B.zfull, 0);
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_bf16(kTM, a.kp);
      int u = 0, issued = -1;
      bool ok = tc_wait(B.zfull, 0, abort_flag, a.status);
      for (int t = 0; ok && t < my_tiles; ++t) {
        const int bsel = t & 1;
        if (!tc_wait(&B.accempty[bsel], ((t >> 1) & 1) ^ 1, abort_flag, a.status)) break;
        const uint32_t d_tmem = tmem + uint32_t(bsel * a.acc_cols);
        for (int c = 0; c < NCH; ++c, ++u) {
          const int i = u % a.nab;
          if (!tc_wait(&B.afull[i], (u / a.nab) & 1, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ahi = smem_u32(base + L.abuf + i * L.abuf_stride);
          const uint32_t alo = ahi + uint32_t(L.lo_off);
          const uint32_t zh = smem_u32(base + L.zh) + uint32_t(c * a.kp * 128);
          const uint32_t zl = smem_u32(base + L.zl) + uint32_t(c * a.kp * 128);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t ao = uint32_t(ks * 32), bo = uint32_t(ks * 32);
            umma_bf16(d_tmem, umma_desc_sw128(ahi + ao), umma_desc_sw128(zh + bo), idesc, (c | ks) != 0);
            umma_bf16(d_tmem, umma_desc_sw128(ahi + ao), umma_desc_sw128(zl + bo), idesc, 1);
            umma_bf16(d_tmem, umma_desc_sw128(alo + ao), umma_desc_sw128(zh + bo), idesc, 1);
          }
          umma_commit(&B.aempty[i]);
          issued = u;
        }
        if (!ok) break;
        umma_commit(&B.accfull[bsel]);
      }
      if (*abort_flag && issued >= 0) {
        // every MMA issued so far has completed once its last commit arrived
        mbar_wait(&B.aempty[issued % a.nab], uint32_t((issued / a.nab) & 1));
      }
    }
  } else if (warp < kEpiWarp0) {
    // ------------------------------------------------ converter warps 2..9
    constexpr int HP = 32;  // columns of a chunk per thread (half of 64)
    const int h = lane >> 4;
    const int r = (warp - 2) * 16 + (lane & 15);
    const bool cosine = a.cosine != 0;
    int u = 0;
    for (int t = 0; t < my_tiles; ++t) {
      const int64_t row = (blockIdx.x + int64_t(t) * gridDim.x) * kTM + r;
      int own = -1, olc = 0;
      bool valid = row < a.n, in_blk = false;
      // squared Euclidean: s0 = ||x'||^2, s1 = ||x' - mu'_c||^2 (exact forms);
      // cosine: x.x, x.g, x.(g + mu'_c), g.g, ||g + mu'_c||^2
      float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0, s4 = s0;
      bool stop = false;
      // the own centroid's 32 columns of the chunk being worked on, loaded one
      // chunk ahead so that the gathers overlap the waits and the split
      float4 zr[HP / 4];
      auto load_z = [&](int c) {
#pragma unroll
        for (int c4 = 0; c4 < HP / 4; ++c4) {
          const int col = c * 64 + h * HP + 4 * c4;
          float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
          if (col < a.dz) {
            if (a.zst)
              z = *reinterpret_cast<const float4*>(zsm + olc * a.zst + col);
            else
              z = __ldg(reinterpret_cast<const float4*>(a.zf + int64_t(kb0 + olc) * a.dz + col));
          }
          zr[c4] = z;
        }
      };
      for (int c = 0; c < NCH; ++c, ++u) {
        const int i = u % a.nab, j = u % a.nxs;
        if (!tc_wait(&B.xfull[j], (u / a.nxs) & 1, abort_flag, a.status) ||
            !tc_wait(&B.aempty[i], ((u / a.nab) & 1) ^ 1, abort_flag, a.status)) {
          stop = true;
          break;
        }
        const unsigned char* xs = base + L.xs + j * L.xs_stride;
        unsigned char* ab = base + L.abuf + i * L.abuf_stride;
        if (c == 0) {
          own = reinterpret_cast<const int32_t*>(xs + raw)[r];
          if (valid && (own < 0 || own >= a.k)) {
            if (h == 0) set_status(a.status, SIL_ELABEL);
            valid = false;
          }
          const int ol = own - kb0;
          in_blk = valid && ol >= 0 && ol < kblk;
          olc = in_blk ? ol : 0;
          load_z(0);
        }
        float x[HP];
#pragma unroll
        for (int c4 = 0; c4 < HP / 4; ++c4) {
          const float4 v = *reinterpret_cast<const float4*>(xs + h * kAtomBytes + sw128(r, c4));
          x[4 * c4 + 0] = v.x;
          x[4 * c4 + 1] = v.y;
          x[4 * c4 + 2] = v.z;
          x[4 * c4 + 3] = v.w;
        }
        // the stage is in registers now: let the producer refill it.  The
        // refill is an async-proxy (TMA) write after these generic-proxy
        // reads, so the reads are fenced against it before the release.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.xempty[j]);
#pragma unroll
        for (int c4 = 0; c4 < HP / 4; ++c4) {
          const int col = c * 64 + h * HP + 4 * c4;  // global column
          const float4 g = *reinterpret_cast<const float4*>(gsm + col);
          const float4 z = zr[c4];
          const float2 xa = make_float2(x[4 * c4], x[4 * c4 + 1]), xb = make_float2(x[4 * c4 + 2], x[4 * c4 + 3]);
          const float2 ga = make_float2(g.x, g.y), gb = make_float2(g.z, g.w);
          if (!cosine) {
            const float2 ca = __fadd2_rn(xa, make_float2(-g.x, -g.y));
            const float2 cb = __fadd2_rn(xb, make_float2(-g.z, -g.w));
            s0 = __ffma2_rn(ca, ca, s0);
            s0 = __ffma2_rn(cb, cb, s0);
            const float2 da = __fadd2_rn(ca, make_float2(-z.x, -z.y));
            const float2 db = __fadd2_rn(cb, make_float2(-z.z, -z.w));
            s1 = __ffma2_rn(da, da, s1);
            s1 = __ffma2_rn(db, db, s1);
          } else {
            const float2 gza = __fadd2_rn(ga, make_float2(z.x, z.y)), gzb = __fadd2_rn(gb, make_float2(z.z, z.w));
            s0 = __ffma2_rn(xa, xa, s0);
            s0 = __ffma2_rn(xb, xb, s0);
            s1 = __ffma2_rn(xa, ga, s1);
            s1 = __ffma2_rn(xb, gb, s1);
            s2 = __ffma2_rn(xa, gza, s2);
            s2 = __ffma2_rn(xb, gzb, s2);
            s3 = __ffma2_rn(ga, ga, s3);
            s3 = __ffma2_rn(gb, gb, s3);
            s4 = __ffma2_rn(gza, gza, s4);
            s4 = __ffma2_rn(gzb, gzb, s4);
          }
        }
        // hi/lo BF16 split of this thread's 32 columns of the chunk
#pragma unroll
        for (int c8 = 0; c8 < HP / 8; ++c8) {
          const int col = h * HP + 8 * c8;  // column within the chunk
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 xv = make_float2(x[8 * c8 + 2 * e], x[8 * c8 + 2 * e + 1]);
            const __nv_bfloat162 hv = __floats2bfloat162_rn(xv.x, xv.y);
            const float2 hf = __bfloat1622float2(hv);
            const float2 rem = __fadd2_rn(xv, make_float2(-hf.x, -hf.y));
            hw[e] = *reinterpret_cast<const uint32_t*>(&hv);
            lw[e] = pack_bf16x2(rem.x, rem.y);
          }
          const int off = sw128(r, col / 8);
          *reinterpret_cast<uint4*>(ab + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(ab + L.lo_off + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        if (c + 1 < NCH) load_z(c + 1);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&B.afull[i]);
      }
      if (stop) break;
      // both halves of the row: fold and form the row terms
      float v0 = s0.x + s0.y, v1 = s1.x + s1.y, v2 = s2.x + s2.y, v3 = s3.x + s3.y, v4 = s4.x + s4.y;
      v0 += __shfl_xor_sync(0xffffffffu, v0, 16);
      v1 += __shfl_xor_sync(0xffffffffu, v1, 16);
      v2 += __shfl_xor_sync(0xffffffffu, v2, 16);
      v3 += __shfl_xor_sync(0xffffffffu, v3, 16);
      v4 += __shfl_xor_sync(0xffffffffu, v4, 16);
      float inv = 1.f, xn2 = v0, aes = v1;
      if (cosine) {
        if (valid && !(v0 > 0.f)) {
          if (h == 0) set_status(a.status, SIL_EZERONORM);
          valid = false;
          in_blk = false;
        }
        inv = v0 > 0.f ? rsqrtf(v0) : 0.f;
        const float xx = v0 * inv * inv;  // ||x_hat||^2 (= 1 up to rounding)
        xn2 = fmaxf(0.f, xx - 2.f * inv * v1 + v3);
        aes = fmaxf(0.f, xx - 2.f * inv * v2 + v4);
      }
      const int s = t % kSideSlots;
      if (!tc_wait(&B.sempty[s], ((t / kSideSlots) & 1) ^ 1, abort_flag, a.status)) break;
      float* side = reinterpret_cast<float*>(base + L.side + s * L.side_stride);
      if (h == 0) {
        float aown = 0.f;
        int code = valid ? kOwnElsewhere : kRowInvalid;
        if (in_blk) {
          const float4 co = clsm[olc];
          aown = fmaf(co.y, aes, co.z);
          code = co.w < 1.5f ? -2 - olc : olc;
        }
        side[r] = xn2;
        side[kTM + r] = aown;
        side[2 * kTM + r] = inv;
        reinterpret_cast<int*>(side)[3 * kTM + r] = code;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&B.sfull[s]);
    }
  } else {
    // ---------------------------------------------- epilogue warps 10..13
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const float rb = tc_cond_radius(a.cl, a.k, gsm, DP, lane);
    float tsum = 0.f;
    for (int t = 0; t < my_tiles; ++t) {
      const int bsel = t & 1, sl = t % kSideSlots;
      if (!tc_wait(&B.accfull[bsel], (t >> 1) & 1, abort_flag, a.status)) break;
      if (!tc_wait(&B.sfull[sl], (t / kSideSlots) & 1, abort_flag, a.status)) break;
      tc_fence_after();
      const float* side = reinterpret_cast<const float*>(base + L.side + sl * L.side_stride);
      const int code = reinterpret_cast<const int*>(side)[3 * kTM + r];
      const bool row_ok = code != kRowInvalid;
      const int own = code >= 0 ? code : (row_ok && code <= -2 ? -2 - code : -1);
      const float sc = -2.f * side[2 * kTM + r];
      const float xn2 = side[r], aown = side[kTM + r], inv = side[2 * kTM + r];
      const uint32_t tbase = tmem + uint32_t(bsel * a.acc_cols) + (uint32_t(q * 32) << 16);
      int kb = -1;
      const float best = tc_lane_min<TRACK, 4>(tbase, a.kp, cbs, sc, own, kb);
      const bool exact = row_ok && best < INFINITY && tc_ill_conditioned(xn2, best, rb);
      if (!TRACK && __any_sync(0xffffffffu, exact)) kb = tc_lane_find(tbase, a.kp, cbs, sc, own, best, exact);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&B.accempty[bsel]);
        mbar_arrive(&B.sempty[sl]);
      }
      const int64_t row = (blockIdx.x + int64_t(t) * gridDim.x) * kTM + r;
      float dk = best < INFINITY ? xn2 + best : INFINITY;
      if (exact && kb >= 0 && row < a.n) {
        // ill-conditioned row: the difference form, with the row read back
        // from global memory (the chunked A buffers hold only part of it)
        const float4 co = clsm[kb];
        const float wn = co.y > 0.f ? co.z / co.y : 0.f;  // W_k / n_k
        dk = wn + tc_row_dist_global<false>(static_cast<const float*>(a.xg) + row * a.ldx, a.d, inv, gsm,
                                            a.zf + int64_t(kb0 + kb) * a.dz);
      }
      if (row < a.n) {
        if (fused) {
          float av = 0.f, bv = INFINITY, sv = 0.f;
          if (row_ok) {
            const bool has_b = dk < INFINITY;
            av = fmaxf(0.f, a.scale * aown);
            bv = has_b ? fmaxf(0.f, a.scale * dk) : INFINITY;
            if (code >= 0 && has_b) {
              sv = sil_eq2(av, bv, a.rms != 0);
            }
            if (!has_b) kb = -1;
          } else {
            kb = -1;
          }
          if (a.s_out) a.s_out[row] = sv;
          if (TRACK && a.sa) {
            a.sa[row] = av;
            a.sb[row] = bv;
            a.skstar[row] = kb;
          }
          tsum += sv;
        } else {
          const int64_t o = int64_t(blockIdx.y) * a.n + row;
          a.pmin[o] = row_ok ? dk : __int_as_float(0x7fc00000);
          if (TRACK && a.parg) a.parg[o] = (row_ok && kb >= 0) ? kb0 + kb : -1;
          if (own >= 0) a.pown[row] = aown;
        }
      }
    }
    if (fused) {
      for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
      float* red = cbs + a.kp;
      if (lane == 0) red[q] = tsum;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (warp == kEpiWarp0 && lane == 0) a.partials[blockIdx.x] = double(red[0]) + red[1] + red[2] + red[3];
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * a.acc_cols)
                 : "memory");
  }
}

// s_i from the per-block results when the clusters span several blocks: the
// minimum over the blocks (lowest cluster index on ties: blocks are visited
// in order and only a strictly smaller value replaces the best), then Eq. 2
// with the singleton and max(a, b) = 0 rules, and one partial sum per CTA.
__global__ void k_tc_combine(int64_t n, int32_t k, int32_t nblk, const int32_t* labels, const float4* cl,
                             float scale, int32_t rms, const float* pmin, const int32_t* parg,
                             const float* pown, float* s_out, float* sa, float* sb, int32_t* skstar,
                             double* partials) {
  float tsum = 0.f;
  for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < n;
       row += int64_t(gridDim.x) * blockDim.x) {
    const int own = labels[row];
    float best = INFINITY, av = 0.f, bv = INFINITY, sv = 0.f;
    int kb = -1;
    bool bad = own < 0 || own >= k;
    for (int g = 0; g < nblk && !bad; ++g) {
      const float v = pmin[int64_t(g) * n + row];
      if (v != v) {
        bad = true;  // NaN marks a row the scoring kernel rejected (zero norm)
      } else if (v < best) {
        best = v;
        if (parg) kb = parg[int64_t(g) * n + row];
      }
    }
    if (!bad) {
      const bool has_b = best < INFINITY;
      av = fmaxf(0.f, scale * pown[row]);
      bv = has_b ? fmaxf(0.f, scale * best) : INFINITY;
      if (has_b && cl[own].w > 1.5f) {
        sv = sil_eq2(av, bv, rms != 0);
      }
      if (!has_b) kb = -1;
    } else {
      kb = -1;
    }
    if (s_out) s_out[row] = sv;
    if (sa) {
      sa[row] = av;
      sb[row] = bv;
      skstar[row] = kb;
    }
    tsum += sv;
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += double(red[w]);
    partials[blockIdx.x] = t;
  }
}

// The labelings of a batched launch whose clusters span several blocks:
// multi[blockIdx.y] names one (its first block's item); each CTA takes the
// rows of slice blockIdx.x of gridDim.x (four per thread in flight) and writes
// the labeling's partial sum partials[b * gridDim.x + blockIdx.x] (the slot
// its fused form would use).
__global__ void __launch_bounds__(1024) k_tc_combine_items(const TcItem* multi, int64_t n, const int32_t* labels,
                                                           int64_t ldl, const float4* cl_all, float scale, int32_t rms,
                                                           const float* planes, const float* own_planes,
                                                           double* partials) {
  const TcItem it = multi[blockIdx.y];
  const int32_t* lab = labels + int64_t(it.b) * ldl;
  const float4* cl = cl_all + it.cl_off;
  const float* p0 = planes + int64_t(it.plane) * n;
  const float* p1 = it.nblk > 1 ? p0 + n : p0;  // a labeling has at most two blocks
  const float* po = own_planes + int64_t(it.own_plane) * n;
  constexpr int U = 4;  // rows per thread in flight: every load of them issued first
  float tsum = 0.f;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x * U + threadIdx.x; base < n;
       base += int64_t(gridDim.x) * blockDim.x * U) {
    int own[U];
    float v0[U], v1[U], ao[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t row = base + int64_t(u) * blockDim.x;
      const bool in = row < n;
      own[u] = in ? lab[row] : -1;
      v0[u] = in ? p0[row] : 0.f;
      v1[u] = in ? p1[row] : 0.f;
      ao[u] = in ? po[row] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      // NaN marks a row the scoring kernel rejected
      const bool bad = own[u] < 0 || own[u] >= it.k || v0[u] != v0[u] || v1[u] != v1[u];
      const float best = fminf(v0[u], v1[u]);
      if (!bad && best < INFINITY && cl[own[u]].w > 1.5f)
        tsum += sil_eq2(fmaxf(0.f, scale * ao[u]), fmaxf(0.f, scale * best), rms != 0);
    }
  }
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += double(red[w]);
    partials[int64_t(it.b) * gridDim.x + blockIdx.x] = t;
  }
}

// Split centroids and per-cluster constants for the tensor-core kernel, one
// row kk (one CTA):
//   zh/zl (bf16 [dp], zero padded) with zh + zl ~ (cs *) mu'_k to ~16 bits,
//   cb = bias_k + 2 g.(zh + zl)_k (+inf for empty clusters and padding).
// With FP8 storage the column scales cs are folded into the split values.
__device__ void tc_pack_row(int kk, const float* zf, const float4* cl, const double* g, const float* cs, int32_t k,
                            int32_t d, int32_t dz, int32_t dp, __nv_bfloat16* zh, __nv_bfloat16* zl, float* cb) {
  __shared__ double red[32];
  double dot = 0.0;
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    const float z = (kk < k && c < dz) ? zf[int64_t(kk) * dz + c] : 0.f;
    const float zs = cs ? (c < d ? z * cs[c] : 0.f) : z;
    const __nv_bfloat16 hh = __float2bfloat16_rn(zs);
    const __nv_bfloat16 ll = __float2bfloat16_rn(zs - __bfloat162float(hh));
    zh[c] = hh;
    zl[c] = ll;
    // The centring term uses the split value the GEMM actually sees, so the
    // split's residual enters d_k only through x' = x - g (zero mean), not as
    // a per-cluster offset g.(mu' - hi - lo).
    if (c < d) {
      const double zz = double(__bfloat162float(hh)) + double(__bfloat162float(ll));
      dot += g[c] * (cs ? (cs[c] != 0.f ? zz / double(cs[c]) : double(z)) : zz);
    }
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dot;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
    float v = INFINITY;
    if (kk < k && cl[kk].w > 0.5f) v = float(double(cl[kk].x) + 2.0 * t);
    *cb = v;
  }
}

// Split centroids of one labeling: rows 0..kpad-1 (one CTA each).
__global__ void k_tc_pack(const float* zf, const float4* cl, const double* g, const float* cs, int32_t k,
                          int32_t d, int32_t dz, int32_t dp, __nv_bfloat16* zh, __nv_bfloat16* zl,
                          float* cb) {
  const int kk = blockIdx.x;
  tc_pack_row(kk, zf, cl, g, cs, k, d, dz, dp, zh + int64_t(kk) * dp, zl + int64_t(kk) * dp, cb + kk);
}

// Split centroids of every labeling of a batched launch: labeling blockIdx.y,
// its rows 0..kp-1 at rows zrow.. of the packed arrays.
__global__ void k_tc_pack_items(const TcItem* items, const float* zf_all, const float4* cl_all, const double* g_all,
                                int32_t d, int32_t dz, int32_t dp, __nv_bfloat16* zh, __nv_bfloat16* zl, float* cb) {
  const TcItem it = items[blockIdx.y];
  const int kk = blockIdx.x;
  if (kk >= it.kp) return;
  const int64_t r = int64_t(it.zrow) + kk;
  tc_pack_row(it.kb0 + kk, zf_all + it.zf_off, cl_all + it.cl_off, g_all + it.g_off, nullptr, it.k, d, dz, dp,
              zh + r * dp, zl + r * dp, cb + r);
}

int pow2_at_least(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

int mode_of(int32_t dtype) { return dtype == SIL_F32 ? kModeF32 : dtype == SIL_BF16 ? kModeBF16 : kModeFP8; }

// Padded row width of the tensor path: 64 or 128 columns in one piece, FP32
// rows of up to 256 columns in 64-column chunks (k_score_tc_wide).
int tc_dp(int32_t d) { return d > 128 ? 256 : d == 32 ? 32 : int(round_up(d, 64)); }
int tc_max_d(int32_t dtype) { return dtype == SIL_F32 ? 256 : 128; }

// Launch plan: cluster-block width kp, ring depths and whether the centroids
// are staged for the own-cluster term.  Candidates are ranked by a small cost
// model -- work per point over the G blocks times penalties for shallow rings
// (an A buffer is held from conversion until the epilogue has read its rows
// back; a single raw stage exposes the TMA latency) and for unstaged
// centroids -- and the cheapest plan whose shared memory fits is taken.
// rank = 1 tracks the argmin in the main pass over the accumulators (the
// kernels built for the backward record); rank = 0 takes the plain minimum
// and rescans for the index only in warps with an ill-conditioned row.  The
// model takes rank = 0; data with mostly ill-conditioned rows (many close
// clusters far from the mean) run faster with rank = 1, which an autotuner
// finds by measurement.
struct TcPlan {
  int kp, nblk, nxs, nab, zst, smem, rank;
};

// Plans chosen by measurement (sil_tensor_plan_set) for one (dtype, d, k);
// they take precedence over the cost model.
struct PlanOverride {
  int32_t dtype, d, k, kp, nab, nxs, stage_z, rank;
};
std::mutex g_plan_mu;
std::vector<PlanOverride> g_plan_over;

// With two converter groups (tiles alternate between them) every slot of a
// ring must always serve the same group, so that a group never waits on the
// next use of a slot whose previous use, by the other group, has not
// completed (an mbarrier parity wait cannot tell the two apart): the A
// buffers, and the raw stages where the converters read them, come in even
// numbers.  (The row-term ring has 4 slots and TMEM 2 accumulators.)
bool tc_rings_ok(int mode, int dp, int kp, int nab, int nxs) {
  if (dp > 128 || tc_conv_groups(mode, dp, kp) == 1) return true;
  return nab % 2 == 0 && (mode == kModeBF16 || nxs % 2 == 0);
}

// Every plan whose shared memory fits, with its modelled cost.
template <class F>
void tc_plan_enumerate(int32_t dtype, int32_t k, int32_t d, F&& visit) {
  const int mode = mode_of(dtype);
  const bool staged = mode != kModeBF16;
  const int dp = tc_dp(d);
  const int dz = int(round_up(d, 4));
  const int kmax = int(std::min<int64_t>(round_up(std::max(k, 16), 16), kMaxBlockN));
  for (int kp = kmax; kp >= 16; kp -= 16) {
    const int nblk = int(cdiv(k, kp));
    for (int nab = 1; nab <= 4; ++nab) {
      for (int nxs = 1; nxs <= (staged ? 3 : 1); ++nxs) {
        if (!tc_rings_ok(mode, dp, kp, nab, nxs)) continue;
        for (int zs = 0; zs < 2; ++zs) {
          const int zst = zs ? dz + 4 : 0;  // padded rows: fewer bank conflicts
          const int smem = tc_smem(mode, dp, kp, nxs, nab, zst).total;
          if (smem > kSmemMax) continue;
          // per block and tile: MMA + epilogue ~ kp columns (the MMA is bound by
          // its A-operand reads below ~64), plus a fixed share for conversion,
          // row terms and the per-block results
          double cost = double(nblk) * (std::max(kp, 64) + dp);
          if (!zst) cost *= 1.12;  // own-centroid rows from L1/L2 instead of shared memory
          const bool two = dp <= 128 && tc_conv_groups(mode, dp, kp) == 2;
          if (two) {
            // two converter groups alternate tiles: each wants a raw stage and
            // an A buffer of its own
            if (staged && nxs < 2) cost *= 1.3;
            if (nab < 2) cost *= 1.8;
          } else {
            if (staged && nxs == 2) cost *= 0.99;  // a second raw stage hides a little TMA latency
            if (!staged && nab == 2) cost *= 1.05;  // BF16: the A ring is the TMA prefetch depth
            if (!staged && nab == 3) cost *= 1.03;
          }
          for (int rank = 0; rank < 2; ++rank) {
            // the narrow kernels hold an A buffer until the epilogue has read
            // its rows back, except FP32 with rank 0 (those rows come from
            // global memory): then one buffer serialises conversion, MMA and
            // epilogue and two overlap them only partly
            const bool held = dp <= 128 && !(mode == kModeF32 && rank == 0);
            double c = cost;
            if (!two && nab < 2) c *= held ? 1.8 : 1.4;
            if (!two && staged && nab == 2) c *= held ? 1.08 : 1.06;  // measured: a third buffer pays ~5 %
            // rank 0 first: at equal cost the model keeps it, and a candidate
            // list pairs the two rank passes of a layout where they tie
            visit(TcPlan{kp, nblk, nxs, nab, zst, smem, rank}, c);
          }
        }
      }
    }
  }
}

bool tc_plan(int32_t dtype, int32_t k, int32_t d, TcPlan* out) {
  const int mode = mode_of(dtype);
  const int dp = tc_dp(d);
  const int dz = int(round_up(d, 4));
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    for (const PlanOverride& o : g_plan_over) {
      if (o.dtype != dtype || o.d != d || o.k != k) continue;
      const int zst = o.stage_z ? dz + 4 : 0;
      const int smem = tc_smem(mode, dp, o.kp, o.nxs, o.nab, zst).total;
      if (smem <= kSmemMax && tc_rings_ok(mode, dp, o.kp, o.nab, o.nxs)) {
        *out = TcPlan{o.kp, int(cdiv(k, o.kp)), o.nxs, o.nab, zst, smem, o.rank};
        return true;
      }
    }
  }
  double best_cost = 0.0;
  bool found = false;
  tc_plan_enumerate(dtype, k, d, [&](const TcPlan& p, double cost) {
    if (!found || cost < best_cost) {
      found = true;
      best_cost = cost;
      *out = p;
    }
  });
  return found;
}

}  // namespace

bool tc_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t k, const void* X,
                 const int32_t* labels) {
  const char* e = getenv("SIL_TC_DISABLE");
  if (e && e[0] == '1') return false;
  if (n <= 0 || n >= (int64_t(1) << 31) || d > tc_max_d(dtype)) return false;
  if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(labels) % 16) return false;
  const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
  if ((ldx * esz) % 16) return false;
  // the TMA box of a row must fit inside the row
  if (dtype == SIL_F32 && d < 32) return false;
  if (dtype == SIL_BF16 && d < 64) return false;
  if (dtype == SIL_FP8_E4M3 && d != 128) return false;
  TcPlan p;
  if (!tc_plan(dtype, k, d, &p)) return false;
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
  return major == 10;
}

cudaError_t launch_selftest_wait(uint32_t* out, cudaStream_t stream) {
  k_selftest_wait<<<1, 96, 0, stream>>>(out);
  return cudaGetLastError();
}

bool tc_plan_query(int32_t dtype, int32_t d, int32_t k, int32_t* block_k, int32_t* n_blocks) {
  if (d > tc_max_d(dtype) || d <= 0 || k <= 0) return false;
  TcPlan p;
  if (!tc_plan(dtype, k, d, &p)) return false;
  *block_k = p.kp;
  *n_blocks = p.nblk;
  return true;
}

int tc_plan_candidates(int32_t dtype, int32_t d, int32_t k, int32_t* plans, int32_t max_plans) {
  if (d > tc_max_d(dtype) || d <= 0 || k <= 0) return 0;
  std::vector<std::pair<double, TcPlan>> all;
  tc_plan_enumerate(dtype, k, d, [&](const TcPlan& p, double cost) { all.emplace_back(cost, p); });
  std::stable_sort(all.begin(), all.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  int n = 0;
  for (const auto& c : all) {
    if (n >= max_plans) break;
    plans[5 * n + 0] = c.second.kp;
    plans[5 * n + 1] = c.second.nab;
    plans[5 * n + 2] = c.second.nxs;
    plans[5 * n + 3] = c.second.zst ? 1 : 0;
    plans[5 * n + 4] = c.second.rank;
    ++n;
  }
  return n;
}

int tc_plan_set(int32_t dtype, int32_t d, int32_t k, int32_t kp, int32_t nab, int32_t nxs, int32_t stage_z,
                int32_t rank) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  for (size_t i = 0; i < g_plan_over.size(); ++i)
    if (g_plan_over[i].dtype == dtype && g_plan_over[i].d == d && g_plan_over[i].k == k) {
      g_plan_over.erase(g_plan_over.begin() + long(i));
      break;
    }
  if (kp == 0) return SIL_OK;  // cleared: back to the cost model
  if (d > tc_max_d(dtype) || kp < 16 || kp > kMaxBlockN || kp % 16 || nab < 1 || nab > 4 || nxs < 1 || nxs > 3 ||
      rank < 0 || rank > 1)
    return SIL_EINVAL;
  const int mode = mode_of(dtype);
  const int zst = stage_z ? int(round_up(d, 4)) + 4 : 0;
  if (!tc_rings_ok(mode, tc_dp(d), kp, nab, mode == kModeBF16 ? 1 : nxs)) return SIL_EINVAL;
  if (tc_smem(mode, tc_dp(d), kp, mode == kModeBF16 ? 1 : nxs, nab, zst).total > kSmemMax)
    return SIL_EUNSUPPORTED;
  g_plan_over.push_back(PlanOverride{dtype, d, k, kp, nab, mode == kModeBF16 ? 1 : nxs, stage_z ? 1 : 0, rank});
  return SIL_OK;
}

size_t tc_pack_bytes(int32_t k, int32_t d) {
  // nblk * kp < k + kp <= k + 256
  const size_t kpad = size_t(round_up(std::max(k, 16), 16)) + kMaxBlockN, dp = size_t(tc_dp(d));
  return 2 * kpad * dp * 2 + kpad * 4 + 256;
}

size_t tc_partial_bytes(int64_t n, int32_t d, int32_t k, int32_t dtype) {
  if (n <= 0 || dtype < SIL_F32 || dtype > SIL_FP8_E4M3 || d > tc_max_d(dtype)) return 0;
  TcPlan p;
  if (!tc_plan(dtype, k, d, &p) || p.nblk == 1) return 0;
  const size_t N = size_t(n), G = size_t(p.nblk);
  return align256(G * N * 4) + align256(G * N * 4) + align256(N * 4);
}

cudaError_t launch_score_tc(const ScoreLaunch& s, const double* g, void* pack, void* partial_ws,
                            size_t partial_bytes, uint32_t* status) {
  TcPlan plan;
  if (!tc_plan(s.dtype, s.k, s.d, &plan)) return cudaErrorInvalidValue;
  auto need = [&](int nblk) {
    const size_t N = size_t(s.n), G = size_t(nblk);
    return nblk > 1 ? align256(G * N * 4) * 2 + align256(N * 4) : size_t(0);
  };
  if (need(plan.nblk) > partial_bytes) {
    // the workspace was sized for another plan (e.g. a larger k of a batch):
    // the cheapest plan whose per-block results fit
    double best = 0.0;
    bool found = false;
    tc_plan_enumerate(s.dtype, s.k, s.d, [&](const TcPlan& p, double cost) {
      if (need(p.nblk) <= partial_bytes && (!found || cost < best)) {
        found = true;
        best = cost;
        plan = p;
      }
    });
    if (!found) return cudaErrorInvalidValue;
  }
  const int mode = mode_of(s.dtype);
  const int dp = tc_dp(s.d);
  const int kp = plan.kp;
  const int kpad = plan.nblk * kp;
  const int dz = int(round_up(s.d, 4));
  __nv_bfloat16* zh = static_cast<__nv_bfloat16*>(pack);
  __nv_bfloat16* zl = zh + size_t(kpad) * dp;
  float* cb = reinterpret_cast<float*>(zl + size_t(kpad) * dp);
  k_tc_pack<<<kpad, 128, 0, s.stream>>>(s.zf, s.cl, g, mode == kModeFP8 ? s.cs : nullptr, s.k, s.d, dz, dp,
                                         zh, zl, cb);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;

  TcMaps maps{};
  const int esz = mode == kModeF32 ? 4 : mode == kModeBF16 ? 2 : 1;
  const CUtensorMapDataType xt = mode == kModeF32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : mode == kModeBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  const uint32_t box_inner = mode == kModeF32 ? 32 : mode == kModeBF16 ? 64 : 128;
  if (!encode_tmap_2d(&maps.x, s.X, xt, esz, uint64_t(s.d), uint64_t(s.n), uint64_t(s.ldx) * esz, box_inner,
                      kTM, CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;
  if (!encode_tmap_1d(&maps.lab, s.labels, CU_TENSOR_MAP_DATA_TYPE_INT32, uint64_t(s.n), kTM))
    return cudaErrorInvalidValue;
  const uint32_t zbox = dp == 32 ? 32 : 64;  // BF16 columns per box (64- or 128-byte rows)
  const CUtensorMapSwizzle zsw = dp == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  if (!encode_tmap_2d(&maps.zh, zh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, uint64_t(dp), uint64_t(kpad),
                      uint64_t(dp) * 2, zbox, uint32_t(kp), zsw) ||
      !encode_tmap_2d(&maps.zl, zl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, uint64_t(dp), uint64_t(kpad),
                      uint64_t(dp) * 2, zbox, uint32_t(kp), zsw))
    return cudaErrorInvalidValue;

  TcK k{};
  k.n = s.n;
  k.d = s.d;
  k.k = s.k;
  k.kp = kp;
  k.nblk = plan.nblk;
  k.acc_cols = pow2_at_least(kp);
  k.dz = dz;
  k.cosine = s.dist == SIL_COSINE;
  k.rms = s.dist == SIL_EUCLIDEAN_RMS;
  k.scale = s.dist == SIL_COSINE ? 0.5f : 1.f;
  k.nxs = plan.nxs;
  k.nab = plan.nab;
  k.zst = plan.zst;
  k.xg = s.X;
  k.ldx = s.ldx;
  k.zf = s.zf;
  k.cl = s.cl;
  k.gf = s.gf;
  k.cb = cb;
  k.cs = s.cs;
  k.s_out = s.s_out;
  k.sa = s.sa;
  k.sb = s.sb;
  k.skstar = s.skstar;
  k.partials = s.partials;
  k.status = status;
  k.zbox_rows = kp;
  k.items = nullptr;
  const bool save = s.sa != nullptr;
  // the kernels built for the backward record track the argmin in the main
  // pass; without the record they serve rank = 1 plans
  const bool track = save || plan.rank == 1;
  if (plan.nblk > 1) {
    const size_t N = size_t(s.n), G = size_t(plan.nblk);
    char* p = static_cast<char*>(partial_ws);
    k.pmin = reinterpret_cast<float*>(p);
    k.parg = save ? reinterpret_cast<int32_t*>(p + align256(G * N * 4)) : nullptr;
    k.pown = reinterpret_cast<float*>(p + 2 * align256(G * N * 4));
  }
  const int64_t ntiles = cdiv(s.n, kTM);
  const int per_block = std::max(1, num_sms() / plan.nblk);
  const dim3 grid(unsigned(std::min<int64_t>(ntiles, per_block)), unsigned(plan.nblk));
  const int cg = dp == 256 ? 1 : tc_conv_groups(mode, dp, kp);
  const int threads = dp == 256 ? kTcThreads : tc_threads(dp, cg);
  // the kernels of one converter group take the own-cluster term a warp per
  // row where the centroids stay in global memory
  k.own_rows = plan.nblk > 1 && plan.zst == 0 && dp != 256 && cg == 1 ? 1 : 0;
  auto launch = [&](auto fn) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, plan.smem, s.stream>>>(k, maps);
    return cudaGetLastError();
  };
  cudaError_t e;
  if (mode == kModeF32) {
    if (dp == 256) {
      e = track ? launch(k_score_tc_wide<true>) : launch(k_score_tc_wide<false>);
    } else if (dp == 32) {
      if (cg == 2) e = track ? launch(k_score_tc<kModeF32, 32, true, 2>) : launch(k_score_tc<kModeF32, 32, false, 2>);
      else e = track ? launch(k_score_tc<kModeF32, 32, true, 1>) : launch(k_score_tc<kModeF32, 32, false, 1>);
    } else if (dp == 64) {
      if (cg == 2) e = track ? launch(k_score_tc<kModeF32, 64, true, 2>) : launch(k_score_tc<kModeF32, 64, false, 2>);
      else e = track ? launch(k_score_tc<kModeF32, 64, true, 1>) : launch(k_score_tc<kModeF32, 64, false, 1>);
    } else {
      e = track ? launch(k_score_tc<kModeF32, 128, true, 1>) : launch(k_score_tc<kModeF32, 128, false, 1>);
    }
  } else if (mode == kModeBF16) {
    if (dp == 64) e = track ? launch(k_score_tc<kModeBF16, 64, true, 1>) : launch(k_score_tc<kModeBF16, 64, false, 1>);
    else e = track ? launch(k_score_tc<kModeBF16, 128, true, 1>) : launch(k_score_tc<kModeBF16, 128, false, 1>);
  } else {
    e = track ? launch(k_score_tc<kModeFP8, 128, true, 1>) : launch(k_score_tc<kModeFP8, 128, false, 1>);
  }
  if (e != cudaSuccess) return e;
  if (plan.nblk == 1) {
    *s.n_partials = int(grid.x);
    return cudaSuccess;
  }
  return launch_tc_combine(s.n, s.k, plan.nblk, s.labels, s.cl, k.scale, k.rms, k.pmin, save ? k.parg : nullptr,
                           k.pown, s.s_out, s.sa, s.sb, s.skstar, s.partials, s.stream, s.n_partials);
}

cudaError_t launch_tc_combine(int64_t n, int32_t k, int32_t nblk, const int32_t* labels, const float4* cl,
                              float scale, int32_t rms, const float* pmin, const int32_t* parg, const float* pown,
                              float* s_out, float* sa, float* sb, int32_t* skstar, double* partials,
                              cudaStream_t stream, int32_t* n_partials) {
  const int cgrid = int(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), kMaxPartials)));
  k_tc_combine<<<cgrid, 256, 0, stream>>>(n, k, nblk, labels, cl, scale, rms, pmin, parg, pown, s_out, sa, sb,
                                          skstar, partials);
  *n_partials = cgrid;
  return cudaGetLastError();
}

bool tc_batched_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t kmax, const void* X,
                         const int32_t* labels, int64_t ldl) {
  if (dtype != SIL_F32 || kmax > 512 || d < 32 || d > 64) return false;
  if (ldl % 4 != 0) return false;  // 16-byte rows of the labels map
  if (!tc_eligible(dtype, n, d, ldx, std::min(kmax, 256), X, labels)) return false;
  return tc_batched_pack_bytes(1, kmax, d) > 0;
}

// Launch plan of the batched launch: row ranges (CTAs per labeling block)
// and A-operand buffers (0: the deepest ring that fits); set by an autotuner.
std::atomic<int> g_batched_ranges{8};
std::atomic<int> g_batched_nab{0};

int tc_batched_ranges() { return g_batched_ranges.load(); }

int tc_batched_plan_set(int32_t ranges, int32_t a_buffers) {
  if (ranges < 1 || ranges > kBatchedMaxRanges || (a_buffers != 0 && a_buffers != 2 && a_buffers != 4))
    return SIL_EINVAL;
  g_batched_ranges.store(ranges);
  g_batched_nab.store(a_buffers);
  return SIL_OK;
}

namespace {
// ring depths of the batched launch for rows of dp columns and blocks of up to
// 256 clusters (wider labelings are split into two blocks)
// The deepest A ring that fits (or the one asked for), with the block's
// centroids staged in shared memory for the converters' own-cluster term and
// the difference form of ill-conditioned rows when they fit beside it.
bool tc_batched_plan(int dp, int dz, int* nab, int* nxs, int* smem, int* zst) {
  const int want = g_batched_nab.load();
  for (int staged = 1; staged >= 0; --staged) {
    const int zs = staged ? dz + 4 : 0;
    for (int b = 4; b >= 2; b -= 2) {
      if (want && b != want) continue;
      const int sm = tc_smem(kModeF32, dp, 256, 2, b, zs).total;
      if (sm <= kSmemMax) {
        *nab = b;
        *nxs = 2;
        *smem = sm;
        *zst = zs;
        return true;
      }
    }
  }
  return false;
}
}  // namespace

size_t tc_batched_pack_bytes(int32_t batch, int32_t kmax, int32_t d) {
  const int dp = tc_dp(d), kmaxp = int(round_up(std::max(kmax, 16), 16));
  int nab, nxs, smem, zst;
  if (!tc_batched_plan(dp, int(round_up(d, 4)), &nab, &nxs, &smem, &zst)) return 0;
  // the blocks of a labeling (at most two) are at most 31 rows wider than its clusters
  const size_t rows = size_t(batch) * size_t(kmaxp + 32);
  return align256(rows * size_t(dp) * 2) * 2 + align256(rows * 4);
}

cudaError_t launch_score_tc_batched(const void* X, int64_t n, int32_t d, int64_t ldx, const int32_t* labels,
                                    int64_t ldl, int32_t batch, int32_t kmax, int32_t dist, const TcItem* items,
                                    int32_t n_items, int32_t total_zrows, const TcItem* multi, int32_t n_multi,
                                    const float* zf_all, const float4* cl_all, const double* g_all,
                                    const float* gf_all, void* pack, float* planes, float* own_planes,
                                    double* partials, uint32_t* status_all, cudaStream_t stream) {
  const int dp = tc_dp(d), dz = int(round_up(d, 4));
  int nab = 0, nxs = 0, smem = 0, zst = 0;
  if (!tc_batched_plan(dp, dz, &nab, &nxs, &smem, &zst)) return cudaErrorInvalidValue;
  const size_t rows = size_t(batch) * size_t(round_up(std::max(kmax, 16), 16) + 32);
  __nv_bfloat16* zh = static_cast<__nv_bfloat16*>(pack);
  __nv_bfloat16* zl = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(pack) + align256(rows * size_t(dp) * 2));
  float* cb = reinterpret_cast<float*>(static_cast<char*>(pack) + 2 * align256(rows * size_t(dp) * 2));
  k_tc_pack_items<<<dim3(256u, unsigned(n_items)), 128, 0, stream>>>(items, zf_all, cl_all, g_all, d, dz, dp, zh,
                                                                     zl, cb);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  TcMaps maps{};
  const uint32_t zbox = dp == 32 ? 32 : 64;
  const CUtensorMapSwizzle zsw = dp == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  if (!encode_tmap_2d(&maps.x, X, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, uint64_t(d), uint64_t(n), uint64_t(ldx) * 4, 32,
                      kTM, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_2d(&maps.lab, labels, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, uint64_t(n), uint64_t(batch),
                      uint64_t(ldl) * 4, kTM, 1, CU_TENSOR_MAP_SWIZZLE_NONE) ||
      !encode_tmap_2d(&maps.zh, zh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, uint64_t(dp), uint64_t(total_zrows),
                      uint64_t(dp) * 2, zbox, 16, zsw) ||
      !encode_tmap_2d(&maps.zl, zl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, uint64_t(dp), uint64_t(total_zrows),
                      uint64_t(dp) * 2, zbox, 16, zsw))
    return cudaErrorInvalidValue;
  TcK k{};
  k.n = n;
  k.d = d;
  k.k = kmax;
  k.kp = 256;  // shared-memory layout for the widest block
  k.nblk = 1;
  k.acc_cols = 256;
  k.dz = dz;
  k.cosine = dist == SIL_COSINE;
  k.rms = dist == SIL_EUCLIDEAN_RMS;
  k.scale = dist == SIL_COSINE ? 0.5f : 1.f;
  k.nxs = nxs;
  k.nab = nab;
  k.zst = zst;
  k.xg = X;
  k.ldx = ldx;
  k.zf = zf_all;
  k.cl = cl_all;
  k.gf = gf_all;
  k.cb = cb;
  k.partials = partials;
  k.pmin = planes;
  k.pown = own_planes;
  k.status = status_all;
  k.zbox_rows = 16;
  k.items = items;
  const unsigned ranges = unsigned(tc_batched_ranges());
  const dim3 grid(ranges, unsigned(n_items));
  const int cg = tc_conv_groups(kModeF32, dp, 256);
  auto launch = [&](auto fn, int threads) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, threads, smem, stream>>>(k, maps);
    return cudaGetLastError();
  };
  cudaError_t e;
  if (dp == 32)
    e = cg == 2 ? launch(k_score_tc<kModeF32, 32, true, 2, true>, tc_threads(32, 2))
                : launch(k_score_tc<kModeF32, 32, true, 1, true>, tc_threads(32, 1));
  else
    e = cg == 2 ? launch(k_score_tc<kModeF32, 64, true, 2, true>, tc_threads(64, 2))
                : launch(k_score_tc<kModeF32, 64, true, 1, true>, tc_threads(64, 1));
  if (e != cudaSuccess || n_multi == 0) return e;
  k_tc_combine_items<<<dim3(ranges, unsigned(n_multi)), 1024, 0, stream>>>(multi, n, labels, ldl, cl_all, k.scale,
                                                                         k.rms, planes, own_planes, partials);
  return cudaGetLastError();
}

}  // namespace sil
