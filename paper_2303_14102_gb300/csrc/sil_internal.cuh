// Internal declarations shared by the translation units of libsil.
//
// Layout conventions (device memory):
//   X        row-major n x d in its storage type, row stride ldx elements
//   labels   int32[n]
//   count    int64[k], s1 f64[k*d], s2 f64[k]   (the pass-1 aggregates)
//   ws       caller workspace carved by ws_layout() below
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sil.h"

namespace sil {

constexpr int kScoreThreads = 256;   // threads per SIMT pass-2 CTA
constexpr int kMaxPartials = 8192;   // per-CTA partial sums of s_i
constexpr int kSmemBudget = 100 * 1024;  // dynamic shared memory per CTA we aim for

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Streaming multiprocessors of the current device (queried once per device
// and cached; 152 on a GB300).  Persistent grids are sized from it.
int num_sms();

// Eq. 2 from a point's mean distances a (own cluster) and b (nearest other
// cluster), both >= 0: 0 when max(a, b) = 0.  With rms set, a and b are means
// of squared Euclidean distances and Eq. 2 takes their square roots -- the
// approximation of the Euclidean Silhouette that the Limitations section
// suggests (the square root of each point-to-cluster mean distance).
__device__ __forceinline__ float sil_eq2(float a, float b, bool rms) {
  if (rms) {
    a = sqrtf(fmaxf(a, 0.f));
    b = sqrtf(fmaxf(b, 0.f));
  }
  const float m = fmaxf(a, b);
  return m > 0.f ? (a <= b ? 1.f - a / b : b / a - 1.f) : 0.f;
}

// Per-cluster constants for pass 2, one float4 per cluster:
//   x = bias  = ||mu'_k||^2 + W_k/n_k   (+inf when n_k = 0)
//   y = an    = n_k / (n_k - 1)          (0 when n_k < 2)
//   z = aw    = W_k / (n_k - 1)          (0 when n_k < 2)
//   w = n_k as float
// mu'_k = mu_k - g is the centroid in coordinates centred on the global mean
// g, W_k = sum ||x - mu_k||^2 is the within-cluster scatter.

struct WsLayout {
  size_t misc;      // uint32 flags[64]
  size_t rs;        // float[k*dz]       per-cluster shift (reference point)
  size_t g;         // double[dz]        global centre
  size_t gf;        // float[dz]
  size_t zf;        // float[k*dz]       centred centroids mu'
  size_t cl;        // float4[k]         per-cluster constants
  size_t invnorm;   // float[n]          1/||x_i|| (cosine, when pass 1 is column-sliced)
  size_t partials;  // double[kMaxPartials]
  size_t bw_w;      // double[2k]        backward: A_k then B_k
  size_t bw_p;      // double[2k*d]      backward: P'_k then Q'_k
  size_t bw_ab;     // float[2n]         backward: alpha_i then beta_i
  size_t bw_f;      // float[k*dz + k]   backward: W_c rows then C_c
  size_t saved;     // 12 bytes * n      recomputed forward record
  size_t bk;        // uint32[3 * 2k + 1] pass-1 bucket counts, starts, cursors
  size_t bidx;      // uint32[2n]        pass-1 row indices in bucket order
  size_t bw;        // float[2n]         pass-1 weights in bucket order (backward)
  size_t zbf;       // bf16 centroid tiles for the tensor path
  size_t tcp;       // tensor path with several cluster blocks: per-block minima
  size_t batch;     // batched aggregates
  // batched tensor-core launch (several labelings, k_max <= 512): per labeling
  // status words, items, finalized constants, packed centroids, CTA sums
  size_t bst, bitems, bmulti, bzf, bcl, bg, bgf, bpack, bpart, bplanes, bown;
  size_t total;
};

WsLayout ws_layout(int64_t n, int32_t d, int32_t k, int32_t dtype, int32_t dist, int32_t batch);

// ---------------------------------------------------------------- loaders
template <int DT>
struct Elem;
template <>
struct Elem<SIL_F32> {
  using T = float;
  static __device__ __forceinline__ float get(const T* p, int64_t i) { return p[i]; }
};
template <>
struct Elem<SIL_BF16> {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float get(const T* p, int64_t i) { return __bfloat162float(p[i]); }
};
template <>
struct Elem<SIL_FP8_E4M3> {
  using T = __nv_fp8_e4m3;
  static __device__ __forceinline__ float get(const T* p, int64_t i) { return float(p[i]); }
};

// Four consecutive elements of row `row` starting at column `col` (col % 4 == 0),
// columns >= d read as 0.  `vec` promises that X, ldx are aligned for one
// vector load of four elements.
template <int DT>
__device__ __forceinline__ float4 load4(const void* Xv, int64_t row, int col, int d, int64_t ldx,
                                        const float* cs, bool vec) {
  using T = typename Elem<DT>::T;
  const T* X = static_cast<const T*>(Xv);
  const int64_t base = row * ldx + col;
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (vec && col + 3 < d) {
    if constexpr (DT == SIL_F32) {
      r = __ldg(reinterpret_cast<const float4*>(X + base));
    } else if constexpr (DT == SIL_BF16) {
      uint2 u = __ldg(reinterpret_cast<const uint2*>(X + base));
      __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162*>(&u.x);
      __nv_bfloat162 hi = *reinterpret_cast<__nv_bfloat162*>(&u.y);
      float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
      r = make_float4(a.x, a.y, b.x, b.y);
    } else {
      uint32_t u = __ldg(reinterpret_cast<const unsigned int*>(X + base));
      const __nv_fp8_e4m3* q = reinterpret_cast<const __nv_fp8_e4m3*>(&u);
      r = make_float4(float(q[0]), float(q[1]), float(q[2]), float(q[3]));
    }
  } else {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (col + j < d) v[j] = Elem<DT>::get(X, base + j);
    r = make_float4(v[0], v[1], v[2], v[3]);
  }
  if constexpr (DT == SIL_FP8_E4M3) {
    if (col + 0 < d) r.x *= __ldg(cs + col + 0);
    if (col + 1 < d) r.y *= __ldg(cs + col + 1);
    if (col + 2 < d) r.z *= __ldg(cs + col + 2);
    if (col + 3 < d) r.w *= __ldg(cs + col + 3);
  }
  return r;
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bit) {
  if (st) atomicOr(st, bit);
}

// ------------------------------------------------------------ host launchers
struct AggLaunch {
  const void* X;
  int32_t dtype;
  int64_t n;
  int32_t d;
  int64_t ldx;
  const float* cs;
  const int32_t* labels;   // bucket id of entry 0 of each row
  const int32_t* labels2;  // dual mode: bucket id (minus k) of entry 1, nullable
  const float* w1;         // weights of entry 0 (nullable: unweighted)
  const float* w2;         // weights of entry 1 (dual)
  int32_t k;
  int32_t dist;
  float* rs;               // out: shift [k][dz] (the reference point of each cluster)
  const float* invnorm;    // nullable
  unsigned long long* count;
  double* s1;
  double* s2;
  double* wsum;
  uint32_t* status;
  // counting-sort scratch (workspace): per bucket counts, starts (nb + 1) and
  // cursors; the sorted row indices and weights (one per entry)
  uint32_t* bcount;
  uint32_t* bstart;
  uint32_t* cursor;
  uint32_t* idx;
  float* widx;
  cudaStream_t stream;
};

// Enqueue 1/||x_i|| for every row (cosine, column-sliced pass 1).
cudaError_t launch_invnorm(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                           const float* cs, float* invnorm, uint32_t* status, cudaStream_t stream);
// Whether pass 1 splits the rows into column slices, so that the cosine norm
// must come from launch_invnorm.
bool agg_needs_invnorm(int32_t dtype, int32_t d);
// Counting sort of the rows by label (the first steps of pass 1): bcount[k],
// bstart[k + 1] (bstart[k] = rows with a valid label), cursor[k] scratch, idx
// = row indices in label order; a label outside [0, k) sets SIL_ELABEL and its
// row is left out.
cudaError_t launch_label_sort(const int32_t* labels, int64_t n, int32_t k, uint32_t* bcount, uint32_t* bstart,
                              uint32_t* cursor, uint32_t* idx, uint32_t* status, cudaStream_t stream);
// The exact Euclidean Silhouette by the quadratic method: workspace bytes,
// the largest d served, and the launch (s_out, sa/sb/skstar nullable).
size_t euclid_ws_bytes(int64_t n, int32_t d, int32_t k);
int euclid_max_d();
cudaError_t launch_euclid(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* cs,
                          const int32_t* labels, int32_t k, float* s_out, float* sa, float* sb, int32_t* skstar,
                          void* ws, uint32_t* user_status, double* S_out, cudaStream_t st);
// Enqueue pass 1 (outputs must be zeroed or hold sums to add to).
cudaError_t launch_aggregate(const AggLaunch& a);

struct FinLaunch {
  const unsigned long long* count;
  const double* s1;
  const double* s2;
  int32_t k;
  int32_t d;
  int32_t dist;
  double* g;
  float* gf;
  float* zf;
  float4* cl;
  uint32_t* status;  // workspace status word
  cudaStream_t stream;
};
cudaError_t launch_finalize(const FinLaunch& f);

// One labeling of a batched tensor-core launch (CTA row blockIdx.y): its
// cluster count, block width (MMA N, up to 512 as two MMAs), first row in the
// packed centroids of all labelings, and offsets of its finalized constants
// (float4 cluster terms, FP32 centred centroids, global centre).
struct TcItem {
  int32_t b;       // labeling (row of labels, status word, partial-sum slots)
  int32_t k, nblk; // clusters of the labeling and its blocks
  int32_t kb0, kp; // first cluster of this block and its width (MMA N)
  int32_t zrow;    // first row of this block in the packed centroids
  int32_t cl_off, zf_off, g_off;  // the labeling's finalized constants
  int32_t plane, own_plane;       // several blocks: result planes (else -1)
};

struct ScoreLaunch {
  const void* X;
  int32_t dtype;
  int64_t n;
  int32_t d;
  int64_t ldx;
  const float* cs;
  const int32_t* labels;
  int32_t k;
  int32_t dist;
  const float* zf;
  const float4* cl;
  const float* gf;
  float* s_out;
  float* sa;
  float* sb;
  int32_t* skstar;
  double* partials;
  int32_t* n_partials;  // host out: number of partials written
  uint32_t* status;     // workspace status word
  cudaStream_t stream;
};
cudaError_t launch_score_simt(ScoreLaunch& s);
// Tensor-core pass 2 (tcgen05): eligibility, bytes of its packed centroids
// (inside the workspace) and the launch (status = workspace status word).
bool tc_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t k, const void* X,
                 const int32_t* labels);
size_t tc_pack_bytes(int32_t k, int32_t d);
// Host-only: the cluster-block plan (false when none fits), the feasible
// plans ranked by the cost model (4 ints each: block_k, A buffers, X
// stages, staged centroids), and a measured choice for one shape.
bool tc_plan_query(int32_t dtype, int32_t d, int32_t k, int32_t* block_k, int32_t* n_blocks);
int tc_plan_candidates(int32_t dtype, int32_t d, int32_t k, int32_t* plans, int32_t max_plans);
int tc_plan_set(int32_t dtype, int32_t d, int32_t k, int32_t kp, int32_t nab, int32_t nxs, int32_t stage_z,
                int32_t rank);
// Bytes of the per-block results when k needs several cluster blocks (else 0).
size_t tc_partial_bytes(int64_t n, int32_t d, int32_t k, int32_t dtype);
// One CTA whose waits run out on purpose (failure-detection self-test), out[3].
cudaError_t launch_selftest_wait(uint32_t* out, cudaStream_t stream);
cudaError_t launch_score_tc(const ScoreLaunch& s, const double* g, void* pack, void* partial_ws,
                            size_t partial_bytes, uint32_t* status);
// Minimum over the cluster blocks of per-block nearest distances (pmin, parg:
// [nblk][n]; pown: a_i from the own cluster's block), then Eq. 2 and one
// partial sum per CTA (their number into *n_partials).
cudaError_t launch_tc_combine(int64_t n, int32_t k, int32_t nblk, const int32_t* labels, const float4* cl,
                              float scale, int32_t rms, const float* pmin, const int32_t* parg, const float* pown,
                              float* s_out, float* sa, float* sb, int32_t* skstar, double* partials,
                              cudaStream_t stream, int32_t* n_partials);
// TF32-ranked tensor-core pass 2 for FP32 rows of 32..64 columns (b_i and a_i
// exact in FP32): eligibility, bytes of its packed centroids and of its
// per-block results inside the workspace, and the launch.
bool t32_serves(int32_t dtype, int32_t d, int32_t k);  // host-only: the shape has a plan
bool t32_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t k, const void* X,
                  const int32_t* labels);
size_t t32_pack_bytes(int32_t k, int32_t d);
size_t t32_partial_bytes(int64_t n, int32_t d, int32_t k);
cudaError_t launch_score_tf32(const ScoreLaunch& s, const double* g, void* pack, void* partial_ws,
                              size_t partial_bytes, uint32_t* status);
// Batched tensor-core pass 2: every labeling in one launch (grid.y = labeling,
// grid.x = row ranges).  Eligibility (k_max <= 512, FP32 rows of 32 or 64
// columns padded, 16-byte aligned X, labels rows and strides), and the launch
// from finalized constants of all labelings (items on the device); partials
// get batch x (*ranges) sums.  Host-side plan: ranges per labeling.
bool tc_batched_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t kmax, const void* X,
                         const int32_t* labels, int64_t ldl);
int tc_batched_ranges();
constexpr int kBatchedMaxRanges = 64;
int tc_batched_plan_set(int32_t ranges, int32_t a_buffers);
size_t tc_batched_pack_bytes(int32_t batch, int32_t kmax, int32_t d);
cudaError_t launch_score_tc_batched(const void* X, int64_t n, int32_t d, int64_t ldx, const int32_t* labels,
                                    int64_t ldl, int32_t batch, int32_t kmax, int32_t dist, const TcItem* items,
                                    int32_t n_items, int32_t total_zrows, const TcItem* multi, int32_t n_multi,
                                    const float* zf_all, const float4* cl_all, const double* g_all,
                                    const float* gf_all, void* pack, float* planes, float* own_planes,
                                    double* partials, uint32_t* status_all, cudaStream_t stream);
// S_out[b] = (sum of partials[b * np .. b * np + np)) / n, NaN when status[b]
// is non-zero (OR-ed into user_status).
cudaError_t launch_reduce_S_batched(const double* partials, int32_t np, int64_t n, int32_t batch,
                                    const uint32_t* status, uint32_t* user_status, double* S_out,
                                    cudaStream_t stream);
// S = sum_c n_c S_c / sum_c n_c over m row chunks (device arrays).
cudaError_t launch_chunk_mean(const double* S_chunks, const int64_t* n_chunks, int32_t m, double* S_out,
                              cudaStream_t stream);
// S = sum(partials)/n, NaN when the workspace status word is non-zero; the
// word is OR-ed into user_status.
cudaError_t launch_reduce_S(const double* partials, int32_t np, int64_t n, const uint32_t* ws_status,
                            uint32_t* user_status, double* S_out, cudaStream_t stream);
cudaError_t launch_publish_status(const uint32_t* ws_status, uint32_t* user_status,
                                  cudaStream_t stream);

struct BackLaunch {
  const void* X;
  int32_t dtype;
  int64_t n;
  int32_t d;
  int64_t ldx;
  const float* cs;
  const int32_t* labels;
  int32_t k;
  int32_t dist;
  const float* zf;
  const float4* cl;
  const float* gf;
  const float* rs;
  const float* sa;
  const float* sb;
  const int32_t* skstar;
  const double* grad_S;
  float* dX;
  int64_t lddx;
  cudaStream_t stream;
  // nullable: the dual pass 1's sort (rows and alpha in bucket order, bucket
  // starts) and beta per row, for the gradient kernel that walks that order
  const uint32_t* idx = nullptr;
  const float* widx = nullptr;
  const uint32_t* bstart = nullptr;
  const float* w2 = nullptr;
};
// alpha_i / beta_i per point written into w1/w2 (float[n] each).
cudaError_t launch_backward_weights(const BackLaunch& b, float* w1, float* w2);
// Wf[c] = P'_c + Q'_c, Cf[c] = A_c + B_c from the dual weighted aggregates.
cudaError_t launch_backward_prep(const double* bw_w, const double* bw_p, int32_t k, int32_t d,
                                 float* Wf, float* Cf, cudaStream_t stream);
cudaError_t launch_backward_grad(const BackLaunch& b, const float* Wf, const float* Cf);

}  // namespace sil
