// The C ABI of libsil (declared in include/sil.h): argument validation,
// workspace carving and the sequence of kernel launches of each entry point.
// No allocation, no synchronisation: every call only enqueues work on the
// caller's stream.
#include <atomic>
#include <cstdlib>
#include <cmath>

#include "sil_internal.cuh"

namespace sil {

int num_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];  // 0 = not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev < kMaxDev) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
  v = std::min(v, kMaxPartials);  // grids sized from it write one partial sum per CTA
  if (dev < kMaxDev) cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

WsLayout ws_layout(int64_t n, int32_t d, int32_t k, int32_t dtype, int32_t dist, int32_t batch) {
  (void)dist;
  const size_t dz = size_t(round_up(d, 4));
  const size_t K = size_t(k), N = size_t(n);
  WsLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align256(bytes);
    return at;
  };
  L.misc = take(64 * 4);
  L.rs = take(K * dz * 4);
  L.g = take(dz * 8);
  L.gf = take(dz * 4);
  L.zf = take(K * dz * 4);
  L.cl = take(K * 16);
  L.invnorm = take(N * 4);
  L.partials = take(size_t(kMaxPartials) * 8);
  L.bw_w = take(2 * K * 8);
  L.bw_p = take(2 * K * size_t(d) * 8);
  L.bw_ab = take(2 * N * 4);
  L.bw_f = take((K * dz + K) * 4);
  L.saved = take(N * 12);
  L.bk = take((3 * 2 * K + 1) * 4);
  L.bidx = take(2 * N * 4);
  L.bw = take(2 * N * 4);
  L.zbf = take(std::max(tc_pack_bytes(k, d), t32_pack_bytes(k, d)));
  L.tcp = take(std::max(tc_partial_bytes(n, d, k, dtype), dtype == SIL_F32 ? t32_partial_bytes(n, d, k) : size_t(0)));
  L.batch = take(K * (size_t(d) + 2) * 8);
  // one launch for every labeling's pass 2 (shapes the batched kernel serves)
  const size_t pack = batch > 1 && dtype == SIL_F32 && k <= 512 ? tc_batched_pack_bytes(batch, k, d) : 0;
  if (pack) {
    const size_t B = size_t(batch), KP = size_t(round_up(std::max(k, 16), 16));
    L.bst = take(B * 4);
    L.bitems = take(2 * B * sizeof(TcItem));  // at most two blocks per labeling
    L.bmulti = take(B * sizeof(TcItem));
    L.bzf = take(B * KP * dz * 4);
    L.bcl = take(B * KP * 16);
    L.bg = take(B * dz * 8);
    L.bgf = take(B * dz * 4);
    L.bpack = take(pack);
    L.bpart = take(B * size_t(kBatchedMaxRanges) * 8);
    // nearest distance per (block, point) and a_i per point of the labelings
    // with two blocks
    L.bplanes = take(2 * B * N * 4);
    L.bown = take(B * N * 4);
  }
  L.total = o;
  return L;
}

}  // namespace sil

using namespace sil;

namespace {

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

int check_common(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* cs,
                 const int32_t* labels, int32_t k, int32_t dist) {
  if (n < 0 || d <= 0 || k <= 0 || ldx < d) return SIL_EINVAL;
  if (dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return SIL_EINVAL;
  if (dist != SIL_SQEUCLIDEAN && dist != SIL_COSINE && dist != SIL_EUCLIDEAN_RMS) return SIL_EINVAL;
  if (n > 0 && (X == nullptr || labels == nullptr)) return SIL_EINVAL;
  if (dtype == SIL_FP8_E4M3 && cs == nullptr) return SIL_EINVAL;
  if (k > (1 << 22) || d > (1 << 16)) return SIL_EUNSUPPORTED;
  if (n >= (int64_t(1) << 31)) return SIL_EUNSUPPORTED;  // row indices of the pass-1 sort are 32-bit
  return SIL_OK;
}

int check_ws(void* ws, size_t ws_bytes, int64_t n, int32_t d, int32_t k, int32_t dtype, int32_t dist,
             int32_t batch) {
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return SIL_EWORKSPACE;
  if (ws_bytes < ws_layout(n, d, k, dtype, dist, batch).total) return SIL_EWORKSPACE;
  return SIL_OK;
}

inline int cu(cudaError_t e) { return e == cudaSuccess ? SIL_OK : SIL_ECUDA; }

#define SIL_TRY(expr)              \
  do {                             \
    int rc_ = (expr);              \
    if (rc_ != SIL_OK) return rc_; \
  } while (0)

// Counting-sort scratch of pass 1 inside the workspace (sized for 2k buckets
// and 2n entries, the backward pass's dual form).
void set_sort_scratch(AggLaunch* a, void* ws, const WsLayout& L, int32_t k, int64_t n) {
  (void)n;
  uint32_t* bk = at<uint32_t>(ws, L.bk);
  a->bcount = bk;
  a->cursor = bk + 2 * size_t(k);
  a->bstart = bk + 4 * size_t(k);
  a->idx = at<uint32_t>(ws, L.bidx);
  a->widx = at<float>(ws, L.bw);
}

// Pass 1 into (count, s1, s2), status into the workspace word (or wst).
int run_aggregate(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* cs,
                  const int32_t* labels, int32_t k, int32_t dist, int64_t* count, double* s1,
                  double* s2, bool accumulate, void* ws, const WsLayout& L, cudaStream_t st,
                  uint32_t* wst = nullptr) {
  if (!wst) wst = at<uint32_t>(ws, L.misc);
  if (!accumulate) {
    SIL_TRY(cu(cudaMemsetAsync(count, 0, size_t(k) * 8, st)));
    SIL_TRY(cu(cudaMemsetAsync(s1, 0, size_t(k) * size_t(d) * 8, st)));
    SIL_TRY(cu(cudaMemsetAsync(s2, 0, size_t(k) * 8, st)));
  }
  if (n == 0) return SIL_OK;
  float* rs = at<float>(ws, L.rs);
  const float* invnorm = nullptr;
  if (dist == SIL_COSINE && agg_needs_invnorm(dtype, d)) {
    SIL_TRY(cu(launch_invnorm(X, dtype, n, d, ldx, cs, at<float>(ws, L.invnorm), wst, st)));
    invnorm = at<float>(ws, L.invnorm);
  }
  AggLaunch a{};
  a.X = X;
  a.dtype = dtype;
  a.n = n;
  a.d = d;
  a.ldx = ldx;
  a.cs = cs;
  a.labels = labels;
  a.k = k;
  a.dist = dist;
  a.rs = rs;
  a.invnorm = invnorm;
  a.count = reinterpret_cast<unsigned long long*>(count);
  a.s1 = s1;
  a.s2 = s2;
  a.status = wst;
  set_sort_scratch(&a, ws, L, k, n);
  a.stream = st;
  return cu(launch_aggregate(a));
}

int run_finalize(const int64_t* count, const double* s1, const double* s2, int32_t k, int32_t d,
                 int32_t dist, void* ws, const WsLayout& L, cudaStream_t st) {
  FinLaunch f{};
  f.count = reinterpret_cast<const unsigned long long*>(count);
  f.s1 = s1;
  f.s2 = s2;
  f.k = k;
  f.d = d;
  f.dist = dist;
  f.g = at<double>(ws, L.g);
  f.gf = at<float>(ws, L.gf);
  f.zf = at<float>(ws, L.zf);
  f.cl = at<float4>(ws, L.cl);
  f.status = at<uint32_t>(ws, L.misc);
  f.stream = st;
  return cu(launch_finalize(f));
}

// The automatic path takes the TF32-ranked kernel for few clusters: it has
// no converter warps (the lower cost per point), but sweeps the ranked
// values twice (the higher cost per cluster).  Measured on 1e7 rows of 64
// columns, pass 2 in ms (split-precision / TF32): K = 2 0.71 / 0.50,
// 16 0.72 / 0.62, 32 0.75 / 0.72, 64 0.79 / 0.85, 100 0.93 / 1.08.
constexpr int32_t kTf32AutoMaxK = 48;

bool takes_tf32(int32_t path, const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                const int32_t* labels, int32_t k) {
  return (path == SIL_PATH_TENSOR_TF32 || (path == SIL_PATH_AUTO && k <= kTf32AutoMaxK)) &&
         t32_eligible(dtype, n, d, ldx, k, X, labels);
}

// Pass 2 over finalized constants; writes partial sums, returns their count.
int run_score(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* cs,
              const int32_t* labels, int32_t k, int32_t dist, float* s_out, float* sa, float* sb,
              int32_t* skstar, int32_t path, void* ws, const WsLayout& L, cudaStream_t st,
              int32_t* np) {
  const bool tf32_ok = takes_tf32(path, X, dtype, n, d, ldx, labels, k);
  const bool tc_ok = (path == SIL_PATH_AUTO || path == SIL_PATH_TENSOR) &&
                     tc_eligible(dtype, n, d, ldx, k, X, labels);
  if ((path == SIL_PATH_TENSOR && !tc_ok) || (path == SIL_PATH_TENSOR_TF32 && !tf32_ok)) return SIL_EUNSUPPORTED;
  ScoreLaunch s{};
  s.X = X;
  s.dtype = dtype;
  s.n = n;
  s.d = d;
  s.ldx = ldx;
  s.cs = cs;
  s.labels = labels;
  s.k = k;
  s.dist = dist;
  s.zf = at<float>(ws, L.zf);
  s.cl = at<float4>(ws, L.cl);
  s.gf = at<float>(ws, L.gf);
  s.s_out = s_out;
  s.sa = sa;
  s.sb = sb;
  s.skstar = skstar;
  s.partials = at<double>(ws, L.partials);
  s.n_partials = np;
  s.status = at<uint32_t>(ws, L.misc);
  s.stream = st;
  if (tf32_ok)
    return cu(launch_score_tf32(s, at<double>(ws, L.g), at<void>(ws, L.zbf), at<void>(ws, L.tcp),
                                L.batch - L.tcp, s.status));
  if (tc_ok)
    return cu(launch_score_tc(s, at<double>(ws, L.g), at<void>(ws, L.zbf), at<void>(ws, L.tcp),
                              L.batch - L.tcp, s.status));
  return cu(launch_score_simt(s));
}

}  // namespace

extern "C" {

size_t sil_workspace_size(int64_t n, int32_t d, int32_t k, int32_t dtype, int32_t dist,
                          int32_t batch) {
  if (n < 0 || d <= 0 || k <= 0) return 0;
  return ws_layout(n, d, k, dtype, dist, batch < 1 ? 1 : batch).total;
}

size_t sil_saved_size(int64_t n) { return n < 0 ? 0 : size_t(n) * 12; }

int sil_aggregate(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                  const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
                  int64_t* count, double* s1, double* s2, uint32_t flags, void* ws,
                  size_t ws_bytes, uint32_t* dev_status, void* stream) {
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, k, dist));
  if (!count || !s1 || !s2) return SIL_EINVAL;
  SIL_TRY(check_ws(ws, ws_bytes, n, d, k, dtype, dist, 1));
  const WsLayout L = ws_layout(n, d, k, dtype, dist, 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = at<uint32_t>(ws, L.misc);
  SIL_TRY(cu(cudaMemsetAsync(wst, 0, 4, st)));
  SIL_TRY(run_aggregate(X, dtype, n, d, ldx, col_scale, labels, k, dist, count, s1, s2,
                        (flags & SIL_AGG_ACCUMULATE) != 0, ws, L, st));
  return cu(launch_publish_status(wst, dev_status, st));
}

int sil_score(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
              const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
              const int64_t* count, const double* s1, const double* s2, float* s_out,
              double* S_out, void* saved, int32_t path, void* ws, size_t ws_bytes,
              uint32_t* dev_status, void* stream) {
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, k, dist));
  if (!count || !s1 || !s2) return SIL_EINVAL;
  if (path < SIL_PATH_AUTO || path > SIL_PATH_TENSOR_TF32) return SIL_EINVAL;
  SIL_TRY(check_ws(ws, ws_bytes, n, d, k, dtype, dist, 1));
  const WsLayout L = ws_layout(n, d, k, dtype, dist, 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = at<uint32_t>(ws, L.misc);
  SIL_TRY(cu(cudaMemsetAsync(wst, 0, 4, st)));
  SIL_TRY(run_finalize(count, s1, s2, k, d, dist, ws, L, st));
  float* sa = nullptr;
  float* sb = nullptr;
  int32_t* skstar = nullptr;
  if (saved) {
    sa = static_cast<float*>(saved);
    sb = sa + n;
    skstar = reinterpret_cast<int32_t*>(sb + n);
  }
  int32_t np = 0;
  SIL_TRY(run_score(X, dtype, n, d, ldx, col_scale, labels, k, dist, s_out, sa, sb, skstar, path, ws,
                    L, st, &np));
  return cu(launch_reduce_S(at<double>(ws, L.partials), np, n, wst, dev_status, S_out, st));
}

int sil_silhouette(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* col_scale,
                   const int32_t* labels, int32_t k, int32_t dist, int64_t* count, double* s1, double* s2,
                   float* s_out, double* S_out, void* saved, int32_t path, void* ws, size_t ws_bytes,
                   uint32_t* dev_status, void* stream) {
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, k, dist));
  if (!count || !s1 || !s2) return SIL_EINVAL;
  if (path < SIL_PATH_AUTO || path > SIL_PATH_TENSOR_TF32) return SIL_EINVAL;
  SIL_TRY(check_ws(ws, ws_bytes, n, d, k, dtype, dist, 1));
  const WsLayout L = ws_layout(n, d, k, dtype, dist, 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = at<uint32_t>(ws, L.misc);
  SIL_TRY(cu(cudaMemsetAsync(wst, 0, 4, st)));
  SIL_TRY(run_aggregate(X, dtype, n, d, ldx, col_scale, labels, k, dist, count, s1, s2, false, ws, L, st));
  SIL_TRY(run_finalize(count, s1, s2, k, d, dist, ws, L, st));
  float* sa = nullptr;
  float* sb = nullptr;
  int32_t* skstar = nullptr;
  if (saved) {
    sa = static_cast<float*>(saved);
    sb = sa + n;
    skstar = reinterpret_cast<int32_t*>(sb + n);
  }
  int32_t np = 0;
  SIL_TRY(run_score(X, dtype, n, d, ldx, col_scale, labels, k, dist, s_out, sa, sb, skstar, path, ws, L, st, &np));
  return cu(launch_reduce_S(at<double>(ws, L.partials), np, n, wst, dev_status, S_out, st));
}

int sil_score_backward(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                       const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
                       const int64_t* count, const double* s1, const double* s2,
                       const void* saved, const double* grad_S, float* dX, int64_t lddx,
                       void* ws, size_t ws_bytes, uint32_t* dev_status, void* stream) {
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, k, dist));
  if (!count || !s1 || !s2 || (n > 0 && !dX) || lddx < d) return SIL_EINVAL;
  if (dist == SIL_EUCLIDEAN_RMS) return SIL_EUNSUPPORTED;  // no gradient for the approximation
  SIL_TRY(check_ws(ws, ws_bytes, n, d, k, dtype, dist, 1));
  const WsLayout L = ws_layout(n, d, k, dtype, dist, 1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = at<uint32_t>(ws, L.misc);
  SIL_TRY(cu(cudaMemsetAsync(wst, 0, 4, st)));
  if (n == 0) return cu(launch_publish_status(wst, dev_status, st));
  SIL_TRY(run_finalize(count, s1, s2, k, d, dist, ws, L, st));
  float* rs = at<float>(ws, L.rs);
  // rs is written by the dual pass 1 below, before the gradient kernel reads it
  const float* sa;
  const float* sb;
  const int32_t* skstar;
  if (saved) {
    sa = static_cast<const float*>(saved);
  } else {
    float* wsa = at<float>(ws, L.saved);
    int32_t np = 0;
    SIL_TRY(run_score(X, dtype, n, d, ldx, col_scale, labels, k, dist, nullptr, wsa, wsa + n,
                      reinterpret_cast<int32_t*>(wsa + 2 * n), SIL_PATH_AUTO, ws, L, st, &np));
    sa = wsa;
  }
  sb = sa + n;
  skstar = reinterpret_cast<const int32_t*>(sb + n);

  BackLaunch b{};
  b.X = X;
  b.dtype = dtype;
  b.n = n;
  b.d = d;
  b.ldx = ldx;
  b.cs = col_scale;
  b.labels = labels;
  b.k = k;
  b.dist = dist;
  b.zf = at<float>(ws, L.zf);
  b.cl = at<float4>(ws, L.cl);
  b.gf = at<float>(ws, L.gf);
  b.rs = rs;
  b.sa = sa;
  b.sb = sb;
  b.skstar = skstar;
  b.grad_S = grad_S;
  b.dX = dX;
  b.lddx = lddx;
  b.stream = st;
  float* w1 = at<float>(ws, L.bw_ab);
  float* w2 = w1 + n;
  SIL_TRY(cu(launch_backward_weights(b, w1, w2)));

  double* bw_w = at<double>(ws, L.bw_w);
  double* bw_p = at<double>(ws, L.bw_p);
  SIL_TRY(cu(cudaMemsetAsync(bw_w, 0, size_t(2) * k * 8, st)));
  SIL_TRY(cu(cudaMemsetAsync(bw_p, 0, size_t(2) * k * size_t(d) * 8, st)));
  const float* invnorm = nullptr;
  if (dist == SIL_COSINE && agg_needs_invnorm(dtype, d)) {
    SIL_TRY(cu(launch_invnorm(X, dtype, n, d, ldx, col_scale, at<float>(ws, L.invnorm), wst, st)));
    invnorm = at<float>(ws, L.invnorm);
  }
  AggLaunch a{};
  a.X = X;
  a.dtype = dtype;
  a.n = n;
  a.d = d;
  a.ldx = ldx;
  a.cs = col_scale;
  a.labels = labels;
  a.labels2 = skstar;
  a.w1 = w1;
  a.w2 = w2;
  a.k = k;
  a.dist = dist;
  a.rs = rs;
  a.invnorm = invnorm;
  a.s1 = bw_p;
  a.wsum = bw_w;
  a.status = wst;
  set_sort_scratch(&a, ws, L, k, n);
  a.stream = st;
  SIL_TRY(cu(launch_aggregate(a)));
  float* Wf = at<float>(ws, L.bw_f);
  float* Cf = Wf + size_t(k) * size_t(round_up(d, 4));
  SIL_TRY(cu(launch_backward_prep(bw_w, bw_p, k, d, Wf, Cf, st)));
  b.idx = a.idx;
  b.widx = a.widx;
  b.bstart = a.bstart;
  b.w2 = w2;
  SIL_TRY(cu(launch_backward_grad(b, Wf, Cf)));
  return cu(launch_publish_status(wst, dev_status, st));
}

}  // extern "C"

namespace {

// Items of the batched launch, handed to the device by value (kernel
// parameters), so that a captured graph holds them too.
constexpr int kItemChunk = 64;
struct ItemChunk {
  TcItem v[kItemChunk];
};
__global__ void k_set_items(ItemChunk c, int32_t count, TcItem* dst) {
  if (int(threadIdx.x) < count) dst[threadIdx.x] = c.v[threadIdx.x];
}

// Every labeling's pass 1 and finalisation, then one tensor-core launch for
// all their pass 2 and one reduction to the B means.
int run_batched_single_launch(const void* X, int64_t n, int32_t d, int64_t ldx, const int32_t* labels, int64_t ldl,
                              const int32_t* k_host, int32_t batch, int32_t kmax, int32_t dist, double* S_out,
                              void* ws, const WsLayout& L, uint32_t* dev_status, cudaStream_t st) {
  const int64_t dz = round_up(d, 4), kmaxp = round_up(std::max(kmax, 16), 16);
  uint32_t* bst = at<uint32_t>(ws, L.bst);
  TcItem* items = at<TcItem>(ws, L.bitems);
  TcItem* multi = at<TcItem>(ws, L.bmulti);
  float* bzf = at<float>(ws, L.bzf);
  float4* bcl = at<float4>(ws, L.bcl);
  double* bg = at<double>(ws, L.bg);
  float* bgf = at<float>(ws, L.bgf);
  SIL_TRY(cu(cudaMemsetAsync(bst, 0, size_t(batch) * 4, st)));
  int64_t* count = at<int64_t>(ws, L.batch);
  double* s1 = reinterpret_cast<double*>(count + kmax);
  double* s2 = s1 + size_t(kmax) * d;
  int32_t zrows = 0, n_items = 0, n_multi = 0, n_planes = 0;
  ItemChunk chunk{}, mchunk{};
  int32_t in_chunk = 0, in_mchunk = 0;
  auto flush = [&](ItemChunk& c, int32_t& cnt, TcItem* dst, int32_t done) -> int {
    if (cnt == 0) return SIL_OK;
    k_set_items<<<1, kItemChunk, 0, st>>>(c, cnt, dst + (done - cnt));
    cnt = 0;
    return cu(cudaGetLastError());
  };
  for (int32_t b = 0; b < batch; ++b) {
    const int32_t kb = k_host[b];
    const int32_t* lab = labels + b * ldl;
    SIL_TRY(run_aggregate(X, SIL_F32, n, d, ldx, nullptr, lab, kb, dist, count, s1, s2, false, ws, L, st, bst + b));
    FinLaunch f{};
    f.count = reinterpret_cast<const unsigned long long*>(count);
    f.s1 = s1;
    f.s2 = s2;
    f.k = kb;
    f.d = d;
    f.dist = dist;
    f.g = bg + b * dz;
    f.gf = bgf + b * dz;
    f.zf = bzf + b * kmaxp * dz;
    f.cl = bcl + b * kmaxp;
    f.status = bst + b;
    f.stream = st;
    SIL_TRY(cu(launch_finalize(f)));
    // blocks of at most 256 clusters (the MMA N), balanced
    const int32_t nblk = int32_t(cdiv(kb, 256));
    const int32_t kp = int32_t(round_up(std::max<int64_t>(cdiv(kb, nblk), 16), 16));
    const int32_t plane0 = nblk > 1 ? n_planes : -1, own_plane = nblk > 1 ? n_multi : -1;
    for (int32_t j = 0; j < nblk; ++j) {
      TcItem& it = chunk.v[in_chunk++];
      it.b = b;
      it.k = kb;
      it.nblk = nblk;
      it.kb0 = j * kp;
      it.kp = kp;
      it.zrow = zrows;
      it.cl_off = int32_t(b * kmaxp);
      it.zf_off = int32_t(b * kmaxp * dz);
      it.g_off = int32_t(b * dz);
      it.plane = nblk > 1 ? plane0 + j : -1;
      it.own_plane = own_plane;
      zrows += kp;
      ++n_items;
      if (j == 0 && nblk > 1) mchunk.v[in_mchunk++] = it;
      if (in_chunk == kItemChunk) SIL_TRY(flush(chunk, in_chunk, items, n_items));
    }
    if (nblk > 1) {
      n_planes += nblk;
      ++n_multi;
      if (in_mchunk == kItemChunk) SIL_TRY(flush(mchunk, in_mchunk, multi, n_multi));
    }
  }
  SIL_TRY(flush(chunk, in_chunk, items, n_items));
  SIL_TRY(flush(mchunk, in_mchunk, multi, n_multi));
  SIL_TRY(cu(launch_score_tc_batched(X, n, d, ldx, labels, ldl, batch, kmax, dist, items, n_items, zrows, multi,
                                     n_multi, bzf, bcl, bg, bgf, at<void>(ws, L.bpack), at<float>(ws, L.bplanes),
                                     at<float>(ws, L.bown), at<double>(ws, L.bpart), bst, st)));
  return cu(launch_reduce_S_batched(at<double>(ws, L.bpart), tc_batched_ranges(), n, batch, bst, dev_status, S_out,
                                    st));
}

}  // namespace

extern "C" {

int sil_score_batched(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                      const float* col_scale, const int32_t* labels, int64_t ldl,
                      const int32_t* k_host, int32_t batch, int32_t dist, double* S_out,
                      void* ws, size_t ws_bytes, uint32_t* dev_status, void* stream) {
  if (batch <= 0 || !k_host || !S_out || ldl < n) return SIL_EINVAL;
  int32_t kmax = 0;
  for (int32_t b = 0; b < batch; ++b) {
    if (k_host[b] <= 0) return SIL_EINVAL;
    kmax = k_host[b] > kmax ? k_host[b] : kmax;
  }
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, kmax, dist));
  SIL_TRY(check_ws(ws, ws_bytes, n, d, kmax, dtype, dist, batch));
  const WsLayout L = ws_layout(n, d, kmax, dtype, dist, batch);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t* wst = at<uint32_t>(ws, L.misc);
  if (L.bpack && batch > 1 && n > 0 && !(getenv("SIL_BATCH_PER_LABELING") && getenv("SIL_BATCH_PER_LABELING")[0] == '1') &&
      tc_batched_eligible(dtype, n, d, ldx, kmax, X, labels, ldl))
    return run_batched_single_launch(X, n, d, ldx, labels, ldl, k_host, batch, kmax, dist, S_out, ws, L, dev_status,
                                     st);
  int64_t* count = at<int64_t>(ws, L.batch);
  double* s1 = reinterpret_cast<double*>(count + kmax);
  double* s2 = s1 + size_t(kmax) * d;
  for (int32_t b = 0; b < batch; ++b) {
    const int32_t kb = k_host[b];
    const int32_t* lab = labels + b * ldl;
    SIL_TRY(cu(cudaMemsetAsync(wst, 0, 4, st)));
    SIL_TRY(run_aggregate(X, dtype, n, d, ldx, col_scale, lab, kb, dist, count, s1, s2, false, ws, L,
                          st));
    SIL_TRY(run_finalize(count, s1, s2, kb, d, dist, ws, L, st));
    int32_t np = 0;
    SIL_TRY(run_score(X, dtype, n, d, ldx, col_scale, lab, kb, dist, nullptr, nullptr, nullptr,
                      nullptr, SIL_PATH_AUTO, ws, L, st, &np));
    SIL_TRY(cu(launch_reduce_S(at<double>(ws, L.partials), np, n, wst, dev_status, S_out + b, st)));
  }
  return SIL_OK;
}

size_t sil_euclidean_workspace_size(int64_t n, int32_t d, int32_t k) {
  if (n < 0 || d <= 0 || k <= 0) return 0;
  return euclid_ws_bytes(n, d, k);
}

int sil_score_euclidean(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* col_scale,
                        const int32_t* labels, int32_t k, float* s_out, double* S_out, void* saved, void* ws,
                        size_t ws_bytes, uint32_t* dev_status, void* stream) {
  SIL_TRY(check_common(X, dtype, n, d, ldx, col_scale, labels, k, SIL_SQEUCLIDEAN));
  if (!S_out) return SIL_EINVAL;
  if (d > euclid_max_d()) return SIL_EUNSUPPORTED;
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < euclid_ws_bytes(n, d, k))
    return SIL_EWORKSPACE;
  float* sa = nullptr;
  float* sb = nullptr;
  int32_t* skstar = nullptr;
  if (saved) {
    sa = static_cast<float*>(saved);
    sb = sa + n;
    skstar = reinterpret_cast<int32_t*>(sb + n);
  }
  return cu(launch_euclid(X, dtype, n, d, ldx, col_scale, labels, k, s_out, sa, sb, skstar, ws, dev_status, S_out,
                          static_cast<cudaStream_t>(stream)));
}

int sil_tensor_plan(int32_t dtype, int32_t d, int32_t k, int32_t* block_k, int32_t* n_blocks) {
  if (!block_k || !n_blocks || d <= 0 || k <= 0) return SIL_EINVAL;
  if (dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return SIL_EINVAL;
  return tc_plan_query(dtype, d, k, block_k, n_blocks) ? SIL_OK : SIL_EUNSUPPORTED;
}

int sil_tensor_kernel(int32_t dtype, int32_t d, int32_t k) {
  if (d <= 0 || k <= 0 || dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return 0;
  int out = t32_serves(dtype, d, k) ? SIL_TENSOR_KERNEL_TF32 : 0;
  int32_t bk = 0, nb = 0;
  const bool box_ok = (dtype == SIL_F32 && d >= 32) || (dtype == SIL_BF16 && d >= 64) ||
                      (dtype == SIL_FP8_E4M3 && d == 128);
  if (box_ok && tc_plan_query(dtype, d, k, &bk, &nb)) out |= SIL_TENSOR_KERNEL_SPLIT;
  return out;
}

int sil_batched_plan_set(int32_t ranges, int32_t a_buffers) { return tc_batched_plan_set(ranges, a_buffers); }

int sil_chunk_mean(const double* S_chunks, const int64_t* n_chunks, int32_t m, double* S_out, void* stream) {
  if (m <= 0 || !S_chunks || !n_chunks || !S_out) return SIL_EINVAL;
  return cu(launch_chunk_mean(S_chunks, n_chunks, m, S_out, static_cast<cudaStream_t>(stream)));
}

int sil_tensor_plan_candidates(int32_t dtype, int32_t d, int32_t k, int32_t* plans, int32_t max_plans,
                               int32_t* n_plans) {
  if (!plans || !n_plans || max_plans < 0 || d <= 0 || k <= 0) return SIL_EINVAL;
  if (dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return SIL_EINVAL;
  *n_plans = tc_plan_candidates(dtype, d, k, plans, max_plans);
  return SIL_OK;
}

int sil_tensor_plan_set(int32_t dtype, int32_t d, int32_t k, int32_t block_k, int32_t a_buffers,
                        int32_t x_stages, int32_t stage_centroids, int32_t rank_pass) {
  if (d <= 0 || k <= 0 || dtype < SIL_F32 || dtype > SIL_FP8_E4M3) return SIL_EINVAL;
  return tc_plan_set(dtype, d, k, block_k, a_buffers, x_stages, stage_centroids, rank_pass);
}

int sil_selftest_bounded_wait(uint32_t* dev_out, void* stream) {
  if (dev_out == nullptr) return SIL_EINVAL;
  return cu(launch_selftest_wait(dev_out, static_cast<cudaStream_t>(stream)));
}

const char* sil_status_string(int32_t status) {
  switch (status) {
    case SIL_OK: return "SIL_OK";
    case SIL_EINVAL: return "SIL_EINVAL: invalid argument";
    case SIL_ELABEL: return "SIL_ELABEL: label outside [0, k)";
    case SIL_EDEGENERATE: return "SIL_EDEGENERATE: fewer than two non-empty clusters";
    case SIL_EZERONORM: return "SIL_EZERONORM: cosine distance of an all-zero row";
    case SIL_ECUDA: return "SIL_ECUDA: CUDA launch or memset failed";
    case SIL_ETIMEOUT: return "SIL_ETIMEOUT: a bounded device wait gave up";
    case SIL_EWORKSPACE: return "SIL_EWORKSPACE: workspace missing, misaligned or too small";
    case SIL_EUNSUPPORTED: return "SIL_EUNSUPPORTED: not served by this library";
    default: return "unknown status";
  }
}

int32_t sil_version(void) { return 100; }

}  // extern "C"
