// The exact Euclidean Silhouette by the standard quadratic method (Sec. II:
// Eq. 1-3 with the plain Euclidean distance ||x_i - x_j||), for the metric the
// linear method cannot serve exactly (Limitations section: the square root of
// a sum is not a sum of square roots, so no per-cluster aggregate gives it).
//
//   a_i = sum over j in C_c, j != i of ||x_i - x_j|| / (n_c - 1)
//   b_i = min over non-empty k != c of sum over j in C_k of ||x_i - x_j|| / n_k
//
// O(n^2 d) work: meant for datasets of up to ~1e5 points (and as a GPU
// cross-check of the O(n^2) definition at sizes the CPU cannot reach).
//
// Every distance is taken in the difference form sqrt(sum_l (x_il - x_jl)^2)
// in FP32, so no distance suffers the cancellation of ||x||^2 + ||y||^2 -
// 2 x.y (a tensor-core GEMM would supply only that expanded form, whose
// rounding bias does not average out of the per-cluster sums).
//
// Layout of the work.  The points are counting-sorted by label (the kernels
// of pass 1) and gathered into FP32 rows in that order, so every cluster is
// one contiguous run of columns.  The columns are split into P groups of
// whole clusters with about equal numbers of points, so that small n still
// gives enough CTAs: CTA (row block, group) owns 128 rows (one per thread,
// kept in registers) and streams its group's columns through shared memory in
// tiles of 64 points; each thread keeps one running sum for the cluster run
// it is in (FP32 over at most one tile, FP64 across tiles) and folds it into
// a_i or the group's running minimum when the run ends.  Run boundaries
// depend only on the column, so every branch is uniform across the CTA.  A
// combine kernel then takes each row's minimum over the groups (Eq. 3: b_i is
// a minimum over clusters, so it splits over any partition of them) and
// finishes s_i.
#include <algorithm>

#include "sil_internal.cuh"

namespace sil {

namespace {

constexpr int kBfThreads = 128;
constexpr int kBfTile = 64;  // columns (points) per shared-memory tile

// Rows of X in label order, as FP32 with dz = round_up(d, 4) columns (zero
// padded); the original row index and the label in that order.
// Rows whose label is outside [0, k) were left out by the sort (and flagged):
// only the first bstart[k] sorted positions are filled.
template <int DT>
__global__ void k_bf_gather(const void* X, int32_t k, int32_t d, int32_t dz, int64_t ldx, const float* cs,
                            bool vec, const uint32_t* bstart, const uint32_t* idx, const int32_t* labels, float* xs,
                            int32_t* ls) {
  const int nq = dz / 4;
  const int64_t total = int64_t(bstart[k]) * nq;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t p = e / nq;
    const int q = int(e - p * nq);
    const uint32_t row = idx[p];
    reinterpret_cast<float4*>(xs + p * dz)[q] = load4<DT>(X, row, 4 * q, d, ldx, cs, vec);
    if (q == 0) ls[p] = labels[row];
  }
}

struct BfK {
  int64_t n;
  int32_t dz, k, groups;
  const float* xs;
  const int32_t* ls;
  const uint32_t* idx;
  const uint32_t* bstart;  // [k + 1] first sorted position of each label
  const uint32_t* gstart;  // [groups + 1] first sorted position of each column group
  float* pmin;             // [groups][n] smallest mean distance to a cluster of the group (not own)
  int32_t* parg;           // [groups][n] that cluster
  float* pown;             // [n] a_i, from the group holding the own cluster
};

// Column groups: group g starts at the first cluster whose run starts at or
// after g * ceil(nv / P); empty groups are allowed.
__global__ void k_bf_groups(const uint32_t* bstart, int32_t k, int32_t P, uint32_t* gstart) {
  const int g = threadIdx.x;
  if (g > P) return;
  const uint32_t nv = bstart[k];
  if (g == P) {
    gstart[P] = nv;
    return;
  }
  const uint64_t target = (uint64_t(nv) + P - 1) / P * uint64_t(g);
  int lo = 0, hi = k;  // first c in [0, k] with bstart[c] >= target
  while (lo < hi) {
    const int mid = (lo + hi) / 2;
    if (bstart[mid] >= target) hi = mid;
    else lo = mid + 1;
  }
  gstart[g] = bstart[lo];
}

template <int DMAX>
__global__ void __launch_bounds__(kBfThreads) k_euclid_bf(BfK a) {
  __shared__ __align__(16) float ys[kBfTile * DMAX];
  __shared__ int32_t yl[kBfTile];
  const int dz = a.dz;
  const int g = blockIdx.y;
  const int64_t nv = a.bstart[a.k];  // sorted positions filled: rows with a valid label
  const int64_t c0 = a.gstart[g], c1 = a.gstart[g + 1];
  const int64_t p = int64_t(blockIdx.x) * kBfThreads + threadIdx.x;
  const bool valid = p < nv;
  const int own = valid ? a.ls[p] : -1;
  float x[DMAX];
#pragma unroll
  for (int c = 0; c < DMAX; c += 4) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid && c < dz) v = *reinterpret_cast<const float4*>(a.xs + p * dz + c);
    x[c] = v.x;
    x[c + 1] = v.y;
    x[c + 2] = v.z;
    x[c + 3] = v.w;
  }
  double run = 0.0, aown = -1.0;
  float tile = 0.f, bmin = INFINITY;
  int kb = -1, cur = -1;  // cur: the cluster whose run the column pointer is in (uniform)
  // folds the finished run of cluster c into a_i or the group's minimum
  auto fold = [&](int c) {
    if (c < 0) return;
    const double tot = run + double(tile);
    if (c == own) {
      aown = tot;
    } else {
      const float m = float(tot / double(a.bstart[c + 1] - a.bstart[c]));
      if (m < bmin) {  // runs come in increasing label order: ties keep the lowest index
        bmin = m;
        kb = c;
      }
    }
    run = 0.0;
    tile = 0.f;
  };
  for (int64_t j0 = c0; j0 < c1; j0 += kBfTile) {
    const int nj = int(std::min<int64_t>(kBfTile, c1 - j0));
    __syncthreads();  // the previous tile is consumed
    for (int e = threadIdx.x; e < nj * (dz / 4); e += kBfThreads) {
      const int jj = e / (dz / 4), q = e - jj * (dz / 4);
      reinterpret_cast<float4*>(ys + jj * DMAX)[q] = reinterpret_cast<const float4*>(a.xs + (j0 + jj) * dz)[q];
    }
    for (int jj = threadIdx.x; jj < nj; jj += kBfThreads) yl[jj] = a.ls[j0 + jj];
    __syncthreads();
    for (int jj = 0; jj < nj;) {
      const int c = yl[jj];
      if (c != cur) {
        fold(cur);
        cur = c;
      }
      if (jj + 1 < nj && yl[jj + 1] == c) {
        // two columns of the same run: four independent chains of FMAs
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
        const float* y = ys + jj * DMAX;
#pragma unroll
        for (int col = 0; col < DMAX; col += 4) {
          if (col >= dz) break;
          const float4 u = *reinterpret_cast<const float4*>(y + col);
          const float4 v = *reinterpret_cast<const float4*>(y + DMAX + col);
          const float2 xa = make_float2(x[col], x[col + 1]), xb = make_float2(x[col + 2], x[col + 3]);
          const float2 ua = __fadd2_rn(xa, make_float2(-u.x, -u.y)), ub = __fadd2_rn(xb, make_float2(-u.z, -u.w));
          const float2 va = __fadd2_rn(xa, make_float2(-v.x, -v.y)), vb = __fadd2_rn(xb, make_float2(-v.z, -v.w));
          a0 = __ffma2_rn(ua, ua, a0);
          a1 = __ffma2_rn(ub, ub, a1);
          b0 = __ffma2_rn(va, va, b0);
          b1 = __ffma2_rn(vb, vb, b1);
        }
        const float du = (a0.x + a1.x) + (a0.y + a1.y), dv = (b0.x + b1.x) + (b0.y + b1.y);
        tile += du > 0.f ? du * rsqrtf(du) : 0.f;  // ||x_i - x_j||; 0 for i = j
        tile += dv > 0.f ? dv * rsqrtf(dv) : 0.f;
        jj += 2;
      } else {
        // two independent partial sums halve the dependent chain of FMAs
        float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
        const float* y = ys + jj * DMAX;
#pragma unroll
        for (int col = 0; col < DMAX; col += 4) {
          if (col >= dz) break;
          const float4 yv = *reinterpret_cast<const float4*>(y + col);
          const float2 da = __fadd2_rn(make_float2(x[col], x[col + 1]), make_float2(-yv.x, -yv.y));
          const float2 db = __fadd2_rn(make_float2(x[col + 2], x[col + 3]), make_float2(-yv.z, -yv.w));
          acc0 = __ffma2_rn(da, da, acc0);
          acc1 = __ffma2_rn(db, db, acc1);
        }
        const float d2 = (acc0.x + acc1.x) + (acc0.y + acc1.y);
        tile += d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
        jj += 1;
      }
    }
    // FP32 sums over at most one tile, FP64 across tiles
    run += double(tile);
    tile = 0.f;
  }
  fold(cur);
  if (!valid) return;
  const uint32_t row = a.idx[p];
  a.pmin[int64_t(g) * a.n + row] = bmin;
  a.parg[int64_t(g) * a.n + row] = bmin < INFINITY ? kb : -1;
  if (aown >= 0.0) {
    const uint32_t nc = a.bstart[own + 1] - a.bstart[own];
    a.pown[row] = nc > 1 ? float(aown / double(nc - 1)) : 0.f;
  }
}

// s_i from the per-group results (row order of X): the smallest mean distance
// over the groups (lowest cluster index on ties: groups hold increasing
// labels and only a strictly smaller value replaces the best), a_i, Eq. 2,
// one partial sum per CTA.  Rows with a label outside [0, k) get s_i = 0.
__global__ void k_bf_combine(int64_t n, int32_t k, int32_t groups, const int32_t* labels, const uint32_t* bstart,
                             const float* pmin, const int32_t* parg, const float* pown, float* s_out, float* sa,
                             float* sb, int32_t* skstar, double* partials, uint32_t* status) {
  __shared__ float red[32];
  float tsum = 0.f;
  for (int64_t row = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; row < n;
       row += int64_t(gridDim.x) * blockDim.x) {
    const int own = labels[row];
    float sv = 0.f, av = 0.f, bv = INFINITY;
    int kb = -1;
    if (own >= 0 && own < k) {
      for (int g = 0; g < groups; ++g) {
        const float v = pmin[int64_t(g) * n + row];
        if (v < bv) {
          bv = v;
          kb = parg[int64_t(g) * n + row];
        }
      }
      av = pown[row];
      if (bv == INFINITY) set_status(status, SIL_EDEGENERATE);  // no other non-empty cluster
      if (bstart[own + 1] - bstart[own] > 1 && bv < INFINITY) sv = sil_eq2(av, bv, false);
    }
    if (s_out) s_out[row] = sv;
    if (sa) {
      sa[row] = av;
      sb[row] = bv;
      skstar[row] = kb;
    }
    tsum += sv;
  }
  for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += double(red[w]);
    partials[blockIdx.x] = t;
  }
}

// Column groups for n points: enough CTAs (row blocks x groups) for about
// four per SM, at most kBfMaxGroups.
constexpr int kBfMaxGroups = 16;
int bf_groups(int64_t n) {
  const int64_t rb = std::max<int64_t>(1, cdiv(n, kBfThreads));
  return int(std::max<int64_t>(1, std::min<int64_t>(kBfMaxGroups, cdiv(int64_t(4) * num_sms(), rb))));
}

}  // namespace

size_t euclid_ws_bytes(int64_t n, int32_t d, int32_t k) {
  const size_t N = size_t(n), dz = size_t(round_up(d, 4)), K = size_t(k), P = kBfMaxGroups;
  return align256(64 * 4)                      // status word
         + align256((3 * K + 1) * 4)           // bucket counts, starts, cursors
         + align256((P + 1) * 4)               // column-group starts
         + align256(N * 4) * 2                 // sorted row indices, labels in that order
         + align256(N * dz * 4)                // rows in label order (FP32)
         + align256(P * N * 4) * 2 + align256(N * 4)  // per-group minima and clusters, a_i
         + align256(size_t(kMaxPartials) * 8);  // per-CTA partial sums
}

int euclid_max_d() { return 128; }

cudaError_t launch_euclid(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* cs,
                          const int32_t* labels, int32_t k, float* s_out, float* sa, float* sb, int32_t* skstar,
                          void* ws, uint32_t* user_status, double* S_out, cudaStream_t st) {
  const size_t N = size_t(n), dz = size_t(round_up(d, 4)), K = size_t(k), PM = kBfMaxGroups;
  char* p = static_cast<char*>(ws);
  uint32_t* status = reinterpret_cast<uint32_t*>(p);
  p += align256(64 * 4);
  uint32_t* bcount = reinterpret_cast<uint32_t*>(p);
  uint32_t* bstart = bcount + K;
  uint32_t* cursor = bstart + K + 1;
  p += align256((3 * K + 1) * 4);
  uint32_t* gstart = reinterpret_cast<uint32_t*>(p);
  p += align256((PM + 1) * 4);
  uint32_t* idx = reinterpret_cast<uint32_t*>(p);
  p += align256(N * 4);
  int32_t* ls = reinterpret_cast<int32_t*>(p);
  p += align256(N * 4);
  float* xs = reinterpret_cast<float*>(p);
  p += align256(N * dz * 4);
  float* pmin = reinterpret_cast<float*>(p);
  p += align256(PM * N * 4);
  int32_t* parg = reinterpret_cast<int32_t*>(p);
  p += align256(PM * N * 4);
  float* pown = reinterpret_cast<float*>(p);
  p += align256(N * 4);
  double* partials = reinterpret_cast<double*>(p);

  cudaError_t e = cudaMemsetAsync(status, 0, 4, st);
  if (e != cudaSuccess) return e;
  int32_t np = 0;
  if (n > 0) {
    if ((e = launch_label_sort(labels, n, k, bcount, bstart, cursor, idx, status, st)) != cudaSuccess) return e;
    const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
    const bool vec = (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
    const unsigned grid = unsigned(std::min<int64_t>(cdiv(int64_t(N) * int64_t(dz / 4), 256), int64_t(num_sms()) * 16));
    switch (dtype) {
      case SIL_F32: k_bf_gather<SIL_F32><<<grid, 256, 0, st>>>(X, k, d, int(dz), ldx, cs, vec, bstart, idx, labels, xs, ls); break;
      case SIL_BF16: k_bf_gather<SIL_BF16><<<grid, 256, 0, st>>>(X, k, d, int(dz), ldx, cs, vec, bstart, idx, labels, xs, ls); break;
      default: k_bf_gather<SIL_FP8_E4M3><<<grid, 256, 0, st>>>(X, k, d, int(dz), ldx, cs, vec, bstart, idx, labels, xs, ls); break;
    }
    const int P = bf_groups(n);
    k_bf_groups<<<1, 32, 0, st>>>(bstart, k, P, gstart);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    BfK bk{};
    bk.n = n;
    bk.dz = int32_t(dz);
    bk.k = k;
    bk.groups = P;
    bk.xs = xs;
    bk.ls = ls;
    bk.idx = idx;
    bk.bstart = bstart;
    bk.gstart = gstart;
    bk.pmin = pmin;
    bk.parg = parg;
    bk.pown = pown;
    const dim3 bgrid(unsigned(cdiv(n, kBfThreads)), unsigned(P));
    if (dz <= 16) k_euclid_bf<16><<<bgrid, kBfThreads, 0, st>>>(bk);
    else if (dz <= 32) k_euclid_bf<32><<<bgrid, kBfThreads, 0, st>>>(bk);
    else if (dz <= 64) k_euclid_bf<64><<<bgrid, kBfThreads, 0, st>>>(bk);
    else k_euclid_bf<128><<<bgrid, kBfThreads, 0, st>>>(bk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int cgrid = int(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), kMaxPartials)));
    k_bf_combine<<<cgrid, 256, 0, st>>>(n, k, P, labels, bstart, pmin, parg, pown, s_out, sa, sb, skstar, partials,
                                        status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    np = cgrid;
  }
  return launch_reduce_S(partials, np, n, status, user_status, S_out, st);
}

}  // namespace sil
