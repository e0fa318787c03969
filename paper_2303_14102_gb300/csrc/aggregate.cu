// Pass 1: the segmented per-cluster reduction (Sec. III-A Eq. 5-9 with the
// footnote that Y and Psi come from one joint pass; Sec. III-B Eq. 15-16).
//
// Design (GB300): the reduction is HBM-bound -- one read of X and the labels
// -- so it is SIMT work whose only job is to stream X at full bandwidth with
// as few instructions per byte as possible.  A per-tile sort of the labels
// costs the same whatever K is, and with many clusters almost every row of a
// tile is its own segment; so the rows are counting-sorted by cluster ONCE,
// on the labels alone (4 bytes a row), and the reduction then walks the
// sorted order:
//   1. k_bucket_count    histogram of the labels (privatised in shared memory)
//   2. k_bucket_scan     exclusive scan -> bucket starts; the int64 counts
//   3. k_bucket_scatter  row indices (and weights) in bucket order; each CTA
//                        reserves one contiguous range per bucket it touches
//   4. k_gather_reduce   every warp takes a contiguous run of the sorted
//                        order; its lanes read whole rows with 16-byte loads
//                        (a row is one contiguous burst, so DRAM sees full
//                        sectors whatever the order of the rows), sum x - r_k
//                        in FP32 registers while the bucket stays the same,
//                        and add into the FP64 outputs once per run.
// Values are accumulated shifted by a per-cluster reference point r_k (the
// first row of cluster k in the sorted order), which keeps the FP32
// partials well conditioned when clusters sit far from the origin; a run's
// sums are un-shifted in FP64 when they are added:
//   s1 += sum(x - r) + m r,   s2 += sum||x - r||^2 + 2 r.sum(x - r) + m ||r||^2.
// The same kernels, with per-row weights and two bucket entries per row
// (bucket c_i and bucket k + k*_i), form the segmented sums of the backward
// pass; those are left shifted (sum w (x - r_c), with the shift of cluster c
// for both of its buckets) and come with sum w per bucket.
#include <climits>
#include <cstdlib>

#include "sil_internal.cuh"
#include "tma.cuh"

namespace sil {

namespace {

constexpr int kHistSmem = 12288;    // buckets privatised in shared memory by the count kernel
constexpr int kScatterSmem = 4096;  // buckets privatised by the scatter kernel
// entries per thread of the scatter kernel: with eight, at six CTAs per SM
// (40 registers), the at-scale scatter took 49 us against 98 us with 16 at
// two CTAs per SM (119 registers)
constexpr int kScatterIPT = 8;
constexpr int kScanThreads = 1024;
constexpr int kGatherThreads = 256;
constexpr int kGatherTmaWarps = 14;  // most warps of the TMA row-gather kernel

// One CTA per cluster: rs[k][c] = x_r for the first row r of cluster k in
// the sorted order (normalised for cosine), 0 when the cluster is empty.
template <int DT>
__global__ void k_shift_build(const void* X, int32_t d, int64_t ldx, const float* cs, const uint32_t* idx,
                              const uint32_t* bstart, int32_t dist, float* rs, int32_t dz) {
  __shared__ float red[32];
  const int kk = blockIdx.x;
  const bool empty = bstart[kk + 1] <= bstart[kk];
  const int64_t r = empty ? 0 : int64_t(idx[bstart[kk]]);
  float* out = rs + int64_t(kk) * dz;
  if (empty) {
    for (int c = threadIdx.x; c < dz; c += blockDim.x) out[c] = 0.f;
    return;
  }
  float ss = 0.f;
  for (int c = threadIdx.x * 4; c < dz; c += blockDim.x * 4) {
    float4 v = load4<DT>(X, r, c, d, ldx, cs, false);
    ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
  }
  float scale = 1.f;
  if (dist == SIL_COSINE) {
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
      red[0] = t;
    }
    __syncthreads();
    scale = red[0] > 0.f ? rsqrtf(red[0]) : 0.f;
  }
  for (int c = threadIdx.x * 4; c < dz; c += blockDim.x * 4) {
    float4 v = load4<DT>(X, r, c, d, ldx, cs, false);
    out[c + 0] = v.x * scale;
    out[c + 1] = v.y * scale;
    out[c + 2] = v.z * scale;
    out[c + 3] = v.w * scale;
  }
}

// One warp per row: invnorm[i] = 1/||x_i|| (0 and SIL_EZERONORM for a zero row).
template <int DT>
__global__ void k_invnorm(const void* X, int64_t n, int32_t d, int64_t ldx, const float* cs,
                          bool vec, float* invnorm, uint32_t* status) {
  const int lane = threadIdx.x & 31;
  int64_t row = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (; row < n; row += nwarps) {
    float ss = 0.f;
    for (int c = lane * 4; c < d; c += 128) {
      float4 v = load4<DT>(X, row, c, d, ldx, cs, vec);
      ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) {
      if (ss > 0.f) {
        invnorm[row] = rsqrtf(ss);
      } else {
        invnorm[row] = 0.f;
        set_status(status, SIL_EZERONORM);
      }
    }
  }
}

// ------------------------------------------------------------ bucket sort
// Entry e < n is row e in bucket labels[e]; in dual mode entry n + i is row i
// in bucket k + labels2[i] (labels2[i] = -1: no second entry).
struct Entries {
  int64_t n;
  int32_t k;
  const int32_t* lab1;
  const int32_t* lab2;
  const float* w1;
  const float* w2;
  uint32_t* status;
  __device__ __forceinline__ int bucket(int64_t e, bool report) const {
    if (e < n) {
      const int l = lab1[e];
      if (l >= 0 && l < k) return l;
      if (report) set_status(status, SIL_ELABEL);
      return -1;
    }
    const int l = lab2[e - n];
    if (l >= 0 && l < k) return k + l;
    if (report && l != -1) set_status(status, SIL_ELABEL);
    return -1;
  }
  // The raw label of entry e, and its bucket (-1: none); `bad` records an
  // out-of-range label (the caller reports it once, after its loads).
  __device__ __forceinline__ int label(int64_t e) const { return e < n ? __ldg(lab1 + e) : __ldg(lab2 + (e - n)); }
  __device__ __forceinline__ int bucket_of(int64_t e, int l, bool& bad) const {
    if (l >= 0 && l < k) return e < n ? l : k + l;
    if (e < n || l != -1) bad = true;
    return -1;
  }
  __device__ __forceinline__ uint32_t row(int64_t e) const { return uint32_t(e < n ? e : e - n); }
  __device__ __forceinline__ float weight(int64_t e) const { return e < n ? w1[e] : w2[e - n]; }
};

// Lanes with the same bucket reserve consecutive slots with one atomic on
// that bucket's counter; returns this lane's slot (the counter's old value
// plus the lane's rank among its peers).  b < 0: no slot.
__device__ __forceinline__ unsigned warp_reserve(int b, unsigned* counter_of_b) {
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, b);
  const int leader = __ffs(peers) - 1;
  unsigned old = 0;
  if (b >= 0 && lane == leader) old = atomicAdd(counter_of_b, unsigned(__popc(peers)));
  old = __shfl_sync(0xffffffffu, old, leader);
  return old + unsigned(__popc(peers & ((1u << lane) - 1u)));
}

__global__ void __launch_bounds__(256) k_bucket_count(Entries en, int64_t E, int32_t nb, uint32_t* bcount) {
  extern __shared__ uint32_t hist[];
  const bool priv = nb <= kHistSmem;
  if (priv)
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  constexpr int UNR = 8;  // labels in flight per thread
  // entries are below 2^32 (the callers check): 32-bit positions
  const uint32_t stride = gridDim.x * blockDim.x, E32 = uint32_t(E);
  // the loop bound is uniform per warp, so every lane reaches the warp collectives
  bool bad = false;
  for (uint64_t base = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x - lane; base < E;
       base += uint64_t(stride) * UNR) {
    // every label load is issued before any is used (a status write between
    // them would keep the compiler from overlapping the loads)
    int l[UNR], b[UNR];
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      const uint64_t e = base + uint64_t(i) * stride + lane;
      l[i] = e < E32 ? en.label(int64_t(e)) : -1;
    }
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      const uint64_t e = base + uint64_t(i) * stride + lane;
      b[i] = e < E32 ? en.bucket_of(int64_t(e), l[i], bad) : -1;
    }
    // shared-memory counters take one fire-and-forget increment per label;
    // global ones are aggregated per warp first
#pragma unroll
    for (int i = 0; i < UNR; ++i) {
      if (priv) {
        if (b[i] >= 0) atomicAdd(&hist[b[i]], 1u);
      } else {
        warp_reserve(b[i], b[i] >= 0 ? &bcount[b[i]] : nullptr);
      }
    }
  }
  if (bad) set_status(en.status, SIL_ELABEL);
  if (priv) {
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
      if (hist[b]) atomicAdd(&bcount[b], hist[b]);
  }
}

// One CTA: bstart[b] = sum of bcount[< b], bstart[nb] = total, cursor = bstart;
// count_out[b] += bcount[b] for the first k buckets when count_out is given.
__global__ void __launch_bounds__(kScanThreads) k_bucket_scan(const uint32_t* bcount, int32_t nb, int32_t k,
                                                              uint32_t* bstart, uint32_t* cursor,
                                                              unsigned long long* count_out) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  __shared__ uint32_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
    const int b = b0 + tid;
    const uint32_t c = b < nb ? bcount[b] : 0u;
    if (count_out && b < k) count_out[b] += c;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t off = carry;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (b < nb) {
      bstart[b] = off + incl - c;
      cursor[b] = off + incl - c;
    }
    __syncthreads();
    if (tid == kScanThreads - 1) carry = off + incl;
    __syncthreads();
  }
  if (tid == 0) bstart[nb] = carry;
}

// Each CTA places kScatterIPT * 256 consecutive entries.  With few buckets it
// counts them in shared memory first and reserves one range per bucket with
// a single global atomic (the hot buckets of skewed size distributions would
// otherwise serialise on their cursor), then lays its entries out in bucket
// order in shared memory, so that the index (and weight) writes are runs of
// consecutive addresses -- one per bucket the CTA touches -- instead of
// 4-byte scatters.
constexpr int kScatterTile = 256 * kScatterIPT;

// Dynamic shared memory of the scatter kernel: counts/starts and range bases
// per bucket, then the staged entries (rows, bucket ids, weights).
size_t scatter_smem(int32_t nb, bool weighted) {
  if (nb > kScatterSmem) return 0;
  return size_t(4) * (2 * size_t(nb) + kScatterTile) + size_t(2) * kScatterTile +
         (weighted ? size_t(4) * kScatterTile : 0);
}

__global__ void __launch_bounds__(256, 6) k_bucket_scatter(Entries en, int64_t E, int32_t nb, uint32_t* cursor,
                                                         uint32_t* idx, float* widx) {
  extern __shared__ __align__(16) uint32_t ssm[];
  const bool priv = nb <= kScatterSmem;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = int64_t(blockIdx.x) * kScatterTile;
  if (!priv) {
    for (int i = 0; i < kScatterIPT; ++i) {
      const int64_t e = c0 + int64_t(i) * 256 + tid;
      const int b = e < E ? en.bucket(e, false) : -1;
      const unsigned pos = warp_reserve(b, b >= 0 ? &cursor[b] : nullptr);
      if (b >= 0) {
        idx[pos] = en.row(e);
        if (widx) widx[pos] = en.weight(e);
      }
    }
    return;
  }
  uint32_t* lh = ssm;                // [nb] counts, then local starts
  uint32_t* lbase = ssm + nb;        // [nb] first global position of each range
  uint32_t* srow = lbase + nb;       // [tile] rows in local bucket order
  uint16_t* sbk = reinterpret_cast<uint16_t*>(srow + kScatterTile);  // their buckets
  float* swt = reinterpret_cast<float*>(sbk + kScatterTile);           // their weights
  __shared__ uint32_t wtot[8], total;
  for (int b = tid; b < nb; b += 256) lh[b] = 0;
  __syncthreads();
  int bk[kScatterIPT];
  unsigned rk[kScatterIPT];
#pragma unroll
  for (int i = 0; i < kScatterIPT; ++i) {  // all label loads first, then the reservations
    const int64_t e = c0 + int64_t(i) * 256 + tid;
    bk[i] = e < E ? en.bucket(e, false) : -1;
  }
  // ranks within the CTA: one shared-memory atomic per entry (independent,
  // so they pipeline); lanes hitting one counter get distinct values
#pragma unroll
  for (int i = 0; i < kScatterIPT; ++i) rk[i] = bk[i] >= 0 ? atomicAdd(&lh[bk[i]], 1u) : 0u;
  __syncthreads();
  for (int b = tid; b < nb; b += 256) {
    const uint32_t c = lh[b];
    lbase[b] = c ? atomicAdd(&cursor[b], c) : 0u;
  }
  __syncthreads();
  // local starts: exclusive scan of the counts (each thread a run of buckets)
  const int per = (nb + 255) / 256;
  const int b0 = min(nb, tid * per), b1 = min(nb, b0 + per);
  uint32_t run = 0;
  for (int b = b0; b < b1; ++b) run += lh[b];
  uint32_t incl = run;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  uint32_t off = incl - run;
  for (int w = 0; w < warp; ++w) off += wtot[w];
  if (tid == 255) total = off + run;
  for (int b = b0; b < b1; ++b) {
    const uint32_t c = lh[b];
    lh[b] = off;
    off += c;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScatterIPT; ++i) {
    if (bk[i] < 0) continue;
    const int64_t e = c0 + int64_t(i) * 256 + tid;
    const uint32_t p = lh[bk[i]] + rk[i];
    srow[p] = en.row(e);
    sbk[p] = uint16_t(bk[i]);
    if (widx) swt[p] = en.weight(e);
  }
  __syncthreads();
  const uint32_t tot = total;
  for (uint32_t p = tid; p < tot; p += 256) {
    const int b = sbk[p];
    const uint32_t pos = lbase[b] + (p - lh[b]);
    idx[pos] = srow[p];
    if (widx) widx[pos] = swt[p];
  }
}

// --------------------------------------------------------- gather-reduce
struct GatherK {
  const unsigned char* X;
  int64_t n;
  int32_t d;
  int64_t ldx_bytes;
  const float* cs;
  int32_t k;
  int32_t nb;
  int32_t dz;
  const uint32_t* idx;
  const float* widx;  // weights in sorted order (weighted mode), else null
  const uint32_t* bstart;
  const float* rs;
  const float* invnorm;  // 1/||x|| per row (cosine with column slices), else null
  int32_t cosine;
  int32_t vec;  // 16-byte loads allowed (X and the row stride 16-byte aligned)
  int32_t G;    // lanes per row (power of two)
  int32_t lgG;
  int32_t nch;       // 16-byte chunks in a row (whole row)
  int32_t ch_slice;  // chunks per column slice (= G * CPL, or fewer in the last)
  int64_t wchunk;    // sorted entries per warp work item
  int64_t nitems;
  int32_t rb;        // TMA-gather kernel: bytes of one row slot in shared memory
  int32_t stages;    // TMA-gather kernel: 32-row blocks in flight per warp
  double* s1;
  double* s2;
  double* wsum;
  uint32_t* status;
};

template <int DT>
struct Chunk;
template <>
struct Chunk<SIL_F32> {
  static constexpr int Q = 4;
  static __device__ __forceinline__ void cvt(const uint4& u, float* v) {
    v[0] = __uint_as_float(u.x);
    v[1] = __uint_as_float(u.y);
    v[2] = __uint_as_float(u.z);
    v[3] = __uint_as_float(u.w);
  }
};
template <>
struct Chunk<SIL_BF16> {
  static constexpr int Q = 8;
  static __device__ __forceinline__ void cvt(const uint4& u, float* v) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[i]));
      v[2 * i] = f.x;
      v[2 * i + 1] = f.y;
    }
  }
};
template <>
struct Chunk<SIL_FP8_E4M3> {
  static constexpr int Q = 16;
  static __device__ __forceinline__ void cvt(const uint4& u, float* v) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const __half2_raw hr =
            __nv_cvt_fp8x2_to_halfraw2(__nv_fp8x2_storage_t((w[i] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
        const float2 f = __half22float2(__half2(hr));
        v[4 * i + 2 * h] = f.x;
        v[4 * i + 2 * h + 1] = f.y;
      }
    }
  }
};

// 16 bytes of row `row` starting at element `col` (chunk aligned); elements
// at or past d read as 0.
template <int DT>
__device__ __forceinline__ uint4 load_chunk(const GatherK& a, uint32_t row, int col) {
  using T = typename Elem<DT>::T;
  constexpr int Q = Chunk<DT>::Q;
  const unsigned char* p = a.X + int64_t(row) * a.ldx_bytes + int64_t(col) * int64_t(sizeof(T));
  if (a.vec && col + Q <= a.d) return __ldg(reinterpret_cast<const uint4*>(p));
  // ragged last chunk or unaligned layout: element by element, packed into
  // the same little-endian words a 16-byte load would give
  constexpr int esz = int(sizeof(T));
  uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int t = 0; t < Q; ++t) {
    if (col + t < a.d) {
      uint32_t bits;
      if constexpr (esz == 4) bits = *reinterpret_cast<const uint32_t*>(p + 4 * t);
      else if constexpr (esz == 2) bits = *reinterpret_cast<const uint16_t*>(p + 2 * t);
      else bits = p[t];
      w[(t * esz) / 4] |= bits << (8 * ((t * esz) % 4));
    }
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// End of a run of bucket b: fold the row groups (lanes with the same chunk
// position hold the same columns), un-shift in FP64 and add to the outputs.
// Every lane of the warp must call it.
template <int DT, int CPL, bool WEIGHTED>
__device__ __forceinline__ void run_flush(const GatherK& a, int b, float2* acc, const float2* rsh, double sqd,
                                          float wacc, double mrows, const int* colb, const int* colend, int G,
                                          int rg, int lane) {
  constexpr int Q = Chunk<DT>::Q;
  constexpr int EL2 = CPL * Q / 2;
  for (int o = G; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < EL2; ++i) {
      acc[i].x += __shfl_xor_sync(0xffffffffu, acc[i].x, o);
      acc[i].y += __shfl_xor_sync(0xffffffffu, acc[i].y, o);
    }
    if (WEIGHTED) wacc += __shfl_xor_sync(0xffffffffu, wacc, o);
  }
  // weighted: every lane now holds the run's total weight in wacc
  const double m = WEIGHTED ? double(wacc) : mrows;
  double s2p = WEIGHTED ? 0.0 : sqd;
  if (rg == 0) {
#pragma unroll
    for (int i = 0; i < EL2; ++i) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = (2 * i + h) / Q, t = (2 * i + h) % Q;
        const int col = colb[j] + t;
        if (col >= colend[j]) continue;
        const double r = -double(h ? rsh[i].y : rsh[i].x), sv = h ? acc[i].y : acc[i].x;
        // weighted (backward) sums stay shifted: the gradient kernel works
        // with sum w (x - r) and sum w directly
        atomicAdd(a.s1 + int64_t(b) * a.d + col, WEIGHTED ? sv : sv + m * r);
        if (!WEIGHTED) s2p += 2.0 * r * sv + m * r * r;
      }
    }
  }
  if (!WEIGHTED) {
    for (int o = 16; o > 0; o >>= 1) s2p += __shfl_xor_sync(0xffffffffu, s2p, o);
    if (lane == 0) atomicAdd(a.s2 + b, s2p);
  } else if (lane == 0 && blockIdx.y == 0) {
    atomicAdd(a.wsum + b, m);
  }
}

// Shift of bucket b for this lane's elements (negated), packed in pairs.
template <int DT, int CPL>
__device__ __forceinline__ void load_shift(const GatherK& a, int b, const int* colb, const int* colend, float2* rsh) {
  constexpr int Q = Chunk<DT>::Q;
  constexpr int EL2 = CPL * Q / 2;
  const int kc = b < a.k ? b : b - a.k;  // cluster whose reference point shifts this bucket
#pragma unroll
  for (int i = 0; i < EL2; ++i) {
    float r[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = (2 * i + h) / Q, t = (2 * i + h) % Q;
      const int col = colb[j] + t;
      r[h] = col < colend[j] ? __ldg(a.rs + int64_t(kc) * a.dz + col) : 0.f;
    }
    rsh[i] = make_float2(-r[0], -r[1]);
  }
}

// One warp walks its work items of the sorted order.  Lane layout: G lanes
// per row (lane % G = first 16-byte chunk, CPL chunks per lane, G apart), 32/G
// rows side by side; every lane issues the loads of RPL rows before it
// consumes any, so a warp keeps 32/G * RPL rows (a few KB) in flight.  The
// run's sorted indices arrive 32 at a time in one coalesced load, one block
// ahead, and lanes take their rows from it by shuffle.  Per run of one bucket
// the lanes keep FP32 sums of the shifted values (packed FP32x2 arithmetic);
// at the end of the run the row groups are folded with shuffles and the run
// is added to the FP64 outputs.
template <int DT, int CPL, bool WEIGHTED, bool COS>
__global__ void __launch_bounds__(kGatherThreads, 2) k_gather_reduce(GatherK a) {
  constexpr int Q = Chunk<DT>::Q;
  constexpr int EL = CPL * Q;        // elements per lane
  constexpr int EL2 = EL / 2;        // packed pairs
  constexpr int RPL = 8 / CPL;  // rows in flight per lane (eight 16-byte loads)
  const int lane = threadIdx.x & 31;
  const int G = a.G, R = 32 >> a.lgG;
  const int rg = lane >> a.lgG, cl = lane & (G - 1);
  const int ch0 = int(blockIdx.y) * a.ch_slice;  // first chunk of this column slice
  const int chn = min(a.ch_slice, a.nch - ch0);  // chunks of this slice
  const uint32_t total = a.bstart[a.nb];
  // column of element t of this lane's chunk j: colb[j] + t, valid while < colend[j]
  int colb[CPL], colend[CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int ch = cl + G * j;
    colb[j] = (ch0 + ch) * Q;
    colend[j] = ch < chn ? min(a.d, colb[j] + Q) : colb[j];
  }
  float2 csc[EL2];
#pragma unroll
  for (int i = 0; i < EL2; ++i) {
    float c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = (2 * i + h) / Q, t = (2 * i + h) % Q;
      c[h] = (DT == SIL_FP8_E4M3 && colb[j] + t < colend[j]) ? __ldg(a.cs + colb[j] + t) : 1.f;
    }
    csc[i] = make_float2(c[0], c[1]);
  }

  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t item = gw; item < a.nitems; item += nw) {
    const int64_t e0 = item * a.wchunk;
    const int64_t e1 = min(int64_t(total), e0 + a.wchunk);
    if (e0 >= e1) break;
    // bucket holding e0: the last b with bstart[b] <= e0
    int lo = 0, hi = a.nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.bstart + mid) <= uint32_t(e0)) lo = mid;
      else hi = mid - 1;
    }
    int b = lo;
    int64_t cur = e0;
    while (cur < e1) {
      while (__ldg(a.bstart + b + 1) <= uint32_t(cur)) ++b;  // skip empty buckets
      const int64_t se = min(e1, int64_t(__ldg(a.bstart + b + 1)));
      float2 rsh[EL2], acc[EL2];
      load_shift<DT, CPL>(a, b, colb, colend, rsh);
#pragma unroll
      for (int i = 0; i < EL2; ++i) acc[i] = make_float2(0.f, 0.f);
      // squared terms: FP32 within a block of 32 entries, FP64 across blocks
      // (short FP32 chains keep the sum of squares free of drift)
      float2 sq2 = make_float2(0.f, 0.f);
      double sqd = 0.0;
      float wacc = 0.f;
      int64_t blk = cur;
      uint32_t iv = blk + lane < se ? __ldg(a.idx + blk + lane) : 0u;
      float wvb = (WEIGHTED && blk + lane < se) ? __ldg(a.widx + blk + lane) : 0.f;
      while (blk < se) {
        const int64_t nxt = blk + 32;
        const uint32_t ivn = nxt + lane < se ? __ldg(a.idx + nxt + lane) : 0u;
        const float wvn = (WEIGHTED && nxt + lane < se) ? __ldg(a.widx + nxt + lane) : 0.f;
        const int cnt = int(min(int64_t(32), se - blk));
        for (int p0 = 0; p0 < cnt; p0 += R * RPL) {
          uint4 raw[RPL][CPL];
          uint32_t rowv[RPL];
          bool ok[RPL];
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int pos = p0 + u * R + rg;
            ok[u] = pos < cnt;
            rowv[u] = __shfl_sync(0xffffffffu, iv, pos & 31);
#pragma unroll
            for (int j = 0; j < CPL; ++j)
              raw[u][j] = (ok[u] && colb[j] < colend[j]) ? load_chunk<DT>(a, rowv[u], colb[j]) : make_uint4(0, 0, 0, 0);
          }
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            float w = 1.f;
            if (WEIGHTED) w = __shfl_sync(0xffffffffu, wvb, (p0 + u * R + rg) & 31);
            float v[EL];
#pragma unroll
            for (int j = 0; j < CPL; ++j) Chunk<DT>::cvt(raw[u][j], v + j * Q);
            float2 v2[EL2];
#pragma unroll
            for (int i = 0; i < EL2; ++i) {
              v2[i] = make_float2(v[2 * i], v[2 * i + 1]);
              if (DT == SIL_FP8_E4M3) v2[i] = __fmul2_rn(v2[i], csc[i]);
            }
            float sc = 1.f;
            if (COS) {
              if (a.invnorm) {
                sc = ok[u] ? __ldg(a.invnorm + rowv[u]) : 0.f;
              } else {
                float2 ss = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < EL2; ++i) ss = __ffma2_rn(v2[i], v2[i], ss);
                float s1 = ss.x + ss.y;
                for (int o = 1; o < G; o <<= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                if (ok[u] && !(s1 > 0.f) && cl == 0) set_status(a.status, SIL_EZERONORM);
                sc = s1 > 0.f ? rsqrtf(s1) : 0.f;
              }
            }
            if (ok[u]) {
              const float2 sc2 = make_float2(sc, sc);
#pragma unroll
              for (int i = 0; i < EL2; ++i) {
                float2 t = __ffma2_rn(sc2, v2[i], rsh[i]);  // sc x - r
                if (WEIGHTED) {
                  t = __fmul2_rn(t, make_float2(w, w));
                } else {
                  sq2 = __ffma2_rn(t, t, sq2);
                }
                acc[i] = __fadd2_rn(acc[i], t);
              }
              if (WEIGHTED) wacc += w;
            }
          }
        }
        sqd += double(sq2.x) + double(sq2.y);
        sq2 = make_float2(0.f, 0.f);
        iv = ivn;
        wvb = wvn;
        blk = nxt;
      }
      run_flush<DT, CPL, WEIGHTED>(a, b, acc, rsh, sqd, wacc, WEIGHTED ? 0.0 : double(se - cur), colb, colend, G, rg, lane);
      cur = se;
    }
  }
}

// The same reduction with the rows brought into shared memory by the tensor
// memory accelerator's row gather (cp.async.bulk.tensor ... tile::gather4,
// four rows by index per instruction): every warp owns a ring of `stages`
// 32-row blocks and keeps all but one of them in flight while it sums the
// oldest one, so the bytes in flight per SM no longer depend on registers.
// A block may cross bucket boundaries; rows are summed into the bucket they
// belong to and the run is flushed where the bucket changes.  Waits are
// bounded: on a timeout the warp flags SIL_ETIMEOUT, waits (bounded) for its
// own copies in flight and stops.
template <int DT, int CPL, bool WEIGHTED, bool COS>
__global__ void __launch_bounds__(kGatherTmaWarps * 32, 1) k_gather_reduce_tma(GatherK a, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr int Q = Chunk<DT>::Q;
  constexpr int EL = CPL * Q;
  constexpr int EL2 = EL / 2;
  constexpr int esz = int(sizeof(typename Elem<DT>::T));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int S = a.stages;
  const int SB = 32 * a.rb;
  unsigned char* ring = base + size_t(warp) * S * SB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + size_t(nwarp) * S * SB) + warp * S;
  if (lane < S) mbar_init(&bars[lane], 1);
  fence_mbar_init();
  __syncwarp();
  const int G = a.G, R = 32 >> a.lgG;
  const int rg = lane >> a.lgG, cl = lane & (G - 1);
  const int RS = R < 32 ? R * (32 / R >= 2 ? 2 : 1) : 32;  // rows per step (two per lane group when they fit)
  const uint32_t total = a.bstart[a.nb];
  int colb[CPL], colend[CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const int ch = cl + G * j;
    colb[j] = ch * Q;
    colend[j] = ch < a.nch ? min(a.d, colb[j] + Q) : colb[j];
  }
  float2 csc[EL2];
#pragma unroll
  for (int i = 0; i < EL2; ++i) {
    float c[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = (2 * i + h) / Q, t = (2 * i + h) % Q;
      c[h] = (DT == SIL_FP8_E4M3 && colb[j] + t < colend[j]) ? __ldg(a.cs + colb[j] + t) : 1.f;
    }
    csc[i] = make_float2(c[0], c[1]);
  }

  uint32_t gblk = 0;  // blocks this warp has consumed (ring position and phase)
  const int64_t gw = int64_t(blockIdx.x) * nwarp + warp;
  const int64_t nw = int64_t(gridDim.x) * nwarp;
  for (int64_t item = gw; item < a.nitems; item += nw) {
    const int64_t e0 = item * a.wchunk;
    const int64_t e1 = min(int64_t(total), e0 + a.wchunk);
    if (e0 >= e1) break;
    const int nblk = int(cdiv(e1 - e0, 32));
    // rows of block t (dummy rows past e1 repeat the block's first row)
    auto block_rows = [&](int t) -> uint32_t {
      const int64_t e = e0 + int64_t(t) * 32 + lane;
      const uint32_t r = e < e1 ? __ldg(a.idx + e) : 0xFFFFFFFFu;
      const uint32_t r0 = __shfl_sync(0xffffffffu, r, 0);
      return r == 0xFFFFFFFFu ? r0 : r;
    };
    auto issue = [&](int t, uint32_t rows) {
      const int slot = int((gblk + uint32_t(t)) % uint32_t(S));
      uint32_t rr[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) rr[q] = __shfl_sync(0xffffffffu, rows, (4 * lane + q) & 31);
      if (lane == 0) mbar_arrive_expect_tx(&bars[slot], uint32_t(SB));
      __syncwarp();
      if (lane < 8)
        tma_gather4(ring + size_t(slot) * SB + size_t(lane) * 4 * a.rb, &xmap, 0, int32_t(rr[0]), int32_t(rr[1]),
                    int32_t(rr[2]), int32_t(rr[3]), &bars[slot]);
    };
    const int pre = nblk < S ? nblk : S;
    for (int t = 0; t < pre; ++t) issue(t, block_rows(t));
    uint32_t pending = pre < nblk ? block_rows(pre) : 0u;

    // bucket holding e0
    int lo = 0, hi = a.nb - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.bstart + mid) <= uint32_t(e0)) lo = mid;
      else hi = mid - 1;
    }
    int b = lo;
    int64_t blo = e0;                                            // first entry of the current run
    int64_t bend = min(e1, int64_t(__ldg(a.bstart + b + 1)));  // end of the current run
    float2 rsh[EL2], acc[EL2];
    load_shift<DT, CPL>(a, b, colb, colend, rsh);
#pragma unroll
    for (int i = 0; i < EL2; ++i) acc[i] = make_float2(0.f, 0.f);
    float2 sq2 = make_float2(0.f, 0.f);  // squared terms: FP32 within a block, FP64 across
    double sqd = 0.0;
    float wacc = 0.f;

    for (int t = 0; t < nblk; ++t) {
      const int slot = int((gblk + uint32_t(t)) % uint32_t(S));
      const uint32_t par = ((gblk + uint32_t(t)) / uint32_t(S)) & 1u;
      const int64_t eb = e0 + int64_t(t) * 32;
      const float wblk = (WEIGHTED && eb + lane < e1) ? __ldg(a.widx + eb + lane) : 0.f;
      if (!mbar_wait(&bars[slot], par)) {
        if (lane == 0) set_status(a.status, SIL_ETIMEOUT);
        // blocks t .. min(nblk, t + S) - 1 were issued and not consumed
        for (int u = t; u < nblk && u < t + S; ++u)
          mbar_wait(&bars[(gblk + uint32_t(u)) % uint32_t(S)], ((gblk + uint32_t(u)) / uint32_t(S)) & 1u);
        return;
      }
      const unsigned char* blkp = ring + size_t(slot) * SB;
      for (int p0 = 0; p0 < 32; p0 += RS) {
        constexpr int RPL = 2;
        uint4 raw[RPL][CPL];
        int64_t ev[RPL];
        bool in_blk[RPL];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int p = p0 + u * R + rg;
          ev[u] = eb + p;
          in_blk[u] = (u * R < RS) && p < 32 && ev[u] < e1;
#pragma unroll
          for (int j = 0; j < CPL; ++j)
            raw[u][j] = (in_blk[u] && colb[j] < colend[j])
                            ? *reinterpret_cast<const uint4*>(blkp + size_t(p) * a.rb + size_t(colb[j]) * esz)
                            : make_uint4(0, 0, 0, 0);
        }
        float2 v2[RPL][EL2];
        float scv[RPL], wv[RPL];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          float v[EL];
#pragma unroll
          for (int j = 0; j < CPL; ++j) Chunk<DT>::cvt(raw[u][j], v + j * Q);
#pragma unroll
          for (int i = 0; i < EL2; ++i) {
            v2[u][i] = make_float2(v[2 * i], v[2 * i + 1]);
            if (DT == SIL_FP8_E4M3) v2[u][i] = __fmul2_rn(v2[u][i], csc[i]);
          }
          scv[u] = 1.f;
          if (COS) {
            float2 ss = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < EL2; ++i) ss = __ffma2_rn(v2[u][i], v2[u][i], ss);
            float s1 = ss.x + ss.y;
            for (int o = 1; o < G; o <<= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            if (in_blk[u] && !(s1 > 0.f) && cl == 0) set_status(a.status, SIL_EZERONORM);
            scv[u] = s1 > 0.f ? rsqrtf(s1) : 0.f;
          }
          wv[u] = WEIGHTED ? __shfl_sync(0xffffffffu, wblk, (p0 + u * R + rg) & 31) : 1.f;
        }
        // rows of this step go to the run they belong to; the step may cross runs
        const int64_t slast = min(eb + p0 + RS, e1) - 1;  // last entry of the step
        while (true) {
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            if (!(in_blk[u] && ev[u] >= blo && ev[u] < bend)) continue;
            const float2 sc2 = make_float2(scv[u], scv[u]);
#pragma unroll
            for (int i = 0; i < EL2; ++i) {
              float2 tt = __ffma2_rn(sc2, v2[u][i], rsh[i]);  // sc x - r
              if (WEIGHTED) {
                tt = __fmul2_rn(tt, make_float2(wv[u], wv[u]));
              } else {
                sq2 = __ffma2_rn(tt, tt, sq2);
              }
              acc[i] = __fadd2_rn(acc[i], tt);
            }
            if (WEIGHTED) wacc += wv[u];
          }
          if (slast < bend) break;
          // the run ends inside this step: add it and start the next bucket
          run_flush<DT, CPL, WEIGHTED>(a, b, acc, rsh, sqd + double(sq2.x) + double(sq2.y), wacc,
                                       double(bend - blo), colb, colend, G, rg, lane);
          sqd = 0.0;
          blo = bend;
          while (__ldg(a.bstart + b + 1) <= uint32_t(blo)) ++b;
          bend = min(e1, int64_t(__ldg(a.bstart + b + 1)));
          load_shift<DT, CPL>(a, b, colb, colend, rsh);
#pragma unroll
          for (int i = 0; i < EL2; ++i) acc[i] = make_float2(0.f, 0.f);
          sq2 = make_float2(0.f, 0.f);
          wacc = 0.f;
        }
      }
      sqd += double(sq2.x) + double(sq2.y);
      sq2 = make_float2(0.f, 0.f);
      // every lane is done with the slot before the TMA (async proxy)
      // refills it: fence the generic-proxy reads, then sync the warp
      fence_proxy_async_smem();
      __syncwarp();
      if (t + S < nblk) {
        issue(t + S, pending);
        pending = t + S + 1 < nblk ? block_rows(t + S + 1) : 0u;
      }
    }
    if (bend > blo)
      run_flush<DT, CPL, WEIGHTED>(a, b, acc, rsh, sqd + double(sq2.x) + double(sq2.y), wacc, double(bend - blo), colb,
                                   colend, G, rg, lane);
    gblk += uint32_t(nblk);
  }
}

// One wave of resident CTAs; each warp takes about four work items of the
// sorted order.
template <int DT, int CPL, bool WEIGHTED, bool COS>
cudaError_t launch_gather_t(GatherK g, int64_t E, int slices, cudaStream_t st) {
  auto fn = k_gather_reduce<DT, CPL, WEIGHTED, COS>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGatherThreads, 0);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, per_sm);
  const int64_t ctas = std::max<int64_t>(1, int64_t(num_sms()) * per_sm / slices);
  const int64_t warps = ctas * (kGatherThreads / 32);
  g.wchunk = round_up(std::max<int64_t>(128, cdiv(E, warps * 4)), 32);
  g.nitems = cdiv(E, g.wchunk);
  const dim3 grid(unsigned(std::min<int64_t>(ctas, cdiv(g.nitems, kGatherThreads / 32))), unsigned(slices));
  fn<<<grid, kGatherThreads, 0, st>>>(g);
  return cudaGetLastError();
}

// Rows into shared memory by TMA row gather: one persistent CTA per SM,
// `warps` warps each with a ring of `stages` 32-row blocks.
template <int DT, int CPL, bool WEIGHTED, bool COS>
cudaError_t launch_gather_tma_t(GatherK g, const CUtensorMap& map, int64_t E, int warps, int smem,
                                cudaStream_t st) {
  auto fn = k_gather_reduce_tma<DT, CPL, WEIGHTED, COS>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t wtot = int64_t(num_sms()) * warps;
  g.wchunk = round_up(std::max<int64_t>(256, cdiv(E, wtot * 2)), 32);
  g.nitems = cdiv(E, g.wchunk);
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(num_sms(), cdiv(g.nitems, warps))));
  fn<<<grid, warps * 32, smem, st>>>(g, map);
  return cudaGetLastError();
}

template <int DT, int CPL>
cudaError_t launch_gather_tma_mode(const GatherK& g, const CUtensorMap& map, int64_t E, int warps, int smem,
                                   cudaStream_t st) {
  const bool w = g.widx != nullptr;
  if (g.cosine)
    return w ? launch_gather_tma_t<DT, CPL, true, true>(g, map, E, warps, smem, st)
             : launch_gather_tma_t<DT, CPL, false, true>(g, map, E, warps, smem, st);
  return w ? launch_gather_tma_t<DT, CPL, true, false>(g, map, E, warps, smem, st)
           : launch_gather_tma_t<DT, CPL, false, false>(g, map, E, warps, smem, st);
}

template <int DT, int CPL>
cudaError_t launch_gather_mode(const GatherK& g, int64_t E, int slices, cudaStream_t st) {
  const bool w = g.widx != nullptr;
  if (g.cosine) return w ? launch_gather_t<DT, CPL, true, true>(g, E, slices, st) : launch_gather_t<DT, CPL, false, true>(g, E, slices, st);
  return w ? launch_gather_t<DT, CPL, true, false>(g, E, slices, st) : launch_gather_t<DT, CPL, false, false>(g, E, slices, st);
}

// Largest number of 16-byte chunks one lane handles (16 elements per lane).
int max_cpl(int32_t dtype) { return dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1; }
int elem_bytes(int32_t dtype) { return dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1; }

}  // namespace

bool agg_needs_invnorm(int32_t dtype, int32_t d) {
  const int q = 16 / elem_bytes(dtype);
  return cdiv(d, q) > 32 * max_cpl(dtype);
}

cudaError_t launch_invnorm(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                           const float* cs, float* invnorm, uint32_t* status, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const int esz = elem_bytes(dtype);
  const bool vec = (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
  const unsigned grid = unsigned(std::min<int64_t>(cdiv(n, 8), int64_t(num_sms()) * 16));
  switch (dtype) {
    case SIL_F32: k_invnorm<SIL_F32><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
    case SIL_BF16: k_invnorm<SIL_BF16><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
    default: k_invnorm<SIL_FP8_E4M3><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_label_sort(const int32_t* labels, int64_t n, int32_t k, uint32_t* bcount, uint32_t* bstart,
                              uint32_t* cursor, uint32_t* idx, uint32_t* status, cudaStream_t stream) {
  if (n >= (int64_t(1) << 32)) return cudaErrorInvalidValue;
  Entries en{n, k, labels, nullptr, nullptr, nullptr, status};
  cudaError_t e = cudaMemsetAsync(bcount, 0, size_t(k) * 4, stream);
  if (e != cudaSuccess) return e;
  const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256 * 8), int64_t(num_sms()) * 8)));
  const size_t smem = k <= kHistSmem ? size_t(k) * 4 : 0;
  k_bucket_count<<<grid, 256, smem, stream>>>(en, n, k, bcount);
  k_bucket_scan<<<1, kScanThreads, 0, stream>>>(bcount, k, k, bstart, cursor, nullptr);
  const size_t ssmem = scatter_smem(k, false);
  if ((e = cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(scatter_smem(kScatterSmem, true)))) != cudaSuccess)
    return e;
  k_bucket_scatter<<<unsigned(cdiv(n, kScatterTile)), 256, ssmem, stream>>>(en, n, k, cursor, idx, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_aggregate(const AggLaunch& L) {
  if (L.n == 0) return cudaSuccess;
  const bool dual = L.labels2 != nullptr;
  const int64_t E = dual ? 2 * L.n : L.n;
  const int nb = dual ? 2 * L.k : L.k;
  if (E >= (int64_t(1) << 32)) return cudaErrorInvalidValue;
  Entries en{L.n, L.k, L.labels, L.labels2, L.w1, L.w2, L.status};

  // 1-3: counting sort of the entries by bucket
  cudaError_t e = cudaMemsetAsync(L.bcount, 0, size_t(nb) * 4, L.stream);
  if (e != cudaSuccess) return e;
  {
    const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>(cdiv(E, 256 * 8), int64_t(num_sms()) * 8)));
    const size_t smem = nb <= kHistSmem ? size_t(nb) * 4 : 0;
    k_bucket_count<<<grid, 256, smem, L.stream>>>(en, E, nb, L.bcount);
  }
  k_bucket_scan<<<1, kScanThreads, 0, L.stream>>>(L.bcount, nb, L.k, L.bstart, L.cursor, dual ? nullptr : L.count);
  if ((e = cudaFuncSetAttribute(k_bucket_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(scatter_smem(kScatterSmem, true)))) != cudaSuccess)
    return e;
  k_bucket_scatter<<<unsigned(cdiv(E, kScatterTile)), 256, scatter_smem(nb, L.w1 != nullptr), L.stream>>>(
      en, E, nb, L.cursor, L.idx, L.w1 ? L.widx : nullptr);
  // reference points: the first row of each cluster's bucket (buckets k + c
  // of the dual form share cluster c's)
  {
    const int dz = int(round_up(L.d, 4));
    switch (L.dtype) {
      case SIL_F32:
        k_shift_build<SIL_F32><<<L.k, 128, 0, L.stream>>>(L.X, L.d, L.ldx, L.cs, L.idx, L.bstart, L.dist, L.rs, dz);
        break;
      case SIL_BF16:
        k_shift_build<SIL_BF16><<<L.k, 128, 0, L.stream>>>(L.X, L.d, L.ldx, L.cs, L.idx, L.bstart, L.dist, L.rs, dz);
        break;
      default:
        k_shift_build<SIL_FP8_E4M3><<<L.k, 128, 0, L.stream>>>(L.X, L.d, L.ldx, L.cs, L.idx, L.bstart, L.dist, L.rs,
                                                                dz);
        break;
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // 4: gather-reduce over the sorted order
  const int esz = elem_bytes(L.dtype);
  const int q = 16 / esz;
  GatherK g{};
  g.X = static_cast<const unsigned char*>(L.X);
  g.n = L.n;
  g.d = L.d;
  g.ldx_bytes = L.ldx * esz;
  g.cs = L.cs;
  g.k = L.k;
  g.nb = nb;
  g.dz = int(round_up(L.d, 4));
  g.idx = L.idx;
  g.widx = L.w1 ? L.widx : nullptr;
  g.bstart = L.bstart;
  g.rs = L.rs;
  g.invnorm = L.invnorm;
  g.cosine = L.dist == SIL_COSINE;
  g.vec = (reinterpret_cast<uintptr_t>(L.X) % 16 == 0) && (g.ldx_bytes % 16 == 0);
  g.nch = int(cdiv(L.d, q));
  // TMA row gather when a whole row is one box of at most 512 bytes (rows
  // padded to 32 bytes keep every 4-row destination 128-byte aligned), except
  // for FP8 rows: their register-load kernel measured faster (1e7-row FP8
  // D = 128 pass 1: 0.94 vs 1.18 ms; BF16 and FP32 rows the other way round);
  // SIL_AGG_LDG=1 in the environment keeps the register-load kernel
  const char* force_ldg = getenv("SIL_AGG_LDG");
  const int dbox = int(round_up(L.d, 32 / esz));
  const int rb = dbox * esz;
  const bool tma = !(force_ldg && force_ldg[0] == '1') && L.dtype != SIL_FP8_E4M3 && g.vec && dbox <= 256 &&
                   rb <= 512;
  // up to 16 elements per lane, as few lanes per row as that allows; rows
  // read from shared memory take at least 8 lanes (128 contiguous bytes per
  // 8-lane phase: no bank conflicts)
  const int mc = max_cpl(L.dtype);
  int G = 1;
  if (tma)
    while (G < 8 && G < g.nch) G <<= 1;
  while (G < 32 && G * mc < g.nch) G <<= 1;
  int cpl = int(std::min<int64_t>(mc, cdiv(g.nch, G)));
  if (cpl == 3) cpl = 4;
  g.G = G;
  g.lgG = 0;
  while ((1 << g.lgG) < G) ++g.lgG;
  g.ch_slice = G * cpl;
  const int slices = int(cdiv(g.nch, g.ch_slice));
  if (slices > 1 && g.cosine && L.invnorm == nullptr) return cudaErrorInvalidValue;
  g.s1 = L.s1;
  g.s2 = L.s2;
  g.wsum = L.wsum;
  g.status = L.status;
  if (tma && slices == 1) {
    CUtensorMap map;
    const CUtensorMapDataType tt = L.dtype == SIL_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : L.dtype == SIL_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    if (encode_tmap_2d(&map, L.X, tt, esz, uint64_t(L.d), uint64_t(L.n), uint64_t(g.ldx_bytes), uint32_t(dbox), 1,
                       CU_TENSOR_MAP_SWIZZLE_NONE)) {
      // the consumer warps pace this kernel (at_scale: 8 warps x 3 stages
      // 0.76 ms, 12 x 2 0.63 ms, 14 x 2 0.61 ms, 4 x 6 1.20 ms): as many warps
      // as the shared memory holds with two 32-row blocks each, up to 14,
      // then as many stages as fit
      const int sb = 32 * rb;
      const int budget = 227 * 1024 - 1024 - 512;
      const int warps = std::max(1, std::min(kGatherTmaWarps, budget / (2 * sb)));
      const int stages = std::max(2, std::min(8, budget / (warps * sb)));
      g.rb = rb;
      g.stages = stages;
      const int smem = warps * stages * sb + warps * stages * 8 + 1024;
      switch (L.dtype) {
        case SIL_F32:
          return cpl == 1   ? launch_gather_tma_mode<SIL_F32, 1>(g, map, E, warps, smem, L.stream)
                 : cpl == 2 ? launch_gather_tma_mode<SIL_F32, 2>(g, map, E, warps, smem, L.stream)
                            : launch_gather_tma_mode<SIL_F32, 4>(g, map, E, warps, smem, L.stream);
        case SIL_BF16:
          return cpl == 1 ? launch_gather_tma_mode<SIL_BF16, 1>(g, map, E, warps, smem, L.stream)
                          : launch_gather_tma_mode<SIL_BF16, 2>(g, map, E, warps, smem, L.stream);
        default:
          return launch_gather_tma_mode<SIL_FP8_E4M3, 1>(g, map, E, warps, smem, L.stream);
      }
    }
  }
  switch (L.dtype) {
    case SIL_F32:
      return cpl == 1   ? launch_gather_mode<SIL_F32, 1>(g, E, slices, L.stream)
             : cpl == 2 ? launch_gather_mode<SIL_F32, 2>(g, E, slices, L.stream)
                        : launch_gather_mode<SIL_F32, 4>(g, E, slices, L.stream);
    case SIL_BF16:
      return cpl == 1 ? launch_gather_mode<SIL_BF16, 1>(g, E, slices, L.stream)
                      : launch_gather_mode<SIL_BF16, 2>(g, E, slices, L.stream);
    default:
      return launch_gather_mode<SIL_FP8_E4M3, 1>(g, E, slices, L.stream);
  }
}

}  // namespace sil
