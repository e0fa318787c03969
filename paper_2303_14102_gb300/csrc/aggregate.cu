// Pass 1: the segmented per-cluster reduction (Sec. III-A Eq. 5-9 with the
// footnote that Y and Psi come from one joint pass; Sec. III-B Eq. 15-16).
//
// Design (GB300): the reduction is HBM-bound -- one read of X and labels --
// so the kernel is SIMT, with no tensor-core reshaping.  A CTA owns a
// contiguous row range and a column slice (and, for very many clusters, a
// bucket slice).  Rows are staged in shared memory one tile of 128 rows at a
// time -- by TMA (cp.async.bulk.tensor) into a ring of stages that runs ahead
// of the computation, or, when the layout does not allow a tensor map, by
// synchronous coalesced 128-bit loads; the tile's labels are counting-sorted in
// shared memory (integer shared atomics only) so that every (cluster, 4-column
// chunk) pair present in the tile is summed by ONE thread in registers and
// added once into a per-CTA FP32 accumulator in shared memory -- no float
// atomics, no warp-divergent scatter.  Values are accumulated shifted by a
// per-cluster reference point r_k (a point of that cluster), which keeps the
// FP32 partials well conditioned even when clusters sit far from the origin;
// the partials are un-shifted and folded into the FP64 outputs once per CTA:
//   s1 += sum(x - r) + m r,   s2 += sum||x - r||^2 + 2 r.sum(x - r) + m ||r||^2.
// The same kernel, with per-row weights and two bucket entries per row, forms
// the segmented sums of the backward pass.
#include <climits>
#include <cstdlib>

#include "sil_internal.cuh"
#include "tma.cuh"

namespace sil {

namespace {

__global__ void k_rep_init(int32_t* rep, int32_t k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) rep[i] = INT_MAX;
}

__global__ void k_rep_find(const int32_t* labels, int64_t m, int32_t k, int32_t* rep) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < m) {
    int32_t l = labels[i];
    if (l >= 0 && l < k) atomicMin(&rep[l], int32_t(i));
  }
}

// One CTA per cluster: rs[k][c] = x_rep (normalised for cosine), 0 when the
// cluster has no point among the rows searched.
template <int DT>
__global__ void k_shift_build(const void* X, int32_t d, int64_t ldx, const float* cs,
                              const int32_t* rep, int32_t dist, float* rs, int32_t dz) {
  __shared__ float red[32];
  const int kk = blockIdx.x;
  const int32_t r = rep[kk];
  float* out = rs + int64_t(kk) * dz;
  if (r == INT_MAX) {
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

struct AggK {
  const void* X;
  int64_t n;
  int32_t d;
  int64_t ldx;
  const float* cs;
  const int32_t* lab1;
  const int32_t* lab2;
  const float* w1;
  const float* w2;
  int32_t k;
  int32_t kb;  // total buckets: k, or 2k in dual mode
  int32_t cosine;
  int32_t vec;
  const float* rs;
  int32_t dz;
  const float* invnorm;
  int32_t dsp;    // columns per slice (multiple of 4)
  int32_t nslc;   // column slices
  int32_t kbs;    // buckets per bucket slice
  int64_t rows_per_cta;
  int32_t stages;      // TMA kernel: pipeline depth
  int32_t stage_bytes; // TMA kernel: bytes of one stage
  unsigned long long* count;
  double* s1;
  double* s2;
  double* wsum;
  uint32_t* status;
};

// Tensor maps of the TMA-fed kernel (X tile, labels, second labels, weights).
struct AggMaps {
  CUtensorMap x, lab1, lab2, w1, w2;
};

// Byte offsets of the per-CTA shared state (the part both kernels share).
struct AggSmem {
  int acc, acc2, macc, mint, cnt, slot, ebk, epos, ew, order, nel, bstart, bsize, segq, inv, wtot, nne,
      total;
};

constexpr int kSeg = 8;  // rows per accumulation segment

__host__ __device__ inline AggSmem agg_smem(int dsp, int kbs, bool dual, bool weighted) {
  const int R = kAggRows, E = dual ? 2 * R : R, c4 = dsp / 4;
  AggSmem s;
  int o = 0;
  s.acc = o; o += kbs * dsp * 4;
  s.acc2 = o; o += weighted ? 0 : kbs * c4 * 4;
  s.macc = o; o += kbs * 4;
  s.mint = o; o += kbs * 4;
  s.cnt = o; o += kbs * 4;
  s.slot = o; o += kbs * 4;
  s.ebk = o; o += E * 4;
  s.epos = o; o += E * 4;
  s.ew = o; o += E * 4;
  s.order = o; o += E * 4;
  s.nel = o; o += E * 4;
  s.bstart = o; o += (E + 1) * 4;
  s.bsize = o; o += E * 4;
  s.segq = o; o += (E + E / kSeg + 1) * 4;
  s.inv = o; o += R * 4;
  s.wtot = o; o += 32 * 4;
  s.nne = o; o += 16;
  s.total = (o + 127) & ~127;
  return s;
}

struct AggState {
  float* acc;
  float4* acc4;
  float* acc2;
  float* macc;
  int* mint;
  int* cnt;
  int* slot;
  int* ebk;
  int* epos;
  float* ew;
  int* order;
  int* nel;
  int* bstart;
  int* bsize;
  int* segq;  // segment -> (bucket position << 8 | segment index)
  float* inv;
  int* wtot;
  int* nne;  // [0] = non-empty bucket count (being built), [1] = abort flag, [2] = count of this tile
};

__device__ inline AggState agg_state(unsigned char* smem, const AggSmem& L) {
  AggState S;
  S.acc = reinterpret_cast<float*>(smem + L.acc);
  S.acc4 = reinterpret_cast<float4*>(smem + L.acc);
  S.acc2 = reinterpret_cast<float*>(smem + L.acc2);
  S.macc = reinterpret_cast<float*>(smem + L.macc);
  S.mint = reinterpret_cast<int*>(smem + L.mint);
  S.cnt = reinterpret_cast<int*>(smem + L.cnt);
  S.slot = reinterpret_cast<int*>(smem + L.slot);
  S.ebk = reinterpret_cast<int*>(smem + L.ebk);
  S.epos = reinterpret_cast<int*>(smem + L.epos);
  S.ew = reinterpret_cast<float*>(smem + L.ew);
  S.order = reinterpret_cast<int*>(smem + L.order);
  S.nel = reinterpret_cast<int*>(smem + L.nel);
  S.bstart = reinterpret_cast<int*>(smem + L.bstart);
  S.bsize = reinterpret_cast<int*>(smem + L.bsize);
  S.segq = reinterpret_cast<int*>(smem + L.segq);
  S.inv = reinterpret_cast<float*>(smem + L.inv);
  S.wtot = reinterpret_cast<int*>(smem + L.wtot);
  S.nne = reinterpret_cast<int*>(smem + L.nne);
  return S;
}

// Geometry of one CTA's work item.
struct AggItem {
  int cslice, col0, dlim, c4, c4e, kb0, kbn;
  int64_t row_begin, row_end;
};

__device__ inline AggItem agg_item(const AggK& a) {
  AggItem it;
  it.cslice = blockIdx.x % a.nslc;
  const int kslice = blockIdx.x / a.nslc;
  it.col0 = it.cslice * a.dsp;
  it.dlim = min(a.d, it.col0 + a.dsp);  // columns of this slice are [col0, dlim)
  it.c4 = a.dsp / 4;
  it.c4e = int(cdiv(it.dlim - it.col0, 4));  // chunks holding columns < dlim
  it.kb0 = kslice * a.kbs;
  it.kbn = min(a.kbs, a.kb - it.kb0);  // buckets of this slice
  it.row_begin = int64_t(blockIdx.y) * a.rows_per_cta;
  it.row_end = min(a.n, it.row_begin + a.rows_per_cta);
  return it;
}

__device__ inline void agg_zero(const AggState& S, const AggItem& it, int dsp, bool weighted) {
  const int tid = threadIdx.x, T = blockDim.x;
  for (int i = tid; i < it.kbn * dsp; i += T) S.acc[i] = 0.f;
  if (!weighted)
    for (int i = tid; i < it.kbn * it.c4; i += T) S.acc2[i] = 0.f;
  for (int i = tid; i < it.kbn; i += T) {
    S.macc[i] = 0.f;
    S.mint[i] = 0;
    S.cnt[i] = 0;
  }
  if (tid == 0) {
    S.nne[0] = 0;
    S.nne[1] = 0;
  }
}

// Tile source of the generic kernel: FP32 rows already in shared memory,
// labels and weights read from global memory.
struct SrcGeneric {
  const float4* xs4;
  int c4;
  const int32_t* lab1;
  const int32_t* lab2;
  const float* w1;
  const float* w2;
  int64_t r0;
  __device__ float4 chunk(int r, int c) const { return xs4[r * c4 + c]; }
  __device__ int label1(int r) const { return lab1[r0 + r]; }
  __device__ int label2(int r) const { return lab2[r0 + r]; }
  __device__ float weight1(int r) const { return w1[r0 + r]; }
  __device__ float weight2(int r) const { return w2[r0 + r]; }
};

// Tile source of the TMA kernel: raw storage rows, labels and weights all in
// one pipeline stage of shared memory.
template <int DT>
struct SrcTma {
  using T = typename Elem<DT>::T;
  const T* xs;
  int dsp;
  const int32_t* lab1;
  const int32_t* lab2;
  const float* w1;
  const float* w2;
  const float* cs;
  int col0, dlim;
  __device__ float4 chunk(int r, int c) const {
    const T* p = xs + r * dsp + 4 * c;
    float4 v;
    if constexpr (DT == SIL_F32) {
      v = *reinterpret_cast<const float4*>(p);
    } else if constexpr (DT == SIL_BF16) {
      const uint2 u = *reinterpret_cast<const uint2*>(p);
      const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
      const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
      v = make_float4(a.x, a.y, b.x, b.y);
    } else {
      const uint32_t u = *reinterpret_cast<const uint32_t*>(p);
      const __nv_fp8_e4m3* q = reinterpret_cast<const __nv_fp8_e4m3*>(&u);
      v = make_float4(float(q[0]), float(q[1]), float(q[2]), float(q[3]));
      const int col = col0 + 4 * c;
      v.x *= col + 0 < dlim ? __ldg(cs + col + 0) : 0.f;
      v.y *= col + 1 < dlim ? __ldg(cs + col + 1) : 0.f;
      v.z *= col + 2 < dlim ? __ldg(cs + col + 2) : 0.f;
      v.w *= col + 3 < dlim ? __ldg(cs + col + 3) : 0.f;
    }
    return v;
  }
  __device__ int label1(int r) const { return lab1[r]; }
  __device__ int label2(int r) const { return lab2[r]; }
  __device__ float weight1(int r) const { return w1[r]; }
  __device__ float weight2(int r) const { return w2[r]; }
};

// One 128-row tile: bucket the rows by label (counting sort in shared memory),
// then one thread per (non-empty bucket, 4-column chunk) sums the bucket's
// rows in registers and adds the result once into the CTA accumulator.
// Counters are reset inside; the caller syncs before the next tile (and
// before its staging buffer is refilled).
template <bool DUAL, bool WEIGHTED, class Src>
__device__ int agg_sort(const AggK& a, const AggState& S, const AggItem& it, const Src& src,
                        int rows, int64_t r0) {
  constexpr int R = kAggRows, T = kAggThreads, E = DUAL ? 2 * R : R;
  const int tid = threadIdx.x;
  const bool in_cta_norm = a.cosine && a.invnorm == nullptr;  // full rows are in this tile
  // (b) bucket entries and row scales
  for (int e = tid; e < E; e += T) {
    const int r = e < R ? e : e - R;
    int lb = -1;
    float w = 1.f;
    if (r < rows) {
      const int lab = (e < R) ? src.label1(r) : src.label2(r);
      if (lab >= 0 && lab < a.k) {
        const int bucket = (e < R) ? lab : a.k + lab;
        if (bucket >= it.kb0 && bucket < it.kb0 + it.kbn) lb = bucket - it.kb0;
        if (WEIGHTED) w = (e < R) ? src.weight1(r) : src.weight2(r);
      } else if (e < R || lab != -1) {
        // a label outside [0, k); -1 marks "no neighbour" in the second entry
        set_status(a.status, SIL_ELABEL);
      }
    }
    // one shared atomic per distinct bucket per warp: lanes with the same
    // bucket rank themselves inside the warp and the lowest one reserves
    // positions for all of them
    const unsigned peers = __match_any_sync(0xffffffffu, lb);
    const int leader = __ffs(peers) - 1;
    const int lane = tid & 31;
    int p = 0;
    if (lb >= 0 && lane == leader) {
      p = atomicAdd(&S.cnt[lb], __popc(peers));
      if (p == 0) {
        const int q = atomicAdd(&S.nne[0], 1);
        S.nel[q] = lb;
        S.slot[lb] = q;
      }
    }
    p = __shfl_sync(0xffffffffu, p, leader);
    if (lb >= 0) S.epos[e] = p + __popc(peers & ((1u << lane) - 1u));
    S.ebk[e] = lb;
    S.ew[e] = w;
  }
  if (a.cosine) {
    if (in_cta_norm) {
      const int warp = tid >> 5, lane = tid & 31;
      for (int r = warp; r < R; r += T / 32) {
        float ss = 0.f;
        for (int c = lane; c < it.c4e; c += 32) {
          const float4 v = src.chunk(r, c);
          ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (lane == 0) {
          if (r < rows && !(ss > 0.f)) set_status(a.status, SIL_EZERONORM);
          S.inv[r] = ss > 0.f ? rsqrtf(ss) : 0.f;
        }
      }
    } else {
      for (int r = tid; r < R; r += T) S.inv[r] = r < rows ? a.invnorm[r0 + r] : 0.f;
    }
  }
  __syncthreads();
  // (c) block-wide exclusive scan over the non-empty buckets (one thread per
  // bucket, m <= E <= T), of the packed pair (rows << 16 | segments of kSeg
  // rows); it also writes the segment -> bucket table and resets the counters
  const int m = S.nne[0];
  {
    const int warp = tid >> 5, lane = tid & 31;
    const int c = tid < m ? S.cnt[S.nel[tid]] : 0;
    const int v = (c << 16) | ((c + kSeg - 1) / kSeg);
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) S.wtot[warp] = incl;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += S.wtot[w];
    const int ex = off + incl - v;
    if (tid < m) {
      const int lb = S.nel[tid];
      S.bstart[tid] = ex >> 16;
      S.bsize[tid] = c;
      S.cnt[lb] = 0;
      const int s0 = ex & 0xFFFF, ns = v & 0xFFFF;
      for (int sg = 0; sg < ns; ++sg) S.segq[s0 + sg] = (tid << 8) | sg;
    }
    if (tid == T - 1) S.nne[2] = (off + incl) & 0xFFFF;  // total number of segments
  }
  __syncthreads();
  if (tid == 0) S.nne[0] = 0;  // everybody has read m
  // (d) scatter entries into bucket order
  for (int e = tid; e < E; e += T) {
    const int lb = S.ebk[e];
    if (lb >= 0) S.order[S.bstart[S.slot[lb]] + S.epos[e]] = e;
  }
  __syncthreads();
  return S.nne[2];  // segments of at most kSeg rows over the non-empty buckets
}

// Accumulation into the per-CTA shared accumulators: one thread per
// (non-empty bucket, 4-column chunk of this slice).
template <bool DUAL, bool WEIGHTED, class Src>
__device__ void agg_tile(const AggK& a, const AggState& S, const AggItem& it, const Src& src,
                         int rows, int64_t r0) {
  constexpr int R = kAggRows, T = kAggThreads;
  const int tid = threadIdx.x;
  const int nseg = agg_sort<DUAL, WEIGHTED>(a, S, it, src, rows, r0);
  // one thread per (segment of at most kSeg rows of one bucket, 4-column
  // chunk): short independent chains; the segments of a bucket longer than
  // kSeg rows meet in shared memory through float atomics
  for (int p = tid; p < nseg * it.c4e; p += T) {
    const int sidx = p / it.c4e, c = p - sidx * it.c4e;
    const int sq_ = S.segq[sidx];
    const int q = sq_ >> 8, sg = sq_ & 255;
    const int lb = S.nel[q];
    const int bg = it.kb0 + lb;
    const int kc = bg < a.k ? bg : bg - a.k;  // cluster whose reference point shifts this bucket
    const float4 rr =
        *reinterpret_cast<const float4*>(a.rs + int64_t(kc) * a.dz + it.col0 + 4 * c);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    float sq = 0.f, wsum = 0.f;
    const int size = S.bsize[q];
    const int jb = S.bstart[q] + sg * kSeg;
    const int je = min(S.bstart[q] + size, jb + kSeg);
    int eidx[kSeg];
#pragma unroll
    for (int u = 0; u < kSeg; ++u) eidx[u] = S.order[min(jb + u, je - 1)];
#pragma unroll
    for (int u = 0; u < kSeg; ++u) {
      if (jb + u >= je) break;
      const int e = eidx[u];
      const int r = DUAL ? (e < R ? e : e - R) : e;
      const float4 x = src.chunk(r, c);
      const float sc = a.cosine ? S.inv[r] : 1.f;
      float4 v;
      v.x = fmaf(sc, x.x, -rr.x);
      v.y = fmaf(sc, x.y, -rr.y);
      v.z = fmaf(sc, x.z, -rr.z);
      v.w = fmaf(sc, x.w, -rr.w);
      if (WEIGHTED) {
        const float w = S.ew[e];
        v.x *= w; v.y *= w; v.z *= w; v.w *= w;
        wsum += w;
      } else {
        sq = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, sq))));
      }
      s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
    }
    float* accp = S.acc + (lb * it.c4 + c) * 4;
    if (size <= kSeg) {  // the only segment of its bucket: plain read-modify-write
      float4 t = S.acc4[lb * it.c4 + c];
      t.x += s.x; t.y += s.y; t.z += s.z; t.w += s.w;
      S.acc4[lb * it.c4 + c] = t;
      if (!WEIGHTED) S.acc2[lb * it.c4 + c] += sq;
      if (c == 0) {
        S.mint[lb] += size;
        if (WEIGHTED) S.macc[lb] += wsum;
      }
    } else {
      atomicAdd(accp + 0, s.x);
      atomicAdd(accp + 1, s.y);
      atomicAdd(accp + 2, s.z);
      atomicAdd(accp + 3, s.w);
      if (!WEIGHTED) atomicAdd(S.acc2 + lb * it.c4 + c, sq);
      if (c == 0) {
        if (sg == 0) S.mint[lb] += size;
        if (WEIGHTED) atomicAdd(S.macc + lb, wsum);
      }
    }
  }
}

// Un-shift in FP64 and add the CTA's sums into the outputs.
template <bool WEIGHTED>
__device__ void agg_flush(const AggK& a, const AggState& S, const AggItem& it) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int dsl = it.dlim - it.col0;
  for (int i = tid; i < it.kbn * dsl; i += T) {
    const int lb = i / dsl, col = i - lb * dsl;
    const int mm = S.mint[lb];
    if (mm == 0) continue;
    const int kg = it.kb0 + lb;
    double v = double(S.acc[lb * a.dsp + col]);
    if (!WEIGHTED) v += double(mm) * double(a.rs[int64_t(kg) * a.dz + it.col0 + col]);
    atomicAdd(a.s1 + int64_t(kg) * a.d + it.col0 + col, v);
  }
  for (int lb = tid; lb < it.kbn; lb += T) {
    const int mm = S.mint[lb];
    if (mm == 0) continue;
    const int kg = it.kb0 + lb;
    if (WEIGHTED) {
      if (it.cslice == 0) atomicAdd(a.wsum + kg, double(S.macc[lb]));
    } else {
      double t = 0.0;
      for (int c = 0; c < it.c4e; ++c) t += double(S.acc2[lb * it.c4 + c]);
      for (int col = 0; col < dsl; ++col) {
        const double r = a.rs[int64_t(kg) * a.dz + it.col0 + col];
        t += 2.0 * r * double(S.acc[lb * a.dsp + col]) + double(mm) * r * r;
      }
      atomicAdd(a.s2 + kg, t);
      if (it.cslice == 0) atomicAdd(a.count + kg, (unsigned long long)mm);
    }
  }
}

// Generic pass 1: synchronous coalesced loads (any alignment, any ldx).
template <int DT, bool DUAL, bool WEIGHTED>
__global__ void __launch_bounds__(kAggThreads) k_aggregate(AggK a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int R = kAggRows, T = kAggThreads;
  const int tid = threadIdx.x;
  const AggSmem L = agg_smem(a.dsp, a.kbs, DUAL, WEIGHTED);
  const AggState S = agg_state(smem, L);
  float4* xs4 = reinterpret_cast<float4*>(smem + L.total);  // [R][dsp] FP32 tile
  const AggItem it = agg_item(a);
  agg_zero(S, it, a.dsp, WEIGHTED);
  __syncthreads();
  for (int64_t r0 = it.row_begin; r0 < it.row_end; r0 += R) {
    const int rows = int((it.row_end - r0) < int64_t(R) ? (it.row_end - r0) : int64_t(R));
    for (int q = tid; q < R * it.c4; q += T) {
      const int r = q / it.c4, c = q - r * it.c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) v = load4<DT>(a.X, r0 + r, it.col0 + 4 * c, it.dlim, a.ldx, a.cs, a.vec);
      xs4[q] = v;
    }
    __syncthreads();
    const SrcGeneric src{xs4, it.c4, a.lab1, a.lab2, a.w1, a.w2, r0};
    agg_tile<DUAL, WEIGHTED>(a, S, it, src, rows, r0);
    __syncthreads();
  }
  agg_flush<WEIGHTED>(a, S, it);
}

// TMA-fed pass 1: a ring of `stages` shared-memory buffers filled by
// cp.async.bulk.tensor (X tile, labels, weights) while earlier tiles are
// processed.  Thread 0 refills a buffer as soon as every thread is done with
// it.  Waits are bounded: on a timeout the CTA flags SIL_ETIMEOUT, waits
// (bounded) for its own copies in flight and returns without flushing.
template <int DT, bool DUAL, bool WEIGHTED>
__global__ void __launch_bounds__(kAggThreads) k_aggregate_tma(AggK a, const __grid_constant__ AggMaps maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  using T = typename Elem<DT>::T;
  constexpr int R = kAggRows;
  constexpr int esz = sizeof(T);
  const int tid = threadIdx.x;
  const AggSmem L = agg_smem(a.dsp, a.kbs, DUAL, WEIGHTED);
  const AggState S = agg_state(smem, L);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.total);
  unsigned char* stage0 = smem + L.total + 128;  // stage buffers, 128-byte aligned
  const AggItem it = agg_item(a);
  const int64_t nrows = it.row_end > it.row_begin ? it.row_end - it.row_begin : 0;
  const int ntiles = int(cdiv(nrows, R));
  const int xbytes = R * a.dsp * esz;
  const int nvec = 1 + (DUAL ? 1 : 0) + (WEIGHTED ? (DUAL ? 2 : 1) : 0);
  const uint32_t tx = uint32_t(xbytes + nvec * R * 4);

  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  agg_zero(S, it, a.dsp, WEIGHTED);
  __syncthreads();

  auto issue = [&](int t) {
    const int s = t % a.stages;
    unsigned char* buf = stage0 + s * a.stage_bytes;
    const int32_t row = int32_t(it.row_begin + int64_t(t) * R);
    mbar_arrive_expect_tx(&bars[s], tx);
    tma_load_2d(buf, &maps.x, it.col0, row, &bars[s]);
    unsigned char* v = buf + xbytes;
    tma_load_1d(v, &maps.lab1, row, &bars[s]);
    v += R * 4;
    if (DUAL) {
      tma_load_1d(v, &maps.lab2, row, &bars[s]);
      v += R * 4;
    }
    if (WEIGHTED) {
      tma_load_1d(v, &maps.w1, row, &bars[s]);
      v += R * 4;
      if (DUAL) tma_load_1d(v, &maps.w2, row, &bars[s]);
    }
  };
  if (tid == 0) {
    fence_proxy_async_smem();
    for (int t = 0; t < ntiles && t < a.stages; ++t) issue(t);
  }

  int t = 0;
  bool aborted = false;
  for (; t < ntiles; ++t) {
    const int s = t % a.stages;
    if (!mbar_wait(&bars[s], uint32_t((t / a.stages) & 1))) {
      // This thread gave up.  It still runs the tile (on whatever the buffer
      // holds; every index stays in bounds) so that all threads meet the same
      // barriers, and the whole CTA stops uniformly after the tile.
      S.nne[1] = 1;
      set_status(a.status, SIL_ETIMEOUT);
    }
    const int64_t r0 = it.row_begin + int64_t(t) * R;
    const int rows = int((it.row_end - r0) < int64_t(R) ? (it.row_end - r0) : int64_t(R));
    const unsigned char* buf = stage0 + s * a.stage_bytes;
    const int32_t* v = reinterpret_cast<const int32_t*>(buf + xbytes);
    SrcTma<DT> src;
    src.xs = reinterpret_cast<const T*>(buf);
    src.dsp = a.dsp;
    src.lab1 = v;
    src.lab2 = DUAL ? v + R : nullptr;
    src.w1 = WEIGHTED ? reinterpret_cast<const float*>(v + (DUAL ? 2 : 1) * R) : nullptr;
    src.w2 = (WEIGHTED && DUAL) ? reinterpret_cast<const float*>(v + 3 * R) : nullptr;
    src.cs = a.cs;
    src.col0 = it.col0;
    src.dlim = it.dlim;
    agg_tile<DUAL, WEIGHTED>(a, S, it, src, rows, r0);
    __syncthreads();
    if (S.nne[1]) {  // a thread timed out on this tile's barrier
      aborted = true;
      ++t;
      break;
    }
    if (tid == 0 && t + a.stages < ntiles) {
      fence_proxy_async_smem();
      issue(t + a.stages);
    }
  }
  if (aborted) {
    // every thread stops; thread 0 waits (bounded) for this CTA's copies in flight
    __syncthreads();
    if (tid == 0) {
      // tiles t-1 .. t-2+stages were issued and not consumed: one per stage
      const int first = t - 1;
      const int end = ntiles < first + a.stages ? ntiles : first + a.stages;
      for (int u = first; u < end; ++u) mbar_wait(&bars[u % a.stages], uint32_t((u / a.stages) & 1));
    }
    __syncthreads();
    return;
  }
  agg_flush<WEIGHTED>(a, S, it);
}

// Column slices of at least 32 columns keep each row read a whole number of
// 32-byte DRAM sectors (bf16/fp32); a CTA may use up to 200 KB to get there.
void agg_plan(int32_t d, int32_t kb, bool dual, bool weighted, int* dsp_out, int* kbs_out) {
  const int dz = int(round_up(d, 4));
  const int dmax = dz < 256 ? dz : 256;  // the accumulation phase covers at most 64 chunks
  const int budgets[2] = {kSmemBudget, 200 * 1024};
  const int min_dsp = dz < 32 ? dz : 32;
  auto total = [&](int dsp, int kbs) {  // generic kernel: shared state + one FP32 tile
    return agg_smem(dsp, kbs, dual, weighted).total + kAggRows * dsp * 4;
  };
  for (int budget : budgets) {
    int dsp = dmax;
    while (dsp > min_dsp && total(dsp, kb) > budget) dsp = std::max(min_dsp, int(round_up(dsp / 2, 4)));
    if (total(dsp, kb) <= budget) {
      *dsp_out = dsp;
      *kbs_out = kb;
      return;
    }
  }
  // very many buckets: narrowest slice, then split the buckets
  int dsp = min_dsp;
  int kbs = kb;
  while (kbs > 1 && total(dsp, kbs) > 200 * 1024) kbs = (kbs + 1) / 2;
  *dsp_out = dsp;
  *kbs_out = kbs;
}

bool vec_ok(const void* X, int32_t dtype, int64_t ldx) {
  const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
  return (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
}

inline bool aligned16(const void* p) { return p == nullptr || reinterpret_cast<uintptr_t>(p) % 16 == 0; }

}  // namespace

bool agg_needs_invnorm(int32_t d, int32_t k, bool dual) {
  int dsp, kbs;
  agg_plan(d, dual ? 2 * k : k, dual, dual, &dsp, &kbs);
  return dsp < round_up(d, 4);
}

cudaError_t launch_shift(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                         const float* cs, const int32_t* labels, int32_t k, int32_t dist,
                         int32_t* rep, float* rs, cudaStream_t stream) {
  const int dz = int(round_up(d, 4));
  k_rep_init<<<unsigned(cdiv(k, 256)), 256, 0, stream>>>(rep, k);
  const int64_t m = n < kRepRows ? n : kRepRows;
  if (m > 0) k_rep_find<<<unsigned(cdiv(m, 256)), 256, 0, stream>>>(labels, m, k, rep);
  const int th = 128;
  switch (dtype) {
    case SIL_F32: k_shift_build<SIL_F32><<<k, th, 0, stream>>>(X, d, ldx, cs, rep, dist, rs, dz); break;
    case SIL_BF16: k_shift_build<SIL_BF16><<<k, th, 0, stream>>>(X, d, ldx, cs, rep, dist, rs, dz); break;
    default: k_shift_build<SIL_FP8_E4M3><<<k, th, 0, stream>>>(X, d, ldx, cs, rep, dist, rs, dz); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_invnorm(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                           const float* cs, float* invnorm, uint32_t* status, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  const bool vec = vec_ok(X, dtype, ldx);
  const unsigned grid = unsigned(std::min<int64_t>(cdiv(n, 8), int64_t(kNumSMs) * 16));
  switch (dtype) {
    case SIL_F32: k_invnorm<SIL_F32><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
    case SIL_BF16: k_invnorm<SIL_BF16><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
    default: k_invnorm<SIL_FP8_E4M3><<<grid, 256, 0, stream>>>(X, n, d, ldx, cs, vec, invnorm, status); break;
  }
  return cudaGetLastError();
}

namespace {

template <int DT, bool DUAL, bool WEIGHTED>
cudaError_t launch_generic_t(const AggK& k, dim3 grid, int smem, cudaStream_t stream) {
  auto fn = k_aggregate<DT, DUAL, WEIGHTED>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kAggThreads, smem, stream>>>(k);
  return cudaGetLastError();
}

template <int DT, bool DUAL, bool WEIGHTED>
cudaError_t launch_tma_t(const AggK& k, const AggMaps& maps, dim3 grid, int smem, cudaStream_t stream) {
  auto fn = k_aggregate_tma<DT, DUAL, WEIGHTED>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kAggThreads, smem, stream>>>(k, maps);
  return cudaGetLastError();
}

template <bool DUAL, bool WEIGHTED>
cudaError_t dispatch(int dtype, bool tma, const AggK& k, const AggMaps& maps, dim3 grid, int smem,
                     cudaStream_t st) {
  switch (dtype) {
    case SIL_F32:
      return tma ? launch_tma_t<SIL_F32, DUAL, WEIGHTED>(k, maps, grid, smem, st)
                 : launch_generic_t<SIL_F32, DUAL, WEIGHTED>(k, grid, smem, st);
    case SIL_BF16:
      return tma ? launch_tma_t<SIL_BF16, DUAL, WEIGHTED>(k, maps, grid, smem, st)
                 : launch_generic_t<SIL_BF16, DUAL, WEIGHTED>(k, grid, smem, st);
    default:
      return tma ? launch_tma_t<SIL_FP8_E4M3, DUAL, WEIGHTED>(k, maps, grid, smem, st)
                 : launch_generic_t<SIL_FP8_E4M3, DUAL, WEIGHTED>(k, grid, smem, st);
  }
}

// Tensor maps for the TMA kernel; false when the layout does not allow them.
bool make_maps(const AggLaunch& L, const AggK& k, AggMaps* maps) {
  const int esz = L.dtype == SIL_F32 ? 4 : L.dtype == SIL_BF16 ? 2 : 1;
  const CUtensorMapDataType xt = L.dtype == SIL_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : L.dtype == SIL_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  if ((k.dsp * esz) % 16 != 0 || k.dsp > 256 || k.dsp > L.d) return false;
  if (!aligned16(L.labels) || !aligned16(L.labels2) || !aligned16(L.w1) || !aligned16(L.w2)) return false;
  if (!encode_tmap_2d(&maps->x, L.X, xt, esz, uint64_t(L.d), uint64_t(L.n), uint64_t(L.ldx) * esz,
                      uint32_t(k.dsp), uint32_t(kAggRows), CU_TENSOR_MAP_SWIZZLE_NONE))
    return false;
  if (!encode_tmap_1d(&maps->lab1, L.labels, CU_TENSOR_MAP_DATA_TYPE_INT32, uint64_t(L.n), kAggRows))
    return false;
  maps->lab2 = maps->lab1;
  maps->w1 = maps->lab1;
  maps->w2 = maps->lab1;
  if (L.labels2 &&
      !encode_tmap_1d(&maps->lab2, L.labels2, CU_TENSOR_MAP_DATA_TYPE_INT32, uint64_t(L.n), kAggRows))
    return false;
  if (L.w1 && !encode_tmap_1d(&maps->w1, L.w1, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, uint64_t(L.n), kAggRows))
    return false;
  if (L.w2 && !encode_tmap_1d(&maps->w2, L.w2, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, uint64_t(L.n), kAggRows))
    return false;
  return true;
}

}  // namespace

// Selects the TMA kernel when the layout allows (set SIL_AGG_GENERIC=1 in the
// environment to force the generic kernel).
cudaError_t launch_aggregate(const AggLaunch& L) {
  if (L.n == 0) return cudaSuccess;
  const bool dual = L.labels2 != nullptr;
  const bool weighted = L.w1 != nullptr;
  AggK k{};
  k.X = L.X;
  k.n = L.n;
  k.d = L.d;
  k.ldx = L.ldx;
  k.cs = L.cs;
  k.lab1 = L.labels;
  k.lab2 = L.labels2;
  k.w1 = L.w1;
  k.w2 = L.w2;
  k.k = L.k;
  k.kb = dual ? 2 * L.k : L.k;
  k.cosine = L.dist == SIL_COSINE;
  k.vec = vec_ok(L.X, L.dtype, L.ldx);
  k.rs = L.rs;
  k.dz = int(round_up(L.d, 4));
  k.invnorm = L.invnorm;
  int dsp, kbs;
  agg_plan(L.d, k.kb, dual, weighted, &dsp, &kbs);
  const int esz = L.dtype == SIL_F32 ? 4 : L.dtype == SIL_BF16 ? 2 : 1;
  const int box_mult = 16 / esz;  // TMA box rows must be whole 16-byte units
  if (dsp % box_mult != 0 && round_up(dsp, box_mult) <= 256) dsp = int(round_up(dsp, box_mult));
  k.dsp = dsp;
  k.kbs = kbs;
  k.nslc = int(cdiv(L.d, dsp));
  const int nkslc = int(cdiv(k.kb, kbs));
  if (k.cosine && k.nslc > 1 && L.invnorm == nullptr) return cudaErrorInvalidValue;
  k.count = L.count;
  k.s1 = L.s1;
  k.s2 = L.s2;
  k.wsum = L.wsum;
  k.status = L.status;

  const int fixed = agg_smem(dsp, kbs, dual, weighted).total;
  const int nvec = 1 + (dual ? 1 : 0) + (weighted ? (dual ? 2 : 1) : 0);
  const int stage = int(round_up(kAggRows * dsp * esz + nvec * kAggRows * 4, 128));
  const char* force_generic = getenv("SIL_AGG_GENERIC");
  AggMaps maps{};
  bool tma = !(force_generic && force_generic[0] == '1') && L.n < (int64_t(1) << 31);
  int stages = 0, smem = 0;
  if (tma) {
    // two CTAs per SM when two stages fit twice, else one CTA with up to four stages
    const int two_cta = (220 * 1024) / 2;
    if (fixed + 128 + 2 * stage <= two_cta) {
      stages = std::min(4, (two_cta - fixed - 128) / stage);
    } else {
      stages = std::min(4, (220 * 1024 - fixed - 128) / stage);
    }
    tma = stages >= 2 && make_maps(L, k, &maps);
    smem = fixed + 128 + stages * stage;
  }
  if (!tma) smem = fixed + kAggRows * dsp * 4;
  k.stages = stages;
  k.stage_bytes = stage;
  const int per_sm = std::max(1, std::min(4, (220 * 1024) / std::max(smem, 1)));
  const int64_t tiles = cdiv(L.n, kAggRows);
  const int64_t slices = int64_t(k.nslc) * nkslc;
  int64_t row_blocks = std::max<int64_t>(1, (int64_t(kNumSMs) * per_sm * (tma ? 1 : 2)) / slices);
  row_blocks = std::min<int64_t>(row_blocks, tiles);
  row_blocks = std::min<int64_t>(row_blocks, 65535);
  k.rows_per_cta = cdiv(tiles, row_blocks) * kAggRows;
  row_blocks = cdiv(L.n, k.rows_per_cta);
  const dim3 grid(static_cast<unsigned>(slices), static_cast<unsigned>(row_blocks));
  if (dual) return dispatch<true, true>(L.dtype, tma, k, maps, grid, smem, L.stream);
  if (weighted) return dispatch<false, true>(L.dtype, tma, k, maps, grid, smem, L.stream);
  return dispatch<false, false>(L.dtype, tma, k, maps, grid, smem, L.stream);
}

}  // namespace sil
