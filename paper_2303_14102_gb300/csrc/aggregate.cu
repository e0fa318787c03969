// Pass 1: the segmented per-cluster reduction (Sec. III-A Eq. 5-9 with the
// footnote that Y and Psi come from one joint pass; Sec. III-B Eq. 15-16).
//
// Design (GB300): the reduction is HBM-bound -- one read of X and labels --
// so the kernel is SIMT, with no tensor-core reshaping.  A CTA owns a
// contiguous row range and a column slice (and, for very many clusters, a
// bucket slice).  Rows are staged in shared memory one tile of 128 rows at a
// time with coalesced 128-bit loads; the tile's labels are counting-sorted in
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

#include "sil_internal.cuh"

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
  unsigned long long* count;
  double* s1;
  double* s2;
  double* wsum;
  uint32_t* status;
};

struct AggSmem {
  // byte offsets into dynamic shared memory
  int xs, acc, acc2, macc, mint, cnt, slot, ebk, epos, ew, order, nel, bstart, inv, wtot, nne,
      total;
};

__host__ __device__ inline AggSmem agg_smem(int dsp, int kbs, bool dual, bool weighted) {
  const int R = kAggRows, E = dual ? 2 * R : R, c4 = dsp / 4;
  AggSmem s;
  int o = 0;
  s.xs = o; o += R * dsp * 4;
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
  s.inv = o; o += R * 4;
  s.wtot = o; o += 32 * 4;
  s.nne = o; o += 16;
  s.total = (o + 15) & ~15;
  return s;
}

template <int DT, bool DUAL, bool WEIGHTED>
__global__ void __launch_bounds__(kAggThreads) k_aggregate(AggK a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int R = kAggRows, T = kAggThreads, E = DUAL ? 2 * R : R;
  const int tid = threadIdx.x;
  const int c4 = a.dsp / 4;
  const AggSmem L = agg_smem(a.dsp, a.kbs, DUAL, WEIGHTED);
  float* xs = reinterpret_cast<float*>(smem + L.xs);
  float4* xs4 = reinterpret_cast<float4*>(smem + L.xs);
  float4* acc4 = reinterpret_cast<float4*>(smem + L.acc);
  float* acc = reinterpret_cast<float*>(smem + L.acc);
  float* acc2 = reinterpret_cast<float*>(smem + L.acc2);
  float* macc = reinterpret_cast<float*>(smem + L.macc);
  int* mint = reinterpret_cast<int*>(smem + L.mint);
  int* cnt = reinterpret_cast<int*>(smem + L.cnt);
  int* slot = reinterpret_cast<int*>(smem + L.slot);
  int* ebk = reinterpret_cast<int*>(smem + L.ebk);
  int* epos = reinterpret_cast<int*>(smem + L.epos);
  float* ew = reinterpret_cast<float*>(smem + L.ew);
  int* order = reinterpret_cast<int*>(smem + L.order);
  int* nel = reinterpret_cast<int*>(smem + L.nel);
  int* bstart = reinterpret_cast<int*>(smem + L.bstart);
  float* inv = reinterpret_cast<float*>(smem + L.inv);
  int* wtot = reinterpret_cast<int*>(smem + L.wtot);
  int* nne = reinterpret_cast<int*>(smem + L.nne);

  const int cslice = blockIdx.x % a.nslc;
  const int kslice = blockIdx.x / a.nslc;
  const int col0 = cslice * a.dsp;
  const int dlim = min(a.d, col0 + a.dsp);       // columns of this slice are [col0, dlim)
  const int kb0 = kslice * a.kbs;
  const int kbn = min(a.kbs, a.kb - kb0);          // buckets of this slice
  const int c4e = int(cdiv(dlim - col0, 4));        // chunks holding columns < dlim
  const int64_t row_begin = int64_t(blockIdx.y) * a.rows_per_cta;
  const int64_t row_end = min(a.n, row_begin + a.rows_per_cta);
  const bool in_cta_norm = a.cosine && a.invnorm == nullptr;  // full rows are in this CTA

  for (int i = tid; i < kbn * a.dsp; i += T) acc[i] = 0.f;
  if (!WEIGHTED)
    for (int i = tid; i < kbn * c4; i += T) acc2[i] = 0.f;
  for (int i = tid; i < kbn; i += T) {
    macc[i] = 0.f;
    mint[i] = 0;
    cnt[i] = 0;
  }
  if (tid == 0) *nne = 0;
  __syncthreads();

  for (int64_t r0 = row_begin; r0 < row_end; r0 += R) {
    const int rows = int((row_end - r0) < int64_t(R) ? (row_end - r0) : int64_t(R));
    // (a) the tile's column slice, dequantised to FP32
    for (int q = tid; q < R * c4; q += T) {
      const int r = q / c4, c = q - r * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) v = load4<DT>(a.X, r0 + r, col0 + 4 * c, dlim, a.ldx, a.cs, a.vec);
      xs4[q] = v;
    }
    __syncthreads();
    // (b) bucket entries and row scales
    for (int e = tid; e < E; e += T) {
      const int r = e < R ? e : e - R;
      int lb = -1;
      float w = 1.f;
      if (r < rows) {
        const int64_t row = r0 + r;
        int32_t lab = (e < R) ? a.lab1[row] : a.lab2[row];
        if (lab >= 0 && lab < a.k) {
          const int bucket = (e < R) ? lab : a.k + lab;
          if (bucket >= kb0 && bucket < kb0 + kbn) lb = bucket - kb0;
          if (WEIGHTED) w = (e < R) ? a.w1[row] : a.w2[row];
        } else if (e < R || lab != -1) {
          // a label outside [0, k); -1 marks "no neighbour" in the second entry
          set_status(a.status, SIL_ELABEL);
        }
      }
      if (lb >= 0) {
        const int p = atomicAdd(&cnt[lb], 1);
        if (p == 0) {
          const int q = atomicAdd(nne, 1);
          nel[q] = lb;
          slot[lb] = q;
        }
        epos[e] = p;
      }
      ebk[e] = lb;
      ew[e] = w;
    }
    if (a.cosine) {
      if (in_cta_norm) {
        const int warp = tid >> 5, lane = tid & 31;
        for (int r = warp; r < R; r += T / 32) {
          float ss = 0.f;
          for (int c = lane; c < a.dsp; c += 32) ss += xs[r * a.dsp + c] * xs[r * a.dsp + c];
          for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
          if (lane == 0) {
            if (r < rows && !(ss > 0.f)) set_status(a.status, SIL_EZERONORM);
            inv[r] = ss > 0.f ? rsqrtf(ss) : 0.f;
          }
        }
      } else {
        for (int r = tid; r < R; r += T) inv[r] = r < rows ? a.invnorm[r0 + r] : 0.f;
      }
    }
    __syncthreads();
    // (c) exclusive scan of the bucket sizes over the non-empty list
    const int m = *nne;
    {
      const int warp = tid >> 5, lane = tid & 31;
      int v = (tid < m) ? cnt[nel[tid]] : 0;
      int incl = v;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      int off = 0;
      for (int w = 0; w < warp; ++w) off += wtot[w];
      if (tid < m) bstart[tid] = off + incl - v;
    }
    __syncthreads();
    // (d) scatter entries into bucket order
    for (int e = tid; e < E; e += T) {
      const int lb = ebk[e];
      if (lb >= 0) order[bstart[slot[lb]] + epos[e]] = e;
    }
    __syncthreads();
    // (e) one thread per (non-empty bucket, 4-column chunk of this slice)
    for (int p = tid; p < m * c4e; p += T) {
      const int q = p / c4e, c = p - q * c4e;
      const int lb = nel[q];
      const int kc = (kb0 + lb) % a.k;  // cluster whose reference point shifts this bucket
      const float4 rr = *reinterpret_cast<const float4*>(a.rs + int64_t(kc) * a.dz + col0 + 4 * c);
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
      float sq = 0.f, wsum = 0.f;
      const int jb = bstart[q], je = jb + cnt[lb];
#pragma unroll 4
      for (int j = jb; j < je; ++j) {
        const int e = order[j];
        const int r = e < R ? e : e - R;
        const float4 x = xs4[r * c4 + c];
        const float sc = a.cosine ? inv[r] : 1.f;
        float4 v;
        v.x = fmaf(sc, x.x, -rr.x);
        v.y = fmaf(sc, x.y, -rr.y);
        v.z = fmaf(sc, x.z, -rr.z);
        v.w = fmaf(sc, x.w, -rr.w);
        if (WEIGHTED) {
          const float w = ew[e];
          v.x *= w; v.y *= w; v.z *= w; v.w *= w;
          wsum += w;
        } else {
          sq = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, sq))));
        }
        s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
      }
      float4 t = acc4[lb * c4 + c];
      t.x += s.x; t.y += s.y; t.z += s.z; t.w += s.w;
      acc4[lb * c4 + c] = t;
      if (!WEIGHTED) acc2[lb * c4 + c] += sq;
      if (c == 0) {
        mint[lb] += je - jb;
        if (WEIGHTED) macc[lb] += wsum;
      }
    }
    __syncthreads();
    // (f) reset the counters used by this tile
    for (int q = tid; q < m; q += T) cnt[nel[q]] = 0;
    if (tid == 0) *nne = 0;
    // the __syncthreads after the next tile load orders this reset before reuse
  }
  __syncthreads();

  // flush: un-shift in FP64 and add into the outputs
  const int dsl = dlim - col0;
  for (int i = tid; i < kbn * dsl; i += T) {
    const int lb = i / dsl, col = i - lb * dsl;
    const int mm = mint[lb];
    if (mm == 0) continue;
    const int kg = kb0 + lb;
    double v = double(acc[lb * a.dsp + col]);
    if (!WEIGHTED) v += double(mm) * double(a.rs[int64_t(kg) * a.dz + col0 + col]);
    atomicAdd(a.s1 + int64_t(kg) * a.d + col0 + col, v);
  }
  for (int lb = tid; lb < kbn; lb += T) {
    const int mm = mint[lb];
    if (mm == 0) continue;
    const int kg = kb0 + lb;
    if (WEIGHTED) {
      if (cslice == 0) atomicAdd(a.wsum + kg, double(macc[lb]));
    } else {
      double t = 0.0;
      for (int c = 0; c < c4e; ++c) t += double(acc2[lb * c4 + c]);
      for (int col = 0; col < dsl; ++col) {
        const double r = a.rs[int64_t(kg) * a.dz + col0 + col];
        t += 2.0 * r * double(acc[lb * a.dsp + col]) + double(mm) * r * r;
      }
      atomicAdd(a.s2 + kg, t);
      if (cslice == 0) atomicAdd(a.count + kg, (unsigned long long)mm);
    }
  }
}

// Choose (dsp, kbs) so that one CTA's shared memory stays within budget.
// Column slices of at least 32 columns keep each row read a whole number of
// 32-byte DRAM sectors (bf16/fp32); a CTA may use up to 200 KB to get there.
void agg_plan(int32_t d, int32_t kb, bool dual, bool weighted, int* dsp_out, int* kbs_out) {
  const int dz = int(round_up(d, 4));
  const int budgets[2] = {kSmemBudget, 200 * 1024};
  const int min_dsp = dz < 32 ? dz : 32;
  for (int budget : budgets) {
    int dsp = dz;
    while (dsp > min_dsp && agg_smem(dsp, kb, dual, weighted).total > budget)
      dsp = std::max(min_dsp, int(round_up(dsp / 2, 4)));
    if (agg_smem(dsp, kb, dual, weighted).total <= budget) {
      *dsp_out = dsp;
      *kbs_out = kb;
      return;
    }
  }
  // very many buckets: narrowest slice, then split the buckets
  int dsp = min_dsp;
  int kbs = kb;
  while (kbs > 1 && agg_smem(dsp, kbs, dual, weighted).total > 200 * 1024) kbs = (kbs + 1) / 2;
  *dsp_out = dsp;
  *kbs_out = kbs;
}

bool vec_ok(const void* X, int32_t dtype, int64_t ldx) {
  const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
  return (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
}

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

template <int DT, bool DUAL, bool WEIGHTED>
static cudaError_t launch_agg_t(const AggK& k, dim3 grid, int smem, cudaStream_t stream) {
  auto fn = k_aggregate<DT, DUAL, WEIGHTED>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kAggThreads, smem, stream>>>(k);
  return cudaGetLastError();
}

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
  const int smem = agg_smem(dsp, kbs, dual, weighted).total;
  const int per_sm = std::max(1, std::min(4, (220 * 1024) / std::max(smem, 1)));
  const int64_t tiles = cdiv(L.n, kAggRows);
  const int64_t slices = int64_t(k.nslc) * nkslc;
  int64_t row_blocks = std::max<int64_t>(1, (int64_t(kNumSMs) * per_sm * 2) / slices);
  row_blocks = std::min<int64_t>(row_blocks, tiles);
  row_blocks = std::min<int64_t>(row_blocks, 65535);
  k.rows_per_cta = cdiv(tiles, row_blocks) * kAggRows;
  row_blocks = cdiv(L.n, k.rows_per_cta);
  const dim3 grid(static_cast<unsigned>(slices), static_cast<unsigned>(row_blocks));
  switch (L.dtype) {
    case SIL_F32:
      return dual ? launch_agg_t<SIL_F32, true, true>(k, grid, smem, L.stream)
                  : weighted ? launch_agg_t<SIL_F32, false, true>(k, grid, smem, L.stream)
                             : launch_agg_t<SIL_F32, false, false>(k, grid, smem, L.stream);
    case SIL_BF16:
      return dual ? launch_agg_t<SIL_BF16, true, true>(k, grid, smem, L.stream)
                  : weighted ? launch_agg_t<SIL_BF16, false, true>(k, grid, smem, L.stream)
                             : launch_agg_t<SIL_BF16, false, false>(k, grid, smem, L.stream);
    default:
      return dual ? launch_agg_t<SIL_FP8_E4M3, true, true>(k, grid, smem, L.stream)
                  : weighted ? launch_agg_t<SIL_FP8_E4M3, false, true>(k, grid, smem, L.stream)
                             : launch_agg_t<SIL_FP8_E4M3, false, false>(k, grid, smem, L.stream);
  }
}

}  // namespace sil
