// Finalisation of the aggregates and the SIMT form of pass 2.
//
// Pass 2 (Sec. III-A Eq. 10-11; Sec. III-B Eq. 17-18) in the centred
// coordinates x' = x - g, mu'_k = mu_k - g, with g the global mean (the
// Silhouette is translation invariant for the squared Euclidean distance):
//   mean distance to cluster k != c:  ||x'||^2 + bias_k - 2 x'.mu'_k,
//       bias_k = ||mu'_k||^2 + W_k/n_k   (Eq. 11 rearranged: Psi_k/n_k - ||g||^2 ...)
//   mean distance to the other members of c:
//       a = n_c/(n_c-1) ||x' - mu'_c||^2 + W_c/(n_c-1)
// where W_k = Psi_k - ||Y_k||^2/n_k is the within-cluster scatter.  The cosine
// distance is half the squared Euclidean distance of the unit vectors
// x_hat (1 - x_hat.y_hat = ||x_hat - y_hat||^2 / 2), so with x replaced by
// x_hat and every distance scaled by 1/2 the same kernel evaluates Eq. 18
// (the aggregates of Eq. 16 play the role of Y).  The own-cluster term uses
// the difference form, the other clusters the dot-product form of the paper.
//
// The SIMT kernel keeps each thread's point(s) in registers and the centroids
// in shared memory; every centroid element is a broadcast 128-bit shared load
// feeding 4 x PPT FFMAs.  N x K distances are never stored: each thread keeps
// the running minimum and its argmin.
#include <algorithm>
#include <cmath>

#include "sil_internal.cuh"

namespace sil {

namespace {

// ---------------------------------------------------------------- finalize
// g = (sum_k Y_k) / (sum_k n_k); one warp-column per output column.
__global__ void k_fin_global(const unsigned long long* count, const double* s1, int32_t k,
                             int32_t d, int32_t dz, double* g, float* gf, uint32_t* status) {
  __shared__ double part[32][33];
  __shared__ unsigned long long wn[32];
  __shared__ int wnon[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // total count and non-empty clusters: warp sums, then one thread (no
  // 64-bit shared atomics on one word from every thread)
  unsigned long long my = 0;
  int mynon = 0;
  for (int kk = threadIdx.x; kk < k; kk += blockDim.x) {
    my += count[kk];
    mynon += count[kk] > 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    my += __shfl_xor_sync(0xffffffffu, my, o);
    mynon += __shfl_xor_sync(0xffffffffu, mynon, o);
  }
  if (lane == 0) {
    wn[warp] = my;
    wnon[warp] = mynon;
  }
  const int c = blockIdx.x * 32 + lane;
  // four independent partial sums per lane keep several loads in flight
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (c < d) {
    int kk = warp;
    for (; kk + 3 * nwarp < k; kk += 4 * nwarp)
#pragma unroll
      for (int u = 0; u < 4; ++u) s[u] += s1[int64_t(kk + u * nwarp) * d + c];
    for (; kk < k; kk += nwarp) s[0] += s1[int64_t(kk) * d + c];
  }
  part[warp][lane] = (s[0] + s[1]) + (s[2] + s[3]);
  __syncthreads();
  unsigned long long ntot = 0;
  int nnon = 0;
  for (int w = 0; w < nwarp; ++w) {
    ntot += wn[w];
    nnon += wnon[w];
  }
  if (warp == 0 && c < dz) {
    double t = 0.0;
    for (int w = 0; w < nwarp; ++w) t += part[w][lane];
    const double gv = (c < d && ntot > 0) ? t / double(ntot) : 0.0;
    g[c] = gv;
    gf[c] = float(gv);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && nnon < 2) set_status(status, SIL_EDEGENERATE);
}

// One CTA per cluster: mu'_k (float, centred), and the constants of pass 2.
__global__ void k_fin_clusters(const unsigned long long* count, const double* s1, const double* s2,
                               int32_t d, int32_t dz, const double* g, float* zf, float4* cl) {
  __shared__ double red[2][32];
  const int kk = blockIdx.x;
  const unsigned long long n = count[kk];
  float* z = zf + int64_t(kk) * dz;
  if (n == 0) {
    for (int c = threadIdx.x; c < dz; c += blockDim.x) z[c] = 0.f;
    if (threadIdx.x == 0) cl[kk] = make_float4(INFINITY, 0.f, 0.f, 0.f);
    return;
  }
  const double inv_n = 1.0 / double(n);
  double mu2 = 0.0, mc2 = 0.0;
  for (int c = threadIdx.x; c < dz; c += blockDim.x) {
    double mu = c < d ? s1[int64_t(kk) * d + c] * inv_n : 0.0;
    double mc = mu - g[c];
    z[c] = float(mc);
    mu2 += mu * mu;
    mc2 += mc * mc;
  }
  for (int o = 16; o > 0; o >>= 1) {
    mu2 += __shfl_xor_sync(0xffffffffu, mu2, o);
    mc2 += __shfl_xor_sync(0xffffffffu, mc2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = mu2;
    red[1][threadIdx.x >> 5] = mc2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    double W = s2[kk] - double(n) * a;  // within-cluster scatter
    if (W < 0.0) W = 0.0;
    const double bias = b + W * inv_n;
    const float an = n > 1 ? float(double(n) / double(n - 1)) : 0.f;
    const float aw = n > 1 ? float(W / double(n - 1)) : 0.f;
    cl[kk] = make_float4(float(bias), an, aw, float(n));
  }
}

// ------------------------------------------------------------------ scoring
struct ScoreK {
  const void* X;
  int64_t n;
  int32_t d;
  int64_t ldx;
  const float* cs;
  const int32_t* labels;
  int32_t k;
  int32_t dz;
  const float* zf;
  const float4* cl;
  const float* gf;
  int32_t cosine;
  int32_t rms;  // Eq. 2 on the square roots of a and b (approximate Euclidean)
  float scale;
  int32_t vec;
  float* s_out;
  float* sa;
  float* sb;
  int32_t* skstar;
  double* partials;
  uint32_t* status;
  int32_t kc;  // clusters per shared-memory chunk
};

__device__ __forceinline__ float silhouette_value(float a, float b, bool defined, bool rms) {
  return defined ? sil_eq2(a, b, rms) : 0.f;
}

__device__ __forceinline__ void block_partial(float v, double* out) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t += double(red[w]);
    *out = t;
  }
}

// DMAX: compile-time bound on the padded dimension (x lives in registers);
// PPT: points per thread.
template <int DT, int DMAX, int PPT>
__global__ void __launch_bounds__(kScoreThreads) k_score_simt(ScoreK a) {
  extern __shared__ __align__(16) float sm[];
  constexpr int T = kScoreThreads, NQ = DMAX / 4;
  const int dz = a.dz, kc = a.kc;
  float* zs = sm;                                              // [kc][dz] + DMAX zero pad
  float4* cls = reinterpret_cast<float4*>(zs + kc * dz + DMAX);  // [kc]
  float* gs = reinterpret_cast<float*>(cls + kc);              // [DMAX]
  const int tid = threadIdx.x;
  const bool one_chunk = kc >= a.k;

  for (int c = tid; c < DMAX; c += T) gs[c] = c < dz ? a.gf[c] : 0.f;
  for (int c = tid; c < DMAX; c += T) zs[kc * dz + c] = 0.f;
  if (one_chunk) {
    for (int i = tid; i < a.k * dz; i += T) zs[i] = a.zf[i];
    for (int i = tid; i < a.k; i += T) cls[i] = a.cl[i];
  }
  __syncthreads();

  float tsum = 0.f;
  for (int64_t base = int64_t(blockIdx.x) * (T * PPT); base < a.n;
       base += int64_t(gridDim.x) * (T * PPT)) {
    float x[PPT][DMAX];
    int own[PPT];
    bool ok[PPT];
    float xn2[PPT], best[PPT];
    int kbest[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = base + tid + j * T;
      ok[j] = p < a.n;
      own[j] = -1;
      if (ok[j]) {
        own[j] = a.labels[p];
        if (own[j] < 0 || own[j] >= a.k) {
          set_status(a.status, SIL_ELABEL);
          ok[j] = false;
          own[j] = -1;
        }
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok[j] && 4 * q < a.d) v = load4<DT>(a.X, p, 4 * q, a.d, a.ldx, a.cs, a.vec);
        x[j][4 * q] = v.x;
        x[j][4 * q + 1] = v.y;
        x[j][4 * q + 2] = v.z;
        x[j][4 * q + 3] = v.w;
      }
      float inv = 1.f;
      if (a.cosine) {
        float ss = 0.f;
#pragma unroll
        for (int c = 0; c < DMAX; ++c) ss = fmaf(x[j][c], x[j][c], ss);
        if (ok[j] && !(ss > 0.f)) {
          set_status(a.status, SIL_EZERONORM);
          ok[j] = false;
        }
        inv = ss > 0.f ? rsqrtf(ss) : 0.f;
      }
      float n2 = 0.f;
#pragma unroll
      for (int c = 0; c < DMAX; ++c) {
        const float v = fmaf(x[j][c], inv, -gs[c]);
        x[j][c] = v;
        n2 = fmaf(v, v, n2);
      }
      xn2[j] = n2;
      best[j] = INFINITY;
      kbest[j] = -1;
    }

    for (int k0 = 0; k0 < a.k; k0 += kc) {
      const int kcur = min(kc, a.k - k0);
      if (!one_chunk) {
        __syncthreads();
        for (int i = tid; i < kcur * dz; i += T) zs[i] = a.zf[int64_t(k0) * dz + i];
        for (int i = tid; i < kcur; i += T) cls[i] = a.cl[k0 + i];
        __syncthreads();
      }
#pragma unroll 1
      for (int kk = 0; kk < kcur; ++kk) {
        const float4* zr = reinterpret_cast<const float4*>(zs + kk * dz);
        float d0[PPT], d1[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) d0[j] = d1[j] = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const float4 z = zr[q];
#pragma unroll
          for (int j = 0; j < PPT; ++j) {
            d0[j] = fmaf(x[j][4 * q], z.x, d0[j]);
            d1[j] = fmaf(x[j][4 * q + 1], z.y, d1[j]);
            d0[j] = fmaf(x[j][4 * q + 2], z.z, d0[j]);
            d1[j] = fmaf(x[j][4 * q + 3], z.w, d1[j]);
          }
        }
        const float bias = cls[kk].x;
        const int kg = k0 + kk;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
          const float v = fmaf(-2.f, d0[j] + d1[j], bias);
          if (kg != own[j] && v < best[j]) {
            best[j] = v;
            kbest[j] = kg;
          }
        }
      }
    }

#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int64_t p = base + tid + j * T;
      if (p >= a.n) continue;
      float av = 0.f, bv = INFINITY, sv = 0.f;
      int kb = -1;
      if (ok[j]) {
        const float4 co = a.cl[own[j]];
        const float4* zo = reinterpret_cast<const float4*>(a.zf + int64_t(own[j]) * dz);
        float ss = 0.f;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          if (4 * q < dz) {
            const float4 z = __ldg(zo + q);
            const float e0 = x[j][4 * q] - z.x, e1 = x[j][4 * q + 1] - z.y;
            const float e2 = x[j][4 * q + 2] - z.z, e3 = x[j][4 * q + 3] - z.w;
            ss = fmaf(e0, e0, fmaf(e1, e1, fmaf(e2, e2, fmaf(e3, e3, ss))));
          }
        }
        av = fmaxf(0.f, a.scale * fmaf(co.y, ss, co.z));
        kb = kbest[j];
        bv = kb >= 0 ? fmaxf(0.f, a.scale * (xn2[j] + best[j])) : INFINITY;
        sv = silhouette_value(av, bv, co.w > 1.5f && kb >= 0, a.rms);
      }
      if (a.s_out) a.s_out[p] = sv;
      if (a.sa) {
        a.sa[p] = av;
        a.sb[p] = bv;
        a.skstar[p] = kb;
      }
      tsum += sv;
    }
  }
  block_partial(tsum, a.partials + blockIdx.x);
}

// Wide rows (d > 128): each thread's row is staged in shared memory.
template <int DT>
__global__ void __launch_bounds__(64) k_score_simt_wide(ScoreK a) {
  extern __shared__ __align__(16) float sm[];
  constexpr int T = 64;
  const int dz = a.dz, kc = a.kc, rs = dz + 4;  // row stride in floats (16-byte skew)
  float* zs = sm;                                          // [kc][dz]
  float4* cls = reinterpret_cast<float4*>(zs + kc * dz);   // [kc]
  float* xsm = reinterpret_cast<float*>(cls + kc);         // [T][rs]
  const int tid = threadIdx.x;
  const bool one_chunk = kc >= a.k;
  if (one_chunk) {
    for (int i = tid; i < a.k * dz; i += T) zs[i] = a.zf[i];
    for (int i = tid; i < a.k; i += T) cls[i] = a.cl[i];
  }
  __syncthreads();
  float tsum = 0.f;
  float* xr = xsm + tid * rs;
  for (int64_t base = int64_t(blockIdx.x) * T; base < a.n; base += int64_t(gridDim.x) * T) {
    const int64_t p = base + tid;
    bool ok = p < a.n;
    int own = -1;
    if (ok) {
      own = a.labels[p];
      if (own < 0 || own >= a.k) {
        set_status(a.status, SIL_ELABEL);
        ok = false;
        own = -1;
      }
    }
    float ss = 0.f;
    for (int c = 0; c < dz; c += 4) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok) v = load4<DT>(a.X, p, c, a.d, a.ldx, a.cs, a.vec);
      *reinterpret_cast<float4*>(xr + c) = v;
      ss += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
    float inv = 1.f;
    if (a.cosine) {
      if (ok && !(ss > 0.f)) {
        set_status(a.status, SIL_EZERONORM);
        ok = false;
      }
      inv = ss > 0.f ? rsqrtf(ss) : 0.f;
    }
    float n2 = 0.f;
    for (int c = 0; c < dz; ++c) {
      const float v = fmaf(xr[c], inv, -a.gf[c]);
      xr[c] = v;
      n2 = fmaf(v, v, n2);
    }
    float best = INFINITY;
    int kbest = -1;
    for (int k0 = 0; k0 < a.k; k0 += kc) {
      const int kcur = min(kc, a.k - k0);
      if (!one_chunk) {
        __syncthreads();
        for (int i = tid; i < kcur * dz; i += T) zs[i] = a.zf[int64_t(k0) * dz + i];
        for (int i = tid; i < kcur; i += T) cls[i] = a.cl[k0 + i];
        __syncthreads();
      }
      for (int kk = 0; kk < kcur; ++kk) {
        const float4* zr = reinterpret_cast<const float4*>(zs + kk * dz);
        const float4* xv = reinterpret_cast<const float4*>(xr);
        float d0 = 0.f, d1 = 0.f;
        for (int q = 0; q < dz / 4; ++q) {
          const float4 z = zr[q], xx = xv[q];
          d0 = fmaf(xx.x, z.x, d0);
          d1 = fmaf(xx.y, z.y, d1);
          d0 = fmaf(xx.z, z.z, d0);
          d1 = fmaf(xx.w, z.w, d1);
        }
        const float v = fmaf(-2.f, d0 + d1, cls[kk].x);
        const int kg = k0 + kk;
        if (kg != own && v < best) {
          best = v;
          kbest = kg;
        }
      }
    }
    if (p < a.n) {
      float av = 0.f, bv = INFINITY, sv = 0.f;
      int kb = -1;
      if (ok) {
        const float4 co = a.cl[own];
        const float* zo = a.zf + int64_t(own) * dz;
        float s2 = 0.f;
        for (int c = 0; c < dz; ++c) {
          const float e = xr[c] - zo[c];
          s2 = fmaf(e, e, s2);
        }
        av = fmaxf(0.f, a.scale * fmaf(co.y, s2, co.z));
        kb = kbest;
        bv = kb >= 0 ? fmaxf(0.f, a.scale * (n2 + best)) : INFINITY;
        sv = silhouette_value(av, bv, co.w > 1.5f && kb >= 0, a.rms);
      }
      if (a.s_out) a.s_out[p] = sv;
      if (a.sa) {
        a.sa[p] = av;
        a.sb[p] = bv;
        a.skstar[p] = kb;
      }
      tsum += sv;
    }
  }
  block_partial(tsum, a.partials + blockIdx.x);
}

// S = sum of the partials / n in a fixed order; NaN when a flag was raised.
__global__ void __launch_bounds__(256) k_reduce_S(const double* partials, int32_t np, int64_t n,
                                                  const uint32_t* ws_status, uint32_t* user_status, double* S_out) {
  __shared__ double wred[8];
  // four independent sums per thread keep the loads of up to kMaxPartials
  // partials in flight; shuffles, then the eight warp sums in order (a fixed
  // order for a given np: deterministic)
  double t4[4] = {0.0, 0.0, 0.0, 0.0};
  const int stride = int(blockDim.x);
  int i = threadIdx.x;
  for (; i + 3 * stride < np; i += 4 * stride)
#pragma unroll
    for (int u = 0; u < 4; ++u) t4[u] += partials[i + u * stride];
  for (; i < np; i += stride) t4[0] += partials[i];
  double t = (t4[0] + t4[1]) + (t4[2] + t4[3]);
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) tot += wred[w];
    const uint32_t st = *ws_status;
    if (user_status && st) atomicOr(user_status, st);
    if (S_out) *S_out = (st == 0 && n > 0) ? tot / double(n) : NAN;
  }
}

// S over row chunks from the chunk means: sum_c n_c S_c / sum_c n_c in FP64
// (one CTA, fixed order); NaN if any chunk mean is NaN.
__global__ void k_chunk_mean(const double* S_chunks, const int64_t* n_chunks, int32_t m, double* S_out) {
  __shared__ double rs[256];
  __shared__ double rn[256];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    s += S_chunks[i] * double(n_chunks[i]);
    c += double(n_chunks[i]);
  }
  rs[threadIdx.x] = s;
  rn[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o) {
      rs[threadIdx.x] += rs[threadIdx.x + o];
      rn[threadIdx.x] += rn[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *S_out = rn[0] > 0.0 ? rs[0] / rn[0] : NAN;
}

// One CTA per labeling: S_b from its np partial sums (fixed order).
__global__ void k_reduce_S_batched(const double* partials, int32_t np, int64_t n, const uint32_t* status,
                                   uint32_t* user_status, double* S_out) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  double t = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) t += partials[int64_t(b) * np + i];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (int(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t st = status[b];
    if (user_status && st) atomicOr(user_status, st);
    S_out[b] = (st == 0 && n > 0) ? red[0] / double(n) : NAN;
  }
}

__global__ void k_publish_status(const uint32_t* ws_status, uint32_t* user_status) {
  if (threadIdx.x == 0 && user_status) {
    const uint32_t st = *ws_status;
    if (st) atomicOr(user_status, st);
  }
}

template <int DT, int DMAX, int PPT>
cudaError_t launch_simt_t(ScoreK& k, cudaStream_t stream, int32_t* np) {
  const int dz = k.dz;
  const int fixed = (DMAX + DMAX) * 4;  // zero pad + g
  const int per_cluster = dz * 4 + 16;
  int kc = std::max(1, (kSmemBudget - fixed) / per_cluster);
  kc = std::min(kc, k.k);
  k.kc = kc;
  const int smem = kc * per_cluster + fixed + 16;
  auto fn = k_score_simt<DT, DMAX, PPT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = cdiv(k.n, int64_t(kScoreThreads) * PPT);
  const int per_sm = std::max(1, std::min(2, (220 * 1024) / smem));
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(groups, int64_t(num_sms()) * per_sm), kMaxPartials)));
  fn<<<grid, kScoreThreads, smem, stream>>>(k);
  *np = grid;
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_wide_t(ScoreK& k, cudaStream_t stream, int32_t* np) {
  const int dz = k.dz;
  const int xbytes = 64 * (dz + 4) * 4;
  const int per_cluster = dz * 4 + 16;
  int kc = std::max(1, (kSmemBudget - xbytes) / per_cluster);
  kc = std::min(kc, k.k);
  k.kc = kc;
  const int smem = kc * per_cluster + xbytes + 16;
  auto fn = k_score_simt_wide<DT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t groups = cdiv(k.n, 64);
  const int per_sm = std::max(1, std::min(8, (220 * 1024) / smem));
  const int grid = int(std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(groups, int64_t(num_sms()) * per_sm), kMaxPartials)));
  fn<<<grid, 64, smem, stream>>>(k);
  *np = grid;
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_simt_dt(ScoreK& k, cudaStream_t stream, int32_t* np) {
  if (k.dz <= 16) return launch_simt_t<DT, 16, 2>(k, stream, np);
  if (k.dz <= 32) return launch_simt_t<DT, 32, 2>(k, stream, np);
  if (k.dz <= 64) return launch_simt_t<DT, 64, 2>(k, stream, np);
  if (k.dz <= 128) return launch_simt_t<DT, 128, 1>(k, stream, np);
  return launch_wide_t<DT>(k, stream, np);
}

bool vec_ok_s(const void* X, int32_t dtype, int64_t ldx) {
  const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
  return (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
}

}  // namespace

cudaError_t launch_finalize(const FinLaunch& f) {
  const int dz = int(round_up(f.d, 4));
  k_fin_global<<<unsigned(cdiv(dz, 32)), 1024, 0, f.stream>>>(f.count, f.s1, f.k, f.d, dz, f.g, f.gf,
                                                              f.status);
  k_fin_clusters<<<f.k, 128, 0, f.stream>>>(f.count, f.s1, f.s2, f.d, dz, f.g, f.zf, f.cl);
  return cudaGetLastError();
}

cudaError_t launch_score_simt(ScoreLaunch& s) {
  ScoreK k{};
  k.X = s.X;
  k.n = s.n;
  k.d = s.d;
  k.ldx = s.ldx;
  k.cs = s.cs;
  k.labels = s.labels;
  k.k = s.k;
  k.dz = int(round_up(s.d, 4));
  k.zf = s.zf;
  k.cl = s.cl;
  k.gf = s.gf;
  k.cosine = s.dist == SIL_COSINE;
  k.rms = s.dist == SIL_EUCLIDEAN_RMS;
  k.scale = s.dist == SIL_COSINE ? 0.5f : 1.f;
  k.vec = vec_ok_s(s.X, s.dtype, s.ldx);
  k.s_out = s.s_out;
  k.sa = s.sa;
  k.sb = s.sb;
  k.skstar = s.skstar;
  k.partials = s.partials;
  k.status = s.status;
  if (s.n == 0) {
    *s.n_partials = 0;
    return cudaSuccess;
  }
  switch (s.dtype) {
    case SIL_F32: return launch_simt_dt<SIL_F32>(k, s.stream, s.n_partials);
    case SIL_BF16: return launch_simt_dt<SIL_BF16>(k, s.stream, s.n_partials);
    default: return launch_simt_dt<SIL_FP8_E4M3>(k, s.stream, s.n_partials);
  }
}

cudaError_t launch_reduce_S(const double* partials, int32_t np, int64_t n, const uint32_t* ws_status,
                            uint32_t* user_status, double* S_out, cudaStream_t stream) {
  k_reduce_S<<<1, 256, 0, stream>>>(partials, np, n, ws_status, user_status, S_out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_S_batched(const double* partials, int32_t np, int64_t n, int32_t batch,
                                    const uint32_t* status, uint32_t* user_status, double* S_out,
                                    cudaStream_t stream) {
  k_reduce_S_batched<<<batch, 256, 0, stream>>>(partials, np, n, status, user_status, S_out);
  return cudaGetLastError();
}

cudaError_t launch_chunk_mean(const double* S_chunks, const int64_t* n_chunks, int32_t m, double* S_out,
                              cudaStream_t stream) {
  k_chunk_mean<<<1, 256, 0, stream>>>(S_chunks, n_chunks, m, S_out);
  return cudaGetLastError();
}

cudaError_t launch_publish_status(const uint32_t* ws_status, uint32_t* user_status,
                                  cudaStream_t stream) {
  if (!user_status) return cudaSuccess;
  k_publish_status<<<1, 32, 0, stream>>>(ws_status, user_status);
  return cudaGetLastError();
}

}  // namespace sil
