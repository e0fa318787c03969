// Backward pass: dS/dX with the labels fixed and b_i's argmin k*_i held at
// its value (the min of b_i and the max of Eq. 1 taken as subgradients).
// The paper has no backward pass; the derivation (written out in the design
// notes) gives, with
//   alpha_i = (ds_i/da_i) / (n_c - 1),   beta_i = (ds_i/db_i) / n_{k*_i},
//   A_k = sum_{c(i)=k} alpha_i,  P_k = sum_{c(i)=k} alpha_i v_i,
//   B_k = sum_{k*_i=k} beta_i,   Q_k = sum_{k*_i=k} beta_i v_i,
// (v = x for the squared Euclidean distance, v = x_hat for cosine):
//   sq-Euclidean  dS/dx_m = (2/N)[alpha_m n_c (x_m - mu_c) + beta_m n_k* (x_m - mu_k*)
//                                + A_c x_m - P_c + B_c x_m - Q_c]
//   cosine        g = -(1/N)[alpha_m n_c mu_c + beta_m n_k* mu_k* + P_c + Q_c]
//                 dS/dx_m = (g - x_hat (x_hat.g)) / ||x_m||
// with c = c(m), k* = k*_m, mu the cluster means (of x_hat for cosine).
// The four segmented sums come from ONE extra pass over X: the pass-1 kernel
// in its weighted dual-entry form (each row adds alpha_i v_i to bucket c(i)
// and beta_i v_i to bucket k + k*_i), again shifted by the per-cluster
// reference points.  A second pass writes dX, one warp per row, walking the
// rows in that pass's sort order so that a cluster's vectors are loaded once
// per run of its rows.
#include "sil_internal.cuh"

namespace sil {

namespace {

__device__ __forceinline__ void silhouette_partials(float a, float b, float* dsa, float* dsb) {
  const float m = fmaxf(a, b);
  if (!(m > 0.f)) {
    *dsa = 0.f;
    *dsb = 0.f;
  } else if (a <= b) {
    *dsa = -1.f / b;
    *dsb = a / (b * b);
  } else {
    *dsa = -b / (a * a);
    *dsb = 1.f / a;
  }
}

// alpha and beta of one point from its saved (a, b, k*).
__device__ __forceinline__ void point_weights(int64_t i, const int32_t* labels, int32_t k,
                                              const float4* cl, const float* sa, const float* sb,
                                              const int32_t* skstar, float* alpha, float* beta,
                                              int* c_out, int* ks_out) {
  const int c = labels[i];
  const int ks = skstar[i];
  *alpha = 0.f;
  *beta = 0.f;
  *c_out = c;
  *ks_out = ks;
  if (c < 0 || c >= k || ks < 0 || ks >= k) return;
  const float nc = cl[c].w;
  if (nc < 1.5f) return;
  float dsa, dsb;
  silhouette_partials(sa[i], sb[i], &dsa, &dsb);
  *alpha = dsa / (nc - 1.f);
  *beta = dsb / cl[ks].w;
}

__global__ void k_bw_weights(int64_t n, const int32_t* labels, int32_t k, const float4* cl,
                             const float* sa, const float* sb, const int32_t* skstar, float* w1,
                             float* w2) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    float al, be;
    int c, ks;
    point_weights(i, labels, k, cl, sa, sb, skstar, &al, &be, &c, &ks);
    w1[i] = al;
    w2[i] = be;
  }
}

// Per cluster: W_c = P'_c + Q'_c (float), C_c = A_c + B_c.
__global__ void k_bw_prep(const double* bw_w, const double* bw_p, int32_t k, int32_t d, int32_t dz,
                          float* Wf, float* Cf) {
  const int c = blockIdx.x;
  for (int l = threadIdx.x; l < dz; l += blockDim.x)
    Wf[int64_t(c) * dz + l] =
        l < d ? float(bw_p[int64_t(c) * d + l] + bw_p[int64_t(k + c) * d + l]) : 0.f;
  if (threadIdx.x == 0) Cf[c] = float(bw_w[c] + bw_w[k + c]);
}

struct GradK {
  const void* X;
  int64_t n;
  int32_t d;
  int32_t dz;
  int64_t ldx;
  const float* cs;
  const int32_t* labels;
  int32_t k;
  int32_t cosine;
  int32_t vec;
  const float4* cl;
  const float* zf;
  const float* gf;
  const float* rs;
  const float* Wf;
  const float* Cf;
  const float* sa;
  const float* sb;
  const int32_t* skstar;
  const double* grad_S;
  float* dX;
  int64_t lddx;
  int32_t vec_out;  // dX rows 16-byte aligned
  // rows in the order of the dual pass 1's sort (entries of the first k
  // buckets: row, alpha, bucket starts), beta per row, and the work split
  const uint32_t* idx;
  const float* widx;
  const float* w2;
  const uint32_t* bstart;
  int64_t wchunk;
  int64_t nitems;
};

// The per-row term of dS/dx_m for the squared Euclidean distance (four
// columns l0 .. l0 + 3 of row m):
//   scale [C_c (x - r_c) - W_c + an (x - g - mu'_c) + bn (x - g - mu'_k*)]
// with an = alpha n_c, bn = beta n_k*; W_c holds P'_c + Q'_c (shifted by r_c).
__device__ __forceinline__ float4 grad_sqeuclid4(float4 x, float4 g, float4 r, float4 w, float4 zc, float4 zk,
                                                 float Cc, float an, float bn, float scale) {
  const float xv[4] = {x.x, x.y, x.z, x.w}, gv[4] = {g.x, g.y, g.z, g.w};
  const float rv[4] = {r.x, r.y, r.z, r.w}, wv[4] = {w.x, w.y, w.z, w.w};
  const float cv[4] = {zc.x, zc.y, zc.z, zc.w}, kv[4] = {zk.x, zk.y, zk.z, zk.w};
  float o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float xc = xv[j] - gv[j];
    float v = Cc * (xv[j] - rv[j]) - wv[j];
    v = fmaf(an, xc - cv[j], v);
    v = fmaf(bn, xc - kv[j], v);
    o[j] = scale * v;
  }
  return make_float4(o[0], o[1], o[2], o[3]);
}

// Cosine: g_l = -(1/N)[an (mu'_c + g) + bn (mu'_k* + g) + W_c + C_c r_c]
// (mu' + g the mean of x_hat), for four columns.
__device__ __forceinline__ float4 grad_cos_g4(float4 g, float4 r, float4 w, float4 zc, float4 zk, float Cc,
                                              float an, float bn, float inv_n) {
  const float G[4] = {g.x, g.y, g.z, g.w}, R[4] = {r.x, r.y, r.z, r.w};
  const float W[4] = {w.x, w.y, w.z, w.w}, C[4] = {zc.x, zc.y, zc.z, zc.w};
  const float Kv[4] = {zk.x, zk.y, zk.z, zk.w};
  float o[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float v = fmaf(Cc, R[j], W[j]);
    v = fmaf(an, C[j] + G[j], v);
    v = fmaf(bn, Kv[j] + G[j], v);
    o[j] = -v * inv_n;
  }
  return make_float4(o[0], o[1], o[2], o[3]);
}

// dX in the order of the dual pass 1's sort: the rows of one cluster c come
// one after another, so each warp keeps c's vectors (r_c, W_c, mu'_c) in
// registers for the run and per row loads only the row, its nearest other
// cluster's mu'_k* and three scalars -- instead of five cluster vectors per
// row.  A warp takes a contiguous range of sorted entries, 32 at a time
// (row ids and alpha in one coalesced load), two rows per step with every
// load of both issued first.  NV = 16-byte chunks per lane (d <= 128 NV).
// Rows with a label outside [0, k) are not in the order (SIL_ELABEL is set
// by pass 1): their dX rows are left as they are.
template <int DT, int NV, bool COS>
__global__ void __launch_bounds__(256, NV == 1 ? 3 : 2) k_bw_grad_sorted(GradK a) {
  constexpr int RPS = 2;  // rows per step (four, or the vectors read from L1 per row, measured slower)
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const double gsd = a.grad_S ? *a.grad_S : 1.0;
  const float inv_n = float(1.0 / double(a.n));
  const uint32_t total = a.bstart[a.k];
  auto ld4 = [&](const float* base, int v) {
    const int l0 = 4 * lane + 128 * v;
    return l0 < a.dz ? __ldg(reinterpret_cast<const float4*>(base + l0)) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  float4 g[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) g[v] = ld4(a.gf, v);
  for (int64_t item = gw; item < a.nitems; item += nw) {
    const int64_t e0 = item * a.wchunk;
    const int64_t e1 = min(int64_t(total), e0 + a.wchunk);
    if (e0 >= e1) break;
    // bucket holding e0: the last c with bstart[c] <= e0
    int lo = 0, hi = a.k - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(a.bstart + mid) <= uint32_t(e0)) lo = mid;
      else hi = mid - 1;
    }
    int c = lo;
    int64_t cend = int64_t(__ldg(a.bstart + c + 1));
    float4 rc[NV], wc[NV], zc[NV];
    float Cc = 0.f, nc = 0.f;
    auto load_cluster = [&]() {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        rc[v] = ld4(a.rs + int64_t(c) * a.dz, v);
        wc[v] = ld4(a.Wf + int64_t(c) * a.dz, v);
        zc[v] = ld4(a.zf + int64_t(c) * a.dz, v);
      }
      Cc = __ldg(a.Cf + c);
      nc = __ldg(&a.cl[c]).w;
    };
    load_cluster();
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int cnt = int(min(int64_t(32), e1 - eb));
      const bool mine = lane < cnt;
      const uint32_t my_row = mine ? __ldg(a.idx + eb + lane) : 0u;
      const float my_al = mine ? __ldg(a.widx + eb + lane) : 0.f;
      const int my_ks = mine ? __ldg(a.skstar + my_row) : -1;
      const float my_be = mine ? __ldg(a.w2 + my_row) : 0.f;
      for (int j = 0; j < cnt; j += RPS) {
        const int nr = min(RPS, cnt - j);
        uint32_t row[RPS];
        float al[RPS], be[RPS], nk[RPS];
        float4 x[RPS][NV], zk[RPS][NV];
#pragma unroll
        for (int u = 0; u < RPS; ++u) {
          const int src = j + (u < nr ? u : 0);
          row[u] = __shfl_sync(0xffffffffu, my_row, src);
          const int ks = __shfl_sync(0xffffffffu, my_ks, src);
          al[u] = __shfl_sync(0xffffffffu, my_al, src);
          be[u] = __shfl_sync(0xffffffffu, my_be, src);
          const bool has_k = ks >= 0 && ks < a.k;
          const int kk = has_k ? ks : 0;
          nk[u] = has_k ? __ldg(&a.cl[kk]).w : 0.f;
          if (!has_k) be[u] = 0.f;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int l0 = 4 * lane + 128 * v;
            x[u][v] = l0 < a.dz ? load4<DT>(a.X, int64_t(row[u]), l0, a.d, a.ldx, a.cs, a.vec)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            zk[u][v] = ld4(a.zf + int64_t(kk) * a.dz, v);
          }
        }
#pragma unroll
        for (int u = 0; u < RPS; ++u) {
          if (u >= nr) break;
          const int64_t pos = eb + j + u;
          if (pos >= cend) {  // the run of cluster c ends: the next non-empty bucket
            while (int64_t(__ldg(a.bstart + c + 1)) <= pos) ++c;
            cend = int64_t(__ldg(a.bstart + c + 1));
            load_cluster();
          }
          const float an = al[u] * nc, bn = be[u] * nk[u];
          float* out = a.dX + int64_t(row[u]) * a.lddx;
          float4 o[NV];
          if (!COS) {
            const float scale = float(gsd) * 2.f * inv_n;
#pragma unroll
            for (int v = 0; v < NV; ++v)
              o[v] = grad_sqeuclid4(x[u][v], g[v], rc[v], wc[v], zc[v], zk[u][v], Cc, an, bn, scale);
          } else {
            float ss = 0.f;
#pragma unroll
            for (int v = 0; v < NV; ++v)
              ss += x[u][v].x * x[u][v].x + x[u][v].y * x[u][v].y + x[u][v].z * x[u][v].z + x[u][v].w * x[u][v].w;
            for (int s = 16; s > 0; s >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, s);
            const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
            float4 gv[NV];
            float proj = 0.f;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              gv[v] = grad_cos_g4(g[v], rc[v], wc[v], zc[v], zk[u][v], Cc, an, bn, inv_n);
              const int l0 = 4 * lane + 128 * v;
              const float xs[4] = {x[u][v].x, x[u][v].y, x[u][v].z, x[u][v].w};
              const float gs[4] = {gv[v].x, gv[v].y, gv[v].z, gv[v].w};
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (l0 + q < a.d) proj = fmaf(xs[q] * inv, gs[q], proj);
            }
            for (int s = 16; s > 0; s >>= 1) proj += __shfl_xor_sync(0xffffffffu, proj, s);
            const float sc = float(gsd) * inv;
#pragma unroll
            for (int v = 0; v < NV; ++v)
              o[v] = make_float4(sc * (gv[v].x - x[u][v].x * inv * proj), sc * (gv[v].y - x[u][v].y * inv * proj),
                                 sc * (gv[v].z - x[u][v].z * inv * proj), sc * (gv[v].w - x[u][v].w * inv * proj));
          }
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int l0 = 4 * lane + 128 * v;
            if (l0 >= a.d) continue;
            if (a.vec_out && l0 + 3 < a.d) {
              *reinterpret_cast<float4*>(out + l0) = o[v];
            } else {
              const float ov[4] = {o[v].x, o[v].y, o[v].z, o[v].w};
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (l0 + q < a.d) out[l0 + q] = ov[q];
            }
          }
        }
      }
    }
  }
}

// One warp per row of dX, in row order (rows of more than 256 columns; the
// kernel above serves the others).  Latency-bound (each warp waits on its
// row's loads): six CTAs per SM (40 registers) measured faster than four (53)
// or eight (32, with spills).
template <int DT>
__global__ void __launch_bounds__(256, 6) k_bw_grad(GradK a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const double gsd = a.grad_S ? *a.grad_S : 1.0;
  const float inv_n = float(1.0 / double(a.n));
  for (int64_t m = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; m < a.n; m += nw) {
    float al, be;
    int c, ks;
    point_weights(m, a.labels, a.k, a.cl, a.sa, a.sb, a.skstar, &al, &be, &c, &ks);
    float* out = a.dX + m * a.lddx;
    if (c < 0 || c >= a.k) {
      for (int l = lane; l < a.d; l += 32) out[l] = 0.f;
      continue;
    }
    const bool has_k = ks >= 0 && ks < a.k;
    const int kk = has_k ? ks : c;
    const float nc = a.cl[c].w, nk = a.cl[kk].w;
    const float Cc = a.Cf[c];
    const float* zc = a.zf + int64_t(c) * a.dz;
    const float* zk = a.zf + int64_t(kk) * a.dz;
    const float* rc = a.rs + int64_t(c) * a.dz;
    const float* Wc = a.Wf + int64_t(c) * a.dz;
    if (!a.cosine) {
      const float scale = float(gsd) * 2.f * inv_n;
      const float an = al * nc, bn = has_k ? be * nk : 0.f;
      for (int l0 = 4 * lane; l0 < a.dz; l0 += 128) {
        // the per-cluster vectors are dz long (zero padded, 16-byte rows):
        // one 16-byte load each
        const float4 x = load4<DT>(a.X, m, l0, a.d, a.ldx, a.cs, a.vec);
        const float4 g4 = __ldg(reinterpret_cast<const float4*>(a.gf + l0));
        const float4 r4 = __ldg(reinterpret_cast<const float4*>(rc + l0));
        const float4 w4 = __ldg(reinterpret_cast<const float4*>(Wc + l0));
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(zc + l0));
        const float4 k4 = __ldg(reinterpret_cast<const float4*>(zk + l0));
        const float xv[4] = {x.x, x.y, x.z, x.w}, gv[4] = {g4.x, g4.y, g4.z, g4.w};
        const float rv[4] = {r4.x, r4.y, r4.z, r4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w};
        const float cv[4] = {c4.x, c4.y, c4.z, c4.w}, kv[4] = {k4.x, k4.y, k4.z, k4.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float xc = xv[j] - gv[j];
          float v = Cc * (xv[j] - rv[j]) - wv[j];
          v = fmaf(an, xc - cv[j], v);
          v = fmaf(bn, xc - kv[j], v);
          o[j] = scale * v;
        }
        if (a.vec_out && l0 + 3 < a.d) {
          *reinterpret_cast<float4*>(out + l0) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (l0 + j < a.d) out[l0 + j] = o[j];
        }
      }
    } else {
      float ss = 0.f;
      for (int l0 = 4 * lane; l0 < a.dz; l0 += 128) {
        const float4 x = load4<DT>(a.X, m, l0, a.d, a.ldx, a.cs, a.vec);
        ss += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
      // g_l = -(1/N)[al nc muh_c + be nk muh_k + W_c + C_c rhat_c],  muh = mu' + g
      // (16-byte loads of the dz-long, zero-padded per-cluster vectors)
      const float an = al * nc, bn = has_k ? be * nk : 0.f;
      auto gvec = [&](int l0, float (&gv)[4]) {
        const float4 g4 = __ldg(reinterpret_cast<const float4*>(a.gf + l0));
        const float4 r4 = __ldg(reinterpret_cast<const float4*>(rc + l0));
        const float4 w4 = __ldg(reinterpret_cast<const float4*>(Wc + l0));
        const float4 c4 = __ldg(reinterpret_cast<const float4*>(zc + l0));
        const float4 k4 = __ldg(reinterpret_cast<const float4*>(zk + l0));
        const float G[4] = {g4.x, g4.y, g4.z, g4.w}, R[4] = {r4.x, r4.y, r4.z, r4.w};
        const float W[4] = {w4.x, w4.y, w4.z, w4.w}, C[4] = {c4.x, c4.y, c4.z, c4.w};
        const float Kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float g = fmaf(Cc, R[j], W[j]);
          g = fmaf(an, C[j] + G[j], g);
          g = fmaf(bn, Kv[j] + G[j], g);
          gv[j] = -g * inv_n;
        }
      };
      float proj = 0.f;
      for (int l0 = 4 * lane; l0 < a.dz; l0 += 128) {
        const float4 x = load4<DT>(a.X, m, l0, a.d, a.ldx, a.cs, a.vec);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        float gv[4];
        gvec(l0, gv);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (l0 + j < a.d) proj = fmaf(xv[j] * inv, gv[j], proj);
      }
      for (int o = 16; o > 0; o >>= 1) proj += __shfl_xor_sync(0xffffffffu, proj, o);
      const float sc = float(gsd) * inv;
      for (int l0 = 4 * lane; l0 < a.dz; l0 += 128) {
        const float4 x = load4<DT>(a.X, m, l0, a.d, a.ldx, a.cs, a.vec);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        float gv[4], o[4];
        gvec(l0, gv);
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = sc * (gv[j] - xv[j] * inv * proj);
        if (a.vec_out && l0 + 3 < a.d) {
          *reinterpret_cast<float4*>(out + l0) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (l0 + j < a.d) out[l0 + j] = o[j];
        }
      }
    }
  }
}

bool vec_ok_b(const void* X, int32_t dtype, int64_t ldx) {
  const int esz = dtype == SIL_F32 ? 4 : dtype == SIL_BF16 ? 2 : 1;
  return (reinterpret_cast<uintptr_t>(X) % (4 * esz) == 0) && (ldx % 4 == 0);
}

}  // namespace

cudaError_t launch_backward_weights(const BackLaunch& b, float* w1, float* w2) {
  if (b.n == 0) return cudaSuccess;
  const unsigned grid = unsigned(std::min<int64_t>(cdiv(b.n, 256), int64_t(num_sms()) * 8));
  k_bw_weights<<<grid, 256, 0, b.stream>>>(b.n, b.labels, b.k, b.cl, b.sa, b.sb, b.skstar, w1, w2);
  return cudaGetLastError();
}

cudaError_t launch_backward_prep(const double* bw_w, const double* bw_p, int32_t k, int32_t d,
                                 float* Wf, float* Cf, cudaStream_t stream) {
  const int dz = int(round_up(d, 4));
  k_bw_prep<<<k, 128, 0, stream>>>(bw_w, bw_p, k, d, dz, Wf, Cf);
  return cudaGetLastError();
}

cudaError_t launch_backward_grad(const BackLaunch& b, const float* Wf, const float* Cf) {
  if (b.n == 0) return cudaSuccess;
  GradK g{};
  g.X = b.X;
  g.n = b.n;
  g.d = b.d;
  g.dz = int(round_up(b.d, 4));
  g.ldx = b.ldx;
  g.cs = b.cs;
  g.labels = b.labels;
  g.k = b.k;
  g.cosine = b.dist == SIL_COSINE;
  g.vec = vec_ok_b(b.X, b.dtype, b.ldx);
  g.cl = b.cl;
  g.zf = b.zf;
  g.gf = b.gf;
  g.rs = b.rs;
  g.Wf = Wf;
  g.Cf = Cf;
  g.sa = b.sa;
  g.sb = b.sb;
  g.skstar = b.skstar;
  g.grad_S = b.grad_S;
  g.dX = b.dX;
  g.lddx = b.lddx;
  g.vec_out = (reinterpret_cast<uintptr_t>(b.dX) % 16 == 0) && (b.lddx % 4 == 0);
  const int nv = int(cdiv(g.dz, 128));
  if (b.idx && nv <= 2) {
    // rows in the order of the dual pass 1's sort
    g.idx = b.idx;
    g.widx = b.widx;
    g.w2 = b.w2;
    g.bstart = b.bstart;
    const int per_sm = nv == 1 ? 3 : 2;  // CTAs per SM (the launch bounds)
    const int64_t warps = int64_t(num_sms()) * per_sm * 8;
    g.wchunk = round_up(std::max<int64_t>(64, cdiv(b.n, warps * 4)), 32);
    g.nitems = cdiv(b.n, g.wchunk);
    const unsigned sgrid =
        unsigned(std::max<int64_t>(1, std::min<int64_t>(int64_t(num_sms()) * per_sm, cdiv(g.nitems, 8))));
    auto go = [&](auto fn) {
      fn<<<sgrid, 256, 0, b.stream>>>(g);
      return cudaGetLastError();
    };
    const bool cs = g.cosine != 0;
    switch (b.dtype) {
      case SIL_F32:
        return nv == 1 ? (cs ? go(k_bw_grad_sorted<SIL_F32, 1, true>) : go(k_bw_grad_sorted<SIL_F32, 1, false>))
                       : (cs ? go(k_bw_grad_sorted<SIL_F32, 2, true>) : go(k_bw_grad_sorted<SIL_F32, 2, false>));
      case SIL_BF16:
        return nv == 1 ? (cs ? go(k_bw_grad_sorted<SIL_BF16, 1, true>) : go(k_bw_grad_sorted<SIL_BF16, 1, false>))
                       : (cs ? go(k_bw_grad_sorted<SIL_BF16, 2, true>) : go(k_bw_grad_sorted<SIL_BF16, 2, false>));
      default:
        return nv == 1 ? (cs ? go(k_bw_grad_sorted<SIL_FP8_E4M3, 1, true>)
                             : go(k_bw_grad_sorted<SIL_FP8_E4M3, 1, false>))
                       : (cs ? go(k_bw_grad_sorted<SIL_FP8_E4M3, 2, true>)
                             : go(k_bw_grad_sorted<SIL_FP8_E4M3, 2, false>));
    }
  }
  const unsigned grid = unsigned(std::min<int64_t>(cdiv(b.n, 8), int64_t(num_sms()) * 16));
  switch (b.dtype) {
    case SIL_F32: k_bw_grad<SIL_F32><<<grid, 256, 0, b.stream>>>(g); break;
    case SIL_BF16: k_bw_grad<SIL_BF16><<<grid, 256, 0, b.stream>>>(g); break;
    default: k_bw_grad<SIL_FP8_E4M3><<<grid, 256, 0, b.stream>>>(g); break;
  }
  return cudaGetLastError();
}

}  // namespace sil
