// Pass 2 for FP32 rows of 32..64 columns on the tensor cores in TF32, with
// every reported distance exact in FP32.
//
// The K dot products x_i . mu'_k of Eq. 10/11 (and x_i . Omega_k of Eq.
// 17/18, through x_hat) are the GEMM X . Z^T.  The FP32 tile that TMA writes
// into shared memory with the 128-byte swizzle is already the K-major operand
// layout of tcgen05.mma kind::tf32, so the tensor core reads the rows exactly
// as they arrive: nothing converts or splits them.  TF32 keeps 10 mantissa
// bits of each operand, so the GEMM only RANKS the clusters; the values
// reported are recomputed in FP32 in the difference form:
//   a_i = an_c ||x' - mu'_c||^2 + aw_c                 (own cluster, n_c - 1)
//   b_i = min over candidates k of ||x' - mu'_k||^2 + W_k / n_k
// with x' = x inv - g (inv = 1/||x|| for cosine, else 1; g the global mean).
//
// Candidates.  The ranked value of cluster k is v_k = cb_k - 2 inv acc_k with
// acc_k the TF32 product x . mu'_k and cb_k = ||mu'_k||^2 + W_k/n_k + 2 g.mu'_k,
// so that v_k + ||x'||^2 is the mean squared distance of Eq. 11.  Each TF32
// operand is within 2^-10 (relative) of its FP32 value, so every product is
// within 2^-9 (1 + 2^-11) of x_l mu'_kl, and with FP32 accumulation of at most
// 64 terms |acc_k - x.mu'_k| <= 2^-9 (1 + 2^-7) ||x|| ||mu'_k|| (Cauchy-
// Schwarz).  With R = max_k ||mu'_k|| over the block and C = max |cb_k|,
//   |v_k - v_k(exact)| <= E = 2^-8 (1 + 2^-6) inv ||x|| R + 2^-22 (C + 2 inv ||x|| R),
// the last term covering the FP32 roundings of cb_k and of the FMA.  If k* is
// the true nearest cluster and m the smallest ranked value over k != own,
// v_k* <= v_k*(exact) + E <= v_j(exact) + E <= v_j + 2E for every j, so k* is
// among the clusters with v_k <= m + 2E.  All of them are recomputed exactly
// and b_i is the smallest; on the at-scale recipe that is one or two
// clusters per point.
//
// One persistent CTA per SM (grid.y = cluster blocks of at most 256; with
// several blocks each writes its block's nearest exact distance per point and
// the combine kernel of the split-precision path finishes s_i), warp-
// specialised:
//   warp 0       TMA producer: the block's centroids (FP32, swizzled) once,
//                then X tiles (128 rows) and their labels into a ring of stages
//   warp 1       TMEM allocation and single-thread tcgen05.mma issue
//   warps 2..    G epilogue groups of 4 warps; group g takes tiles g, g + G, ...
//                and owns TMEM accumulator g.  Each thread owns one row: it
//                copies the row from the stage into registers (and releases
//                the stage once the MMA is done with it), forms the exact a_i,
//                reads the K ranked values from TMEM twice (minimum, then the
//                candidate mask), recomputes the candidates and finishes s_i.
// Every wait is bounded (SIL_ETIMEOUT); on a timeout every role stops,
// in-flight copies and MMAs are waited for (bounded) and TMEM is freed.
#include <algorithm>
#include <cstdlib>

#include "sil_internal.cuh"
#include "tcgen05.cuh"
#include "tma.cuh"

namespace sil {

namespace {

constexpr int kTM = 128;               // rows per tile = TMEM lanes
constexpr int kAtom = kTM * 128;       // 128 rows x 128 bytes (32 FP32 columns), 128-byte swizzle
constexpr int kMaxBlockN = 256;        // clusters per block (MMA N)
constexpr int kSmemMax = 227 * 1024;
constexpr int kMaxStages = 8;
constexpr int kOwnElsewhere = -1;
constexpr int kRowInvalid = -0x7fffffff - 1;

// Shared memory (byte offsets from a 1024-aligned base).
struct T32Smem {
  int z, xs, xs_stride, cb, cl, g, red, bars, total;
};

__host__ __device__ inline T32Smem t32_smem(int dp, int kp, int ns, int groups) {
  const int nat = dp / 32;
  T32Smem s;
  int o = 0;
  s.z = o;
  o += nat * kp * 128;  // kp is a multiple of 16: every atom stays 1024-aligned
  o = (o + 1023) & ~1023;
  s.xs = o;
  s.xs_stride = nat * kAtom + 1024;  // + the tile's labels (512 bytes), keeps 1024 alignment
  o += ns * s.xs_stride;
  s.cb = o;
  o += kp * 4;
  o = (o + 15) & ~15;
  s.cl = o;
  o += kp * 16;
  s.g = o;
  o += dp * 4;
  s.red = o;
  o += 32 * 4;
  o = (o + 15) & ~15;
  s.bars = o;
  o += 8 * (2 * ns + 2 * groups + 1) + 16;  // + TMEM base, abort flag
  s.total = o + 1024;                       // slack for aligning the dynamic base
  return s;
}

struct T32K {
  int64_t n;
  int32_t d, k, kp, nblk, acc_cols, tmem_cols, ns, dz;
  int32_t cosine, rms;
  float scale;
  const float* cb;     // [nblk * kp] ranking constants (+inf: empty or padding)
  const float4* clp;   // [nblk * kp] {an, aw, W/n, n}
  const float* zn;     // [nblk * kp] ||mu'_k||
  const float* gf;     // [dz] global centre
  float* s_out;
  float* sa;
  float* sb;
  int32_t* skstar;
  double* partials;
  float* pmin;    // [nblk][n] nearest exact distance of the block, NaN for a rejected row
  int32_t* parg;  // [nblk][n] its cluster (backward record)
  float* pown;    // [n] a_i before scaling, from the own cluster's block
  uint32_t* status;
};

struct T32Maps {
  CUtensorMap x, lab, z;
};

// ||x - z_k||^2 for the row in registers (DP values) and centroid row kr of
// the swizzled block in shared memory (zero padded past d).
template <int DP>
__device__ __forceinline__ float t32_dist(const float (&x)[DP], const unsigned char* zs, int kp, int kr) {
  float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
#pragma unroll
  for (int at = 0; at < DP / 32; ++at) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float4 z = *reinterpret_cast<const float4*>(zs + at * kp * 128 + sw128(kr, c));
      const float2 da = __fadd2_rn(make_float2(x[32 * at + 4 * c], x[32 * at + 4 * c + 1]), make_float2(-z.x, -z.y));
      const float2 db =
          __fadd2_rn(make_float2(x[32 * at + 4 * c + 2], x[32 * at + 4 * c + 3]), make_float2(-z.z, -z.w));
      acc0 = __ffma2_rn(da, da, acc0);
      acc1 = __ffma2_rn(db, db, acc1);
    }
  }
  return (acc0.x + acc1.x) + (acc0.y + acc1.y);
}

// Smallest ranked value v_k = cb_k + sc acc_k over the block's columns
// k != own of this warp's 32 TMEM lanes (accumulator at tb); 16 NLD columns
// per round trip (NLD loads in flight, one wait).  Warp-collective.
template <int NLD>
__device__ __forceinline__ float t32_min(uint32_t tb, int kp, const float* cbs, float sc, int own) {
  float best = INFINITY;
  const float2 sc2 = make_float2(sc, sc);
#pragma unroll
  for (int c0 = 0; c0 < kMaxBlockN; c0 += 16 * NLD) {
    if (c0 >= kp) break;
    uint32_t rv[NLD][16];
#pragma unroll
    for (int j = 0; j < NLD; ++j)
      if (c0 + 16 * j < kp) tmem_ld16_async(tb + uint32_t(c0 + 16 * j), rv[j]);
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
        for (int e = 0; e < 4; ++e)
          if (c0 + 16 * j + 4 * q4 + e != own) best = fminf(best, vals[e]);
      }
    }
  }
  return best;
}

// Candidate mask: bit e of mk[w] is set for column k = 32 w + e when
// v_k <= thr and k != own (KW words cover the block).  Warp-collective
// (every lane loads; lanes with nothing to find pass thr = -inf).
template <int NLD, int KW>
__device__ __forceinline__ void t32_mask(uint32_t tb, int kp, const float* cbs, float sc, int own, float thr,
                                         uint32_t (&mk)[KW]) {
  const float2 sc2 = make_float2(sc, sc);
#pragma unroll
  for (int w = 0; w < KW; ++w) mk[w] = 0u;
#pragma unroll
  for (int c0 = 0; c0 < 32 * KW; c0 += 16 * NLD) {
    if (c0 >= kp) break;
    uint32_t rv[NLD][16];
#pragma unroll
    for (int j = 0; j < NLD; ++j)
      if (c0 + 16 * j < kp) tmem_ld16_async(tb + uint32_t(c0 + 16 * j), rv[j]);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < NLD; ++j) {
      const int cj = c0 + 16 * j;  // 16 columns: one half of word cj / 32
      if (cj >= kp) break;
      reg_fence16(rv[j]);
      const float4* cb4 = reinterpret_cast<const float4*>(cbs + cj);
      uint32_t m = 0u;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const float4 cq = cb4[q4];
        const float2 va = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[j][4 * q4]), __uint_as_float(rv[j][4 * q4 + 1])),
                                     make_float2(cq.x, cq.y));
        const float2 vb = __ffma2_rn(sc2, make_float2(__uint_as_float(rv[j][4 * q4 + 2]), __uint_as_float(rv[j][4 * q4 + 3])),
                                     make_float2(cq.z, cq.w));
        const float vals[4] = {va.x, va.y, vb.x, vb.y};
#pragma unroll
        for (int e = 0; e < 4; ++e) m |= (vals[e] <= thr ? 1u : 0u) << (4 * q4 + e);
      }
      mk[cj / 32] |= m << (cj % 32);
    }
  }
  // the own cluster is never a candidate for b_i
#pragma unroll
  for (int w = 0; w < KW; ++w) mk[w] &= (own >> 5) == w ? ~(1u << (own & 31)) : ~0u;
}

// Lowest set column of the mask (and clears it); -1 when empty.
template <int KW>
__device__ __forceinline__ int t32_pop(uint32_t (&mk)[KW]) {
  int k = -1;
#pragma unroll
  for (int w = KW - 1; w >= 0; --w)
    if (mk[w] != 0u) k = 32 * w + __ffs(int(mk[w])) - 1;
  const uint32_t keep = ~(1u << (k & 31));
#pragma unroll
  for (int w = 0; w < KW; ++w) mk[w] &= (k >> 5) == w ? keep : ~0u;  // k = -1 matches no word
  return k;
}

template <int DP, int G, int KW>
__global__ void __launch_bounds__(64 + 128 * G, 1) k_score_tf32(T32K a, const __grid_constant__ T32Maps maps) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  constexpr int NAT = DP / 32;
  const T32Smem L = t32_smem(DP, a.kp, a.ns, G);
  uint64_t* xfull = reinterpret_cast<uint64_t*>(base + L.bars);
  uint64_t* xempty = xfull + a.ns;
  uint64_t* accfull = xempty + a.ns;
  uint64_t* accempty = accfull + G;
  uint64_t* zfull = accempty + G;
  uint32_t* tmem_base = reinterpret_cast<uint32_t*>(zfull + 1);
  volatile int* abort_flag = reinterpret_cast<int*>(tmem_base + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntiles = cdiv(a.n, kTM);
  const int my_tiles = blockIdx.x < ntiles ? int(cdiv(ntiles - blockIdx.x, gridDim.x)) : 0;
  const int kb0 = int(blockIdx.y) * a.kp;
  const int kblk = min(a.kp, a.k - kb0);
  const bool fused = a.nblk == 1;
  float* cbs = reinterpret_cast<float*>(base + L.cb);
  float4* cls = reinterpret_cast<float4*>(base + L.cl);
  float* gsm = reinterpret_cast<float*>(base + L.g);
  float* red = reinterpret_cast<float*>(base + L.red);

  if (threadIdx.x == 0) {
    for (int i = 0; i < a.ns; ++i) {
      mbar_init(&xfull[i], 1);
      mbar_init(&xempty[i], 4);  // the 4 warps of the group that read the tile
    }
    for (int i = 0; i < G; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], 4);
    }
    mbar_init(zfull, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < a.kp; i += blockDim.x) {
    cbs[i] = a.cb[kb0 + i];
    cls[i] = a.clp[kb0 + i];
  }
  for (int i = threadIdx.x; i < DP; i += blockDim.x) gsm[i] = i < a.dz ? a.gf[i] : 0.f;
  if (warp == 0) {
    // R and C of the candidate band over this block's clusters
    float rmax = 0.f, cmax = 0.f;
    for (int i = lane; i < kblk; i += 32) {
      rmax = fmaxf(rmax, a.zn[kb0 + i]);
      const float c = a.cb[kb0 + i];
      if (c < INFINITY) cmax = fmaxf(cmax, fabsf(c));
    }
    for (int o = 16; o > 0; o >>= 1) {
      rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    if (lane == 0) {
      red[30] = rmax;
      red[31] = cmax;
    }
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_base)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_base;
  const int lab_off = NAT * kAtom;

  if (warp == 0) {
    // ------------------------------------------------------- TMA producer
    if (lane == 0) {
      mbar_arrive_expect_tx(zfull, uint32_t(NAT * a.kp * 128));
      for (int at = 0; at < NAT; ++at) tma_load_2d(base + L.z + at * a.kp * 128, &maps.z, at * 32, kb0, zfull);
      int t = 0;
      for (; t < my_tiles; ++t) {
        const int s = t % a.ns;
        if (!tc_wait(&xempty[s], ((t / a.ns) & 1) ^ 1, abort_flag, a.status)) break;
        unsigned char* xs = base + L.xs + s * L.xs_stride;
        const int32_t row0 = int32_t((blockIdx.x + int64_t(t) * gridDim.x) * kTM);
        mbar_arrive_expect_tx(&xfull[s], uint32_t(NAT * kAtom + kTM * 4));
        for (int at = 0; at < NAT; ++at) tma_load_2d(xs + at * kAtom, &maps.x, at * 32, row0, &xfull[s]);
        tma_load_1d(xs + lab_off, &maps.lab, row0, &xfull[s]);
      }
      if (*abort_flag) {
        // wait (bounded) for every copy issued and not consumed
        const int first = t - a.ns > 0 ? t - a.ns : 0;
        for (int u = first; u < t; ++u) mbar_wait(&xfull[u % a.ns], uint32_t((u / a.ns) & 1));
        mbar_wait(zfull, 0);
      }
    }
  } else if (warp == 1) {
    // --------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_tf32(kTM, a.kp);
      const uint32_t zs = smem_u32(base + L.z);
      int t = 0;
      bool ok = tc_wait(zfull, 0, abort_flag, a.status);
      for (; ok && t < my_tiles; ++t) {
        const int s = t % a.ns, acc = t % G;
        if (!tc_wait(&xfull[s], (t / a.ns) & 1, abort_flag, a.status)) break;
        if (!tc_wait(&accempty[acc], ((t / G) & 1) ^ 1, abort_flag, a.status)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem + uint32_t(acc * a.acc_cols);
        const uint32_t xa = smem_u32(base + L.xs + s * L.xs_stride);
#pragma unroll
        for (int at = 0; at < NAT; ++at) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {  // K-steps of 8 TF32 = 32 bytes of each row
            umma_tf32(d_tmem, umma_desc_sw128(xa + uint32_t(at * kAtom + ks * 32)),
                      umma_desc_sw128(zs + uint32_t(at * a.kp * 128 + ks * 32)), idesc, (at | ks) != 0);
          }
        }
        umma_commit(&accfull[acc]);
      }
      if (*abort_flag && t > 0) {
        // the last committed accumulator must be complete before TMEM is freed
        const int u = t - 1;
        mbar_wait(&accfull[u % G], uint32_t((u / G) & 1));
      }
    }
  } else {
    // ------------------------------------------------- epilogue groups
    const int gi = (warp - 2) >> 2;  // group: tiles gi, gi + G, ...; accumulator gi
    const int q = warp & 3;          // the TMEM lane quarter this warp may access
    const int r = q * 32 + lane;     // tile row = TMEM lane
    const float R = red[30], C = red[31];
    const unsigned char* zsm = base + L.z;
    bool zready = false;
    float tsum = 0.f;
    int j = 0;
    for (int t = gi; t < my_tiles; t += G, ++j) {
      const int s = t % a.ns;
      if (!zready) {
        if (!tc_wait(zfull, 0, abort_flag, a.status)) break;
        zready = true;
      }
      if (!tc_wait(&xfull[s], (t / a.ns) & 1, abort_flag, a.status)) break;
      const unsigned char* xs = base + L.xs + s * L.xs_stride;
      const int own = reinterpret_cast<const int32_t*>(xs + lab_off)[r];
      const int64_t row = (blockIdx.x + int64_t(t) * gridDim.x) * kTM + r;
      float x[DP];
#pragma unroll
      for (int at = 0; at < NAT; ++at) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(xs + at * kAtom + sw128(r, c));
          x[32 * at + 4 * c + 0] = v.x;
          x[32 * at + 4 * c + 1] = v.y;
          x[32 * at + 4 * c + 2] = v.z;
          x[32 * at + 4 * c + 3] = v.w;
        }
      }
      bool valid = row < a.n;
      if (valid && (own < 0 || own >= a.k)) {
        set_status(a.status, SIL_ELABEL);
        valid = false;
      }
      float2 xx2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < DP; c += 2) xx2 = __ffma2_rn(make_float2(x[c], x[c + 1]), make_float2(x[c], x[c + 1]), xx2);
      const float xx = xx2.x + xx2.y;
      float inv = 1.f;
      if (a.cosine) {
        if (valid && !(xx > 0.f)) {
          set_status(a.status, SIL_EZERONORM);
          valid = false;
        }
        inv = xx > 0.f ? rsqrtf(xx) : 0.f;
      }
      const float nxi = a.cosine ? 1.f : sqrtf(xx);  // ||x|| inv (the band's scale)
      // x' = x inv - g, in place
      const float2 inv2 = make_float2(inv, inv);
#pragma unroll
      for (int c = 0; c < DP; c += 4) {
        const float4 g = *reinterpret_cast<const float4*>(gsm + c);
        const float2 pa = __ffma2_rn(make_float2(x[c], x[c + 1]), inv2, make_float2(-g.x, -g.y));
        const float2 pb = __ffma2_rn(make_float2(x[c + 2], x[c + 3]), inv2, make_float2(-g.z, -g.w));
        x[c] = pa.x;
        x[c + 1] = pa.y;
        x[c + 2] = pb.x;
        x[c + 3] = pb.y;
      }
      const int ol = own - kb0;
      const bool in_blk = valid && ol >= 0 && ol < kblk;
      float aown = 0.f;
      int code = valid ? kOwnElsewhere : kRowInvalid;
      if (in_blk) {
        const float4 co = cls[ol];
        aown = fmaf(co.x, t32_dist<DP>(x, zsm, a.kp, ol), co.y);
        code = co.w < 1.5f ? -2 - ol : ol;  // singleton: s_i = 0, b_i still reported
      }
      const int olx = in_blk ? ol : -1;  // column excluded from b_i
      if (!tc_wait(&accfull[gi], j & 1, abort_flag, a.status)) break;
      tc_fence_after();
      // the row is in registers and the MMA has read the stage: release it.
      // The refill is an async-proxy (TMA) write after these generic-proxy
      // reads, so the reads are fenced against it first.
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&xempty[s]);
      const uint32_t tb = tmem + uint32_t(gi * a.acc_cols) + (uint32_t(q * 32) << 16);
      const float sc = -2.f * inv;
      constexpr int NLD = G >= 3 ? 1 : 2;  // TMEM loads in flight (registers: the row is held)
      const float m = t32_min<NLD>(tb, a.kp, cbs, sc, olx);
      const float xr = nxi * R;
      const float band = 2.f * (0.00396728515625f * xr + 2.384185791015625e-7f * (C + 2.f * xr));
      const float thr = (valid && m < INFINITY) ? m + band : -INFINITY;
      uint32_t mk[KW];
      t32_mask<NLD, KW>(tb, a.kp, cbs, sc, olx, thr, mk);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accempty[gi]);
      // exact distances of the candidates, lowest index first (ties keep it)
      float dk = INFINITY;
      int kb = -1;
      for (;;) {
        const int kc = t32_pop<KW>(mk);
        if (!__any_sync(0xffffffffu, kc >= 0)) break;
        if (kc >= 0) {
          const float v = cls[kc].z + t32_dist<DP>(x, zsm, a.kp, kc);
          if (v < dk) {
            dk = v;
            kb = kc;
          }
        }
      }
      const bool row_ok = code != kRowInvalid;
      if (row < a.n) {
        if (fused) {
          float av = 0.f, bv = INFINITY, sv = 0.f;
          if (row_ok) {
            const bool has_b = dk < INFINITY;
            av = fmaxf(0.f, a.scale * aown);
            bv = has_b ? fmaxf(0.f, a.scale * dk) : INFINITY;
            if (code >= 0 && has_b) sv = sil_eq2(av, bv, a.rms != 0);
            if (!has_b) kb = -1;
          } else {
            kb = -1;
          }
          if (a.s_out) a.s_out[row] = sv;
          if (a.sa) {
            a.sa[row] = av;
            a.sb[row] = bv;
            a.skstar[row] = kb;
          }
          tsum += sv;
        } else {
          const int64_t o = int64_t(blockIdx.y) * a.n + row;
          a.pmin[o] = row_ok ? dk : __int_as_float(0x7fc00000);
          if (a.parg) a.parg[o] = (row_ok && kb >= 0) ? kb0 + kb : -1;
          if (olx >= 0) a.pown[row] = aown;
        }
      }
    }
    if (fused) {
      for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
      if (lane == 0) red[warp - 2] = tsum;
      asm volatile("bar.sync 1, %0;" ::"n"(128 * G) : "memory");
      if (warp == 2 && lane == 0) {
        double p = 0.0;
        for (int w = 0; w < 4 * G; ++w) p += double(red[w]);
        a.partials[blockIdx.x] = p;
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// Centroids, ranking constants and per-cluster terms of the kernel above
// (one warp per cluster row):
//   z32[k][c] = mu'_k,c (zero padded to dp columns and kpad rows),
//   cb[k] = bias_k + 2 g.mu'_k (+inf for empty clusters and padding),
//   zn[k] = ||mu'_k||, clp[k] = {an_k, aw_k, W_k / n_k, n_k}.
__global__ void k_t32_pack(const float* zf, const float4* cl, const double* g, int32_t k, int32_t d, int32_t dz,
                           int32_t dp, float* z32, float* cb, float* zn, float4* clp) {
  const int kk = blockIdx.x;
  double dot = 0.0;
  float nrm = 0.f;
  for (int c = threadIdx.x; c < dp; c += blockDim.x) {
    const float z = (kk < k && c < dz) ? zf[int64_t(kk) * dz + c] : 0.f;
    z32[int64_t(kk) * dp + c] = z;
    if (c < d) dot += g[c] * double(z);
    nrm = fmaf(z, z, nrm);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dot += __shfl_xor_sync(0xffffffffu, dot, o);
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  }
  if (threadIdx.x == 0) {
    float v = INFINITY;
    float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kk < k) {
      const float4 co = cl[kk];
      if (co.w > 0.5f) v = float(double(co.x) + 2.0 * dot);
      c4 = make_float4(co.y, co.z, co.y > 0.f ? co.z / co.y : 0.f, co.w);
    }
    cb[kk] = v;
    zn[kk] = sqrtf(nrm);
    clp[kk] = c4;
  }
}

struct T32Plan {
  int dp, kp, nblk, acc_cols, tmem_cols, groups, ns, smem;
};

int pow2_ge(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

bool t32_plan(int32_t d, int32_t k, T32Plan* p) {
  if (d < 32 || d > 64 || k < 1) return false;
  T32Plan q{};
  q.dp = d <= 32 ? 32 : 64;
  q.nblk = int(cdiv(k, kMaxBlockN));
  q.kp = int(round_up(cdiv(k, q.nblk), 16));
  q.acc_cols = pow2_ge(q.kp);
  // epilogue groups: as many as TMEM holds accumulators for, at most 4 (rows
  // of 32 columns) or 3 (64 columns: the row is kept in 64 registers)
  q.groups = std::min(q.dp == 32 ? 4 : 3, 512 / q.acc_cols);
  q.tmem_cols = pow2_ge(q.groups * q.acc_cols);
  q.ns = 0;
  for (int ns = kMaxStages; ns >= 2; --ns)
    if (t32_smem(q.dp, q.kp, ns, q.groups).total <= kSmemMax) {
      q.ns = ns;
      break;
    }
  if (q.ns == 0) return false;
  q.smem = t32_smem(q.dp, q.kp, q.ns, q.groups).total;
  *p = q;
  return true;
}

}  // namespace

bool t32_serves(int32_t dtype, int32_t d, int32_t k) {
  T32Plan p;
  return dtype == SIL_F32 && t32_plan(d, k, &p);
}

bool t32_eligible(int32_t dtype, int64_t n, int32_t d, int64_t ldx, int32_t k, const void* X, const int32_t* labels) {
  if (dtype != SIL_F32 || n <= 0 || n >= (int64_t(1) << 31)) return false;
  if (reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(labels) % 16 || (ldx * 4) % 16) return false;
  T32Plan p;
  if (!t32_plan(d, k, &p)) return false;
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
  return major == 10;
}

size_t t32_pack_bytes(int32_t k, int32_t d) {
  if (d < 32 || d > 64) return 0;
  const size_t kpad = size_t(round_up(std::max(k, 16), 16)) + kMaxBlockN;
  const size_t dp = d <= 32 ? 32 : 64;
  return align256(kpad * dp * 4) + 3 * align256(kpad * 4) + align256(kpad * 16);
}

size_t t32_partial_bytes(int64_t n, int32_t d, int32_t k) {
  T32Plan p;
  if (n <= 0 || !t32_plan(d, k, &p) || p.nblk == 1) return 0;
  const size_t N = size_t(n), G = size_t(p.nblk);
  return align256(G * N * 4) * 2 + align256(N * 4);
}

cudaError_t launch_score_tf32(const ScoreLaunch& s, const double* g, void* pack, void* partial_ws,
                              size_t partial_bytes, uint32_t* status) {
  T32Plan plan;
  if (!t32_plan(s.d, s.k, &plan)) return cudaErrorInvalidValue;
  const size_t N = size_t(s.n), NB = size_t(plan.nblk);
  if (plan.nblk > 1 && align256(NB * N * 4) * 2 + align256(N * 4) > partial_bytes) return cudaErrorInvalidValue;
  const int kpad = plan.nblk * plan.kp;
  const int dz = int(round_up(s.d, 4));
  char* pk = static_cast<char*>(pack);
  float* z32 = reinterpret_cast<float*>(pk);
  pk += align256(size_t(kpad) * plan.dp * 4);
  float* cb = reinterpret_cast<float*>(pk);
  pk += align256(size_t(kpad) * 4);
  float* zn = reinterpret_cast<float*>(pk);
  pk += align256(size_t(kpad) * 4);
  pk += align256(size_t(kpad) * 4);  // spare
  float4* clp = reinterpret_cast<float4*>(pk);
  k_t32_pack<<<kpad, 32, 0, s.stream>>>(s.zf, s.cl, g, s.k, s.d, dz, plan.dp, z32, cb, zn, clp);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;

  T32Maps maps{};
  if (!encode_tmap_2d(&maps.x, s.X, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, uint64_t(s.d), uint64_t(s.n),
                      uint64_t(s.ldx) * 4, 32, kTM, CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_tmap_1d(&maps.lab, s.labels, CU_TENSOR_MAP_DATA_TYPE_INT32, uint64_t(s.n), kTM) ||
      !encode_tmap_2d(&maps.z, z32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, uint64_t(plan.dp), uint64_t(kpad),
                      uint64_t(plan.dp) * 4, 32, uint32_t(plan.kp), CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;

  T32K k{};
  k.n = s.n;
  k.d = s.d;
  k.k = s.k;
  k.kp = plan.kp;
  k.nblk = plan.nblk;
  k.acc_cols = plan.acc_cols;
  k.tmem_cols = plan.tmem_cols;
  k.ns = plan.ns;
  k.dz = dz;
  k.cosine = s.dist == SIL_COSINE;
  k.rms = s.dist == SIL_EUCLIDEAN_RMS;
  k.scale = s.dist == SIL_COSINE ? 0.5f : 1.f;
  k.cb = cb;
  k.clp = clp;
  k.zn = zn;
  k.gf = s.gf;
  k.s_out = s.s_out;
  k.sa = s.sa;
  k.sb = s.sb;
  k.skstar = s.skstar;
  k.partials = s.partials;
  k.status = status;
  const bool save = s.sa != nullptr;
  if (plan.nblk > 1) {
    char* p = static_cast<char*>(partial_ws);
    k.pmin = reinterpret_cast<float*>(p);
    k.parg = save ? reinterpret_cast<int32_t*>(p + align256(NB * N * 4)) : nullptr;
    k.pown = reinterpret_cast<float*>(p + 2 * align256(NB * N * 4));
  }
  const int64_t ntiles = cdiv(s.n, kTM);
  const int per_block = std::max(1, num_sms() / plan.nblk);
  const dim3 grid(unsigned(std::min<int64_t>(ntiles, per_block)), unsigned(plan.nblk));
  auto launch = [&](auto fn, int groups) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, 64 + 128 * groups, plan.smem, s.stream>>>(k, maps);
    return cudaGetLastError();
  };
  cudaError_t e = cudaErrorInvalidValue;
  const bool narrow_k = plan.kp <= 128;  // candidate masks of 4 words
  if (plan.dp == 32) {
    if (plan.groups == 4) e = launch(k_score_tf32<32, 4, 4>, 4);  // kp <= 128
    else if (plan.groups == 2) e = launch(k_score_tf32<32, 2, 8>, 2);
  } else {
    if (plan.groups == 3) e = launch(k_score_tf32<64, 3, 4>, 3);  // kp <= 128
    else if (plan.groups == 2) e = narrow_k ? launch(k_score_tf32<64, 2, 4>, 2) : launch(k_score_tf32<64, 2, 8>, 2);
  }
  if (e != cudaSuccess) return e;
  if (plan.nblk == 1) {
    *s.n_partials = int(grid.x);
    return cudaSuccess;
  }
  return launch_tc_combine(s.n, s.k, plan.nblk, s.labels, s.cl, k.scale, k.rms, k.pmin, save ? k.parg : nullptr,
                           k.pown, s.s_out, s.sa, s.sb, s.skstar, s.partials, s.stream, s.n_partials);
}

}  // namespace sil
