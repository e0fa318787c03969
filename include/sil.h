/*
 * sil.h -- C ABI of libsil, a GB300 (sm_103a) implementation of the
 * linear-complexity Silhouette of Gaido, "Distributed Silhouette Algorithm:
 * Evaluating Clustering on Big Data" (arXiv 2303.14102).
 *
 * The Silhouette of a clustering (Sec. II, Eq. 1-2): for every point i with
 * label c, a_i is its mean distance to the other members of c, b_i the
 * smallest mean distance to another non-empty cluster, s_i = (b_i - a_i) /
 * max(a_i, b_i), and S = sum_i s_i / N.  The paper (Sec. III) removes the
 * O(N^2) pairwise work: for the squared Euclidean distance (Eq. 4-11) and the
 * cosine distance (Eq. 12-18) the mean distance from a point to a cluster is a
 * closed form in per-cluster aggregates (count, sum of vectors, sum of
 * squared norms -- or the sum of normalised vectors for cosine), which one
 * pass over the data produces.  This library runs that as two GPU passes:
 *
 *   sil_aggregate       pass 1, a segmented per-cluster reduction (Eq. 6, 8, 16)
 *   sil_score           pass 2, every point against all K aggregates
 *                       (Eq. 11 / Eq. 18), own cluster over N_c - 1, b_i the
 *                       minimum over the other clusters, s_i and the mean S
 *   sil_score_backward  dS/dX with labels fixed (no counterpart in the paper)
 *   sil_score_batched   S for many labelings of the same points
 *   sil_score_euclidean the exact (non-squared) Euclidean Silhouette by the
 *                       quadratic method of Sec. II, for moderate n
 *
 * Conventions shared by every entry point
 *   - Every pointer named as "device" must be memory the current CUDA device
 *     can read/write (cudaMalloc or torch CUDA tensors); "host" pointers are
 *     ordinary process memory.  The caller owns every buffer.  The library
 *     never allocates, never frees and never synchronises: each call only
 *     enqueues kernels (and, where stated, cudaMemsetAsync) on `stream`, a
 *     cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - X is row-major: row i starts at element i*ldx, ldx >= d.  dtype selects
 *     float32, bfloat16 or FP8 E4M3 storage; FP8 takes a per-column positive
 *     scale col_scale[d] (device, float32) and the value a kernel uses is
 *     q * col_scale[l].  Computation is FP32 per point with FP64 aggregates
 *     and an FP64 mean.
 *   - labels are int32 dense ids in [0, k); ids with no point are allowed
 *     and are not clusters.  A label outside [0, k) sets SIL_ELABEL in
 *     *dev_status and the row is ignored.
 *   - Return value: SIL_OK, or a host-side argument error (SIL_EINVAL,
 *     SIL_EWORKSPACE, SIL_EUNSUPPORTED) / launch error (SIL_ECUDA) detected
 *     before or while enqueueing; nothing is enqueued after an error.
 *   - dev_status (device, one uint32, nullable) receives data-dependent
 *     errors OR-ed in as bit flags (SIL_ELABEL, SIL_EDEGENERATE,
 *     SIL_EZERONORM, SIL_ETIMEOUT).  The library never clears it.  When such
 *     a flag is raised by a scoring call, S is written as NaN.  Kernels never
 *     trap or assert.
 *   - ws is a device workspace of at least sil_workspace_size(...) bytes,
 *     256-byte aligned.  Its contents are scratch between calls.
 *   - n < 2^31 (pass 1 sorts 32-bit row indices); larger n returns
 *     SIL_EUNSUPPORTED.
 */
#ifndef SIL_H_
#define SIL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Distance measures of Sec. III-A (squared Euclidean, Eq. 4) and Sec. III-B
 * (cosine distance 1 - cs, Eq. 12), and SIL_EUCLIDEAN_RMS, the approximation
 * of the Euclidean Silhouette that the Limitations section suggests: a_i and
 * b_i are the square roots of the point-to-cluster MEAN SQUARED Euclidean
 * distances (root mean square, >= the mean Euclidean distance), so that b_i's
 * cluster and everything before Eq. 2 are those of SIL_SQEUCLIDEAN (same
 * aggregates, same passes).  The exact Euclidean Silhouette has no aggregate
 * form.  sil_score_backward returns SIL_EUNSUPPORTED for SIL_EUCLIDEAN_RMS,
 * and its saved record holds the squared means. */
typedef enum { SIL_SQEUCLIDEAN = 0, SIL_COSINE = 1, SIL_EUCLIDEAN_RMS = 2 } sil_distance_t;

/* Storage type of X. */
typedef enum { SIL_F32 = 0, SIL_BF16 = 1, SIL_FP8_E4M3 = 2 } sil_dtype_t;

/* Return codes (single values) and device status flags (OR-ed bits). */
typedef enum {
  SIL_OK = 0,
  SIL_EINVAL = 1,        /* bad argument (null pointer, size, ldx < d, ...) */
  SIL_ELABEL = 2,        /* device flag: a label outside [0, k) */
  SIL_EDEGENERATE = 4,   /* device flag: fewer than two non-empty clusters */
  SIL_EZERONORM = 8,     /* device flag: cosine with an all-zero row */
  SIL_ECUDA = 16,        /* a CUDA launch or memset failed */
  SIL_ETIMEOUT = 32,     /* device flag: a bounded wait inside a kernel gave up */
  SIL_EWORKSPACE = 64,   /* ws is NULL, misaligned or smaller than required */
  SIL_EUNSUPPORTED = 128 /* valid arguments this library does not serve */
} sil_status_t;

/* Pass-2 implementation choice for sil_score. */
typedef enum {
  SIL_PATH_AUTO = 0,   /* library picks from (k, d, dtype): the split-precision
                          tensor kernel, or for float32 rows of 32..64 columns
                          and k <= 48 the TF32 kernel (faster there) */
  SIL_PATH_SIMT = 1,   /* FP32 FFMA with the centroids staged in shared memory */
  SIL_PATH_TENSOR = 2, /* tcgen05 tensor-core GEMM with a fused epilogue: the
                          split-precision kernel (BF16 hi/lo operands, a
                          ~FP32-accurate GEMM) */
  SIL_PATH_TENSOR_TF32 = 3 /* float32 rows of 32..64 columns only: clusters
                              ranked by a TF32 GEMM on the rows as stored, then
                              a_i and every cluster inside the GEMM's provable
                              error band recomputed exactly in FP32 */
} sil_path_t;

/* Flags of sil_aggregate. */
#define SIL_AGG_ACCUMULATE 1u /* add into count/s1/s2 instead of overwriting */

/* Bytes of workspace any call below needs for these sizes (batch = number of
 * labelings for sil_score_batched, 1 otherwise; k = the largest k). */
size_t sil_workspace_size(int64_t n, int32_t d, int32_t k, int32_t dtype, int32_t dist,
                          int32_t batch);

/* Bytes of the per-point record sil_score can save for the backward pass
 * (a_i and b_i as float32, the b_i argmin cluster as int32: 12 bytes/point). */
size_t sil_saved_size(int64_t n);

/*
 * Pass 1 (Sec. III-A Eq. 5-9 and its footnotes; Sec. III-B Eq. 15-16): the
 * per-cluster aggregates in one pass over X.
 *   count[k] (device int64)   N_k, the number of points with label k
 *   s1[k*d + l] (device f64)  squared Euclidean: Y_{k,l} = sum of x_{il}
 *                             (Eq. 8); cosine: Omega_{k,l} = sum of x_{il} /
 *                             ||x_i|| (Eq. 16)
 *   s2[k] (device f64)        squared Euclidean: Psi_k = sum of ||x_i||^2
 *                             (Eq. 6); cosine: sum of ||x_i/||x_i|| ||^2
 * These are exactly additive over any split of the rows, so aggregates of
 * several calls on disjoint row ranges can be merged by adding them (the
 * per-worker partial sums of the paper's distributed form); with
 * SIL_AGG_ACCUMULATE the call adds into the outputs instead of overwriting
 * them.  The rows are first counting-sorted by label (inside the
 * workspace); each warp then sums a run of one cluster's rows in FP32 on
 * values shifted by a per-cluster reference point and folds the run into
 * FP64 once.
 */
int sil_aggregate(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                  const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
                  int64_t* count, double* s1, double* s2, uint32_t flags, void* ws,
                  size_t ws_bytes, uint32_t* dev_status, void* stream);

/*
 * Pass 2 (Sec. III-A Eq. 10-11, Sec. III-B Eq. 17-18, Sec. II Eq. 1-2): score
 * every point from the aggregates of sil_aggregate over the SAME rows and
 * labels.  For point i with label c:
 *   a_i = mean distance to the other N_c - 1 members of c (0 if N_c = 1)
 *   b_i = min over non-empty k != c of the mean distance to cluster k
 *   s_i = (b_i - a_i) / max(a_i, b_i), 0 when N_c = 1 or max = 0
 *   S   = sum_i s_i / n   (S_out: device, one double; NaN on a data error)
 * s_out (device float[n], nullable) receives s_i.  saved (device,
 * sil_saved_size(n) bytes, nullable) receives a_i, b_i and the argmin of b_i
 * (lowest index on ties) for sil_score_backward.  N x K distances are never
 * stored.  path selects the pass-2 kernel (SIL_PATH_AUTO recommended).
 * Accuracy (FP32 arithmetic, FP64 aggregates and S): the tensor-core path
 * ranks the clusters by the expanded distance ||x'||^2 + bias_k - 2 x'.mu'_k;
 * for points where that form is ill-conditioned ((||x'|| + a bound on
 * ||mu'_k||)^2 above 6 times the point's smallest expanded distance) b_i is
 * recomputed from the nearest cluster in the difference form
 * ||x' - mu'_k||^2 + W_k / n_k, so that the rounding of the tensor-core sums
 * does not bias S.
 */
int sil_score(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
              const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
              const int64_t* count, const double* s1, const double* s2, float* s_out,
              double* S_out, void* saved, int32_t path, void* ws, size_t ws_bytes,
              uint32_t* dev_status, void* stream);

/*
 * Both passes of one labeling in one call: sil_aggregate into (count, s1, s2)
 * (device outputs, overwritten, as sil_aggregate documents them), then
 * sil_score from them on the same workspace, with the same s_out, S_out,
 * saved, path and results as those two calls.
 */
int sil_silhouette(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* col_scale,
                   const int32_t* labels, int32_t k, int32_t dist, int64_t* count, double* s1, double* s2,
                   float* s_out, double* S_out, void* saved, int32_t path, void* ws, size_t ws_bytes,
                   uint32_t* dev_status, void* stream);

/*
 * dS/dX with the labels fixed and b_i's argmin held at its value (the min
 * and max of Eq. 1 taken as subgradients).  grad_S (device, one double,
 * nullable = 1.0) scales the result, dX (device float32, row-major n x d,
 * row stride lddx >= d) receives grad_S * dS/dX.  saved is the record of
 * sil_score on the same inputs, or NULL to recompute it.  Cost: two passes
 * over X plus the write of dX (the pass-2 scores again when saved is NULL).
 */
int sil_score_backward(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                       const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
                       const int64_t* count, const double* s1, const double* s2,
                       const void* saved, const double* grad_S, float* dX, int64_t lddx,
                       void* ws, size_t ws_bytes, uint32_t* dev_status, void* stream);

/*
 * S for `batch` labelings of the same X.  labels is device int32 of
 * batch x n (labeling b at labels + b*ldl), k_host (host int32[batch]) the
 * number of label ids of each labeling, S_out (device double[batch]).
 * Equivalent to sil_aggregate + sil_score per labeling.  For float32 rows of
 * 32..64 columns, k <= 512 and 16-byte aligned rows (ldl a multiple of 4),
 * pass 1 and the finalisation run per labeling and the pass 2 of EVERY
 * labeling runs as one tensor-core launch (a CTA row per labeling block of
 * at most 256 clusters, the CTAs of all labelings streaming the same rows
 * of X); wider labelings' two blocks are combined by one more launch.  Other
 * shapes run the per-labeling launch sequence.  The workspace grows with
 * batch x n (two planes of per-block distances and one of a_i per labeling).
 */
int sil_score_batched(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                      const float* col_scale, const int32_t* labels, int64_t ldl,
                      const int32_t* k_host, int32_t batch, int32_t dist, double* S_out,
                      void* ws, size_t ws_bytes, uint32_t* dev_status, void* stream);

/*
 * The exact Euclidean Silhouette (d(x, y) = ||x - y||, not squared) by the
 * standard quadratic method of Sec. II (Eq. 1-3 evaluated pair by pair), for
 * the metric the linear method cannot serve exactly (Limitations section;
 * SIL_EUCLIDEAN_RMS is that section's linear-time approximation).  O(n^2 d)
 * work: meant for up to ~1e5 points.  For point i with label c:
 *   a_i = sum over the other members j of c of ||x_i - x_j|| / (n_c - 1)
 *   b_i = min over non-empty k != c of sum over j in k of ||x_i - x_j|| / n_k
 *   s_i and S as in sil_score (s_out, S_out, saved with the same layout).
 * Each distance is formed in FP32 from the coordinate differences (no
 * expanded-form cancellation); per-cluster sums are FP32 over runs of at most
 * 64 points and FP64 across them.  The rows are counting-sorted by label and
 * gathered into FP32 inside the workspace (sil_euclidean_workspace_size
 * bytes, 256-byte aligned).  d <= 128, otherwise SIL_EUNSUPPORTED.  A label
 * outside [0, k) sets SIL_ELABEL (its row gets s_i = 0) and fewer than two
 * non-empty clusters SIL_EDEGENERATE; either makes S NaN.  No aggregates are
 * needed: the call is self-contained.
 */
size_t sil_euclidean_workspace_size(int64_t n, int32_t d, int32_t k);
int sil_score_euclidean(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx, const float* col_scale,
                        const int32_t* labels, int32_t k, float* s_out, double* S_out, void* saved, void* ws,
                        size_t ws_bytes, uint32_t* dev_status, void* stream);

/*
 * S of rows scored in m disjoint chunks (Sec. II: S is the mean of s_i over
 * every point), from each chunk's S_out of sil_score: S_chunks (device
 * double[m]) and n_chunks (device int64[m], the chunks' row counts) give
 * *S_out (device double) = sum_c n_c S_c / sum_c n_c in FP64; NaN if a chunk
 * mean is NaN.  Returns SIL_EINVAL for m <= 0 or a NULL pointer.
 */
int sil_chunk_mean(const double* S_chunks, const int64_t* n_chunks, int32_t m, double* S_out, void* stream);

/*
 * Launch plan of the one-launch batched pass 2 (see sil_score_batched), for an
 * autotuner: ranges = CTAs per labeling block (1..64, each streaming an equal
 * share of the rows), a_buffers = A-operand buffers (2 or 4; 0 = the deepest
 * that fits).  Process-wide; returns SIL_EINVAL out of range.  Host-only.
 */
int sil_batched_plan_set(int32_t ranges, int32_t a_buffers);

/* Largest sizes sil_score_noalloc serves. */
#define SIL_NOALLOC_MAX_K 1024
#define SIL_NOALLOC_MAX_D 256

/*
 * sil_score without a workspace argument, for callers that cannot provide
 * device memory at the point they want a score -- for example code inside a
 * host framework that owns all device memory through its own pool, where a
 * raw cudaMalloc can fail or fragment that pool, or a plugin whose host
 * application forbids allocation on its hot path.  The paper has no
 * counterpart: this is a deployment convenience.
 *
 * Same arguments and results as sil_score (SIMT pass 2 only), minus ws and
 * ws_bytes.  Its scratch is one fixed device array inside the library
 * (about 1.1 MB, sized for k <= SIL_NOALLOC_MAX_K and d <= SIL_NOALLOC_MAX_D)
 * that stays reserved until the process exits.  The CUDA driver reserves it
 * when it loads that part of the library on a device: with lazy module
 * loading (the default of current drivers) during the first call on the
 * device, with CUDA_MODULE_LOADING=EAGER when the library is loaded.  So a
 * caller whose memory budget is fixed later makes one call at start-up;
 * after it, calls on that device allocate nothing.  Larger k or d return
 * SIL_EUNSUPPORTED with nothing enqueued.  The first call on a device (and
 * the first after its context is destroyed and re-created, e.g. by
 * cudaDeviceReset) looks up the array's device address with that device
 * current, so make it before any stream capture starts.  All calls on a
 * device share the array: calls whose GPU work overlaps race and must be
 * ordered by the caller.  Each call clears what must start at zero and
 * rewrites the rest.
 */
int sil_score_noalloc(const void* X, int32_t dtype, int64_t n, int32_t d, int64_t ldx,
                      const float* col_scale, const int32_t* labels, int32_t k, int32_t dist,
                      const int64_t* count, const double* s1, const double* s2, float* s_out,
                      double* S_out, void* saved, uint32_t* dev_status, void* stream);

/*
 * The cluster-block plan of the tensor-core pass 2 (sil_score with
 * SIL_PATH_TENSOR or AUTO) for this storage type and shape: *block_k =
 * clusters per block (the MMA N, a multiple of 16, at most 256) and
 * *n_blocks = blocks covering the k clusters.  With more than one block every
 * block is scored by its own CTAs and a combine kernel takes the minimum over
 * blocks (Eq. 3: b_i is a minimum over clusters, so it splits over any
 * partition of them).  Host-only arithmetic: no device is touched and the
 * answer does not say whether the current device can run the path.  Returns
 * SIL_OK, SIL_EINVAL (null outputs, bad dtype, d or k <= 0) or
 * SIL_EUNSUPPORTED (no plan fits in shared memory: d > 256 for float32
 * storage, whose rows wider than 128 columns are taken in 64-column chunks,
 * or d > 128 for BF16 and FP8).
 */
int sil_tensor_plan(int32_t dtype, int32_t d, int32_t k, int32_t* block_k, int32_t* n_blocks);

/*
 * Which tensor-core kernels serve this storage type and shape (on 16-byte
 * aligned X, labels and row stride; other inputs take the SIMT kernel): bit
 * SIL_TENSOR_KERNEL_SPLIT for the split-precision kernel that SIL_PATH_AUTO
 * and SIL_PATH_TENSOR run and whose launch plans the functions below
 * describe, bit SIL_TENSOR_KERNEL_TF32 for the kernel of SIL_PATH_TENSOR_TF32.
 * Host-only arithmetic; invalid arguments give 0.
 */
#define SIL_TENSOR_KERNEL_SPLIT 1
#define SIL_TENSOR_KERNEL_TF32 2
int sil_tensor_kernel(int32_t dtype, int32_t d, int32_t k);

/*
 * Launch plans of the split-precision tensor-core pass 2 (SIL_PATH_AUTO and
 * SIL_PATH_TENSOR) for one storage type and shape, for
 * an autotuner.  sil_tensor_plan_candidates writes up to max_plans feasible
 * plans (host int32[max_plans][5]: block_k, A-operand buffers, raw X stages,
 * 1 if the centroids are staged in shared memory for the own-cluster term,
 * rank_pass), best first by the library's cost model, and their number into
 * *n_plans.  rank_pass = 1 tracks each point's nearest cluster during the
 * pass over the GEMM results; rank_pass = 0 keeps only the minimum and looks
 * the cluster up again for the points whose b_i is recomputed in the
 * difference form (the ill-conditioned ones, see sil_score).  Both give the
 * same results; which is faster depends on how many points that is.
 * sil_tensor_plan_set makes one plan the choice for (dtype, d, k) in this
 * process (block_k = 0 returns the shape to the cost model); it returns
 * SIL_EINVAL for values out of range (including an odd number of A-operand
 * buffers or raw X stages for rows of up to 64 columns, whose kernels split the
 * tiles between two converter warpgroups) and SIL_EUNSUPPORTED when the plan does
 * not fit in shared memory.  Set plans before sizing the workspace: the
 * number of cluster blocks changes sil_workspace_size.  Host-only; safe to
 * call from several threads.
 */
int sil_tensor_plan_candidates(int32_t dtype, int32_t d, int32_t k, int32_t* plans, int32_t max_plans,
                               int32_t* n_plans);
int sil_tensor_plan_set(int32_t dtype, int32_t d, int32_t k, int32_t block_k, int32_t a_buffers,
                        int32_t x_stages, int32_t stage_centroids, int32_t rank_pass);

/*
 * Self-test of the library's failure detection, with no data and no
 * workspace: one small kernel waits on mbarriers that nothing completes,
 * through the same bounded waits the pass-1 and pass-2 kernels use, and
 * reports how each wait ended.  dev_out (device uint32[3], zeroed by the
 * caller) receives: [0] SIL_ETIMEOUT from the pass-2 wait once its limit
 * (1 s) passed; [1] SIL_ETIMEOUT from the pass-1 wait likewise; [2] 1 if a
 * second pass-2 wait, started half a limit later, gave up on the first one's
 * abort signal before its own limit.  The kernel runs about one second and
 * leaves the context usable.  Returns SIL_EINVAL for a NULL dev_out.
 */
int sil_selftest_bounded_wait(uint32_t* dev_out, void* stream);

/* Human-readable name of a return code or of one status flag. */
const char* sil_status_string(int32_t status);

/* Library version, major*10000 + minor*100 + patch. */
int32_t sil_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SIL_H_ */
