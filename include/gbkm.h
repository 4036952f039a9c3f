/*
 * gbkm.h -- C ABI of the GB300 (sm_103a) k-means hot-path library.
 *
 * The library computes the data-parallel core of the high-dimensional k-means
 * pipeline of "Solving k-means on High-dimensional Big Data" (Kappmeier,
 * Schmidt, Schmidt): projection of point blocks onto a low-rank subspace
 * (Section 2.2), k-means++ D^2 seeding (Section 1), Lloyd's assignment and
 * centroid steps (Section 1), clustering-feature sums and the k-means cost
 * (Section 2.1, Section 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Points are the ROWS of a row-major n x d matrix (leading dimension d).
 *    Centers are a row-major k x d FP32 matrix.  Labels are int32 in [0, k).
 *  - Every array argument is a DEVICE pointer owned by the caller, unless the
 *    argument's comment says "host".  Scalar outputs (costs, counters) are
 *    device pointers too, so that a whole Lloyd loop runs without a host
 *    synchronisation.  Optional outputs may be NULL.
 *  - Calls are asynchronous on the context's stream (gbkm_create /
 *    gbkm_set_stream).  The library allocates only its own grow-only
 *    workspace; the first call of a given size may allocate (and synchronise
 *    the stream while it grows), later calls of the same or smaller size do not.
 *  - Return value: GBKM_OK, or a negative gbkm_status.  Argument errors are
 *    detected before any launch and leave every output untouched;
 *    gbkm_last_error() then holds a message.  Conditions detected on the
 *    device (a bounded wait that timed out, a degenerate seeding input) are
 *    recorded in a device status word and reported by the next gbkm_sync().
 *  - n, d, k >= 1 unless stated otherwise; n * d < 2^40; k <= 65536.
 *  - Arithmetic: see each call.  Only cluster sums and costs use FP64.
 */
#ifndef GBKM_H
#define GBKM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbkm_ctx gbkm_ctx;

typedef enum {
    GBKM_OK = 0,
    GBKM_EINVAL = -1,         /* bad argument (size, NULL, alignment, dtype) */
    GBKM_ENOMEM = -2,         /* workspace allocation failed */
    GBKM_ECUDA = -3,          /* a CUDA runtime call failed (message in gbkm_last_error) */
    GBKM_ETIMEOUT = -4,       /* a bounded device-side wait gave up */
    GBKM_EUNSUPPORTED = -5,   /* shape or dtype outside what this build supports */
    GBKM_EDEGENERATE = -6,    /* k-means++: fewer than k points with positive D^2 */
    GBKM_ETOOBIG = -7         /* kmeans_update_noalloc: the problem needs more than its fixed scratch */
} gbkm_status;

typedef enum {
    GBKM_F32 = 0,       /* float */
    GBKM_BF16 = 1,      /* bfloat16, round to nearest even */
    GBKM_FP8E4M3 = 2    /* E4M3 (no inf, max 448) with one power-of-two FP32 scale per row block */
} gbkm_dtype;

typedef enum {
    GBKM_ENGINE_AUTO = 0,     /* tcgen05 where the shape allows it, else SIMT */
    GBKM_ENGINE_SIMT = 1,     /* CUDA-core FFMA tiles (FP32 operands only) */
    GBKM_ENGINE_TCGEN05 = 2   /* tensor-core tiles: TMA -> SMEM -> tcgen05.mma -> TMEM */
} gbkm_engine;

/* options of kmeans_assign */
typedef struct {
    int32_t compute;    /* gbkm_dtype of the distance-GEMM operands */
    int32_t engine;     /* gbkm_engine */
    int32_t recheck;    /* 1 (default): re-resolve certified near-ties exactly from FP32 data */
    int32_t center_terms; /* GBKM_BF16 only: 2 = centers as two BF16 terms (hi + lo, a second MMA),
                             which shrinks the near-tie bound where x's own rounding is small next
                             to the distances; 0 or 1 (default) = one term */
} gbkm_assign_opts;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context; the caller destroys it with gbkm_destroy. */
int gbkm_create(gbkm_ctx **out, int device, void *cuda_stream);
int gbkm_destroy(gbkm_ctx *ctx);
int gbkm_set_stream(gbkm_ctx *ctx, void *cuda_stream);
/* Message of the last error on this context ("" if none).  Owned by ctx. */
const char *gbkm_last_error(const gbkm_ctx *ctx);
/* Wait for the context's stream, then report (and clear) the device status
 * word: GBKM_OK, GBKM_ETIMEOUT, GBKM_EDEGENERATE or GBKM_ECUDA. */
int gbkm_sync(gbkm_ctx *ctx);
/* Number of this library's kernel launches issued on ctx since creation. */
int64_t gbkm_launch_count(const gbkm_ctx *ctx);
/* Library version as major*10000 + minor*100 + patch. */
int gbkm_version(void);

/* ------------------------------------------------------------------ A1: row norms */

/* xnorm[i] = ||x_i||^2 (Section 2.1: the sum-of-squares term of a clustering
 * feature), FP32 output from FP32 products summed in FP32 per lane and a warp
 * tree.  X: n x d FP32.  xnorm: n FP32. */
int kmeans_row_norms(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, float *xnorm);

/* ------------------------------------------------------------------ A0: operand quantisation */

/* Copy of X in a lower-precision operand format (precision form of the
 * distance and projection GEMMs; no paper counterpart).
 *   dtype == GBKM_BF16:    Xq is n x d bfloat16 (round to nearest even); scales, when not
 *     NULL, is n FP32 and receives each row's rounding residual ||x_i - Xq_i|| rounded
 *     up, which kmeans_assign uses for a narrower certified band.
 *   dtype == GBKM_FP8E4M3: Xq is n x d E4M3 bytes; scales is n x ceil(d/128) FP32,
 *     scale = 2^e with e the smallest integer such that the block's max |x| * 2^-e
 *     <= 448 (1 for an all-zero block); x ~= scale * e4m3(q), round to nearest even.
 * X: n x d FP32.  Xq must be 16-byte aligned. */
int kmeans_quantize(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, int32_t dtype,
                    void *Xq, float *scales);

/* ------------------------------------------------------------------ A0 + A1: ingest */

/* Page-locked host memory mapped into every device's address space, for kmeans_ingest
 * sources (the kernel reads it across the CPU-GPU link; no copy-engine transfer).
 * gbkm_host_alloc: *out receives a block of `bytes` bytes, or NULL with GBKM_ENOMEM.
 * gbkm_host_free: releases a block from gbkm_host_alloc (NULL is a no-op; any other
 * pointer returns GBKM_EINVAL).  The caller owns the block and frees it after the
 * last call that reads it has completed. */
int gbkm_host_alloc(size_t bytes, void **out);
int gbkm_host_free(void *p);

/* One read of a block of points feeding the rest of the path (Section 2.1's
 * sum-of-squares term and the BF16 operand copy, as kmeans_row_norms and
 * kmeans_quantize(GBKM_BF16, with scales) compute them):
 *   X_dev = X_src (NULL to skip), xnorm[i] = ||x_i||^2 (NULL to skip),
 *   Xq = bf16(X_src) (NULL to skip), resid[i] = ||x_i - Xq_i|| rounded up (NULL to
 *   skip; needs Xq).
 * X_src: n x d FP32, either device memory or a range inside one gbkm_host_alloc block
 * (checked exactly; any other host memory returns GBKM_EINVAL).  X_dev (16-byte
 * aligned, not X_src): n x d FP32 device memory; Xq (16-byte aligned): n x d bfloat16.
 * The sums run in the same order as those of kmeans_row_norms and kmeans_quantize on a
 * 16-byte-aligned copy, so xnorm, Xq and resid equal theirs bitwise. */
int kmeans_ingest(gbkm_ctx *ctx, const float *X_src, int64_t n, int64_t d, float *X_dev,
                  float *xnorm, void *Xq, float *resid);

/* ------------------------------------------------------------------ A2: block projection */

/* Randomised truncated SVD of a piece (Section 2.2: the best-fit subspace of
 * dimension ell is spanned by the top ell right singular vectors; computed, as in
 * the paper, by the randomised scheme of Halko, Martinsson and Tropp, which reduces
 * the columns by a random matrix, then the rows, and decomposes the small rest;
 * Section 2.3.2: weighted points enter as rows scaled by sqrt(w_i)):
 *   A' = diag(sqrt(w)) A, Y = A' Omega, Q = orth(Y) (CholeskyQR, twice),
 *   B = Q^T A' (s x d), V = the top ell right singular vectors of B.
 *   A: n x d FP32 row-major; w: n FP32 >= 0 or NULL; Omega: d x s FP32 row-major
 *   (the random matrix, e.g. independent N(0, 1) draws; s = ell + oversampling);
 *   16 <= s <= 128, s % 16 == 0, 1 <= ell <= s <= min(n, d).
 *   V: d x ell FP32 out, orthonormal columns in decreasing singular value, each
 *   column's entry of largest magnitude (lowest row on ties) positive.
 *   sigma: ell FP32 out (decreasing) or NULL.
 *   info: 1 int32 (device) or NULL; bit 0: a Cholesky pivot had to be clamped (A'
 *   of rank below s), bit 1: the Jacobi sweeps stopped at their cap (30); bits 8-15:
 *   the number of Jacobi sweeps run.
 * Arithmetic: FP32 products and sums for the passes over A, Gram matrices with
 * double-float accumulation, Cholesky in FP64, one-sided Jacobi in FP32. */
int kmeans_rsvd(gbkm_ctx *ctx, const float *A, int64_t n, int64_t d, const float *w,
                const float *Omega, int64_t s, int64_t ell, float *V, float *sigma,
                int32_t *info);

/* Projection of a block of points onto the span of V (Section 2.2: the best-fit
 * subspace projection A_l = U D_l V^T; here V is given, d x r with orthonormal
 * columns, for example the top-r right singular vectors of a piece):
 *   Y = X V         (n x r FP32, the r-dimensional coordinates)
 *   X_lift = Y V^T  (n x d FP32, the paper's d-dimensional A_l; NULL to skip).
 * X is n x d in dtype xt (GBKM_F32: the tensor cores take X and V in the 3xTF32
 * form, each split into two TF32 terms and multiplied as hi.hi + hi.lo + lo.hi,
 * which gives FP32-faithful products; GBKM_BF16: bfloat16 X against V rounded to
 * bfloat16).  Accumulation is FP32.  r must be a multiple of 16 and <= 256 for
 * the tensor-core engine; other r use the SIMT engine (FP32 X only).  The lift
 * runs on the tensor cores in the 3xTF32 form when d % 16 == 0 and r % 4 == 0. */
int kmeans_project_block(gbkm_ctx *ctx, const void *X, int32_t xt, int64_t n, int64_t d,
                         const float *V, int64_t r, float *Y, float *X_lift);

/* Per-piece bases with the d-dimensional lift (Section 2.2, piecy: the input is read in pieces,
 * each piece A_q is replaced by its projection A_q V_q V_q^T onto its own best-fit subspace of
 * dimension ell, which keeps d coordinates; every piece adds up to ell dimensions to the point set
 * as a whole).  Rows [q * piece_rows, (q + 1) * piece_rows) form piece q (the last may be shorter,
 * but every piece needs at least s rows).  For each piece in order: kmeans_rsvd with the piece's
 * rows (and weights), then kmeans_project_block of the piece onto V_q with the lift.
 *   X: n x d FP32; w: n FP32 or NULL (the weighted SVD of Section 2.3.2; the lift needs no weights);
 *   Omegas: pieces x d x s FP32, piece q's random matrix; s, ell: as in kmeans_rsvd;
 *   X_lift: n x d FP32 out (may not alias X); V_out: pieces x d x ell FP32 out (piece q's basis);
 *   sigma_out: pieces x ell FP32 or NULL; info_out: pieces int32 or NULL (kmeans_rsvd's info).
 * The projection and the lift run on the tensor cores in the 3xTF32 form when ell % 16 == 0 and
 * d % 16 == 0 (FP32-faithful products), else on the CUDA cores.  Allocates the coordinates of one
 * piece (piece_rows x ell FP32) stream-ordered for the call. */
int kmeans_piecy_lift(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, const float *w, int64_t piece_rows,
                      const float *Omegas, int64_t s, int64_t ell, float *X_lift, float *V_out, float *sigma_out,
                      int32_t *info_out);

/* ------------------------------------------------------------------ A3: k-means++ seeding */

/* k-means++ seeding (Section 1).  The first center is row floor(u[0] * n), or,
 * when weights w are given, the first row whose inclusive prefix sum of w
 * exceeds u[0] * sum(w).  Center j >= 1 is the smallest i whose inclusive
 * prefix of p_i = w_i * D^2_i exceeds u[j] * sum(p), D^2_i being the squared
 * distance of x_i to its closest chosen center (if rounding leaves no such i,
 * the last i with p_i > 0).  D^2 is evaluated from direct differences with
 * error-free FP32 transformations (accurate to ~2^-44 relative) and summed in
 * FP64 by a two-level block scan; no host synchronisation between rounds.
 *   X: n x d FP32; w: n FP32 or NULL; u: k FP64 uniforms in [0, 1) (device);
 *   idx_out: k int64 (device); C_out: k x d FP32 (device), the chosen rows.
 * If fewer than k rows have positive w * D^2 the remaining idx_out entries
 * are -1, their C_out rows are left unchanged and gbkm_sync reports
 * GBKM_EDEGENERATE.  Requires k <= n. */
int kmeans_seed_pp(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, const float *w,
                   int64_t k, const double *u, int64_t *idx_out, float *C_out);

/* kmeans_seed_pp with the BF16 copy of X and its rows' rounding residuals at hand (kmeans_quantize
 * or kmeans_ingest with resid): the same picks (bit-identical indices), found with less reading.  A
 * row's distance to the new center is first bounded from below through its BF16 copy,
 * ||x - c|| >= ||bf16(x) - c|| - ||bf16(x) - x|| (evaluated in FP32 with its error bound); when the
 * bound already exceeds the row's D^2 the FP32 row is not read.  Xq: n x d bfloat16, 16-byte
 * aligned, d % 8 == 0 (otherwise the call runs as kmeans_seed_pp); xresid: n FP32, the residuals
 * rounded up.  Other arguments and results as kmeans_seed_pp.  It pays where the bound decides most
 * rows (clusters far apart compared with the rows' rounding); on the mixtures measured here, whose
 * far distances differ by about the bound's slack, it was no faster than kmeans_seed_pp. */
int kmeans_seed_pp_q(gbkm_ctx *ctx, const float *X, const void *Xq, const float *xresid, int64_t n, int64_t d,
                     const float *w, int64_t k, const double *u, int64_t *idx_out, float *C_out);

/* ------------------------------------------------------------------ A4 + A5: assignment */

/* Assignment step of Lloyd's algorithm (Section 1): labels[i] = argmin_j
 * ||x_i - c_j||^2, ties to the lowest j.  Scores ||c_j||^2 - 2 x_i . c_j come
 * from a distance GEMM in the operand format opts->compute:
 *   GBKM_F32:     Xop == X (FP32); SIMT FFMA or tcgen05 3xTF32 (split hi/lo);
 *   GBKM_BF16:    Xop is the bfloat16 copy of X; tcgen05 kind::f16; with
 *                 opts->center_terms == 2 the centers enter as two BF16 terms (hi +
 *                 lo, two MMAs): the rounding of x is then the main error, and the
 *                 bound on a score difference grows with the two centers' distances
 *                 to x instead of with max ||c||;
 *   GBKM_FP8E4M3: Xop is the E4M3 copy with per-row scales (d <= 128 only);
 *                 tcgen05 kind::f8f6f4, scales applied in the epilogue.
 * The fused epilogue keeps, per point, the best score and every center whose score
 * lies within the worst-case error bound of a score difference from it (the
 * certified band).  A point whose band holds more than its best center is a
 * near-tie; with opts->recheck != 0 it is re-resolved from the FP32 data: the band's
 * centers (up to 8) by direct FP32 differences, or, when the band cannot be listed,
 * by a 3xTF32 pass over the gathered points (BF16 / FP8 forms; its own near-ties
 * then take the direct recheck, scanning all k if needed).  Every label equals the
 * exact nearest center except where two centers' distances agree to within the
 * direct recheck's error ((ceil(d/128) + 10) 2^-24 relative).
 *   Xop_scales: per-row scales of an FP8 Xop (n x ceil(d/128)); for a BF16 Xop,
 *     optionally the rows' rounding residuals from kmeans_quantize (n FP32): the band
 *     then uses them in place of the worst case u ||x|| (and, with one-term centers,
 *     the centers' largest residual in place of u ||c||; the bound stays certified);
 *     else NULL.
 *   X: n x d FP32 (always required: recheck and bounds).
 *   xnorm: ||x_i||^2 FP32 from kmeans_row_norms, or NULL (then computed here).
 *   C: k x d FP32.  labels: n int32.  min_d2: n FP32 or NULL, the squared
 *   distance to the chosen center (expanded form, clamped at 0; direct form on
 *   rechecked rows).  n_rechecked: 1 int64 or NULL (device), near-tie rows.
 *   opts: host pointer or NULL (F32, AUTO, recheck on). */
int kmeans_assign(gbkm_ctx *ctx, const void *Xop, const float *Xop_scales, const float *X,
                  const float *xnorm, int64_t n, int64_t d, const float *C, int64_t k,
                  const gbkm_assign_opts *opts, int32_t *labels, float *min_d2,
                  int64_t *n_rechecked);

/* ------------------------------------------------------------------ A6 + A7: update and cost */

/* Centroid step of Lloyd's algorithm (Section 1; Section 2: mu(P) = sum x/|P|)
 * through clustering features (Section 2.1): for every cluster j,
 * N_j = sum w_i, S_j = sum w_i x_i, Q_j = sum w_i ||x_i||^2 over rows labelled j;
 * C_new[j] = S_j / N_j, or C_old[j] when N_j == 0 (empty cluster keeps its center).
 * The rows are grouped by a stable counting sort of the labels (per-segment
 * histograms with warp-aggregated match_any counting; for k <= 2048 one launch
 * scans each cluster's row of the table, else a device-wide scan; a stable
 * scatter), then each cluster's rows are summed in fixed-size chunks with
 * error-free FP32 transformations, the chunk sums folded in runs of 32 chunks and
 * the runs combined in run order (double-float, then FP64): no floating-point
 * atomics, bit-reproducible, and no cluster's sum a chain as long as its rows.
 * Costs from the CF identity (Section 2.1), in FP64:
 *   cost_old = sum_j Q_j - 2 c_old_j . S_j + N_j ||c_old_j||^2 = cost(C_old, labels)
 *   cost_new = sum_j Q_j - ||S_j||^2 / N_j                      = cost(C_new, labels)
 *   X: n x d FP32; w: n FP32 or NULL; labels: n int32 in [0, k);
 *   C_old, C_new: k x d FP32 (may not alias); counts: k FP64 (N_j) or NULL;
 *   cost_old, cost_new: 1 FP64 each or NULL; n_empty: 1 int64 or NULL.
 * Labels outside [0, k) are reported as GBKM_EINVAL by gbkm_sync. */
int kmeans_update(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, const float *w,
                  const int32_t *labels, int64_t k, const float *C_old, float *C_new,
                  double *counts, double *cost_old, double *cost_new, int64_t *n_empty);

/* Fixed device scratch of kmeans_update_noalloc, in bytes (64 MiB). */
#define GBKM_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* kmeans_update for callers that cannot allocate device memory.  The paper has
 * no counterpart: this exists for callers that must not call cudaMalloc, for
 * example code running while the CUDA caching allocator of a host framework is
 * locked, a memory-capped or pre-reserved serving process, or a real-time loop
 * in which an allocation (and the synchronisation it can bring) is not allowed.
 * It computes exactly what kmeans_update computes, with the same kernels and
 * the same results, but needs no gbkm_ctx and allocates nothing: its scratch is
 * a fixed GBKM_NOALLOC_SCRATCH_BYTES block compiled into the library, which
 * every GPU that loads the library holds until the process exits.
 *  - cuda_stream: a cudaStream_t of the CURRENT device (NULL = legacy stream);
 *    the work is queued there, asynchronously.  All other pointers are device
 *    pointers as in kmeans_update and are owned by the caller.
 *  - The first call on a device looks up the scratch block's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    outside any stream capture.
 *  - Every call on a device shares the one scratch block, and the block keeps
 *    the last call's contents (what must start at zero is cleared by the call
 *    itself).  Calls whose work overlaps on the GPU (two streams, two threads)
 *    race on the block and corrupt each other: serialise them.
 *  - Scratch needed: kmeans_update_scratch_bytes(n, d, k) bytes, that is 256 plus these
 *    terms, each rounded up to a multiple of 256: 4 kS (twice), 4 ceil(kS/4096),
 *    4 (k+1) (twice), 4 n, 8 I d, 8 (ceil(I/32) + k) d, 16 I, 8 k (2 + 2 ceil(d/256)),
 *    4 k and 4, with I = ceil(n/128) + k, S = ceil(n/R) and R the smallest power of two
 *    >= R0 with k ceil(n/R) <= 2^23, R0 = 256 for k <= 2048 and 128 above.  A problem
 *    that needs more than GBKM_NOALLOC_SCRATCH_BYTES returns GBKM_ETOOBIG before
 *    anything is queued (n = 200,000, d = 1,024, k = 100 needs ~16.3 MB).
 *  - The scratch block's address is resolved once per device and kept for the life of
 *    the process: after cudaDeviceReset (which unloads the library's device image) this
 *    entry point must not be called again in that process.
 *  - Labels must lie in [0, k); rows with other labels are left out of the sums
 *    (no status word is reported, since there is no context).
 * Returns GBKM_OK, GBKM_EINVAL, GBKM_EUNSUPPORTED, GBKM_ETOOBIG or GBKM_ECUDA. */
int kmeans_update_noalloc(void *cuda_stream, const float *X, int64_t n, int64_t d, const float *w,
                          const int32_t *labels, int64_t k, const float *C_old, float *C_new,
                          double *counts, double *cost_old, double *cost_new, int64_t *n_empty);

/* Bytes of the fixed scratch block that kmeans_update_noalloc needs for an n x d update with
 * k clusters (the formula above); -1 for sizes kmeans_update does not take.  Host
 * arithmetic only: no device is touched.  No paper counterpart. */
int64_t kmeans_update_scratch_bytes(int64_t n, int64_t d, int64_t k);

/* ------------------------------------------------------------------ A8: batched problems */

/* One problem of a batched run.  All pointers are device pointers owned by the caller. */
typedef struct {
    const float *X;      /* n x d FP32 points, 16-byte aligned */
    int64_t n, d, k;     /* d % 16 == 0, 1 <= k <= min(n, 1024) */
    const double *u;     /* seeds x k uniforms in [0, 1): row s drives seed s's k-means++ */
    float *C_out;        /* seeds x k x d: the centers of every seed after the last iteration */
    int32_t *labels_out; /* seeds x n or NULL: labels of the last assignment */
    double *cost_out;    /* seeds x 2 or NULL: cost(C_{T-1}, L) and cost(C_T, L) of the last iteration */
} gbkm_problem;

/* Run k-means++ (Section 1) and then `iters` Lloyd iterations (Section 1) for `count`
 * independent problems x `seeds` seeds each, with the same rules and results as
 * kmeans_seed_pp, kmeans_assign (compute = GBKM_F32 or GBKM_BF16, tcgen05 engine,
 * certified near-ties re-resolved exactly) and kmeans_update.  No paper counterpart
 * as a batch: it runs many instances of the paper's solver at once.  Every phase is
 * one launch over all (problem, seed) pairs: the k-means++ rounds, the assignment
 * (a persistent tcgen05 kernel over the row tiles of all problems, the seeds'
 * centers side by side so one read of X serves every seed), the recheck, and the
 * CF update (one label table and one device-wide scan for all pairs).
 *   probs: host array of `count` problems; 1 <= seeds <= 8; iters >= 0.
 *   flags: bit 0 (GBKM_BATCH_GRAPH): record the whole run into one CUDA graph and
 *          launch it; bit 1 (GBKM_BATCH_AUTOTUNE): choose the center-chunk width of
 *          each problem's shape with kmeans_autotune (else 256).
 * Asynchronous on the context's stream; workspace and per-problem tables are
 * allocated (and the stream synchronised) before anything is queued. */
#define GBKM_BATCH_GRAPH 1
#define GBKM_BATCH_AUTOTUNE 2
int kmeans_batch_run(gbkm_ctx *ctx, const gbkm_problem *probs, int64_t count, int64_t seeds,
                     int64_t iters, int32_t compute, int32_t flags);

/* Relaunch, on the context's stream, the CUDA graph that the last kmeans_batch_run
 * with GBKM_BATCH_GRAPH recorded on this context (no paper counterpart): the same
 * problems, seeds and iteration count, reading and writing the same buffers (X, u,
 * C_out, labels_out, cost_out must still be allocated; their contents may have
 * changed).  The graph keeps its tables in the context's workspace, so any other
 * call on the context that uses the workspace in between invalidates it:
 * GBKM_EINVAL if no graph was recorded or it has been invalidated. */
int kmeans_batch_replay(gbkm_ctx *ctx);

/* The project's tile autotuner (no paper counterpart): times the tcgen05
 * assignment of a synthetic 16,384-point problem of dimension d against ncols
 * centers with center-chunk widths of 64, 128 and 256 columns and returns the
 * fastest in *bn_out (host).  Results are cached per (GPU, compute, d, ncols rounded
 * up to a power of two) for the life of the process and, when the environment
 * variable GBKM_TUNE_CACHE names a file, across processes.  Synchronises. */
int kmeans_autotune(gbkm_ctx *ctx, int32_t compute, int64_t d, int64_t ncols, int32_t *bn_out);

/* The autotuner for the single-problem assignment (no paper counterpart): times kmeans_assign of a
 * synthetic 32,768-point problem of dimension d against k centers over the candidate configurations --
 * the tcgen05 engine with center-chunk widths of 64, 128 and 256 columns (distinct chunkings only) and
 * stage rings of 2, 3 or as many stages as fit in shared memory, and for GBKM_F32 the CUDA-core engine
 * -- and keeps the fastest (host outputs, each may be NULL: *engine_out a gbkm_engine, *bn_out the
 * chunk width, *stages_out the ring depth, 0 for as many as fit).  From then on, kmeans_assign with
 * GBKM_ENGINE_AUTO on a shape of this (GPU, compute, d, k rounded up to a power of two) takes that
 * configuration; labels are exact in every configuration.  Cached per process and, when GBKM_TUNE_CACHE
 * names a file, across processes.  compute: GBKM_F32 or GBKM_BF16.  Synchronises. */
int kmeans_autotune_assign(gbkm_ctx *ctx, int32_t compute, int64_t d, int64_t k, int32_t *engine_out,
                           int32_t *bn_out, int32_t *stages_out);

/* ------------------------------------------------------------------ A9: learned candidate proposal */

/* A small MLP d_in -> hidden -> hidden -> k (GELU after the two hidden layers) that scores the k
 * centers for a point (no paper counterpart).  Parameters are one FP32 vector, layout
 * W1 (hidden x d_in), b1 (hidden), W2 (hidden x hidden), b2 (hidden), W3 (k x hidden), b3 (k),
 * rows = output units; params_bf16 is its BF16 copy (what the tensor cores read).  adam_m /
 * adam_v (same layout, FP32) and wd_mask (same layout, 1 = decayed weight) serve training and may
 * be NULL for inference.  d_in, hidden and k are multiples of 16.  Device pointers except step. */
typedef struct {
    int64_t d_in, hidden, k;
    float *params;
    void *params_bf16;
    float *adam_m, *adam_v;
    const uint8_t *wd_mask;
    int64_t step;  /* host: AdamW step counter, advanced by kmeans_mlp_train_step */
} gbkm_mlp;

/* Number of parameters of the layout above. */
int64_t kmeans_mlp_param_count(int64_t d_in, int64_t hidden, int64_t k);

/* D = A B^T on the tensor cores with a fused epilogue (building block of the MLP):
 * A: M x K, B: N x K, BF16 row-major (K % 8 == 0, N % 16 == 0, 16-byte aligned);
 * Y[i, j] = act(D[i, j] + bias[j]) (act 0: none, 1: GELU), FP32 or BF16 (out_bf16), row stride ldy.
 * bias may be NULL; it enters the FP32 accumulator through the tensor cores as the BF16 head and
 * tail of each bias[j] (2^-17 relative), the same way in every GEMM of the MLP. */
int kmeans_gemm_bf16(gbkm_ctx *ctx, const void *A, const void *B, int64_t M, int64_t N, int64_t K,
                     const float *bias, int32_t act, int32_t out_bf16, void *Y, int64_t ldy);

/* Forward pass on Xh (n x d_in BF16): logits (n x k FP32) and/or topm (1..32) proposed centers
 * per point (n x topm int32, in decreasing logit order, equal logits by increasing index, -1
 * padding), selected inside the logits GEMM's epilogue so that the logits are never stored.
 * group 0 or 1: the topm largest logits; group 16: every aligned group of 16 centers offers only
 * its best center (lowest index on equal logits) and the topm best offers are returned, which
 * keeps the selection to one comparison per group in the epilogue. */
int kmeans_mlp_forward(gbkm_ctx *ctx, const gbkm_mlp *mlp, const void *Xh, int64_t n, float *logits,
                       int32_t *top_idx, int32_t topm, int32_t group);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled decay wd on wd_mask) on the mean
 * softmax cross-entropy of the batch Xh (B x d_in BF16, B % 8 == 0) against labels (B int32 in
 * [0, k)).  Every matrix product of the forward and backward passes runs on the tensor cores.
 * loss_rows (B FP32) and grad_out (param_count FP32, the batch gradient) may be NULL.
 * mlp->step is advanced on the host. */
int kmeans_mlp_train_step(gbkm_ctx *ctx, gbkm_mlp *mlp, const void *Xh, const int32_t *labels, int64_t B,
                          float lr, float wd, float *loss_rows, float *grad_out);

/* s2[j] = (1/4) min_{i != j} ||c_j - c_i||^2 for the k x d centers C (FP32 direct differences):
 * the squared acceptance radius of kmeans_learned_assign's certificate. */
int kmeans_center_separation(gbkm_ctx *ctx, const float *C, int64_t k, int64_t d, float *s2);

/* Assignment step (Section 1) with learned candidates: the MLP proposes topm centers per point
 * (group 16 of kmeans_mlp_forward, in decreasing logit order); their exact FP32 distances are taken
 * in that order until a candidate b has the point certifiably inside the ball of radius s(c_b) (then
 * every other center is strictly farther, so b is the exact label); the points without such a
 * candidate are gathered and get the full scan of kmeans_assign in its BF16 form, whose certified
 * near-tie recheck makes its labels exact too.  The labels are therefore those of the exact method.
 * X: n x d FP32, Xh: its BF16 copy (n x d), C: k x d, s2 from kmeans_center_separation; labels:
 * n int32; n_fallback: 1 int64 (device) or NULL; cand_out: n x topm int32 or NULL.  Synchronises
 * once (to size the fallback scan). */
int kmeans_learned_assign(gbkm_ctx *ctx, const gbkm_mlp *mlp, const float *X, const void *Xh, int64_t n,
                          int64_t d, const float *C, int64_t k, const float *s2, int32_t topm,
                          int32_t *labels, int64_t *n_fallback, int32_t *cand_out);

/* k-means objective (Section 1): cost = sum_i w_i min_j ||x_i - c_j||^2 (FP64),
 * evaluated as an exact FP32-operand assignment followed by the CF identity of
 * Section 2.1 on the resulting clusters.  X: n x d FP32; w: n FP32 or NULL;
 * C: k x d FP32; cost: 1 FP64 (device). */
int kmeans_cost(gbkm_ctx *ctx, const float *X, int64_t n, int64_t d, const float *w,
                const float *C, int64_t k, double *cost);

/* ------------------------------------------------------------------ BICO-style nearest-reference query */

/* Batched weighted nearest-reference query against one snapshot of BICO's clustering features
 * (Section 2.1: the feature (N_j, S_j, Q_j) of a point set holds its total weight, the weighted sum
 * of its points and the weighted sum of their squared lengths, so it knows its centroid
 * mu_j = S_j / N_j and its error c_j = Q_j - ||S_j||^2 / N_j; Section 2.3.1: a weighted point
 * (x, w) stands for w copies of x, its nearest reference point is found once, and feature j
 * takes
 *     w' = w                                                if s ||x - mu_j||^2 - T + c_j <= 0,
 *     w' = max(0, min(w, floor((s T - s c_j) / (s ||x - mu_j||^2 - T + c_j))))  otherwise,
 * copies of it, s = N_j and T the threshold; the paper leaves c_j > T open, where this gives 0).
 * The sequential tree that applies the answers is not part of the call: every point of the batch
 * is answered against the same snapshot.
 *   Xop, Xop_scales, X, xnorm, opts: as in kmeans_assign (X: n x d FP32 points; the operand form
 *     of the distance GEMM; the reference search is the exact assignment step against R).
 *   w: n FP32 weights (whole numbers in BICO's use) or NULL for 1.
 *   R: m x d FP32 reference points (one per feature), m <= 65536.
 *   N: m FP64 (> 0; a feature with N_j <= 0 is treated as empty: d2 = 0 and w' = w),
 *   S: m x d FP64, Q: m FP64: the snapshot.  T: the threshold (>= 0, host value).
 *   ref_out: n int32, the nearest reference (lowest index on ties, exact as kmeans_assign's labels).
 *   d2_out: n FP64 or NULL, ||x_i - mu_j||^2 (FP64 direct differences).
 *   take_out: n FP64, w' (whole copies when w is whole).
 * Arithmetic after the search: FP64, each step of the rule above rounded once, in that order. */
int kmeans_bico_query(gbkm_ctx *ctx, const void *Xop, const float *Xop_scales, const float *X,
                      const float *xnorm, int64_t n, int64_t d, const float *w, const float *R,
                      int64_t m, const double *N, const double *S, const double *Q, double T,
                      const gbkm_assign_opts *opts, int32_t *ref_out, double *d2_out, double *take_out);

#ifdef __cplusplus
}
#endif
#endif /* GBKM_H */
