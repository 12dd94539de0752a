/*
 * rklt.h -- C ABI of the GB300 (sm_103a) rounded-KLT image-compression library.
 *
 * Method: "Low-complexity Rounded KLT Approximation for Image Compression"
 * (Radunz, Bayer, Cintra; arXiv 2111.14239).  Per N x N block A of an 8-bit
 * image the library computes the integer stage C = T A T^T (T = round(alpha K),
 * K the KLT of a first-order Markov process with correlation rho, Sec. 2.1 and
 * Sec. 2.3), the normalised coefficients B = S C S (S from Eq. 1, the Appendix's
 * (u u^T) o (T A T^T) form), keeps the first r coefficients in zig-zag order
 * (Sec. 4.1), reconstructs A' = That^{-1} B' That^{-T} (Sec. 4.1, Appendix), and
 * reduces the squared error to MSE / PSNR with peak 255 (Sec. 4.1, Table 3).
 *
 * Conventions shared by every entry point
 *  - Status: every call returns rklt_status; RKLT_OK (0) on success.  On failure
 *    nothing has been enqueued, and rklt_last_error() (per host thread) holds a
 *    one-line reason.  No C++ exception crosses this boundary.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Device work is enqueued asynchronously on it; the call
 *    returns before the GPU finishes.  Errors raised by a kernel while it runs
 *    (a bounded wait that gave up) are latched on the device and reported by
 *    rklt_device_status().
 *  - Pointers named d_* are device pointers that the CALLER allocates and owns;
 *    h_* are host pointers.  The library never frees caller memory.
 *  - Images: uint8, row-major, H rows of W pixels, row pitch `ld` bytes (ld >= W).
 *    H and W must be multiples of N (disjoint N x N blocks, Sec. 4.1), else
 *    RKLT_ERR_SHAPE.  H = 0 or W = 0 is a valid empty image.
 *  - Blocks are numbered row-major over the (H/N) x (W/N) block grid; batched
 *    calls place image i's blocks after those of images 0..i-1.
 *  - Zig-zag: coefficient (i, j) of a block (i = vertical frequency, j =
 *    horizontal) has zig-zag index z(i, j); the walk visits anti-diagonals i + j
 *    in order, moving down-left on odd ones and up-right on even ones, i.e. the
 *    JPEG order for N = 8.
 *  - Precision: the integer stage is exact (bit-identical to integer
 *    arithmetic); normalisation, inverse and error are FP32 with FP64 per-tile
 *    and per-image accumulation.  FP64 is used on the host only, to build plans.
 */
#ifndef RKLT_H
#define RKLT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rklt_status;
#define RKLT_OK 0
#define RKLT_ERR_ARG 1         /* bad argument (N, rho, alpha, r, NULL pointer, count) */
#define RKLT_ERR_SHAPE 2       /* H or W not a multiple of N, ld < W, bad strides    */
#define RKLT_ERR_DEGENERATE 3  /* T has a zero row, is singular, has an entry outside
                                  {0, +1, -1}, lacks the row parity of the KLT, or an
                                  entry of alpha*K lies within 1e-9 of a rounding tie */
#define RKLT_ERR_CUDA 4        /* a CUDA runtime call failed                          */
#define RKLT_ERR_OOM 5         /* a library-owned device or host allocation failed    */
#define RKLT_ERR_BUDGET 6      /* serving: request exceeds the device-memory budget   */
#define RKLT_ERR_TIMEOUT 7     /* a bounded device-side wait gave up                  */
#define RKLT_ERR_UNSUPPORTED 8 /* valid request the library does not handle          */

/* Thread-local description of the last failure on this host thread. */
const char *rklt_last_error(void);
/* Static name of a status code. */
const char *rklt_status_string(rklt_status s);
/* Library version, major * 10000 + minor * 100 + patch. */
int rklt_version(void);

/* ------------------------------------------------------------------------
 * Plans (Sec. 2.1, Sec. 2.3, Eq. 1) -- built on the host in FP64, uploaded once.
 * ------------------------------------------------------------------------ */

typedef struct rklt_plan rklt_plan;

/* Build the RKLT plan for block size N in {4, 8, 16, 32} and correlation
 * 0 < rho < 1 with the default expansion factor alpha = 2 sqrt(N/8) (alpha = 2
 * for N = 8, Sec. 3).  Steps: omega roots of the Sec. 2.1 equation by
 * bisection, one per interval (i pi/N, (i+1) pi/N); K from the closed form
 * (sign: K[i][0] > 0); T = floor(alpha K + 1/2) (Eq. 2); s_i = 1/sqrt((T T^T)_ii)
 * (Eq. 1); T^{-1} in FP64; zig-zag table.  On success *out owns host tables and
 * nothing on the device (plan tables travel as kernel parameters); release it
 * with rklt_destroy.  Plans are immutable, so concurrent use from several host
 * threads and streams is safe.
 * Errors: RKLT_ERR_ARG (N, rho, out), RKLT_ERR_DEGENERATE, RKLT_ERR_OOM. */
rklt_status rklt_make(int N, double rho, rklt_plan **out);

/* As rklt_make with an explicit expansion factor alpha > 0 (Sec. 2.3). */
rklt_status rklt_make_alpha(int N, double rho, double alpha, rklt_plan **out);

/* Build a plan from a caller-supplied integer matrix T (h_T: N*N int8, row-major,
 * entries in {0, +1, -1}, rows with the parity T[i][N-1-j] = (-1)^i T[i][j]).
 * Used to run the paper's printed matrices (Table 1) directly.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_DEGENERATE, RKLT_ERR_OOM. */
rklt_status rklt_make_from_matrix(int N, const int8_t *h_T, rklt_plan **out);

/* Comparison transforms of the paper (Sec. 4.1, the exact KLT and the DCT rows of
 * its results) as plans for the same pipeline: an orthonormal real N x N matrix M
 * (rows = basis vectors) replaces T-hat, so B = M A M^T with S = I, zonal
 * retention as for the RKLT, and A' = M^T B' M.  Built in FP64 on the host; the
 * kernels run them in FP32 (not integer-exact).  They are accepted by rklt_fused,
 * rklt_fused_batched, rklt_fused_noalloc, rklt_forward, rklt_zonal and
 * rklt_inverse; rklt_forward_int, the uneven batches and rklt_rsweep reject them
 * with RKLT_ERR_UNSUPPORTED.
 *   rklt_make_klt: the exact KLT of the Markov-1 model with correlation rho
 *   (Sec. 2.1, the closed form, rows with K[i][0] > 0).
 *   rklt_make_dct: the orthonormal DCT-II, M[i][j] = c_i cos(pi (2j + 1) i / (2N)),
 *   c_0 = sqrt(1/N), c_i = sqrt(2/N).
 * Errors: RKLT_ERR_ARG (N, rho, out), RKLT_ERR_OOM. */
rklt_status rklt_make_klt(int N, double rho, rklt_plan **out);
rklt_status rklt_make_dct(int N, rklt_plan **out);

/* Kind of a plan: 0 = rounded KLT (integer T), 1 = exact KLT, 2 = DCT-II; -1 for NULL. */
int rklt_plan_kind(const rklt_plan *plan);

/* The plan's analysis matrix in FP64 (h_M: N*N, row-major): T-hat = S T for a
 * rounded plan, M for the comparison transforms.  Errors: RKLT_ERR_ARG. */
rklt_status rklt_plan_matrix(const rklt_plan *plan, double *h_M);

/* Algorithm 1 (Sec. 3), the design procedure of the rounded transforms, as a
 * setup-time service on the host (FP64): for rho = step, 2 step, ..., 1 - step,
 * T' = round(alpha K_rho) (Eq. 2, K from the closed form); each T' that differs from
 * the one before joins the output.  h_T receives up to max_out matrices (N*N int8
 * each, row-major), h_rho_first / h_rho_last (may be NULL) the first and last rho
 * of the grid that produced each; *count the number of distinct matrices.  The
 * rounded entries need not lie in {0, +1, -1} (any alpha is accepted; rklt_make
 * checks that separately).
 * Errors: RKLT_ERR_ARG, RKLT_ERR_DEGENERATE (entries beyond int8),
 * RKLT_ERR_BUDGET (more matrices than max_out; *count still holds the total). */
rklt_status rklt_design_sweep(int N, double alpha, double step, int max_out, int8_t *h_T, double *h_rho_first,
                              double *h_rho_last, int *count);

/* Figures of merit of a plan's analysis matrix M (T-hat = S T, or the exact KLT /
 * DCT) for the Markov-1 model with correlation rho (Sec. 3.1), host FP64; any output
 * may be NULL:  *cg  unified coding gain 10 log10 prod_k (A_k B_k)^(-1/N) with
 * A_k = h_k R h_k^T (h_k row k of M) and B_k = ||g_k||^2 (g_k row k of M^{-1}, as
 * printed);  *eta transform efficiency 100 sum|r_ii| / sum|r_ij|, r = M R M^T;
 * *mse tr((K - M) R (K - M)^T) / N;  *eps pi ||K - M||_F^2.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_DEGENERATE. */
rklt_status rklt_figures(const rklt_plan *plan, double rho, double *cg, double *eta, double *mse, double *eps);

/* Free a plan (NULL is ignored).  Work already enqueued with it is unaffected. */
void rklt_destroy(rklt_plan *plan);

/* Plan introspection into caller-owned host buffers; any output may be NULL.
 * h_T: N*N int8 row-major; h_s: N doubles (diagonal of S); *orthogonal = 1 when
 * T T^T is diagonal (Eq. 1, first branch); *N_out = N; *alpha_out, *rho_out as
 * built (rho = 0 for rklt_make_from_matrix). */
rklt_status rklt_plan_info(const rklt_plan *plan, int8_t *h_T, double *h_s, int *orthogonal,
                           int *N_out, double *alpha_out, double *rho_out);

/* ------------------------------------------------------------------------
 * Split path (Sec. 4.1): forward -> zonal -> inverse -> psnr.
 * ------------------------------------------------------------------------ */

/* Exact integer stage C = T A T^T of every block (Sec. 2.3 with Eq. 2's integer T,
 * applied to disjoint blocks as in Sec. 4.1), int32, raster order inside a
 * block: d_C[blk][i][j] (N*N per block).  |C| <= (nnz per row)^2 * 255.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_forward_int(const rklt_plan *plan, const uint8_t *d_img, int H, int W,
                             int64_t ld, int32_t *d_C, void *stream);

/* Normalised forward transform B = That A That^T = (s s^T) o C of every block
 * (Eq. 1 for S, Sec. 4.1 and the Appendix for the 2-D form), FP32, zig-zag order:
 * d_coef[blk][z] with z = 0..N*N-1.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_forward(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld,
                         float *d_coef, void *stream);

/* Zonal retention (Sec. 4.1): d_out[blk][k] = d_coef[blk][k] for k < r, i.e.
 * the first r zig-zag coefficients of each of nblk blocks, compact.  0 <= r <= N*N.
 * d_out may equal d_coef only when r == N*N.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_CUDA. */
rklt_status rklt_zonal(const rklt_plan *plan, const float *d_coef, int64_t nblk, int r,
                       float *d_out, void *stream);

/* Inverse transform (Sec. 4.1, Appendix): from compact coefficients d_zcoef
 * [blk][r] (zero beyond r), A' = That^{-1} B' That^{-T} per block into d_recon,
 * FP32, H x W with row pitch ld_out floats (ld_out >= W).  Unrounded.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_inverse(const rklt_plan *plan, const float *d_zcoef, int r, int H, int W,
                         float *d_recon, int64_t ld_out, void *stream);

/* Squared error and PSNR (Sec. 4.1, Table 3): *d_sse = sum (A - A')^2 (FP64),
 * *d_psnr = 10 log10(255^2 H W / SSE) (FP32; +inf when SSE = 0; NaN for an empty
 * image).  Both scalars are device memory; reading them is the caller's job.
 * ldr is the pitch of d_recon in floats.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_psnr(const uint8_t *d_img, int64_t ld, const float *d_recon, int64_t ldr,
                      int H, int W, double *d_sse, float *d_psnr, void *stream);

/* ------------------------------------------------------------------------
 * Fused single pass: forward + zonal + inverse + error, nothing in between
 * touches HBM.
 * ------------------------------------------------------------------------ */

/* One image.  Outputs (each optional, NULL to skip except the scalars):
 *   d_zcoef  [blk][r] FP32 compact zig-zag coefficients (as rklt_forward + rklt_zonal);
 *   d_recon  uint8 reconstruction clip(floor(A' + 1/2), 0, 255), pitch ld_recon bytes;
 *   d_sse    FP64 SSE of the unrounded reconstruction; d_psnr FP32 PSNR (as rklt_psnr).
 * The reconstruction uses A' = T^{-1} (M o C) T^{-T}, which equals That^{-1} B' That^{-T}
 * because the diagonal S cancels (Appendix).  When T T^T is diagonal (Eq. 1's
 * orthogonal branch) and the register path serves the call (N = 4; N = 8 with
 * r <= 15), the SSE is taken by Parseval's identity, sum A^2 - sum_retained C_ij^2 /
 * (d_i d_j), in exact integers (one 64-bit sum per tile and per image, divided once
 * by m^2 = lcm(d)^2), with or without d_recon: the error of the unrounded
 * reconstruction without FP32 rounding, identical for every subset of the outputs,
 * and exactly 0 at r = N*N.  Other plans take it from the FP32 reconstruction.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_fused(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld, int r,
                       float *d_zcoef, uint8_t *d_recon, int64_t ld_recon, double *d_sse,
                       float *d_psnr, void *stream);

/* rklt_fused (Sec. 4.1, Appendix) over nimg images of one shape in one launch
 * (the batched form of the per-image pass).  Image i starts at d_img + i*img_stride
 * (bytes); its reconstruction at d_recon + i*recon_stride; its coefficients after
 * those of images 0..i-1; d_sse[i], d_psnr[i] are its scalars.  When the base
 * pointers and pitches are 16-byte aligned the tiles move by TMA (bulk tensor
 * copies through a shared-memory ring); otherwise by vector loads.  Results are
 * bit-identical either way and independent of nimg.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA. */
rklt_status rklt_fused_batched(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W,
                               int64_t ld, int64_t img_stride, int r, float *d_zcoef,
                               uint8_t *d_recon, int64_t ld_recon, int64_t recon_stride,
                               double *d_sse, float *d_psnr, void *stream);

/* ------------------------------------------------------------------------
 * Many images of uneven sizes, each with its own r and plan, in one pass
 * (the batched form of Sec. 4.1's per-image compression).  N = 4 or 8.
 * ------------------------------------------------------------------------ */

/* One image of a batch.  d_img: H x W uint8, pitch ld bytes; image rows must be
 * N-byte aligned (pointer and ld), as must the reconstruction's.  plan: index into
 * the plans array of the call.  d_zcoef: [blocks][r] FP32 compact zig-zag
 * coefficients (as rklt_fused) or NULL.  d_recon: uint8 reconstruction or NULL. */
typedef struct rklt_item {
    const uint8_t *d_img;
    int H, W;
    int64_t ld;
    int plan;
    int r;
    float *d_zcoef;
    uint8_t *d_recon;
    int64_t ld_recon;
} rklt_item;

/* Immediate batched pass: rklt_fused (Sec. 4.1, Appendix) for images of uneven
 * sizes, each with its own plan and r.  Items are grouped by (plan, retained
 * support); per group one launch of a persistent kernel over a flattened queue of
 * 32-block units of all its images (warp per unit, each lane one block, coalesced row
 * accesses), then a per-image SSE / PSNR kernel; with three or more groups, one launch
 * of the queue kernel over every group's units (plans from a constant-memory table,
 * written on first use) and one SSE / PSNR kernel instead, so that a caller issuing
 * many small batches queues few commands.  d_sse[i], d_psnr[i] receive item i's
 * results; they are
 * bit-identical to what a batch of item i alone produces.  Scratch (descriptors,
 * per-unit partials) comes from a stream-ordered pool; the descriptors travel
 * through a library-owned pinned ring (4 MB per device, reused once the copy
 * that read a region has completed), so the call does not wait for work already
 * queued.  h_items may be reused as soon as the call returns.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_UNSUPPORTED (N not 4 or 8,
 * misaligned rows), RKLT_ERR_OOM, RKLT_ERR_CUDA. */
rklt_status rklt_fused_items(const rklt_item *h_items, int n, const rklt_plan *const *plans, int nplans,
                             double *d_sse, float *d_psnr, void *stream);

typedef struct rklt_batch rklt_batch;

/* A reusable batch of rklt_fused_items work (Sec. 4.1 per image): the work queue
 * (library-owned device memory, freed by rklt_batch_destroy) is built once, the
 * launch sequence is captured into a CUDA graph and every rklt_batch_run replays it.
 * Two forms of the work exist: one persistent kernel over the whole flattened
 * queue (every plan and r in one launch: units ordered heaviest first, dealt
 * round-robin to the warps, each dispatching on its image's retained support; then
 * one finalize kernel writes every image's SSE / PSNR -- two kernel nodes), and one
 * launch per (plan, support) group fanned over side streams.  flags bit 0 =
 * autotune: time both forms in several launch shapes (threads per CTA, CTAs per SM)
 * on the batch itself and keep the fastest (rklt_batch_candidates lists what was
 * timed); without it the grouped form runs with 256 threads and one CTA per SM.  (On
 * GB300 the grouped form measured about 1.3x faster for 2000 uneven crops: there
 * each plan's tables are constant-bank operands of the arithmetic, while the queue
 * form must load them by slot index.)  Creation then has run the batch
 * several times, overwriting its outputs, and synchronises the device.  The queue
 * form keeps each plan in a constant-memory slot of the device (16 per block size,
 * written on first use, released by rklt_destroy; destroy a plan only after the
 * work that uses it has finished); when the slots run out the grouped form is used.
 * The device buffers named in h_items and d_sse / d_psnr are baked into the graph:
 * refill them between runs, keep them alive until rklt_batch_destroy.
 * Errors: as rklt_fused_items. */
rklt_status rklt_batch_create(const rklt_item *h_items, int n, const rklt_plan *const *plans, int nplans,
                              double *d_sse, float *d_psnr, int flags, rklt_batch **out);

/* Replay the batch's graph on `stream`.  Errors: RKLT_ERR_ARG, RKLT_ERR_CUDA. */
rklt_status rklt_batch_run(rklt_batch *b, void *stream);

/* The shape the batch runs with: mode 1 = one persistent queue launch, 0 = grouped
 * launches (groups = the number of (plan, support) groups); tuned_us = best timed
 * run (0 without autotune).  Any output pointer may be NULL. */
rklt_status rklt_batch_info(const rklt_batch *b, int *threads, int *ctas_per_sm, int *groups, double *tuned_us,
                            int *mode);

/* The autotuner's timings: for k < min(*count, max_out), candidate k's mode (as
 * rklt_batch_info), threads per CTA, CTAs per SM and time per run in microseconds.
 * *count = number of candidates timed.  Errors: RKLT_ERR_ARG. */
rklt_status rklt_batch_candidates(const rklt_batch *b, int *modes, int *threads, int *ctas_per_sm, double *us,
                                  int max_out, int *count);

/* Wait for the batch's own stream, free its device memory and graph (NULL ignored). */
void rklt_batch_destroy(rklt_batch *b);

/* Request loop (serving).  A server owns one device buffer of budget_bytes (the
 * device-memory budget requests are admitted against), a pinned host mirror of
 * it, nstreams CUDA streams and result slots for batches of up to max_batch
 * requests, at most two batches in flight per stream (a batch waits for a slot, so
 * under load later arrivals join the next batch); plans (rounded plans, all of one
 * N: 4 or 8) stay host-side and travel
 * with each launch.  Creation allocates all of that and runs every kernel both
 * loops can reach once on a small image (so no request pays for module loading);
 * it synchronises the device.  Release with rklt_server_destroy.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_UNSUPPORTED (N), RKLT_ERR_OOM, RKLT_ERR_CUDA. */
typedef struct rklt_server rklt_server;

/* One request: compress + decompress + PSNR (Sec. 4.1 per image) of the H x W
 * uint8 image at h_img (host memory, pitch W, read when the request is admitted)
 * with plans[plan] and r retained coefficients; it arrives arrival_s seconds after
 * the start of the run.  Arrivals must be non-decreasing. */
typedef struct rklt_request {
    double arrival_s;
    const uint8_t *h_img;
    int H, W;
    int plan;
    int r;
} rklt_request;

/* Outcome of one request: the time its launch was issued (admit_s) and its
 * completion time (done_s), both in seconds from the start of the run (the clock
 * of arrival_s); SSE and PSNR (as rklt_fused); status RKLT_OK or RKLT_ERR_BUDGET
 * (the request alone needs more than the budget; rejected). */
typedef struct rklt_result {
    double done_s;
    double admit_s;
    double sse;
    float psnr;
    int status;
} rklt_result;

rklt_status rklt_server_create(const rklt_plan *const *plans, int nplans, size_t budget_bytes, int nstreams,
                               int max_batch, rklt_server **out);

/* Replay n requests in real time on the calling thread and fill results[0..n).
 * mode 0 = continuous batching: a waiting request is admitted (first come, first
 * served) as soon as its input, 8-bit reconstruction and coefficients fit in a
 * first-fit arena over the budget; every request admitted in one pass of the loop
 * goes out in one rklt_fused_items launch on the next stream, so batches overlap
 * on the device; a request completes when its batch's copies back to pinned
 * memory have finished.  mode 1 = one request at a time: copy in, rklt_fused,
 * copy out, synchronise.  h_recon[i] (H x W bytes) and h_coef[i] ([blocks][r]
 * FP32) receive request i's outputs when the arrays and entries are non-NULL.
 * *wall_s = duration of the run.  Calls on one server must not overlap.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_BUDGET (mode 1: a request exceeds
 * the budget), RKLT_ERR_CUDA. */
rklt_status rklt_server_run(rklt_server *s, const rklt_request *reqs, int n, int mode, uint8_t *const *h_recon,
                            float *const *h_coef, rklt_result *results, double *wall_s);

/* Wait for the server's streams and free everything it owns (NULL ignored). */
void rklt_server_destroy(rklt_server *s);

/* Host-only check of the server's first-fit arena (no GPU needed): `steps` random
 * allocations and releases over a 64 KB arena; fails (RKLT_ERR_ARG, message in
 * rklt_last_error) if two live ranges overlap, a range is misaligned, or releasing
 * everything does not coalesce the free list back into one range. */
rklt_status rklt_arena_selftest(unsigned seed, int steps);

/* Host-only check of the worker pool that stages large batches' images into pinned
 * memory (no GPU needed): `rounds` batches of random images with random pitches, cut
 * into row chunks, copied by the pool; fails (RKLT_ERR_ARG, message in
 * rklt_last_error) if a destination row differs from its source or a copy touches
 * the pitch padding.  Starts and joins three worker threads. */
rklt_status rklt_copypool_selftest(unsigned seed, int rounds);

/* r-sweep: for nimg same-shape images and nplans plans (all with the same N, 4 or
 * 8), the SSE and PSNR of the reconstruction that keeps the first r zig-zag
 * coefficients, for every r = 1..N*N (Sec. 4.1 zonal retention swept over r, as
 * in the paper's r in (0, 45) study).  Outputs are [image][plan][r - 1]:
 * d_psnr (required) and d_sse (FP64, may be NULL); r = N*N gives SSE 0 and PSNR +inf.
 * Per block the exact coefficients c_k are formed once and
 * SSE(r) = SSE(r+1) + c_r (c_r G_rr + 2 sum_{l>r} c_l G_rl) with
 * G_kl = H[i_k][i_l] H[j_k][j_l], H = (T T^T)^{-1} (Parseval when T T^T is
 * diagonal); plans with identical T are evaluated once.  Image rows must be N-byte
 * aligned.  Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_UNSUPPORTED, RKLT_ERR_OOM,
 * RKLT_ERR_CUDA. */
rklt_status rklt_rsweep(const rklt_plan *const *plans, int nplans, const uint8_t *d_imgs, int nimg, int H, int W,
                        int64_t ld, int64_t img_stride, double *d_sse, float *d_psnr, void *stream);

/* JPEG-like quantisation with S absorbed into the quantiser (Appendix: Bbar =
 * round(B / Q) = round(C / Qtilde) with Qtilde = Q / (s s^T) and C = T A T^T), in
 * one pass per block: Bbar for the first r zig-zag positions, stored as int32 in
 * d_qcoef[nimg][nblk][r] (may be NULL); the decoder's reconstruction A' = That^{-1}
 * (Bbar o Q) That^{-T} as 8-bit output (d_recon, may be NULL) and its per-image SSE
 * and PSNR (d_sse[nimg], d_psnr[nimg], as rklt_fused, on the unrounded A').
 * h_Q: N*N positive finite doubles, host, row-major (caller-owned; the paper gives
 * no Q).  round(x) = floor(x + 1/2) as in Eq. 2.  The integer decision is taken in
 * binary32: w_ij = fl32(s_i s_j / Q_ij), q = fl32(fl32(C_ij) w_ij), Bbar =
 * floor(q + 1/2) -- the same steps on any hardware, so Bbar is reproducible bit
 * for bit.  Images as rklt_fused_batched (img_stride, recon_stride ignored when
 * nimg = 1), nimg in [1, 65535].  N in {4, 8, 16, 32}, rounded plans only.  Runs
 * in the fused pass's tile pipeline (TMA when pointers and pitches are 16-byte
 * aligned); for N = 16, 32 with small supports on the tensor cores, where C is the
 * same exact integer and the decision the same binary32 steps.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_UNSUPPORTED (an
 * exact-KLT / DCT plan), RKLT_ERR_OOM, RKLT_ERR_CUDA. */
rklt_status rklt_fused_quant(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W, int64_t ld,
                             int64_t img_stride, int r, const double *h_Q, int32_t *d_qcoef, uint8_t *d_recon,
                             int64_t ld_recon, int64_t recon_stride, double *d_sse, float *d_psnr, void *stream);

/* Mean structural similarity of two 8-bit images, the quality measure of the
 * results (Sec. 4.1, Wang et al. 2004): 11 x 11 Gaussian window (sigma 1.5, weights
 * normalised to sum 1), C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2, the mean of the
 * SSIM map over the (H - 10) x (W - 10) positions where the window fits.  Typical
 * use: d_x the original, d_y the 8-bit reconstruction of rklt_fused.  nimg images
 * of H x W with pitches ldx, ldy and image strides (ignored for nimg = 1);
 * d_mssim[nimg] FP64 (NaN when H or W < 11).  FP32 window sums with the values
 * centred at 128, an FP64 mean per image in a fixed order.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_OOM, RKLT_ERR_CUDA. */
rklt_status rklt_mssim(const uint8_t *d_x, const uint8_t *d_y, int nimg, int H, int W, int64_t ldx,
                       int64_t x_stride, int64_t ldy, int64_t y_stride, double *d_mssim, void *stream);

/* rklt_fused_batched and rklt_mssim in one pass (Sec. 4.1: PSNR and SSIM of the
 * reconstruction): the fused pass's outputs (d_zcoef, d_recon optional; d_sse,
 * d_psnr required) plus d_mssim[nimg] (FP64), the MSSIM of each original against its
 * 8-bit reconstruction, computed while the reconstruction is in shared memory, so
 * d_recon may be NULL and the reconstruction never reaches HBM.  Arguments and
 * layouts as rklt_fused_batched; d_mssim device memory.
 * One launch for the register-path plans: N = 4, or N = 8 with r <= 15, T T^T
 * diagonal (the rounded plans of the paper for rho < 0.39 or >= 0.8).  There the
 * coefficients, reconstruction, SSE and PSNR are bit-identical to rklt_fused_batched,
 * the SSIM at every window position bit-identical to rklt_mssim's on that
 * reconstruction, and the mean differs from rklt_mssim's only in the grouping of its
 * FP32 partial sums (about 1e-7).  Other plans run rklt_fused_batched and then
 * rklt_mssim (with a stream-ordered scratch reconstruction when d_recon is NULL).
 * NaN MSSIM when H or W < 11.  The result does not depend on nimg.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_OOM, RKLT_ERR_CUDA. */
rklt_status rklt_fused_mssim(const rklt_plan *plan, const uint8_t *d_img, int nimg, int H, int W, int64_t ld,
                             int64_t img_stride, int r, float *d_zcoef, uint8_t *d_recon, int64_t ld_recon,
                             int64_t recon_stride, double *d_sse, float *d_psnr, double *d_mssim, void *stream);

/* rklt_fused for callers that must not allocate.  (Not part of the paper: this
 * is a deployment variant of the fused pass, with no counterpart in the method.)
 *
 * rklt_fused obtains a small per-call scratch buffer (one error partial of 4 or
 * 8 bytes per 64 x 256 tile, or per 32 x 256 strip when N = 32 and the retained
 * support stays inside i + j < 16) from a stream-ordered memory pool.  Some callers cannot allow that: code
 * running on a real-time path where an allocation may block or synchronise the
 * device, plugins whose host framework owns the whole device-memory budget and
 * leaves no room for a private pool, and callers that must keep every device
 * allocation under their own bookkeeping.  This entry point allocates nothing: no
 * cudaMalloc, cudaFree, pool or library allocation.  Its scratch is one fixed
 * array of 65536 eight-byte slots (512 KB) inside the library's device image,
 * which every GPU that loads the library keeps until the process exits.
 *
 * Arguments, outputs and results are those of rklt_fused (bit-identical).
 * Limit: the image may span at most 65536 tiles (ceil(H/64) * ceil(W/256) <= 65536,
 * e.g. 32768 x 32768; with 32-row strips ceil(H/32) * ceil(W/256) <= 65536); larger
 * images are rejected with RKLT_ERR_ARG before anything is enqueued.
 * Set-up: the first call on each device, made with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture.  Sharing: all calls use the same array and each call
 * overwrites it (no state carries over), so calls that may overlap on the GPU --
 * on different streams, or from several host threads -- race and must be
 * serialised by the caller.
 * Errors: RKLT_ERR_ARG, RKLT_ERR_SHAPE, RKLT_ERR_CUDA, RKLT_ERR_UNSUPPORTED. */
rklt_status rklt_fused_noalloc(const rklt_plan *plan, const uint8_t *d_img, int H, int W, int64_t ld, int r,
                               float *d_zcoef, uint8_t *d_recon, int64_t ld_recon, double *d_sse,
                               float *d_psnr, void *stream);

/* ------------------------------------------------------------------------
 * Device status
 * ------------------------------------------------------------------------ */

/* Synchronises the current device, then returns and clears the library's latched
 * device-side error: RKLT_OK, or RKLT_ERR_TIMEOUT when a bounded wait inside a
 * kernel gave up (the kernel then skipped its remaining work and returned). */
rklt_status rklt_device_status(void);

/* Bound, in microseconds of GPU time (%globaltimer), on every device-side wait
 * (TMA-ring mbarrier waits) of kernels launched after this call from this
 * process; 0 restores the default of 4 seconds.  A wait that exceeds it latches
 * RKLT_ERR_TIMEOUT (see rklt_device_status) and ends its kernel early. */
void rklt_set_wait_timeout_us(uint32_t microseconds);

/* Transport of the fused kernel's tiles for later calls from this process:
 * 0 (default) = TMA bulk tensor copies when pointers and pitches are 16-byte
 * aligned, else plain loads; 1 = plain loads always.  Results are identical;
 * the switch exists so that both transports can be tested on the same data. */
void rklt_set_transport(int mode);

/* Tensor-core engine for 32 x 32 blocks whose retained support lies inside
 * i + j < 16 (r <= 136), for later calls from this process: 0 (default) =
 * warp-level mma.sync with accumulators in registers; 1 = tcgen05.mma with
 * accumulators in tensor memory (one elected thread per warp group issues the
 * MMAs, operands staged in shared memory, 32 x 256-pixel strips).  Both compute
 * the same exact integer stage; coefficients, reconstruction and SSE agree within
 * the FP32 bounds of the tests (the inverse's rounding differs).  Other N and
 * larger r are unaffected. */
void rklt_set_tensor_engine(int mode);

/* Fault injection for tests of the bounded waits: while on (non-zero), the TMA
 * producer of later fused launches issues no tile loads, so the consumers' waits
 * run out after the rklt_set_wait_timeout_us limit; the kernel then returns early
 * without touching its outputs and rklt_device_status() reports RKLT_ERR_TIMEOUT.
 * No memory access is skipped or misdirected; nothing faults. */
void rklt_debug_inject_stall(int on);

#ifdef __cplusplus
}
#endif

#endif /* RKLT_H */
