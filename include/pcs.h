/*
 * pcs.h -- C ABI of libpcs: GB300 (sm_103a) primal-dual reconstruction for
 * susceptibility-based positive-contrast MRI.
 *
 * The library solves, independently for every 2-D slice s of a stack,
 *
 *     chi_s = argmin  lambda/2 || W (D chi - dB) ||_2^2 + || M G chi ||_1      (Eq. (1))
 *
 * with the first-order primal-dual (Chambolle-Pock) iteration of the paper's
 * Sec. II.A pseudocode: zero start, then N times
 *
 *     p    <- (p + sigma (W D chibar - W dB)) / (1 + sigma/lambda)     dual data prox
 *     q    <- clamp(q + sigma M G chibar, -1, 1)                        dual TV prox
 *     chi+ <- chi - tau D W p - tau G^T M q                             primal step
 *     chibar <- 2 chi+ - chi;  chi <- chi+                              over-relaxation
 *
 * Conventions (readings of the paper, which leaves them open):
 *   - slices are H x W, row-major, stacked as [S][H][W]; row index i runs
 *     along y, column index j along x;
 *   - D is the dipole convolution F^-1 D(k) F with D(k) = 1/3 - k_par^2/|k|^2,
 *     D(0) = 0, circular on the slice; B0 lies in-plane along y (rows) unless
 *     pcs_options.b0_axis = 1 (columns);
 *   - G is forward differences with a Neumann boundary; G^T its exact adjoint;
 *   - W = M = mask (0/1); the TV dual prox is the componentwise clamp;
 *   - the primal function is zero, so the primal prox is the identity;
 *   - the iteration count N is fixed and the output is chi_N.
 *
 * All arithmetic of the iteration runs in FP32 on the GPU; the step sizes and
 * kernel tables are computed in FP64 on the host and rounded once.
 *
 * Ownership: the caller owns every input and output buffer and every stream.
 * The library owns its context, its scratch (dual variables, chibar, device
 * tables) and never frees or retains caller memory.  Work is enqueued on the
 * context's stream; functions return after enqueueing unless stated
 * otherwise.  Errors are reported as pcs_status codes only; nothing aborts or
 * throws across this boundary.  pcs_last_error() gives a thread-local text.
 */
#ifndef PCS_H
#define PCS_H

#include <stddef.h>

/* Only the functions below are exported from libpcs.so. */
#if defined(__GNUC__)
#define PCS_API __attribute__((visibility("default")))
#else
#define PCS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcs_ctx pcs_ctx; /* opaque */

typedef enum pcs_status {
    PCS_OK = 0,
    PCS_EINVAL = 1,       /* bad argument: NULL pointer, non-positive lambda/tau/sigma, S > max_slices ... */
    PCS_EUNSUPPORTED = 2, /* slice size or feature without a kernel (see pcs_supported_size,
                             pcs_supported_generic, pcs_supported_volume_3d) */
    PCS_ENOMEM = 3,       /* device allocation failed */
    PCS_ECUDA = 4,        /* a CUDA runtime call failed (no device, launch failure, ...) */
    PCS_ETIMEOUT = 5,     /* a bounded device wait expired (the balanced schedule's; see pcs_check) */
    PCS_EBUSY = 6         /* context in use by another call */
} pcs_status;

typedef struct pcs_options {
    int b0_axis;       /* 0 = B0 along rows / y (default), 1 = along columns / x */
    int cluster_size;  /* 0 = library default for the slice size; else CTAs per slice (1,2,4,8,16) */
    int max_clusters;  /* 0 = as many concurrent clusters as fit; else an upper bound (tuning) */
    int kernel;        /* 0 = library default; 1 = streaming (state in global memory);
                          2 = resident (state kept on chip for all iterations) */
    int threads;       /* 0 = library default; else threads per CTA of a compiled variant */
    int use_graph;     /* 1 = launch each solve as a CUDA graph, captured once per distinct argument
                          set and replayed (needs a non-NULL stream); 0 = direct launch */
    int tv;            /* 0 = anisotropic TV: the dual TV prox clamps each gradient component
                          (the componentwise reading of Eq. (1)'s ||M G chi||_1, default);
                          1 = isotropic TV: it projects each pixel's (qx, qy) onto the unit disc */
    int tile;          /* 0 = library default; else the FFT tile shape of a compiled variant:
                          100 x (complex elements per lane of the row transforms) + those of the
                          column transforms (e.g. 1616, 816, 1608) */
} pcs_options;

/* Diagnostics of one slice at (chi_N, p_N, q_N), in FP64 (see pcs_slice_report doc below). */
typedef struct pcs_slice_report {
    double objective;     /* lambda/2 ||W(D chi - dB)||^2 + ||M G chi||_1 (Eq. (1)) */
    double gap;           /* Fenchel-Young gap: ||p - lambda(W D chi - W dB)||^2/(2 lambda)
                             + sum(|g| - q.g), g = M G chi; >= 0 */
    double stationarity;  /* || D W p + G^T M q ||_2 */
    double data_residual; /* || W (D chi - dB) ||_2 */
    int iters;
    int pad;
} pcs_slice_report;

/* Fill *opt with the defaults (all zero). Returns PCS_EINVAL if opt is NULL. */
PCS_API pcs_status pcs_options_default(pcs_options *opt);

/* Non-zero if H x W slices have a compiled kernel in this build. */
PCS_API int pcs_supported_size(int H, int W);

/*
 * Create a context for slices of H x W and batches of up to max_slices.
 * Computes the dipole-kernel table D(k) (Eq. (1)'s D, with D(0) = 0) and the
 * FFT twiddles in FP64 on the host, uploads them, and allocates the scratch
 * state (chibar, p, qx, qy: 4 x max_slices x H x W floats).
 *   out         receives the context (set to NULL on failure)
 *   opt         NULL for defaults
 *   cuda_stream a cudaStream_t (NULL = legacy default stream) used by every
 *               later call on this context
 * Sizes without a compiled kernel (pcs_supported_size = 0) that
 * pcs_supported_generic accepts, such as 256 x 258, make an any-size context
 * when opt leaves cluster_size, kernel and threads at 0: pcs_solve_slices,
 * pcs_solve_slices_weighted and pcs_solve_slices_host then run the row and
 * column kernels of pcs_solve_slices_generic on the context's scratch and
 * stream (asynchronous, no allocation; use_graph has no effect), rep and
 * pcs_report give the same FP64 report, pcs_opnorm runs the same power
 * iteration with these kernels, and pcs_solve_slices_monitored resumes from
 * the stored state (the spectrum of chibar rebuilt) with frozen slices left
 * alone.
 * Errors: PCS_EINVAL (out NULL, max_slices < 1), PCS_EUNSUPPORTED (size),
 *         PCS_ECUDA (no device), PCS_ENOMEM.
 */
PCS_API pcs_status pcs_create(pcs_ctx **out, int H, int W, int max_slices, const pcs_options *opt,
                      void *cuda_stream);

/* Change the stream later calls enqueue on. */
PCS_API pcs_status pcs_set_stream(pcs_ctx *ctx, void *cuda_stream);

/*
 * Run n_iter primal-dual iterations (Sec. II.A pseudocode) on S independent
 * slices and write chi_N.
 *   field   device, [S][H][W] float32: the normalised local field dB/B0 (ppm)
 *   mask    device, [S][H][W] uint8 0/1: W = M = mask
 *   lambda  regularisation weight of Eq. (1), > 0
 *   tau, sigma  primal and dual steps, > 0 (the paper uses tau = sigma = 1/||K||;
 *               see pcs_opnorm); tau*sigma*||K||^2 <= 1 is the caller's duty
 *   n_iter  >= 0 (0 gives chi = 0)
 *   chi_out device, [S][H][W] float32, caller-owned; also serves as the
 *           primal iterate during the solve (must not alias field)
 *   rep     NULL, or a host array of S reports; when given, the call also
 *           evaluates the FP64 diagnostics and synchronises the stream
 * All device pointers must be 16-byte aligned.  Slices are independent: the
 * result for a slice does not depend on the other slices in the call.
 * Errors: PCS_EINVAL, PCS_ECUDA.
 */
PCS_API pcs_status pcs_solve_slices(pcs_ctx *ctx, const float *field, const unsigned char *mask, int S,
                            double lambda, double tau, double sigma, int n_iter, float *chi_out,
                            pcs_slice_report *rep);

/*
 * pcs_solve_slices with a non-binary data weighting.  Eq. (1) weights the
 * data residual by a matrix W and restricts the TV term by a mask M
 * (Sec. II.A); pcs_solve_slices takes W = M = mask.  Here weight is W
 * (device float32 [S][H][W], 16-byte aligned, values in [0, 1] so that the
 * full-mask step sizes stay valid) and mask is M.  The dual data step becomes
 * p <- (p + sigma W (u - dB)) / (1 + sigma/lambda) and the adjoint transform
 * takes W p.  With weight equal to the 0/1 mask the result is bit-identical
 * to pcs_solve_slices.  rep (optional) reports the weighted objective, gap,
 * stationarity and residual ||W (D chi - dB)||.  Runs on the streaming
 * kernel: a context created for the resident kernel returns PCS_EUNSUPPORTED.
 * Errors as pcs_solve_slices; PCS_EINVAL if weight is NULL or misaligned.
 */
PCS_API pcs_status pcs_solve_slices_weighted(pcs_ctx *ctx, const float *field, const unsigned char *mask,
                                             const float *weight, int S, double lambda, double tau,
                                             double sigma, int n_iter, float *chi_out, pcs_slice_report *rep);

/*
 * Balanced schedule.  When a solve has more slices than the kernel variant can
 * keep resident as clusters (e.g. 64 slices of 256 x 256 on the 512-thread
 * variant, 36 resident clusters), pcs_solve_slices spreads the S x n_iter
 * slice-iterations evenly over the clusters (McNaughton's wrap-around rule):
 * some slices are split in two consecutive parts run by two clusters, the
 * second part continuing from the state the first left in memory (the same
 * continuation as the monitored solves; results are unchanged, bit for bit).
 * The second part waits for a flag the first sets; the wait is bounded
 * (about 2 s) and never expected to run out.  If it does, the cluster returns
 * early, the launch's results are invalid and pcs_check reports it.
 *
 * pcs_check: synchronise the context's stream and return PCS_ETIMEOUT if any
 * earlier solve on it gave up a wait (clearing the report), else PCS_OK
 * (PCS_ECUDA if the stream reports a CUDA error).  The entry points that
 * synchronise the stream themselves (pcs_solve_slices_host, and the solves
 * given a report array) make the same check and return PCS_ETIMEOUT.
 */
PCS_API pcs_status pcs_check(pcs_ctx *ctx);

/*
 * The balanced schedule a solve of S slices x n_iter iterations uses on
 * `clusters` resident clusters (1 <= clusters < S): segments[4k .. 4k+3] =
 * (slice, first iteration, end iteration, flags: 1 = waits for the slice's
 * first part, 2 = releases its continuation), cluster c running segments
 * [offsets[c], offsets[c+1]) in that order.  *n_segments: capacity in, count
 * out; with segments or offsets NULL only the count is returned.  Host only.
 */
PCS_API pcs_status pcs_schedule_plan(int S, int n_iter, int clusters, int *segments, int *n_segments,
                                     int *offsets);

/*
 * Test of the schedule's bounded wait: one warp waits on a flag that nothing
 * sets, with a limit of limit_cycles SM clock cycles, and *gave_up (host) is
 * set to 1 when the wait gave up.  Synchronises cuda_stream.
 */
PCS_API pcs_status pcs_selftest_wait(void *cuda_stream, long long limit_cycles, int *gave_up);

/*
 * Same as pcs_solve_slices, but field, mask and chi_out are HOST buffers
 * (pinned memory gives full copy bandwidth).  Copies the inputs to
 * library-owned device staging buffers, solves, copies chi back and
 * synchronises the stream before returning.  This is the Sec. II.B flow:
 * one host-to-device copy in, one device-to-host copy out.
 */
PCS_API pcs_status pcs_solve_slices_host(pcs_ctx *ctx, const float *field_host,
                                 const unsigned char *mask_host, int S, double lambda, double tau,
                                 double sigma, int n_iter, float *chi_out_host,
                                 pcs_slice_report *rep);

/*
 * FP64 diagnostics of the state left by the last pcs_solve_slices on this
 * context (chi is the caller's chi_out of that call): objective, Fenchel-Young
 * gap, stationarity and data residual per slice (pcs_slice_report).  Runs
 * two extra dipole convolutions per slice on the GPU with FP64 reductions
 * and synchronises the stream.  rep: host array of S entries.
 */
PCS_API pcs_status pcs_report(pcs_ctx *ctx, const float *field, const unsigned char *mask, int S,
                      double lambda, const float *chi, pcs_slice_report *rep);

/*
 * L = ||K||_2 for K = [W D; M G] of each slice's mask, by power iteration on
 * K^T K (pseudocode step 1), power_iters iterations from a fixed
 * pseudo-random start.  mask: device [S][H][W] uint8; L_out: host array [S].
 * Synchronises the stream.
 */
PCS_API pcs_status pcs_opnorm(pcs_ctx *ctx, const unsigned char *mask, int S, int power_iters,
                      double *L_out);

/*
 * All-FP64 solve (precision study): the same fused iteration kernel
 * instantiated with double state, double transforms and double D(k) /
 * twiddle tables (computed in FP64, not rounded).  field and chi_out are
 * device double [S][H][W], mask uint8; tau, sigma, lambda as for
 * pcs_solve_slices.  Allocates and frees its own scratch and synchronises
 * the stream before returning.  Compiled sizes: 64 x 64 and 256 x 256 (others: PCS_EUNSUPPORTED).
 */
PCS_API pcs_status pcs_solve_slices_f64(const double *field, const unsigned char *mask, int H, int W, int S,
                                        double lambda, double tau, double sigma, int n_iter, double *chi_out,
                                        int b0_axis, void *cuda_stream);

/* ---------------------------------------------------------------- preprocessing */

/*
 * The preprocessing step of Sec. II.B (1): from the two acquisitions without
 * (s0) and with (s1) the readout shift T_shift (Sec. II), the local field dB,
 * the weighting W and the mask that Eq. (1) takes.
 *   dB (ppm)  = arg(s1 conj s0) / (2 pi gamma_bar B0 T_shift) * 1e6, gamma_bar =
 *               42.577478518 MHz/T; the wrapped phase in (-pi, pi], no unwrapping;
 *               0 outside the mask
 *   W         = |s0| / max |s0| over the n voxels
 *   mask      = |s0|^2 >= threshold^2 max |s0|^2 (float32, reproducible bit for bit)
 * s0, s1: device complex float32, interleaved (re, im), n_voxels each, 16-byte
 * aligned.  field_out, weight_out: device float32 [n_voxels], 8-byte aligned;
 * mask_out: device uint8 [n_voxels], 2-byte aligned.  Asynchronous on
 * cuda_stream (a small stream-ordered scratch allocation).  Errors: PCS_EINVAL (NULL, misaligned, t_shift or b0 <= 0,
 * threshold < 0), PCS_ECUDA.  n_voxels = 0 is a no-op.
 */
PCS_API pcs_status pcs_field_map(const float *s0, const float *s1, size_t n_voxels, double t_shift_s,
                                 double b0_tesla, double threshold, float *field_out, float *weight_out,
                                 unsigned char *mask_out, void *cuda_stream);

/* ---------------------------------------------------------------- any slice size */

/*
 * pcs_solve_slices for slice sizes outside the compiled kernel variants, such
 * as the 256 x 258 and 128 x 132 slices of the paper's acquisitions (Sec. III):
 * any even H and W in [8, 512] whose prime factors are all <= 61.  Same
 * problem and iteration as pcs_solve_slices (Eq. (1), Sec. II.A; 2-D D and G
 * per slice, slices independent), with W = weight (NULL: W = mask) and M =
 * mask as in pcs_solve_slices_weighted, tv as pcs_solve_volume_3d, and
 * b0_axis 0 (B0 along y, the rows axis) or 1 (along x).  D(k) is evaluated
 * in FP32 from the integer frequencies.  field, weight, chi_out: device float32
 * [S][H][W]; mask: device uint8 [S][H][W]; 4-byte alignment suffices; chi_out
 * must not alias field.  rep (host [S], optional): the per-slice FP64 report
 * of pcs_solve_slices at (chi_N, p_N, q_N).  Allocates its scratch (4 floats
 * and a half spectrum per pixel), frees it and synchronises cuda_stream before
 * returning.
 * Errors: PCS_EINVAL for bad arguments, PCS_EUNSUPPORTED for sizes outside
 * the set above, PCS_ECUDA for CUDA failures.  S = 0 is a no-op.
 */
PCS_API pcs_status pcs_solve_slices_generic(const float *field, const unsigned char *mask, const float *weight,
                                            int S, int H, int W, int b0_axis, double lambda, double tau,
                                            double sigma, int n_iter, int tv, float *chi_out, pcs_slice_report *rep,
                                            void *cuda_stream);

/* 1 if pcs_solve_slices_generic accepts H x W slices, else 0. */
PCS_API int pcs_supported_generic(int H, int W);

/* ---------------------------------------------------------------- 3-D variant */

/*
 * Eq. (1) with the gradient G in all three dimensions and the 3-D dipole
 * convolution of the whole volume (Sec. II.A; the per-slice solver above
 * reads G as 2-D and solves slices independently).  The volume [S][H][W] is
 * one unknown: D(k) = 1/3 - kz^2/|k|^2 with B0 along z (the slice axis),
 * periodic on the S x H x W grid, k_i = (cycles per sample along axis i) /
 * voxel[i] with voxel = {dz, dy, dx} the voxel's edge lengths in any common
 * unit (host, optional: NULL = isotropic; the paper's acquisitions have
 * 0.72 x 0.72 mm pixels and 2 mm slices, Sec. III; each > 0, else
 * PCS_EINVAL); G = unit forward differences
 * along x, y, z with a Neumann boundary; M = mask, and W = mask when weight
 * is NULL, else weight (device float32 [S][H][W], 16-byte aligned, values in
 * [0, 1], as pcs_solve_slices_weighted).  The Sec. II.A
 * iteration runs n_iter times from the zero start (tau, sigma as for
 * pcs_solve_slices; ||K|| <= sqrt(4/9 + 12) for any 0/1 mask, so
 * tau = sigma = 1/3.53 is always valid).  tv: 0 anisotropic (clamp of each of
 * the three components), 1 isotropic (projection onto the unit ball).
 * field, chi_out: device float32 [S][H][W]; mask: device uint8; 16-byte
 * aligned; chi_out must not alias field.  Allocates its scratch (6 floats and
 * a half spectrum per voxel), frees it and synchronises cuda_stream before
 * returning.  rep (host, optional): the FP64 diagnostics of the whole volume
 * at (chi_N, p_N, q_N), the terms of pcs_slice_report with D, G, W, M of this
 * 3-D problem (the objective and the gap summed over all voxels; iters =
 * n_iter); three more slice launches and two z passes, after the solve.
 * Shapes: H = W in {64, 128, 256}, S in {32, 64} (and 128 for H >= 128);
 * others PCS_EUNSUPPORTED.  Errors: PCS_EINVAL for bad arguments, PCS_ECUDA
 * for CUDA failures.
 */
PCS_API pcs_status pcs_solve_volume_3d(const float *field, const unsigned char *mask, const float *weight, int S,
                                       int H, int W, double lambda, double tau, double sigma, int n_iter, int tv,
                                       const double *voxel, float *chi_out, pcs_slice_report *rep,
                                       void *cuda_stream);

/* 1 if pcs_solve_volume_3d has kernels for an S x H x W volume, else 0. */
PCS_API int pcs_supported_volume_3d(int S, int H, int W);

/* ---------------------------------------------------------------- uneven batches */

typedef struct pcs_batch pcs_batch; /* opaque */

/* One volume of a batch: S slices of H x W, its own lambda; device buffers, caller-owned. */
typedef struct pcs_volume {
    int H, W, S, pad;
    double lambda;
    const float *field;        /* device [S][H][W] */
    const unsigned char *mask; /* device [S][H][W] */
    float *chi_out;            /* device [S][H][W] */
} pcs_volume;

/* What the autotuner chose for one slice size, and what it measured. */
typedef struct pcs_tuning {
    int H, W;
    int cluster_size, kernel, threads; /* the chosen variant (kernel: 1 streaming, 2 resident) */
    int n_candidates;
    double L;                          /* ||K||_2 of the full-mask operator; tau = sigma = 1/L */
    double ns_per_voxel_iter[8];       /* trial time of each candidate, in registry order */
    int cand_cluster_size[8], cand_kernel[8], cand_threads[8];
    int tile;                          /* the chosen variant's FFT tile shape (see pcs_options.tile) */
    int cand_tile[8];
    int pad;
} pcs_tuning;

/*
 * Create a batch solver: all slices of all volumes of a call are solved by the
 * fused primal-dual kernels -- one persistent launch per slice size, run one
 * size after another (the most work first; each launch balances its slices
 * over every resident cluster), with the packing of every size's inputs
 * forked onto per-size streams and everything joined back into cuda_stream.  Step sizes are tau = sigma = 1/L(H, W), L the norm
 * of the full-mask operator K (Sec. II.A pseudocode step 1), computed once per
 * size on the GPU.  autotune != 0: the first solve of a new slice size times
 * every compiled kernel variant of that size on that call's slice count
 * (a short trial) and keeps the fastest; otherwise the library default (or
 * the variant opt selects) is used.
 */
PCS_API pcs_status pcs_batch_create(pcs_batch **out, const pcs_options *opt, int autotune, void *cuda_stream);

/*
 * Solve every slice of every volume with n_iter iterations of the Sec. II.A
 * iteration (each volume with its own lambda) and write each volume's chi_out.
 * Enqueued on the batch stream; inputs are copied into per-size packed
 * buffers owned by the batch.  Slice sizes: the compiled ones and those
 * pcs_supported_generic accepts (run by the any-size kernels: row and column
 * launches per iteration instead of one persistent launch; no variants to
 * autotune).  Errors: PCS_EINVAL, PCS_EUNSUPPORTED, PCS_ENOMEM, PCS_ECUDA.
 */
PCS_API pcs_status pcs_batch_solve(pcs_batch *b, const pcs_volume *vols, int n_vols, int n_iter);

/* The tuning record of slice size H x W (PCS_EINVAL if that size was never solved). */
PCS_API pcs_status pcs_batch_tuning(pcs_batch *b, int H, int W, pcs_tuning *out);

/*
 * Synchronise the batch stream and return PCS_ETIMEOUT if a launch of any size
 * class gave up a bounded wait of the balanced schedule (that call's results
 * are invalid; see pcs_check), else PCS_OK.  Clears the reports.
 */
PCS_API pcs_status pcs_batch_check(pcs_batch *b);

/* Release the batch solver. NULL-safe. */
PCS_API void pcs_batch_destroy(pcs_batch *b);

/* ---------------------------------------------------------------- serving loop */

typedef struct pcs_server pcs_server; /* opaque */

typedef struct pcs_server_config {
    size_t hbm_budget_bytes; /* device memory the admitted requests may hold (see pcs_serve_request_bytes);
                                allocated once, as one arena, by pcs_serve_start */
    int slots;               /* requests in flight at once (one CUDA stream each) */
    int n_iter;              /* primal-dual iterations per slice */
    int autotune;            /* pick each slice size's kernel variant by timing (see pcs_batch_create) */
    int b0_axis;             /* as in pcs_options */
    int reserved[4];
} pcs_server_config;

typedef struct pcs_serve_summary {
    long long completed;     /* requests finished */
    long long pending;       /* requests open or running */
    double voxel_iters;      /* sum over finished requests of S*H*W*n_iter */
    double span_s;           /* first open -> last completion */
    double p50_s, p99_s, max_s; /* per-volume latency (open -> last slice back on the host) */
    double peak_bytes;       /* peak bytes of the arena held by admitted requests */
    int peak_inflight, pad;
    long long failed;        /* requests finished with an error status */
} pcs_serve_summary;

/*
 * Start a server: a scheduler thread that admits volume requests by arrival
 * order, slot and memory budget, solves each request's slices as they arrive
 * (chunks of different requests run concurrently on their slots' streams;
 * a request's primal/dual state stays on the device until it completes),
 * and copies chi back into the request's host buffer.  Slices are solved
 * independently, so a volume's chi does not depend on what else is in flight.
 * The budget is allocated here as one device arena (PCS_ENOMEM if it cannot
 * be); admitted requests occupy ranges of it, so the scheduler thread never
 * allocates or frees device memory while serving.  A request whose copy or
 * launch fails finishes alone with an error status (pcs_serve_poll); a
 * sticky CUDA error stops the server and every later poll returns it.
 */
PCS_API pcs_status pcs_serve_start(pcs_server **out, const pcs_server_config *cfg);

/* Set up a slice size ahead of traffic (autotune, step size, tables); info may be NULL. */
PCS_API pcs_status pcs_serve_prepare_size(pcs_server *sv, int H, int W, pcs_tuning *info);

/*
 * Open a request for a volume of S slices of H x W with regularisation lambda.
 * chi_host: host [S][H][W] float32 that receives chi (keep it alive until the
 * request completes).  Returns its id.  PCS_ENOMEM if the volume alone exceeds
 * the budget, PCS_EUNSUPPORTED for a size neither compiled nor accepted by
 * pcs_supported_generic (those run the any-size kernels, each request with its
 * own half-spectrum scratch, counted in the budget).  The first request of a
 * slice size not prepared with pcs_serve_prepare_size sets that size up on the
 * calling thread (autotuning and step size: up to about a second).
 */
PCS_API pcs_status pcs_serve_open(pcs_server *sv, int H, int W, int S, double lambda, float *chi_host,
                                  long long *id);

/*
 * Slices [s0, s0+n) of request id have arrived: host field [n][H][W] float32
 * and mask [n][H][W] uint8 (pinned memory recommended; keep them alive until
 * the request completes).  Slices must be pushed in order.
 */
PCS_API pcs_status pcs_serve_push(pcs_server *sv, long long id, int s0, int n, const float *field_host,
                                  const unsigned char *mask_host);

/*
 * Up to max finished requests since the last poll: ids, latencies (s) and,
 * if status is not NULL, each request's status (PCS_OK, or PCS_ECUDA for a
 * request whose copy or launch failed; its chi is incomplete).  Non-blocking.
 * Returns PCS_ECUDA once the server met a sticky CUDA error.
 */
PCS_API pcs_status pcs_serve_poll(pcs_server *sv, long long *ids, double *latency_s, pcs_status *status, int max,
                                  int *n_out);

/*
 * The serving arena's placement on the host, for inspection and tests (no GPU):
 * an arena of `capacity` bytes replays ops[0..n_ops): ops[k] > 0 allocates that
 * many bytes (rounded up to 256) first fit; ops[k] < 0 releases the range that
 * op -ops[k]-1 allocated (nothing if that allocation was refused; PCS_EINVAL if
 * that op is not an earlier allocation).  offsets[k] receives op k's offset (-1 if it did not
 * fit or was a release); used_after[k] (may be NULL) the bytes in use after it.
 */
PCS_API pcs_status pcs_serve_arena_plan(size_t capacity, const long long *ops, int n_ops, long long *offsets,
                                        size_t *used_after);

/* Device bytes one request of S slices of H x W holds while admitted (its share of the budget). */
PCS_API pcs_status pcs_serve_request_bytes(int H, int W, int S, size_t *bytes);

/*
 * Failure injection on the host (tests): the next launch of request id reports
 * an error code as if the launch call had failed, so that the request fails
 * alone.  No GPU fault is involved.
 */
PCS_API pcs_status pcs_serve_fail_next_launch(pcs_server *sv, long long id);

/* Running statistics (latency quantiles over finished requests). */
PCS_API pcs_status pcs_serve_stats(pcs_server *sv, pcs_serve_summary *out);

/* Stop the scheduler, wait for work in flight, release everything. NULL-safe. */
PCS_API void pcs_serve_stop(pcs_server *sv);

/*
 * Solve without allocating device memory (the paper has no counterpart; this
 * is a deployment aid).  For callers that may not call cudaMalloc once they
 * run -- e.g. a reconstruction plug-in inside a scanner or interventional host
 * application that owns the GPU memory budget, or code running inside another
 * framework's memory pool -- and so cannot use pcs_create.
 *
 * Same iteration and arguments as pcs_solve_slices (H, W, b0_axis and the
 * stream given per call instead of through a context).  Its scratch (dual
 * variables, chibar, kernel tables) lives in static device arrays of fixed
 * size that every GPU loading libpcs holds until process exit (~16.5 MiB):
 * S*H*W may not exceed PCS_NOALLOC_MAX_VOXELS; larger calls fail with
 * PCS_EINVAL and a message.  The first call on a device sets that device up
 * (looks up the arrays' addresses, sets kernel attributes), and the first
 * call of each slice size and b0_axis uploads that size's kernel tables into
 * its own fixed region (waiting for the upload on the stream); a region is
 * never rewritten.  Make those first calls before any stream capture.  All
 * calls share the state arrays and each leaves its state in them; calls that
 * overlap on the GPU race and must be serialised by the caller.  Calls no
 * allocating CUDA or library routine.
 */
#define PCS_NOALLOC_MAX_VOXELS 1048576
PCS_API pcs_status pcs_solve_slices_noalloc(const float *field, const unsigned char *mask, int H, int W,
                                            int S, double lambda, double tau, double sigma, int n_iter,
                                            float *chi_out, int b0_axis, void *cuda_stream);

/*
 * pcs_solve_slices with monitoring: iterate in chunks of check_every
 * iterations; after each chunk evaluate the FP64 diagnostics of every slice
 * (as pcs_report) and, if rel_gap_tol > 0, freeze each slice whose
 * Fenchel-Young gap is <= rel_gap_tol * objective (its chi, p, q stay as they
 * are).  Chunks resume exactly from the stored state, so with
 * rel_gap_tol = 0 the result equals one n_iter-iteration solve bit for bit.
 * rep (host, S entries, required) receives each slice's last diagnostics and
 * its iteration count.  Synchronises the stream.  (The paper's stop is the
 * fixed count; the gap test is this library's optional monitor.)
 */
PCS_API pcs_status pcs_solve_slices_monitored(pcs_ctx *ctx, const float *field, const unsigned char *mask, int S,
                                              double lambda, double tau, double sigma, int n_iter, int check_every,
                                              double rel_gap_tol, float *chi_out, pcs_slice_report *rep);

/* Release the context and everything it owns. NULL-safe. */
PCS_API void pcs_destroy(pcs_ctx *ctx);

/* Thread-local text of the last error on this thread ("" if none). */
PCS_API const char *pcs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PCS_H */
