/*
 * aexp.h -- C ABI of the GB300 (sm_103a) expanded-encoding reconstruction library.
 *
 * The library solves Eq. (1) of Varela-Mattatall, Dubovan et al., "High-resolution
 * single-shot spiral diffusion-weighted imaging at 7T using expanded encoding with
 * compressed sensing" (MRM Technical Note):
 *
 *     x^ = argmin_x  ||A_exp x - y||_2^2 + lambda ||W x||_1                      (Eq. 1)
 *
 * with the matrix-free expanded encoding operator (Sec. 1: static B0 offsets plus
 * field dynamics expanded in spherical harmonics up to 2nd/3rd order; Sec. 2.1):
 *
 *     phi(t, r)   = sum_{l < nl} k_l(t) h_l(r) + omega(r) t
 *     (A x)_c(t)  = sum_r exp(-i phi(t, r)) S_c(r) x(r)
 *     (A^H y)(r)  = sum_c conj(S_c(r)) sum_t exp(+i phi(t, r)) y_c(t)
 *
 * Conventions for every entry point
 * ---------------------------------
 * - All array pointers are DEVICE pointers owned by the caller (allocate them with
 *   cudaMalloc or a framework allocator).  The library never allocates device memory
 *   on these paths; scratch comes from the caller's workspace `ws` of `ws_bytes`
 *   bytes, sized by the matching *_workspace_size() call.  `ws` must be 256-byte
 *   aligned (cudaMalloc memory is).
 * - Complex arrays are complex64: interleaved (re, im) float pairs, 8-byte aligned.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Every
 *   call is asynchronous on that stream; none synchronises the host unless stated.
 * - Image voxel r = iy * nx + ix (row-major, x fastest).  k-space y[c * nt + t].
 * - Return value: AEXP_OK (0) or a negative aexp_status.  On a negative return
 *   nothing was launched.  Errors discovered on the device (a bounded wait that gave
 *   up, a non-finite Lipschitz estimate) are written to a status word inside `ws`
 *   and read with aexp_read_status().
 * - Calls sharing one workspace must be ordered (same stream or explicit events);
 *   concurrent calls need separate workspaces.
 * - Limits: 1 <= nc <= 32, 1 <= nl + (omega != NULL) <= 32, nx, ny, nt >= 1.
 * - Results are bitwise repeatable for a given problem, precision and work-item layout:
 *   every reduction runs in a fixed order, also in the persistent tensor-core kernels.
 */
#ifndef AEXP_H
#define AEXP_H

#include <stddef.h>

#if defined(__GNUC__)
#define AEXP_API __attribute__((visibility("default")))
#else
#define AEXP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aexp_status {
    AEXP_OK = 0,
    AEXP_ERR_INVALID_ARG = -1,     /* null pointer, size out of range, bad enum      */
    AEXP_ERR_MISALIGNED = -2,      /* a pointer breaks its alignment rule           */
    AEXP_ERR_UNSUPPORTED = -3,     /* valid but outside the limits listed above     */
    AEXP_ERR_WORKSPACE = -4,       /* ws_bytes smaller than the size query returned */
    AEXP_ERR_CUDA = -5,            /* a CUDA runtime call failed; see aexp_last_cuda_error() */
    AEXP_ERR_DEVICE_TIMEOUT = -6,  /* a bounded device wait gave up (device status) */
    AEXP_ERR_NONFINITE = -7,       /* NaN/Inf in a device scalar (device status)    */
    AEXP_ERR_NOT_PREPARED = -8     /* workspace was not prepared for this problem   */
} aexp_status;

typedef enum aexp_precision {
    AEXP_FP32 = 0,        /* FP32 CUDA cores: phase, sincos and contraction in FP32   */
    AEXP_BF16_TC = 1,     /* encoding tile in BF16, tcgen05 tensor cores, FP32 accum  */
    AEXP_FP16X2_TC = 2    /* encoding tile and coil images split hi+lo in FP16        */
} aexp_precision;
/* Accuracy (relative L2 error of A x and A^H y against an FP64 evaluation of the operator
 * of Eq. 1, Sec. 2.1):
 *   AEXP_FP32       ~2e-7 .. 1.2e-6;
 *   AEXP_BF16_TC    ~2e-3 for white inputs (each factor rounded to 8 significant bits),
 *                   ~1e-4 .. 3e-4 for smooth images;
 *   AEXP_FP16X2_TC  ~5e-7 .. 3e-6: each operand value is v_hi + 2^-11 v_lo' in FP16,
 *                   products hi*hi + hi*lo + lo*hi on the tensor cores, accumulators
 *                   promoted to FP32 every 8 stages; the coil-weighted image (forward)
 *                   and the k-space data (adjoint) are scaled by a power of two chosen
 *                   from their largest component, so any finite FP32 input is accepted. */

/* How cs_recon obtains lambda: the caller's value, or the paper's rule (Supporting
 * Information S1, Method 2): lambda = sigma / 2 with sigma the maximum of the histogram of
 * the detail-coefficient magnitudes of W A^H y (needs `undecimated`; one level). */
typedef enum aexp_lambda_rule {
    AEXP_LAMBDA_GIVEN = 0,
    AEXP_LAMBDA_RAYLEIGH = 1
} aexp_lambda_rule;

typedef enum aexp_wavelet {
    AEXP_WAVELET_HAAR = 0, /* orthonormal Haar, 2 taps                          */
    AEXP_WAVELET_DB4 = 1   /* orthonormal Daubechies, 4 vanishing moments, 8 taps */
} aexp_wavelet;

/* One 2-D slice problem.  Every pointer is a device pointer; the arrays must stay
 * unchanged between aexp_prepare() and the operator calls that use the workspace. */
typedef struct aexp_problem {
    int nx, ny;           /* image size; nr = nx * ny                                    */
    int nt;               /* k-space samples per coil                                    */
    int nc;               /* receive coils                                               */
    int nl;               /* field terms: spherical harmonics (Sec. 1: up to 3rd order = 16;
                             4th order = 25) and any extra rows such as concomitant fields
                             (Fig. S3d); nl + (omega != NULL) <= 32                      */
    const float *k;       /* [nl][nt] field coefficients k_l(t), rad / m^deg(l)          */
    const float *h;       /* [nl][nr] basis values h_l(r), m^deg(l)                      */
    const float *omega;   /* [nr] static off-resonance (B0 map), rad/s, or NULL          */
    const float *t;       /* [nt] sample times, s (read only when omega != NULL)         */
    const void *S;        /* [nc][nr] complex64 coil sensitivities S_c(r)                */
} aexp_problem;

/* ---------------------------------------------------------------------------
 * Operator: A_exp and A_exp^H (Eq. 1; Sec. 2.1 writes the adjoint as A^T)
 * --------------------------------------------------------------------------- */

/* Bytes of device workspace that a_exp_forward / a_exp_adjoint need for `prob` at
 * `precision`.  Host-only; reads no device memory.  Writes *bytes. */
AEXP_API int aexp_workspace_size(const aexp_problem *prob, int precision, size_t *bytes);

/* Derive the operator's internal layouts from prob into ws: field coefficients in
 * turns as FP32 pairs, basis offsets per 8x8 voxel tile, the per-(tile, sample)
 * reference phase table, coil maps in tile order.  Must precede the operator calls
 * (stream-ordered) and be repeated whenever k, h, omega, t or S change. */
AEXP_API int aexp_prepare(const aexp_problem *prob, int precision, void *ws, size_t ws_bytes, void *stream);

/* The same two calls for a chosen launch shape: the work-item granularity items_per_sm and
 * the kernel tiling tile_variant, with the meanings and ranges of the aexp_recon_opts fields
 * of the same names (0, 0: the defaults, as above; e.g. the choice of aexp_autotune).  The
 * operator calls below run with the shape ws was prepared with.  AEXP_ERR_INVALID_ARG for a
 * value out of range. */
AEXP_API int aexp_workspace_size_tiled(const aexp_problem *prob, int precision, int items_per_sm, int tile_variant,
                                       size_t *bytes);
AEXP_API int aexp_prepare_tiled(const aexp_problem *prob, int precision, int items_per_sm, int tile_variant,
                                void *ws, size_t ws_bytes, void *stream);

/* y = A_exp x.  x: [nr] complex64 image; y: [nc][nt] complex64 (overwritten).
 * ws must have been prepared for prob and precision (aexp_prepare, aexp_prepare_tiled, or
 * a solver call on ws, whose workspace begins with the operator's); the launch shape is the
 * one it was prepared with.  Returns AEXP_ERR_NOT_PREPARED when the host-side record of the
 * last preparation of ws does not match prob and precision. */
AEXP_API int a_exp_forward(const aexp_problem *prob, int precision, const void *x, void *y,
                  void *ws, size_t ws_bytes, void *stream);

/* x = A_exp^H y.  y: [nc][nt] complex64; x: [nr] complex64 (overwritten). */
AEXP_API int a_exp_adjoint(const aexp_problem *prob, int precision, const void *y, void *x,
                  void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Compressed-sensing reconstruction: FISTA on Eq. (1) (Sec. 2.1, balanced FISTA;
 * with an orthonormal W its prox step is exactly the one used here)
 * --------------------------------------------------------------------------- */

typedef struct aexp_recon_opts {
    int precision;          /* aexp_precision of every A / A^H application              */
    int wavelet;            /* aexp_wavelet                                              */
    int levels;             /* wavelet levels J >= 1; the image is zero-padded to a
                               multiple of 2^J per side, W is orthonormal on the padded grid */
    int n_power;            /* power iterations for L_f = 2 lambda_max(A^H A); 0 with
                               lipschitz <= 0 is invalid                                 */
    double lipschitz;       /* > 0: use this L_f and skip the power iteration            */
    const void *x0;         /* [nr] complex64 start image, or NULL for zero              */
    const void *power_init; /* [nr] complex64 power-iteration start, or NULL for A^H y   */
    int use_graph;          /* nonzero: capture the whole loop in one CUDA graph         */
    int undecimated;        /* nonzero: the paper's regulariser W -- the one-level undecimated
                               (stationary) transform with the same filters, a tight frame
                               (W^H W = I); the prox step is W^H soft(W v) ("balanced"
                               FISTA, Sec. 2.1); `levels` is ignored                      */
    int lambda_rule;        /* aexp_lambda_rule                                          */
    double *lambda_out;     /* optional DEVICE double: the lambda used                   */
    int items_per_sm;       /* work-item granularity of the operator launches: the sample
                               (forward) and voxel (adjoint) reductions are split until a
                               launch holds about 152 x items_per_sm blocks or persistent
                               work items (shared among the problems of a batch); 0 = the
                               default (FP32 16, tensor cores 8); aexp_autotune picks one */
    int tile_variant;       /* kernel tiling of the operator launches, 0 = the default, 1 = the
                               alternative.  FP32 form at more than 20 coils (at fewer, 1 acts
                               as 0): two samples per forward thread and two voxels per adjoint
                               thread at 2 blocks per SM (default: one each at 4 blocks per
                               SM).  BF16 form: a 6-deep contraction-operand ring and 4
                               phase-operand stages (default 4 and 3).  FP16 hi+lo form: the
                               phase sums on the CUDA cores (default: on the tensor cores, like
                               the BF16 form).  aexp_autotune picks it; a workspace must be used
                               with the tiling it was prepared for */
} aexp_recon_opts;

/* Fill opts with defaults: FP32, Haar, 3 levels, 30 power iterations, estimate L_f,
 * zero start, A^H y power start, graph capture on, default work-item granularity. */
AEXP_API void aexp_recon_opts_default(aexp_recon_opts *opts);

/* Bytes of workspace cs_recon needs (includes the operator workspace). */
AEXP_API int aexp_recon_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes);

/* x_out = FISTA iterate after `iters` iterations on Eq. (1):
 *   F(x) = ||A x - y||^2 + lambda * sum over detail coefficients |(W pad x)_j|
 * (low-pass weight 0, Supporting Information S1), gradient 2 A^H (A z - y), step 1/L_f,
 * threshold lambda / L_f, momentum t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 in FP64.
 * y: [nc][nt] complex64; x_out: [nr] complex64.  lipschitz_out: optional DEVICE
 * pointer to one double that receives the L_f used.  Prepares ws itself. */
AEXP_API int cs_recon(const aexp_problem *prob, const void *y, float lambda, int iters,
             const aexp_recon_opts *opts, void *x_out, double *lipschitz_out,
             void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Coil compression (Sec. 2.2.1 compresses 32 receive channels to 20 virtual coils to speed the
 * reconstruction up; Sec. 2.2.2 compares 8, 16 and 32; the method is not stated -- here the
 * principal components of the k-space data): C = y y^H in FP64, its eigenvectors by cyclic
 * Jacobi on the device, U = the nv leading ones, each scaled so that its largest component is
 * real and positive; y_out = U^H y ([nv][nt] complex64), S_out = U^H S ([nv][nr] complex64).
 * The compressed problem is prob with nc = nv and S = S_out (the encoding matrix does not
 * depend on the coil).  eig_out: optional DEVICE double [nc], eigenvalues descending.
 * Reads prob->nc, nt, nr and S; nc <= 32, 1 <= nv <= nc.  A Jacobi iteration that has not
 * converged after 40 sweeps leaves AEXP_ERR_NONFINITE in the status word read by
 * aexp_coil_compress_status.
 * --------------------------------------------------------------------------- */
AEXP_API int aexp_coil_compress_workspace_size(int nc, size_t *bytes);
AEXP_API int aexp_coil_compress(const aexp_problem *prob, const void *y, int nv, void *y_out, void *S_out,
                                double *eig_out, void *ws, size_t ws_bytes, void *stream);
AEXP_API int aexp_coil_compress_status(const void *ws, int nc, void *stream, int *status);
/* The same with the Jacobi iteration capped at max_sweeps (1 ..= 40; aexp_coil_compress uses
 * 40): a cap that the iteration does not converge within is reported like a non-converged
 * default run, AEXP_ERR_NONFINITE in the status word. */
AEXP_API int aexp_coil_compress_sweeps(const aexp_problem *prob, const void *y, int nv, int max_sweeps, void *y_out,
                                       void *S_out, double *eig_out, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * The undecimated one-level wavelet on its own (Sec. 2.1; tight frame, subband s = fx + 2 fy
 * with f = lowpass 0 / highpass 1: LL, HL, LH, HH).  in/out: [ny][nx] complex64, coef:
 * [4][ny][nx] complex64 device arrays.  aexp_swt_prox: out = W^H soft_detail(W in, tau),
 * ws of aexp_swt_workspace_size bytes.  aexp_swt_lambda: *lambda_out (device double) =
 * sigma / 2 of the detail coefficients of W img (the lambda rule applied to img).
 * --------------------------------------------------------------------------- */
AEXP_API int aexp_swt_workspace_size(int nx, int ny, size_t *bytes);
AEXP_API int aexp_swt_forward(int nx, int ny, int wavelet, const void *in, void *coef, void *stream);
AEXP_API int aexp_swt_prox(int nx, int ny, int wavelet, float tau, const void *in, void *out, void *ws,
                           size_t ws_bytes, void *stream);
AEXP_API int aexp_swt_lambda(int nx, int ny, int wavelet, const void *img, double *lambda_out, void *ws,
                             size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Least-squares reconstruction: conjugate gradient on the normal equations A^H A x = A^H y
 * (CGLS) from x_0 = 0 with a fixed iteration count -- the paper's LS baseline, stopped early
 * at 20 iterations as implicit regularisation (Sec. 2.1, Supporting Information S2).  y:
 * [nc][nt] complex64; x_out: [nr] complex64.  opts: precision, items_per_sm and use_graph
 * are used, the wavelet and power-iteration fields are ignored.  FP64 device scalars; the
 * whole loop is one CUDA graph (use_graph, non-default stream).  Prepares ws itself.
 * --------------------------------------------------------------------------- */
AEXP_API int aexp_cgls_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes);
AEXP_API int cgls_recon(const aexp_problem *prob, const void *y, int iters, const aexp_recon_opts *opts,
                        void *x_out, void *ws, size_t ws_bytes, void *stream);

/* Estimate L_f = 2 lambda_max(A^H A) with n_power iterations from v0 ([nr] complex64,
 * not modified).  Result to the DEVICE double *lipschitz_out.  ws as for cs_recon. */
AEXP_API int aexp_power_lipschitz(const aexp_problem *prob, int precision, const void *v0, int n_power,
                         double *lipschitz_out, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Autotuning of the operator's launch shape (no counterpart in the paper; it serves the
 * ragged many-problem workload of Sec. 2.2.1's protocol grid).  Candidates: the work-item
 * granularity items_per_sm in {2, 4, 8, 16, 32} times the kernel tilings of the precision
 * (tile_variant 0 and 1 where the form has two, see aexp_recon_opts).  For each candidate
 * the call lays out the workspace, prepares the problem(s) and times one A^H A application
 * with CUDA events, after one warm-up, 5 times (3 for a batch): of `probs[0]` alone when
 * nprob == 1 (the cs_recon layout, any precision), of the whole batch when nprob > 1 (the
 * cs_recon_batched layout, tensor-core precisions only).  The candidate with the smallest
 * median wins, except that the default (items_per_sm 0's value, tile_variant 0) is kept when
 * it is within 1 % of it, so that near-ties do not flip between runs.  The choice goes to
 * *best_items_per_sm and *best_tile_variant, its median time in ms to *best_ms (optional),
 * and is remembered per device, precision and problem shape(s) for the life of the process:
 * a later call for the same shapes returns it without timing.  ws: device memory of
 * aexp_autotune_workspace_size bytes, whose contents are overwritten (a preparation of ws
 * for the operator calls is void afterwards).  The call synchronizes `stream` and returns
 * AEXP_ERR_INVALID_ARG while it is being captured; a device-side error status met while
 * timing is returned as it is.
 * --------------------------------------------------------------------------- */
AEXP_API int aexp_autotune_workspace_size(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts,
                                          size_t *bytes);
AEXP_API int aexp_autotune(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, void *ws,
                           size_t ws_bytes, void *stream, int *best_items_per_sm, int *best_tile_variant,
                           float *best_ms);

/* ---------------------------------------------------------------------------
 * Ragged batches: many independent slice problems (several resolutions, diffusion volumes
 * with their own field coefficients, slices) reconstructed together.  Sec. 2.2.1 acquires
 * 15 protocols x (1 b=0 + 6 directions) x 10 slices, each reconstructed as its own 2-D
 * problem (Sec. 2.1); here every operator application of the whole batch is one persistent
 * tensor-core launch and the complete solve is one CUDA graph.
 * --------------------------------------------------------------------------- */

/* Bytes of workspace cs_recon_batched needs.  probs: HOST array of nprob problems
 * (1 <= nprob <= 4095) whose padded coil and term counts agree (e.g. all 32 coils with
 * 3rd-order terms plus B0); opts->precision must be a tensor-core form. */
AEXP_API int aexp_batch_workspace_size(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts,
                                       size_t *bytes);

/* cs_recon for every problem of the batch, same wavelet, levels, iteration count and
 * power-iteration count; per-problem lambda.  y, x_out: HOST arrays of nprob device
 * pointers ([nc][nt] and [nr] complex64 per problem); lambda: HOST array of nprob floats;
 * lipschitz_out: optional DEVICE array of nprob doubles.  opts->x0 and opts->power_init
 * must be NULL (zero start, A^H y power start).  The first device-side error of any
 * problem is reported by aexp_read_status(ws). */
AEXP_API int cs_recon_batched(const aexp_problem *probs, int nprob, const void *const *y, const float *lambda,
                              int iters, const aexp_recon_opts *opts, void *const *x_out, double *lipschitz_out,
                              void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiation through unrolled FISTA.  Sec. 5 names unrolled CS as future work; these
 * two calls give one FISTA step of Eq. (1) with its state, and the step's vector-Jacobian
 * product, so that a caller can unroll K steps with per-step checkpoints (z_k) and
 * back-propagate to the start image, lambda and every k_l(t) (L_f held fixed).
 * Cotangents follow the real-loss convention dLoss/dRe + i dLoss/dIm.
 * --------------------------------------------------------------------------- */

/* Bytes of workspace for aexp_fista_step / aexp_fista_step_vjp (includes the operator
 * workspace, which must have been prepared with aexp_prepare for prob and opts->precision). */
AEXP_API int aexp_unroll_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes);

/* One step: v = z - (2/L) A^H (A z - y), x_out = crop W^H soft(W pad v, lambda/L),
 * z_out = x_out + beta (x_out - x_prev).  y: [nc][nt]; z, x_prev, x_out, z_out: [nr]
 * complex64 (x_out and z_out must not alias the inputs).  Uses opts->wavelet and levels. */
AEXP_API int aexp_fista_step(const aexp_problem *prob, const aexp_recon_opts *opts, const void *y, float lambda,
                             double lipschitz, const void *z, const void *x_prev, double beta, void *x_out,
                             void *z_out, void *ws, size_t ws_bytes, void *stream);

/* VJP of step k given its checkpoint z = z_k, b_k = beta, b_{k+1} = beta_next and the
 * cotangents zbar_next = zbar_{k+1}, zbar_next2 = zbar_{k+2} (NULL = 0) and xbar_in (extra
 * cotangent of x_k, NULL = 0):  xbar_k = (1+b_k) zbar_{k+1} - b_{k+1} zbar_{k+2} + xbar_in,
 * zbar_out = zbar_k = (I - (2/L) A^H A) crop W^H S'^T W pad xbar_k.  Accumulates (+=)
 * kbar [nl][nt] (float, device, may be NULL) and *lambar (double, device, may be NULL).
 * The start image's cotangent is zbar_1 (b_1 = 0). */
AEXP_API int aexp_fista_step_vjp(const aexp_problem *prob, const aexp_recon_opts *opts, const void *y, float lambda,
                                 double lipschitz, const void *z, double beta, double beta_next, const void *xbar_in,
                                 const void *zbar_next, const void *zbar_next2, void *zbar_out, float *kbar,
                                 double *lambar, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Wavelet step on its own (Eq. 1 regulariser): out = crop(W^H soft(W pad(in), tau))
 * --------------------------------------------------------------------------- */

/* Bytes of workspace aexp_wavelet_prox needs. */
AEXP_API int aexp_wavelet_workspace_size(int nx, int ny, int wavelet, int levels, size_t *bytes);

/* Soft-threshold (w -> w max(0, 1 - tau/|w|)) of the detail coefficients only;
 * in, out: [ny][nx] complex64 (may alias).  tau >= 0. */
AEXP_API int aexp_wavelet_prox(int nx, int ny, int wavelet, int levels, float tau, const void *in,
                      void *out, void *ws, size_t ws_bytes, void *stream);

/* Forward transform only: coef = W pad(in), coef: [Npy][Npx] complex64 in Mallat
 * layout, Npy = ceil(ny / 2^J) 2^J (same for x). */
AEXP_API int aexp_wavelet_forward(int nx, int ny, int wavelet, int levels, const void *in, void *coef,
                         void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Allocation-free wavelet step (no counterpart in the paper)
 * --------------------------------------------------------------------------- */

/* Same result as aexp_wavelet_prox, but without a caller workspace: the scratch (the
 * wavelet pyramid and the intermediate approximation images) is a fixed 4 MiB device
 * array inside the library, reserved on every GPU that loads the library until the
 * process exits.  For callers that cannot allocate device memory at the point of the
 * call -- code running while a CUDA stream is being captured (cudaMalloc is not allowed
 * then), real-time reconstruction services that reserve all GPU memory at start-up and
 * forbid later allocations, and plug-ins whose host framework owns the device allocator.
 * The call itself allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 * - Size limit: the zero-padded image (each side rounded up to a multiple of 2^levels)
 *   must have a pyramid of at most 4 MiB, about 4/3 * npy * npx * 8 bytes, i.e. up to
 *   512 x 512; larger sizes return AEXP_ERR_UNSUPPORTED and launch nothing.
 * - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *   with that device current, and caches it for the life of the process; make that first
 *   call before any stream capture.  A cudaDeviceReset (or anything else that destroys the
 *   device's primary context) makes the cached address stale: do not call this entry point
 *   on that device again in the same process after such a reset.
 * - All calls share the one array and it keeps the last call's contents; each call writes
 *   every scratch byte it reads, so nothing is cleared.  Calls that overlap on the GPU
 *   (different streams, or different host threads on one device) race on the array:
 *   order them, e.g. on one stream.
 * in, out: [ny][nx] complex64 device arrays (may alias); tau >= 0. */
AEXP_API int aexp_wavelet_prox_static(int nx, int ny, int wavelet, int levels, float tau, const void *in,
                                      void *out, void *stream);

/* ---------------------------------------------------------------------------
 * Failure detection probe (no counterpart in the paper)
 * --------------------------------------------------------------------------- */

/* Checks on the device that the library's bounded waits end and report instead of hanging:
 * one block in which one thread waits on an mbarrier phase that nothing completes, through the
 * same bounded wait the operator kernels use but limited to `polls` polls (1 ..= 2^22), and a
 * second thread waits on another such barrier through the tensor-core kernels' wait, which
 * gives up as soon as another thread of its block has.  Afterwards the status word of `ws`
 * (read with aexp_read_status) holds AEXP_ERR_DEVICE_TIMEOUT and the DEVICE ints
 * result[0], result[1] are 1 (each wait gave up).  Nothing is left in flight; the context
 * stays usable.  ws: any 256-byte-aligned device buffer of at least aexp_header_bytes()
 * bytes whose status word is 0 (e.g. a fresh operator workspace). */
AEXP_API int aexp_probe_bounded_wait(int polls, int *result, void *ws, size_t ws_bytes, void *stream);
/* Bytes of the header at the start of every workspace (status word first). */
AEXP_API size_t aexp_header_bytes(void);

/* ---------------------------------------------------------------------------
 * Status
 * --------------------------------------------------------------------------- */

/* Synchronise `stream`, read and clear the device status word in ws (AEXP_OK when
 * no device-side error was recorded since the last read). */
AEXP_API int aexp_read_status(void *ws, void *stream, int *status);

/* Short English description of a status code; never NULL. */
AEXP_API const char *aexp_status_string(int status);

/* The cudaError_t value of the last AEXP_ERR_CUDA on this host thread. */
AEXP_API int aexp_last_cuda_error(void);

/* Library version, e.g. 100 for 0.1.0. */
AEXP_API int aexp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AEXP_H */
