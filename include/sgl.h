/*
 * sgl.h -- C-ABI of the GB300 (sm_103a) implementation of the non-lattice fast
 * SGL Fourier transform (NFSGLFT), its adjoint and its point gradient, after
 * C. Wuelker, "Fast SGL Fourier transforms for scattered data" (arXiv:1809.10786).
 *
 * Notation (paper, Sect. 1):
 *   H_nlm(x) = N_nl R_nl(r) Y_lm(theta, phi), 1 <= n <= B, 0 <= l < n, |m| <= l.
 *   Coefficients are stored in the paper's linear order
 *       mu(n, l, m) = n(n-1)(2n-1)/6 + l(l+1) + m,   0 <= mu < Nc = B(B+1)(2B+1)/6.
 *   The NDSGLFT matrix is Lambda = [H_{n(mu) l(mu) m(mu)}(x_i)]_{i, mu} (Def. of the NDSGLFT);
 *   the forward transform computes f = Lambda fhat, the adjoint fhat' = Lambda^H f.
 *
 * Method (Sect. 6, Thm. on the factorization of Lambda): dense radial and polar
 * conversion products (FP64) turn fhat into the coefficients eta_k of a 3-D
 * trigonometric polynomial in xtilde = [arccos((2r - rho)/rho), theta, phi];
 * a 3-D NFFT (Sect. 2: window deconvolution, oversampled inverse FFT, windowed
 * interpolation) evaluates it at the points.  The adjoint runs the conjugate
 * transposed factors in reverse order (Sect. 6, Cor. on Lambda^H).  The only
 * approximation is the NFFT (Sect. 7).
 *
 * Conventions for every call below:
 *   - Device pointers are CUDA global-memory pointers on the plan's device,
 *     8-byte aligned at least (16-byte aligned recommended).  Host pointers are
 *     ordinary (pageable or pinned) host memory.  The caller owns every buffer
 *     passed in; the library never frees or retains them beyond the call.
 *   - Complex numbers are interleaved (re, im) pairs of double (complex128).
 *     Outputs are always complex128, in both precisions.
 *   - Points are [M][3] double, row-major (x, y, z).
 *   - All device-pointer calls are asynchronous on the plan's stream; results
 *     are ready when that stream reaches the call's position.  Input buffers
 *     must stay valid until then.
 *   - A plan owns its workspace (allocated by sgl_plan_create) and is not
 *     re-entrant: use one plan per stream / host thread at a time.
 *   - Every function returns an sgl_status; none throws or aborts.  On failure
 *     sgl_last_error() returns a message (thread-local, valid until the next
 *     call on that thread).  Errors raised asynchronously on the device (a
 *     non-finite input point) are reported by the next sgl_sync().
 */
#ifndef SGL_H
#define SGL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SGL_OK = 0,
    SGL_ERR_ARG = 1,          /* invalid argument (size, pointer, alignment, enum) */
    SGL_ERR_ALLOC = 2,        /* device or host allocation failed */
    SGL_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SGL_ERR_NONFINITE = 4,    /* a point coordinate was NaN or infinite */
    SGL_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
    SGL_ERR_UNSUPPORTED = 6,  /* valid but not supported by this build (e.g. FFT size) */
    SGL_ERR_STATE = 7         /* call out of order (e.g. forward before set_points) */
} sgl_status;

typedef enum {
    SGL_FP64 = 0,             /* binary64 throughout, except that interpolation, gradient and
                                 spreading run in double-float arithmetic (FP32 pairs, relative
                                 rounding ~2^-48) unless SGL_FLAG_NATIVE_FP64 is set */
    SGL_FP32_MIXED = 1        /* FFT, interpolation and spreading in binary32; conversions,
                                 recurrences and deconvolution factors in binary64 */
} sgl_precision;

typedef enum {
    SGL_WIN_KB = 0,           /* Kaiser-Bessel window (sinh form, shape b = pi(2 - 1/sigma)) */
    SGL_WIN_GAUSS = 1         /* Gaussian window of Sect. 2 (lambda = sigma q / ((2 sigma - 1) pi)) */
} sgl_window;

/* plan flags */
#define SGL_FLAG_HOST_IO 1u   /* also allocate staging buffers for the *_host calls */
#define SGL_FLAG_PROFILE 2u   /* record CUDA events around every stage (read with sgl_profile) */
#define SGL_FLAG_SIMT 4u      /* FP32-mixed: interpolate and take gradients with the CUDA-core kernels only */
#define SGL_FLAG_TC 8u        /* FP32-mixed: use the tensor-core (tcgen05) interpolation and gradient
                                 kernels wherever the plan allows them (q <= 8, windowed axes 0
                                 and 1), not only where they are the faster choice */
#define SGL_FLAG_NATIVE_FP64 16u  /* FP64: run interpolation, gradient and spreading in binary64
                                 arithmetic.  Without it these three loops use double-float
                                 arithmetic (pairs of FP32 numbers with error-free products and
                                 sums, relative rounding of order 2^-48 per operation; window
                                 values, reductions and everything else stay binary64), which
                                 runs several times faster on the FP32 pipes */
#define SGL_FLAG_OVERLAP_POINTS 32u  /* bin the points of sgl_set_points on a plan-owned stream
                                 (rho stays on the plan's stream), so that the binning overlaps
                                 the conversions and the FFT of the next forward; the first
                                 call that reads the bins waits for it.  Results and the stream
                                 semantics of every call are unchanged.  Measured on one GB300
                                 at B = 64, 10^6 points, FP32-mixed, step = set_points + forward
                                 with the gradient + adjoint: 3.344 -> 3.253 ms when the host
                                 waits for every step, but 3.375 -> 3.52 ms when steps are
                                 queued back to back.  FP64 plans compute the points' angles on
                                 the FP64 pipe, where they compete with the conversions.  Not
                                 accepted for batches */
#define SGL_FLAG_GENERIC_FFT 64u  /* run every FFT pass with the generic mixed-radix kernel (tiles of
                                 lines staged in shared memory, one radix stage per pass over
                                 the tile) instead of the register kernels that power-of-two
                                 lengths 64 ... 1024 take by default.  Same results to rounding */
#define SGL_FLAG_FULL_GRID 128u  /* transform the whole kept grid.  By default, where axes 0 and 1 are
                                 windowed, the FFT passes use the symmetries of eta (Sect. 6: even in
                                 kappa0, parity of m in kappa1): the radial pass transforms the
                                 lines kappa1 >= 0 only, and the two angular passes the grid
                                 lines of [0, N0/2] x [0, N1/2], whose mirrors fill the q halo
                                 rows; the adjoint folds in the same places.  Same results to
                                 rounding */

/* stages reported by sgl_profile (index order) */
#define SGL_NUM_STAGES 12

typedef struct sgl_plan sgl_plan;

/* Sizes of a plan (filled by sgl_plan_info). */
typedef struct {
    int B;                    /* bandwidth */
    int q;                    /* window cutoff: half-width in oversampled grid cells (2q taps per axis) */
    int precision;            /* sgl_precision */
    int window;               /* sgl_window */
    int64_t num_coeffs;       /* Nc = B(B+1)(2B+1)/6 */
    int64_t M_max;            /* capacity in points */
    int64_t M;                /* points of the last sgl_set_points */
    int n[3];                 /* conversion grid (4B, 2B, 2B), axes (radial, polar, azimuthal) */
    int N[3];                 /* oversampled FFT grid (>= sigma n, 2-3-5-smooth) */
    int rows[3];              /* grid rows held per axis after the pruned FFT */
    double sigma_eff[3];      /* N[d] / n[d] */
    int64_t workspace_bytes;  /* device bytes owned by the plan */
    int64_t kernel_launches;  /* CUDA kernels this plan has launched so far */
    int tensor_cores;         /* bit 0: interpolation, bit 1: gradient run on the tcgen05 kernels;
                                 bit 2 (spreading) is 0: spreading runs on the CUDA cores */
    int sym_grid;             /* 1: the FFT passes use the symmetry-reduced grid (see
                                 SGL_FLAG_FULL_GRID), 0: they transform every kept line */
} sgl_plan_info_t;

/* Nc = B(B+1)(2B+1)/6 (Sect. 1); -1 if B < 1. */
int64_t sgl_num_coeffs(int B);

/*
 * Create a plan for bandwidth B (1 <= B <= 128) and at most M_max points
 * (0 <= M_max < 2^31).  precision: sgl_precision; window: sgl_window; q: window
 * cutoff, 1 <= q <= 16 (the paper's cutoff parameter, Sect. 2); sigma: requested
 * oversampling factor, 1.5 <= sigma <= 4 (the FFT grid is rounded up to the next
 * even 2-3-5-smooth size per axis, so the effective factor is >= sigma).
 * cuda_stream: a cudaStream_t (NULL: the legacy default stream).  The plan
 * uses the current CUDA device.  Host work: FP64 precompute of the polar
 * conversion matrices (Sect. 6, P_m = W_m D C~ Vtilde L_m^T diag Q) and the window
 * Fourier factors.  On failure *out is NULL and nothing is leaked.
 */
sgl_status sgl_plan_create(sgl_plan **out, int B, int64_t M_max, int precision, int window,
                           int q, double sigma, unsigned flags, void *cuda_stream);

/* Release the plan and all of its device memory (synchronizes its stream). NULL is a no-op. */
void sgl_plan_destroy(sgl_plan *plan);

/* Change the stream later calls are issued on. */
sgl_status sgl_set_stream(sgl_plan *plan, void *cuda_stream);

/* Fill *info with the plan's sizes. */
sgl_status sgl_plan_info(const sgl_plan *plan, sgl_plan_info_t *info);

/*
 * Set the M points (0 <= M <= M_max) the next transforms use: xyz_dev [M][3]
 * (device).  Computes rho = max_i |x_i| on the device (Sect. 7 choice of rho,
 * with a relative margin of 2^-20 so that every point has arccos argument < 1),
 * the transformed points xtilde_i (Sect. 6, eq. of the transformed points) and a
 * spatial bin sort of the points (no host synchronization).  The coordinates
 * are copied; xyz_dev may be reused once the stream passes this call.
 * Non-finite coordinates set a device flag reported by sgl_sync().
 */
sgl_status sgl_set_points(sgl_plan *plan, const double *xyz_dev, int64_t M);
/* (with SGL_FLAG_OVERLAP_POINTS the points are copied into plan memory on the plan's stream
   before the binning forks, so xyz_dev may still be reused once the stream passes this call) */

/* rho used by the plan (synchronizes the stream); SGL_ERR_STATE before set_points. */
sgl_status sgl_get_rho(sgl_plan *plan, double *rho_host);

/*
 * Forward NFSGLFT: vals_dev[i] ~= f(x_i) = sum_mu coef_dev[mu] H_mu(x_i), i < M
 * (Def. of the NDSGLFT; Sect. 6 factorization, Sect. 2 NFFT).
 * coef_dev: complex128 [Nc] in mu order (device); vals_dev: complex128 [M] in the
 * order the points were given (device).  SGL_ERR_STATE before sgl_set_points.
 */
sgl_status sgl_forward(sgl_plan *plan, const double *coef_dev, double *vals_dev);

/*
 * Adjoint NFSGLFT: coef_dev[mu] ~= sum_i conj(H_mu(x_i)) vals_dev[i] (Lambda^H,
 * Sect. 6 corollary).  vals_dev: complex128 [M]; coef_dev: complex128 [Nc], fully
 * overwritten (zeros when M = 0).
 */
sgl_status sgl_adjoint(sgl_plan *plan, const double *vals_dev, double *coef_dev);

/*
 * Point gradient of the forward map:
 *   gxyz_dev[i][d] = Re( conj(gout_dev[i]) * d f(x_i) / d x_{i,d} ),  f = Lambda coef,
 * the vector-Jacobian product of the forward transform with respect to the points
 * (rho held fixed: the exact factorization holds for every rho >= max r).
 * The derivative of the NFFT approximant is taken through the window derivative.
 * coef_dev: complex128 [Nc]; gout_dev: complex128 [M]; gxyz_dev: double [M][3].
 */
sgl_status sgl_grad_points(sgl_plan *plan, const double *coef_dev, const double *gout_dev,
                           double *gxyz_dev);

/*
 * The trigonometric coefficients of Sect. 6 (eq. of the NFFT sum): eta_dev receives
 * eta_k for |k0| <= 2B-2, |k1| <= B-1, |k2| <= B-1 as complex128
 * [4B-3][2B-1][2B-1], index (k0 + 2B-2, k1 + B-1, k2 + B-1), so that
 *   f(x) = sum_k eta_k exp(i <k, xtilde>)  exactly (before any NFFT approximation).
 * Needs sgl_set_points (eta depends on rho).  coef_dev: complex128 [Nc].
 */
sgl_status sgl_trig_coeffs(sgl_plan *plan, const double *coef_dev, double *eta_dev);

/*
 * Forward transform and point gradient together: vals_dev = Lambda coef (as sgl_forward) and
 * gxyz_dev as sgl_grad_points, from one pass of the conversions, the FFT and one windowed
 * sweep (the value is the gradient sweep's s itself), which is what a loss-and-gradient step
 * needs.  coef_dev complex128 [Nc]; gout_dev complex128 [M]; vals_dev complex128 [M];
 * gxyz_dev double [M][3]; all device pointers, 8-byte aligned, on the plan's stream.
 */
sgl_status sgl_forward_grad(sgl_plan *plan, const double *coef_dev, const double *gout_dev,
                            double *vals_dev, double *gxyz_dev);

/*
 * Inverse transform (iNFSGLFT; Sect. 7, end, after the iNFFT of Sect. 2): SGL Fourier
 * coefficients from the M samples vals_dev[i] = f(x_i) at the plan's points, by conjugate
 * gradients on the normal equations with one sgl_forward and one sgl_adjoint per iteration:
 *   method 1 CGNR (normal equations of the first kind; least squares, for M >= Nc),
 *   method 2 CGNE (second kind; minimum-norm solution, for M < Nc),
 *   method 0 picks CGNR if M >= Nc, else CGNE.
 * coef_dev complex128 [Nc]: the initial guess on entry (zeros, or sgl_midpoint_guess), the
 * last iterate on return.  Stops after `iters` iterations or once ||f - Lambda c|| <= tol ||f||.
 * residual_out (host, may be NULL): the final ||f - Lambda c|| / ||f||; iters_out (host, may
 * be NULL): iterations done.  Synchronizes the stream (the step sizes are formed on the host in
 * extended precision from device-reduced norms).  The first call allocates four work vectors
 * (2 M_max + 2 Nc complex128), owned by the plan.
 */
sgl_status sgl_inverse(sgl_plan *plan, const double *vals_dev, double *coef_dev, int iters, double tol,
                       int method, double *residual_out, int *iters_out);

/*
 * Quadrature initial guess for sgl_inverse: coef_dev = Lambda^H (w .* vals), i.e. the rule
 * sum_i w_i f(x_i) conj(H_nlm(x_i)) for the inner product that makes the H_nlm orthonormal
 * (the paper's last test, Sect. 8: the mid-point rule on a Cartesian grid, w_i = h^3 e^{-|x_i|^2}).
 * weights_dev double [M]; vals_dev complex128 [M]; coef_dev complex128 [Nc] (device).
 */
sgl_status sgl_midpoint_guess(sgl_plan *plan, const double *vals_dev, const double *weights_dev, double *coef_dev);

/*
 * Error control.  The factorization of Lambda is exact (Sect. 7, error estimate: the final NFFT
 * is the only approximating step), so for every coefficient vector
 *     max_i |f(x_i) - f~(x_i)| <= bound * ||eta||_1,
 * with eta the trigonometric coefficients of f (sgl_trig_coeffs) and bound the worst error of the
 * windowed interpolation on a single frequency: per axis d, e_d = max over |k| <= K_d and over
 * the fractional grid positions f = (i + 1/2) / 128, i < 128, of
 * |1 - Psi(k)^-1 sum_taps psi(x_j) exp(-2 pi i k x_j / N_d)|,
 * x_j = f + q - 1 - j, and bound = prod_d (1 + e_d) - 1 (the three axes' factors multiply).  This
 * is the quantity the paper's theorem on the NFFT error bounds for the Gaussian window (aliasing
 * plus truncation), evaluated for the plan's own window, q, oversampled grid sizes and frequency
 * ranges.  It bounds the approximation in exact arithmetic, with the maximum over f taken on
 * the 128 sampled positions; the rounding of the plan's precision comes on top (FP32-mixed:
 * about 1e-7 relative).  Host computation, no GPU needed (except sgl_eta_l1).
 *
 * sgl_nfft_error_bound: the bound for a plan that sgl_plan_create(B, ..., window, q, sigma)
 *   would make.  Errors: SGL_ERR_ARG for parameters sgl_plan_create rejects.
 * sgl_plan_error_bound: the same for an existing plan.
 * sgl_choose_cutoff: the smallest q in [1, 16] whose bound is <= tol (error-driven choice of the
 *   cutoff for a target accuracy per unit ||eta||_1); SGL_ERR_UNSUPPORTED if none reaches tol.
 * sgl_eta_l1: ||eta||_1 of coef_dev (complex128 [Nc], device) for the plan's current points (rho
 *   enters eta); synchronizes the stream.  bound * ||eta||_1 bounds this transform's error.
 */
/*
 * sgl_choose_params: error-driven choice of both NFFT parameters.  Over the oversampling factors
 *   sigma in {1.5, 2, 2.5, 3, 4}, takes for each the smallest q whose bound (as sgl_nfft_error_bound)
 *   is <= tol, and returns the pair that a cost model of one forward plus one adjoint transform of M
 *   points rates cheapest: M (2q)^3 c_tap + (stored grid cells) c_cell milliseconds, with per-tap
 *   and per-cell costs of the windowed loops and the FFT passes measured on GB300 for the given
 *   precision (the conversions, which depend on neither parameter, are left out).  sigma, q: the
 *   choice; model_ms (may be NULL): the model's estimate in milliseconds.  SGL_ERR_UNSUPPORTED if
 *   no pair reaches tol; SGL_ERR_ARG for invalid B, M < 0, precision, window or tol <= 0.
 */
sgl_status sgl_nfft_error_bound(int B, int window, int q, double sigma, double *bound);
sgl_status sgl_plan_error_bound(const sgl_plan *plan, double *bound);
sgl_status sgl_choose_cutoff(int B, int window, double sigma, double tol, int *q);
sgl_status sgl_choose_params(int B, int64_t M, int precision, int window, double tol, double *sigma, int *q,
                             double *model_ms);
sgl_status sgl_eta_l1(sgl_plan *plan, const double *coef_dev, double *l1);

/*
 * Host-buffer variants (need SGL_FLAG_HOST_IO): copy the inputs from host memory
 * into the plan's staging buffers, run set_points + forward (or adjoint) on the
 * plan's stream, copy the result back and synchronize the stream before returning.
 * xyz_host [M][3] double; coef_host complex128 [Nc]; vals_host complex128 [M].
 * xyz_host NULL keeps the points of the previous call (no copy, no re-binning); M must then
 * equal their number (SGL_ERR_ARG otherwise, or if no points are set).
 */
sgl_status sgl_forward_host(sgl_plan *plan, const double *xyz_host, int64_t M,
                            const double *coef_host, double *vals_host);
sgl_status sgl_adjoint_host(sgl_plan *plan, const double *xyz_host, int64_t M,
                            const double *vals_host, double *coef_host);
/* gout_host complex128 [M]; gxyz_host double [M][3] (see sgl_grad_points). */
sgl_status sgl_grad_points_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *coef_host,
                                const double *gout_host, double *gxyz_host);
/* vals_host complex128 [M]; gxyz_host double [M][3] (see sgl_forward_grad). */
sgl_status sgl_forward_grad_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *coef_host,
                                 const double *gout_host, double *vals_host, double *gxyz_host);

/*
 * Per-stage device times of a plan created with SGL_FLAG_PROFILE: synchronizes the
 * stream, writes the summed milliseconds (ms_out) and the number of timed calls
 * (count_out) of each of the SGL_NUM_STAGES stages since the last call, then resets.
 * Either output may be NULL.  Stage names: sgl_stage_name(i).
 */
sgl_status sgl_profile(sgl_plan *plan, double *ms_out, int64_t *count_out);
const char *sgl_stage_name(int stage);

/*
 * Allocation-free trigonometric coefficients (the paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory).  Some applications own all
 * of their device memory through their own pool allocator, or run under a fixed memory
 * budget; for them a library call to cudaMalloc/cudaFree may fail or synchronize the
 * device at a bad moment, and sgl_plan_create allocates.  This entry point computes the
 * same eta as sgl_trig_coeffs for the points xyz_dev (rho = max |x_i| with the same
 * 2^-20 margin) without allocating: no cudaMalloc, no cudaFree, no allocating library
 * routine.  Its scratch is one static device array sized for B <= SGL_NOALLOC_MAX_B
 * (about 6.9 MB, the conversion tables of every such B included), which every GPU that
 * loads the library holds until process exit.
 *   B: 1 <= B <= SGL_NOALLOC_MAX_B, otherwise SGL_ERR_ARG with a message naming the limit.
 *   xyz_dev [M][3] double (device, M >= 0; M = 0 gives rho = 1); coef_dev complex128 [Nc]
 *   (device); eta_dev complex128 [4B-3][2B-1][2B-1] (device), layout as in sgl_trig_coeffs.
 *   cuda_stream: the stream the work is issued on (asynchronous, like the plan calls).
 * Set-up: the first call on a device looks up the scratch array's device address on the
 * current device, copies the conversion tables (built once per process in host static
 * storage) into the array on cuda_stream and synchronizes that stream.  That first call
 * returns SGL_ERR_STATE inside a stream capture: make it before capturing.  Later calls
 * issue one memset and the conversion kernels only.
 * All calls share the one scratch array, which keeps the last call's contents (the
 * reduction cell is cleared by each call): calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race on it and must be serialized by the caller.
 * Non-finite coordinates are left out of rho and not reported.
 * sgl_noalloc_max_b() returns SGL_NOALLOC_MAX_B of the loaded library.
 */
#define SGL_NOALLOC_MAX_B 32
int sgl_noalloc_max_b(void);
sgl_status sgl_trig_coeffs_noalloc(int B, const double *xyz_dev, int64_t M, const double *coef_dev,
                                   double *eta_dev, void *cuda_stream);

/*
 * Fault injection for tests of the failure paths (the paper has no counterpart).
 * sgl_test_hooks: hooks bit SGL_TEST_WITHHOLD_ARRIVAL makes the prep warps of the tensor-core
 *   interpolation and gradient kernels withhold their operand arrival, so that the kernel's bounded
 *   waits run out: it issues no tensor-core product, drains its loads, frees its tensor memory and
 *   returns, and the next sgl_sync reports SGL_ERR_TIMEOUT (that call's results are invalid).
 *   wait_cycles: the limit of those waits in clock cycles (0: the default, about a second); hooks 0
 *   and wait_cycles 0 restore normal operation.  SGL_ERR_ARG for unknown bits or wait_cycles < 0.
 * sgl_test_fail_alloc: after >= 0 lets that many further device allocations of the library
 *   succeed and fails the next one (once), as if cudaMalloc had run out of memory; after < 0 turns
 *   the injection off.  Process-wide.
 */
#define SGL_TEST_WITHHOLD_ARRIVAL 1u
sgl_status sgl_test_hooks(sgl_plan *plan, unsigned hooks, int64_t wait_cycles);
sgl_status sgl_test_fail_alloc(int after);

/* Synchronize the plan's stream and report deferred device errors (non-finite points). */
sgl_status sgl_sync(sgl_plan *plan);

/*
 * Batches: n independent transforms, instance i with bandwidth B[i] and at most
 * M_max[i] points, all with the same precision, window, q and sigma, issued together
 * (Def. of the NDSGLFT applied per instance).  The instances are spread over L lanes -- each a
 * stream of its own with FFT work buffers shared by the instances of that lane -- by a cost
 * estimate (longest first onto the least loaded lane), so that small instances run side by side;
 * every batch call forks from the batch's stream into the lanes and joins back, so its results
 * are ordered on the batch's stream like a single call.  L starts at min(n, 8); sgl_batch_set_lanes
 * changes it (1 <= L <= min(n, 32)) and sgl_batch_autotune chooses it by timing.
 * With sgl_batch_use_graph(b, 1) a batch forward or adjoint (fork, every lane's kernels, join) is
 * captured into one CUDA graph the first time and replayed while the pointer arrays and point
 * counts are the same as at capture (a change, new points or new lanes recapture).  Pointer
 * arrays are host arrays of n device pointers, with the per-instance layouts of sgl_forward /
 * sgl_adjoint.  SGL_FLAG_PROFILE and SGL_FLAG_OVERLAP_POINTS are not accepted for batches.
 * sgl_batch_autotune: with cache_path (may be NULL) naming a JSON file that already holds this
 *   batch's entry (keyed on precision, window, q, sigma, n and a hash of the (B, M_max) list), takes
 *   its lane count; otherwise times a forward plus an adjoint (two untimed, three timed, graph mode
 *   as set) for L = 1, 2, 4, 8, 16, 32 (<= n), keeps the fastest and records all timings in the
 *   file.  Needs sgl_batch_set_points; allocates and releases one block of timing inputs.
 *   lanes_out, ms_out (may be NULL): the choice and its time per forward + adjoint (-1 if cached).
 */
typedef struct sgl_batch sgl_batch;
sgl_status sgl_batch_create(sgl_batch **out, int n, const int *B, const int64_t *M_max, int precision, int window,
                            int q, double sigma, unsigned flags, void *cuda_stream);
void sgl_batch_destroy(sgl_batch *batch);
sgl_status sgl_batch_use_graph(sgl_batch *batch, int enable);
sgl_status sgl_batch_set_points(sgl_batch *batch, const double *const *xyz_dev, const int64_t *M);
sgl_status sgl_batch_forward(sgl_batch *batch, const double *const *coef_dev, double *const *vals_dev);
sgl_status sgl_batch_adjoint(sgl_batch *batch, const double *const *vals_dev, double *const *coef_dev);
/* n, graph replays so far, device bytes owned (any output may be NULL) */
sgl_status sgl_batch_info(const sgl_batch *batch, int *n, int64_t *graph_launches, int64_t *workspace_bytes);
sgl_status sgl_batch_set_lanes(sgl_batch *batch, int lanes);
sgl_status sgl_batch_lanes(const sgl_batch *batch, int *lanes);
sgl_status sgl_batch_autotune(sgl_batch *batch, const char *cache_path, int *lanes_out, double *ms_out);
/* synchronize the stream and report deferred device errors of any instance */
sgl_status sgl_batch_sync(sgl_batch *batch);

/* Message of the last failing call on this thread ("" if none). */
const char *sgl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGL_H */
