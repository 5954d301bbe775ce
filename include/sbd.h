/*
 * sbd.h - C ABI of the GB300 Sparse Bessel Decomposition library (libsbd.so).
 *
 * The library computes the approximate 2-D discrete convolution
 *
 *     q_k = sum_{l != k} G(z_k - z_l) f_l,      k = 1..N            (Introduction, Eq. discreteConv)
 *
 * for the Laplace kernel G(x) = -log|x| / (2 pi) and the Helmholtz kernel
 * G(x) = (i/4) H0^(1)(kappa |x|), by the Sparse Bessel Decomposition of
 * M. Averseng, arXiv:1711.07877:
 *
 *   off-line (sbd_plan, Sec. 1 "Off-line part", Sec. 3-5, Sec. 6.1): fit G on
 *     [delta_min, delta_max] by a Fourier-Bessel series sum_p alpha_p e_p, turn each
 *     J0 term into M_p plane waves on a circle of frequencies (circular quadrature),
 *     and assemble the sparse close-correction matrix D of Eq. (defD);
 *   on-line (sbd_matvec, Sec. 1 "On-line part", Sec. 6.2): q = q_far + D f with
 *     q_far = NUFFT_+[z, xi](omega_hat . NUFFT_-[z, xi](f))  (Eq. far convolution).
 *
 * Every on-line step runs in this library's CUDA kernels for sm_103a; nothing
 * falls back to the CPU.  The output satisfies, up to rounding of the chosen
 * form, |q_k - exact_k| <= eps * sum_l |f_l| (Sec. 1, output bound).
 *
 * Conventions for every entry point:
 *   - Return SBD_OK (0) on success and a negative SBD_E* code on error; nothing
 *     is written to outputs on argument errors.  sbd_error_string() names a code
 *     and sbd_last_error_message() gives the calling thread's last detail text.
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library owns the plan and its device memory.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it asynchronously unless stated otherwise.
 *   - Vectors with several right-hand sides are stored right-hand side by
 *     right-hand side: element l of rhs r is at index r * N + l.
 *   - Laplace vectors are float64; Helmholtz vectors are complex128 stored as
 *     interleaved (re, im) float64 pairs.
 */
#ifndef SBD_H
#define SBD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define SBD_OK         0
#define SBD_EINVAL    -1   /* invalid argument (null pointer, size, tolerance, kernel) */
#define SBD_ENOMEM    -2   /* device or host allocation failed */
#define SBD_ECUDA     -3   /* a CUDA runtime call failed (no device, launch error, ...) */
#define SBD_EFIT      -4   /* the SBD fit cannot reach the requested tolerance (Sec. 4.1 floor ~1e-10) */
#define SBD_ETIMEOUT  -5   /* a bounded device wait expired */
#define SBD_ENOTSUP   -6   /* combination not supported by this build */

typedef struct sbd_plan_s* sbd_plan_t;   /* opaque; owned by the library */

/* Kernel G (Introduction; Sec. 4.1 Laplace; Sec. 4.2 Helmholtz). */
typedef enum { SBD_LAPLACE = 0, SBD_HELMHOLTZ = 1, SBD_RADIAL = 2 } sbd_kernel_kind;
typedef struct {
    int32_t kind;      /* sbd_kernel_kind */
    double  kappa;     /* wavenumber (> 0) for SBD_HELMHOLTZ; ignored for SBD_LAPLACE */
} sbd_kernel;

/* Arithmetic of the on-line part.  FP64: spread, FFT, node step and interpolation in
 * float64.  FP32: those steps in float32 (coordinates split as an integer cell plus a
 * float32 fraction computed in float64).  In both forms the close correction D (computed
 * in float64, where G - G_approx cancels) is stored and applied in float64 (float64 f,
 * products and row sums), and the xi = 0 term and the final accumulation are float64.
 * SBD_FLAG_NEAR_FP32 (FP32 form only) instead rounds D to float32 once built and applies
 * it to f rounded to float32: products and per-lane partial sums in float32, the partials
 * of a row added in float64 (half the bytes of D and no FP64 products, at an error of
 * float32 rounding on the near term). */
typedef enum { SBD_FORM_FP64 = 0, SBD_FORM_FP32 = 1 } sbd_form;

typedef struct {
    int32_t form;        /* sbd_form (default SBD_FORM_FP64) */
    int32_t fixed_P;     /* > 0: use exactly this many Bessel terms; 0: the P search of Sec. 1 */
    double  nufft_tol;   /* > 0: tolerance of each type-3 transform; 0: automatic from eps */
    int32_t max_nrhs;    /* largest nrhs a matvec will use (0 = 1); sizes the workspace */
    int32_t flags;       /* 0, or SBD_FLAG_* bits */
    double  delta_max;   /* > 0: the outer radius of the fit (must be >= 2 max |z - c|, else
                            SBD_EINVAL); 0: 2 max |z - c| (R2).  A caller that rounds delta_max
                            and delta_min / delta_max to fixed grids makes repeated fits hit the
                            fit cache below. */
    int32_t host_threads;/* > 0: OpenMP threads for the host part of sbd_plan (fit, tables);
                            0: the OpenMP default.  Servers that build several plans at
                            once give each a share of the cores. */
    int32_t reserved;
} sbd_options;

/* sbd_options.flags: use a Gaussian window at the quadrature nodes (GAUSSIAN_NODES) or
 * for spreading the points (GAUSSIAN_SPREAD) instead of the default ES (exponential of
 * semicircle) window, which needs about half the width at the same accuracy.  The
 * Gaussian's Fourier transform is radial, so its deconvolution is one factor per circle;
 * the ES window's is a factor per node, folded into the node weights at plan time. */
#define SBD_FLAG_GAUSSIAN_NODES 1
#define SBD_FLAG_GAUSSIAN_SPREAD 2
/* Oversampling sigma of the spreading grid (spacing pi / (sigma S), S the largest circle
 * radius).  By default the plan takes 1.5 (ES window of about 10 cells at the FP32
 * tolerance) where the grid at sigma = 2 would have more than 20 cells per point, which
 * shrinks the spreading grid and the FFT rows by a quarter, else 2 (8 cells).  These flags
 * force one or the other; SPREAD_SIGMA_15 with GAUSSIAN_SPREAD, or both flags, is
 * SBD_EINVAL. */
#define SBD_FLAG_SPREAD_SIGMA_2 4
#define SBD_FLAG_SPREAD_SIGMA_15 8
/* Oversampling 1.25 (ES window of about 14 cells at the FP32 tolerance): a further sixth off
 * the grid and FFT sides for wider point stencils.  With another oversampling flag or
 * GAUSSIAN_SPREAD it is SBD_EINVAL. */
#define SBD_FLAG_SPREAD_SIGMA_125 64
/* Close correction D f in float32 (see sbd_form); with SBD_FORM_FP64 it is SBD_EINVAL. */
#define SBD_FLAG_NEAR_FP32 16
/* Uniform-grid multiplier variant of the far part (the fast summation the paper cites as the
 * alternative to its type-3 transforms; no counterpart in its algorithm): each J0 term of the
 * fit is kept whole instead of being turned into a circle of plane waves (Sec. 5), the series
 * G_fit is windowed to the points' differences and periodised on the FFT period, and its
 * Fourier coefficients on the frequency grid (computed in FP64 at plan time) replace the node
 * step by one multiplication per frequency.  D is G - G_fit on the near pairs.  The operator
 * is then the SBD without its quadrature error.  Not with the Gaussian windows;
 * sbd_nufft_minus / sbd_nufft_plus return SBD_ENOTSUP for such a plan. */
#define SBD_FLAG_UNIFORM_GRID 32

/* Plan summary (sbd_plan_info). */
typedef struct {
    int64_t n_points;        /* N */
    int64_t P;               /* Bessel terms of the SBD (Sec. 3.1) */
    int64_t n_circles;       /* P, plus one J0 circle for Helmholtz */
    int64_t n_xi;            /* N_xi = sum_p M_p (Sec. 6.1), the xi = 0 node excluded */
    int64_t nnz;             /* non-zeros of D, the diagonal included */
    int64_t n_coincident;    /* pairs of distinct points at distance 0 (treated as self pairs) */
    int32_t grid_x;          /* side of the spreading grid (cells) */
    int32_t grid_k;          /* side of the stored frequency grid (cells) */
    int32_t fft_n;           /* FFT length per dimension */
    int32_t stencil_x;       /* spreading stencil width (cells per dimension) */
    int32_t stencil_k;       /* node-step stencil width (cells per dimension) */
    int32_t form;            /* sbd_form */
    int32_t kind;            /* sbd_kernel_kind */
    double  delta_max;       /* 2 max_k |z_k - c|, c = bounding-box centre */
    double  delta_min;
    double  scale_R;         /* radius scale of the Bessel circles (delta_max, or k'/kappa for Y0) */
    double  a;               /* delta_min / scale_R */
    double  fit_err;         /* L_inf error of the fit on its sample set of [a, 1] (kernel units) */
    double  nufft_tol;       /* tolerance used for each type-3 transform */
    double  w0_re, w0_im;    /* weight of the xi = 0 term, G(delta_max) for Laplace (Sec. 1) */
    int64_t device_bytes;    /* device memory held by the plan */
    double  plan_seconds;    /* wall time of sbd_plan */
    int64_t n_records;       /* node records stored: N_xi, or N_xi / 2 for Laplace (the
                                antipodal nodes follow by Hermitian symmetry) */
    int32_t node_acc;        /* fused node-kernel variant (sbd_tune): accumulation mode */
    int32_t node_sched;      /* fused node-kernel variant (sbd_tune): record schedule */
    int32_t fft_split;       /* row-FFT phases (sbd_tune): 0 one where it fits, 2 always two */
    int32_t node_binned;     /* 1 when the binned node kernels (acc 3, 4) apply to the plan */
    int64_t n_targets;       /* targets (rows of D, length of q): n_points unless sbd_plan_st */
    int32_t separate_targets;/* 1 for a plan of sbd_plan_st */
    int32_t uniform_grid;    /* 1 for a plan made with SBD_FLAG_UNIFORM_GRID */
    int32_t point_chunk;     /* records per work item of the spreading / interpolation kernels */
    int32_t tuned;           /* 0 untuned, 1 tuned by timing, 2 tuned from the tuning cache */
    int32_t robin;           /* 1: Helmholtz at low kappa delta_max, fitted in the Dini basis of the
                                Robin condition (Sec. 2.3, 4.2) at scale delta_max; 0 otherwise */
} sbd_plan_stats;

/* ---------------------------------------------------------------------------------
 * sbd_plan - off-line part (Sec. 1 "Off-line part"; Sec. 3.2 fit, Sec. 5 circular
 * quadrature, Sec. 6.1 close-correction matrix, Eq. defD).
 *   points     device, N x 2 float64, interleaved (x, y); copied, so the caller may
 *              free it when the call returns.
 *   n          N >= 1.
 *   kernel     Laplace or Helmholtz (kappa > 0).
 *   delta_min  near-field radius, 0 < delta_min < delta_max; pairs with
 *              |z_k - z_l| <= delta_min go to D.
 *   eps        target accuracy in kernel units, 1e-10 <= eps <= 0.1.
 *   opt        NULL for defaults.
 *   out        receives the plan.
 * Synchronises cuda_stream before returning (the plan is ready to use on any
 * stream).  Errors: SBD_EINVAL, SBD_ENOMEM, SBD_ECUDA, SBD_EFIT.
 * ------------------------------------------------------------------------------- */
int sbd_plan(const double* points, int64_t n, sbd_kernel kernel, double delta_min,
             double eps, const sbd_options* opt, void* cuda_stream, sbd_plan_t* out);

/* ---------------------------------------------------------------------------------
 * sbd_plan_st - the off-line part for separate targets and sources (Sec. 7.1 and Table 2:
 * q_k = sum_l G(x_k - y_l) f_l for two independent point sets; the sound-cancelling example
 * of Sec. 7.2 evaluates sources on a separate zone the same way).
 *   targets    device, n_targets x 2 float64 (x_k), copied.
 *   sources    device, n_sources x 2 float64 (y_l), copied.
 *   kernel, delta_min, eps, opt, cuda_stream, out   as for sbd_plan.
 * The fit is the one sbd_plan makes for the union of the two sets (delta_max = 2 max |z - c|
 * over both, c the centre of their joint bounding box), so every |x_k - y_l| is covered.
 * The forward transform takes the sources, the backward one the targets, and D is the
 * n_targets x n_sources matrix of Eq. defD over the pairs with |x_k - y_l| <= delta_min; a
 * target that coincides with a source takes no G term from it (reading R1 carried over: D
 * holds -G_approx(0) there, counted in n_coincident).
 * sbd_matvec / sbd_far / sbd_close / sbd_matvec_graph then read f with n_sources entries per
 * right-hand side and write q with n_targets entries; sbd_nufft_minus takes f on the sources,
 * sbd_nufft_plus writes q on the targets.  sbd_gmres rejects such a plan (not a square system).
 * Errors: as sbd_plan (SBD_EINVAL also for null targets or n_targets < 1).
 * ------------------------------------------------------------------------------- */
int sbd_plan_st(const double* targets, int64_t n_targets, const double* sources, int64_t n_sources,
                sbd_kernel kernel, double delta_min, double eps, const sbd_options* opt, void* cuda_stream,
                sbd_plan_t* out);

/* ---------------------------------------------------------------------------------
 * sbd_plan_radial - the off-line part for a general real radial kernel G (Sec. 4.3):
 * the multi-Dirichlet condition of Sec. 2.2 is enforced at r = delta_max up to order
 * n_enforce by K(s) = sum_t mu_t J0(omega_t s) / J0(omega_t), s = r / delta_max, with
 * omega_t the roots of J1 nearest omega' (the square root of the mean ratio of successive
 * iterates Delta^j G(delta_max), j = 1..n_enforce + 1) and mu solving
 * sum_t (-1)^j omega_t^(2j) mu_t = delta_max^(2j) Delta^j G(delta_max), j = 1..n_enforce;
 * the constant c = G(delta_max) - K(1) is the xi = 0 term, and h = G - K - c is fitted by
 * the SBD of Sec. 3 (right-hand side by quadrature of h').  The far part has one circle per
 * Bessel term of h and one per term of K; D = G - G_approx as for sbd_plan, tabulated in r
 * on [0, delta_min] as log_coef log r + a Chebyshev series (so G - log_coef log r must be
 * smooth on [0, delta_min]).  The kernel is real: f and q are float64, as for Laplace.
 *   kernel->value(r, ctx)         G(r), r > 0.
 *   kernel->deriv(r, ctx)         G'(r), r > 0.
 *   kernel->laplacian(j, r, ctx)  (Delta^j G)(r) for 1 <= j <= n_enforce + 1, Delta =
 *                                 d^2/dr^2 + (1/r) d/dr; may be NULL when n_enforce = 0.
 *   kernel->log_coef              c with G(r) - c log r smooth at r = 0.
 *   kernel->n_enforce             0 .. 8 iterates enforced.
 * The callbacks run on the calling thread, only during this call (never afterwards), and
 * may be called from several OpenMP threads at once (they must be thread safe).  Other
 * arguments as sbd_plan; the plan works with every on-line call except those of the
 * uniform-grid variant (SBD_FLAG_UNIFORM_GRID gives SBD_ENOTSUP) and is never taken from
 * or put in the fit cache.  Errors: as sbd_plan; SBD_EINVAL also for a null kernel or
 * callback, n_enforce outside [0, 8], or a non-finite G(delta_max).
 * ------------------------------------------------------------------------------- */
typedef struct {
    double (*value)(double r, void* ctx);
    double (*deriv)(double r, void* ctx);
    double (*laplacian)(int32_t j, double r, void* ctx);
    void* ctx;
    double log_coef;
    int32_t n_enforce;
} sbd_radial_kernel;

int sbd_plan_radial(const double* points, int64_t n, const sbd_radial_kernel* kernel, double delta_min,
                    double eps, const sbd_options* opt, void* cuda_stream, sbd_plan_t* out);

/* sbd_offline_fit_radial - the fit of sbd_plan_radial alone, on the host (as sbd_offline_fit,
 * with delta_max given): rho / alpha / M receive the circles (P Bessel terms, whose alpha
 * are h's coefficients in the e_p basis, then the n_enforce terms of K: rho = omega_t,
 * alpha = mu_t / J0(omega_t)); *w0_out receives c.  No GPU needed (the Cholesky may use one,
 * see sbd_set_fit_device). */
int sbd_offline_fit_radial(const sbd_radial_kernel* kernel, double delta_min, double delta_max, double eps,
                           int32_t fixed_P, int64_t cap, double* rho, double* alpha, int32_t* M, int64_t* P_out,
                           int64_t* n_circles_out, double* fit_err, double* w0_out);

/* ---------------------------------------------------------------------------------
 * sbd_matvec - on-line part (Sec. 1 "On-line part"; Sec. 6.2; Eq. far convolution):
 * q = NUFFT_+(omega_hat . NUFFT_-(f)) + D f for nrhs right-hand sides.
 *   f, q   device, nrhs x N (float64 for Laplace, complex128 for Helmholtz; for a plan of
 *          sbd_plan_st f has n_sources and q n_targets entries per right-hand side);
 *          q is overwritten, f is read only; f and q must not overlap.
 *   nrhs   1 <= nrhs <= max_nrhs of the plan's options.  Every step takes all nrhs
 *          right-hand sides in one launch (the plan's grids hold max_nrhs of each).
 * Asynchronous on cuda_stream.  The plan's workspace is shared: calls on the same
 * plan must be ordered (one stream, or events); different plans run concurrently.
 * D is held over the plan's internal point order (the spatial order of its spreading
 * records): D f is formed first from f gathered into that order, and each point's
 * value is added as the far part is interpolated to it.  For Laplace the spreading
 * grid is real and the frequency grid Hermitian, so half the transforms and half the
 * quadrature nodes are processed (the rest follow by symmetry).
 * ------------------------------------------------------------------------------- */
int sbd_matvec(sbd_plan_t plan, const void* f, void* q, int32_t nrhs, void* cuda_stream);

/* sbd_matvec_graph - sbd_matvec replayed from a CUDA graph (no counterpart in the paper):
 * the per-kernel launch cost (10 kernels per call, whatever nrhs) matters for small N.  The first
 * call for a given nrhs runs one matvec on plan-owned buffers and captures a second one
 * into a graph; every call then copies f into the plan's input buffer, launches the graph
 * and copies the plan's output buffer to q, on a plan-owned stream ordered after and before
 * cuda_stream with events (so the legacy default stream works too).  Same arguments,
 * layout, results and ordering rules as sbd_matvec; holds two extra N x max_nrhs buffers.
 * Errors: as sbd_matvec, and SBD_ECUDA if capture or instantiation fails. */
int sbd_matvec_graph(sbd_plan_t plan, const void* f, void* q, int32_t nrhs, void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * Batches of instances (no counterpart in the paper): the matvecs of several plans in
 * one CUDA graph, each plan on its own branch, so that one launch runs instances of
 * uneven size side by side on the device.
 *   sbd_batch_create   plans[count] (distinct), nrhs[i] (1..max_nrhs of plan i), device
 *                      buffers f[i], q[i] (layout of sbd_matvec) that stay valid and fixed
 *                      while the batch lives; runs one matvec per plan, then captures the
 *                      graph.  Blocks until done.
 *   sbd_batch_launch   q[i] = matvec of plan i on f[i] for every i, one graph launch,
 *                      asynchronous on cuda_stream.  The plans must not be used elsewhere
 *                      while a launch runs (their workspace is in the graph).
 *   sbd_batch_destroy  frees the graph (not the plans).  NULL-safe.
 * Errors: SBD_EINVAL (null pointers, count < 1, a plan twice, nrhs out of range),
 * SBD_ECUDA (capture or instantiation failed), and those of sbd_matvec.
 * ------------------------------------------------------------------------------- */
typedef struct sbd_batch_s* sbd_batch_t;
int sbd_batch_create(const sbd_plan_t* plans, const int32_t* nrhs, int32_t count, const void* const* f,
                     void* const* q, sbd_batch_t* out);
int sbd_batch_launch(sbd_batch_t batch, void* cuda_stream);
int sbd_batch_destroy(sbd_batch_t batch);

/* ---------------------------------------------------------------------------------
 * sbd_matvec_batched - the matvecs of several plans (instances of uneven size, Laplace and
 * Helmholtz mixed, separate-target plans included) in one call: q[i] = matvec of plans[i]
 * on f[i] with nrhs[i] right-hand sides (Sec. 1 on-line part for each; batching itself has
 * no counterpart in the paper).  The steps that walk points and nodes run once for the
 * whole batch: a persistent cooperative spreading kernel over every (instance, chunk of a
 * tile's points, right-hand-side group), a node-step kernel over every (instance, tile,
 * right-hand side) and a persistent interpolation kernel over every (instance, chunk,
 * right-hand-side group), each taking work items from a counter; the two cooperative ones
 * first clear the grids they accumulate into and meet at a grid-wide barrier.  The FFTs run
 * per instance, each plan on its own stream, and the near part D f on each plan's near stream.
 *   plans     host, count distinct plans of one form (SBD_ENOTSUP otherwise).
 *   f, q      host arrays of count device pointers, layout of sbd_matvec per plan.
 *   nrhs      host, count values, 1 <= nrhs[i] <= max_nrhs of plan i.
 *   count     1 .. 64.
 * Asynchronous on cuda_stream; the plans must not be used elsewhere until it completes.
 * Every device-side wait (the grid barriers) gives up after the limit of
 * sbd_set_device_wait; the kernel then skips its remaining work, the results are invalid,
 * and sbd_device_status reports SBD_ETIMEOUT.
 * Errors: SBD_EINVAL (null pointers, count or nrhs out of range, a plan twice), SBD_ENOTSUP
 * (mixed forms, or a kernel that does not fit an SM), SBD_ECUDA.
 * ------------------------------------------------------------------------------- */
int sbd_matvec_batched(const sbd_plan_t* plans, const void* const* f, void* const* q, const int32_t* nrhs,
                       int32_t count, void* cuda_stream);

/* sbd_set_device_wait - bound of every device-side wait of the batched launches (no
 * counterpart in the paper): a CTA that waits longer than limit_seconds (default 2 s;
 * (0, 600]) at a grid barrier stops waiting, records SBD_ETIMEOUT and returns, so that a
 * fault elsewhere cannot hang the GPU.  phantom_arrivals (0 in use, at most 1024) makes each
 * barrier wait for that many CTAs beyond those launched, which never arrive: a
 * fault-injection knob that lets a test watch the wait run out.  Process-wide; applies to
 * launches made after the call. */
int sbd_set_device_wait(double limit_seconds, int32_t phantom_arrivals);

/* sbd_device_status - synchronises cuda_stream, then returns and clears the process-wide
 * status of the bounded device waits: SBD_OK, or SBD_ETIMEOUT when a wait of a batched
 * launch ran out since the last call (a CUDA error of the synchronisation returns SBD_ECUDA). */
int sbd_device_status(void* cuda_stream);

/* The two halves of sbd_matvec, same arguments and layout:
 *   sbd_far   q = NUFFT_+(omega_hat . NUFFT_-(f))   (Eq. far convolution, incl. the xi = 0 term)
 *   sbd_close q = D f                               (Sec. 1, close correction)                  */
int sbd_far(sbd_plan_t plan, const void* f, void* q, int32_t nrhs, void* cuda_stream);
int sbd_close(sbd_plan_t plan, const void* f, void* q, int32_t nrhs, void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * sbd_nufft_minus - the forward type-3 transform of the plan (Introduction,
 * NUFFT_-[z, xi]): fhat_nu = sum_l exp(-i z_l . xi_nu) f_l at every quadrature node
 * xi_nu, nodes ordered circle by circle (circle p = 0..n_circles-1, m = 0..M_p-1,
 * xi = r_p (cos 2 pi m / M_p, sin 2 pi m / M_p), Eq. defXimp).
 *   f     device, N complex128.      fhat   device, N_xi complex128.
 * sbd_nufft_plus is its adjoint: q_l = sum_nu exp(+i z_l . xi_nu) ghat_nu
 *   ghat  device, N_xi complex128.   q      device, N complex128.
 * Both run in the plan's form; asynchronous on cuda_stream.
 * ------------------------------------------------------------------------------- */
int sbd_nufft_minus(sbd_plan_t plan, const void* f, void* fhat, void* cuda_stream);
int sbd_nufft_plus(sbd_plan_t plan, const void* ghat, void* q, void* cuda_stream);

/* Plan summary; host struct.  Synchronous, no device work. */
int sbd_plan_info(sbd_plan_t plan, sbd_plan_stats* out);

/* Copy the plan's SBD data to host arrays of capacity cap (>= n_circles):
 * rho (J0 roots rho_p, Sec. 2.1), alpha (SBD coefficients on e_p = C_p J0(rho_p r),
 * Sec. 3.1; 0 for the Helmholtz J0 circle), M (nodes per circle, Sec. 5),
 * radius (circle radius in frequency units), weight_re/_im (omega_hat per node,
 * Sec. 6.2, in kernel units).  Any pointer may be NULL.  Synchronous. */
int sbd_plan_export(sbd_plan_t plan, int64_t cap, double* rho, double* alpha, int32_t* M,
                    double* radius, double* weight_re, double* weight_im);

/* Copy D (Eq. defD) to host CSR arrays: rowptr (n_targets + 1), col (nnz), val (nnz float64
 * for Laplace, 2 nnz float64 = complex128 for Helmholtz; a plan made with
 * SBD_FLAG_NEAR_FP32 gives the float32 values it stores, widened).  Rows (targets) and
 * columns (sources) are in the caller's point orders; each row holds its diagonal first
 * (plans of one point set), then its columns in increasing order.  Synchronous. */
int sbd_close_export(sbd_plan_t plan, int64_t* rowptr, int32_t* col, double* val);

/* Release the plan (NULL is accepted).  sbd_destroy first waits for the whole device, so
 * any pending use of the plan on any stream is safe.  sbd_destroy_async waits only for
 * the plan's own graph stream and orders the frees on cuda_stream after the caller's work
 * there: every other use of the plan must already be complete or ordered before that
 * point on cuda_stream.  Plan memory is stream-ordered and returns to the device's memory
 * pool (kept, not released to the system, so that later plans reuse it). */
int sbd_destroy(sbd_plan_t plan);
int sbd_destroy_async(sbd_plan_t plan, void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * sbd_offline_fit - the SBD fit and circle sizes alone, on the host (Sec. 3.2
 * Eq. LinearSystem with the explicit A^P; Sec. 1 P search; Sec. 5 sizes).  Needs no GPU;
 * the full Cholesky of A^P (tolerances below 5e-9) runs on one when sbd_set_fit_device says so.
 *   kernel, delta_min, delta_max, eps   as for sbd_plan (delta_max given directly).
 *   fixed_P      > 0 fixes P, 0 searches.
 *   cap          capacity of rho / alpha / M (>= P, plus 1 for Helmholtz).
 *   P_out        receives P; n_circles_out receives the number of circles.
 *   fit_err      receives the L_inf fit error in kernel units.
 * ------------------------------------------------------------------------------- */
int sbd_offline_fit(sbd_kernel kernel, double delta_min, double delta_max, double eps,
                    int32_t fixed_P, int64_t cap, double* rho, double* alpha, int32_t* M,
                    int64_t* P_out, int64_t* n_circles_out, double* fit_err);

/* ---------------------------------------------------------------------------------
 * sbd_transform_params - the sizes sbd_plan would choose for the type-3 transforms of
 * the far part (Sec. 1 steps (i)-(iii); Sec. 6.2), on the host, without a GPU: the fit
 * (as sbd_offline_fit) and from it the per-transform tolerance, the spreading window,
 * its oversampling and width, the spreading-grid, frequency-grid and FFT sizes.  For
 * sizing device memory before planning, and for choosing options.
 *   kernel, delta_min, delta_max, eps   as for sbd_offline_fit.
 *   n_points     N (>= 1); feeds the automatic spreading oversampling.
 *   half_extent  half the side of the points' bounding box (> 0): the larger of its
 *                half width and half height, as sbd_plan measures it.
 *   opt          NULL for defaults (form, flags, nufft_tol and fixed_P are used).
 *   out          host, receives the sizes.
 * SBD_EINVAL for a null out, n_points < 1, half_extent <= 0, delta_min outside
 * (0, delta_max), eps outside [1e-10, 0.1], invalid options or kernel; SBD_EFIT when the
 * fit cannot reach eps; SBD_ENOTSUP when the FFT length exceeds the row kernels' limit.
 * ------------------------------------------------------------------------------- */
typedef struct {
    double  sigma_s;         /* oversampling of the spreading grid: 1.5 or 2 */
    double  h;               /* spreading-grid spacing, pi / (sigma_s S), S the largest circle radius */
    double  deta;            /* frequency-grid spacing, 2 pi / (fft_n h) */
    double  nufft_tol;       /* tolerance of each type-3 transform */
    int32_t grid_x;          /* side of the spreading grid (cells) */
    int32_t grid_k;          /* side of the stored frequency grid (cells) */
    int32_t fft_n;           /* FFT length per dimension (2 grid_x) */
    int32_t stencil_x;       /* spreading stencil width (cells per dimension) */
    int32_t stencil_k;       /* node stencil width */
    int32_t spread_window;   /* 1 ES, 0 Gaussian */
    int64_t P;               /* Bessel terms */
    int64_t n_circles;       /* circles (P, plus one for Helmholtz) */
    int64_t n_xi;            /* quadrature nodes */
} sbd_transform_stats;
int sbd_transform_params(sbd_kernel kernel, double delta_min, double delta_max, double eps,
                         int64_t n_points, double half_extent, const sbd_options* opt,
                         sbd_transform_stats* out);

/* ---------------------------------------------------------------------------------
 * sbd_fft2 - the library's 2-D complex FFT on its own (the transform the far part
 * uses; exposed for testing): out[j0][j1] = sum_{k0,k1} in[k0][k1]
 * exp(sign * 2 pi i (j0 k0 / n0 + j1 k1 / n1)), unnormalised, row-major n0 x n1.
 *   in, out   device, complex64 (form FP32) or complex128 (form FP64); may alias.
 *   n0, n1    2..65536, each a product of 2, 3 and 5.
 *   sign      -1 or +1.
 * Asynchronous on cuda_stream; allocates a temporary of n0 x n1 elements.
 * ------------------------------------------------------------------------------- */
int sbd_fft2(const void* in, void* out, int32_t n0, int32_t n1, int32_t sign, int32_t form,
             void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * Autotuning of the node step (no counterpart in the paper).  The fused node kernel
 * has variants that compute the same sums: acc 0 adds re and im into two float planes
 * (one shared-memory atomic each), acc 1 (FP32 form only) into one float2 plane with
 * one 64-bit compare-and-swap, acc 2 (FP32 form only) into two int64 fixed-point
 * planes with integer atomics (quantum 2^-50 of a per-tile bound on any contribution);
 * for these sched 0 deals the records of a tile to the lane groups in turn, sched 1
 * gives each group a contiguous run.  acc 3 (FP32 form, node stencil of at most 8
 * cells, every 64 x 64 tile of the frequency grid holding at most 4096 records) takes
 * the records bin by bin (8 x 8 stencil starts; four accumulators, one per bin colour,
 * so that no two warps write one cell and no atomics are needed); for it sched 0 runs
 * 512 threads per CTA, sched 1 1024, one persistent CTA per SM walking the plan's tiles
 * with records.  acc 4 (where acc 3 applies) takes the same bins two at a time per warp,
 * one per half-warp, each half-warp carrying one record at a time with bank-conflict-free
 * accesses (sched as for acc 3).  Results agree to FP32 rounding.
 *   sbd_tune       times every applicable variant on the plan's own records (reps
 *                  launches each, after one warm-up, CUDA events on cuda_stream; the
 *                  frequency workspace is first filled with a constant non-zero value,
 *                  so that concurrent adds to a cell contend as with real data) and
 *                  keeps the fastest.
 *                  ms (host, 12 entries, may be NULL): mean ms per launch of variant
 *                  acc * 2 + sched for acc <= 3 and 10 + sched for acc 4, -1 where not
 *                  applicable; ms[8], ms[9]: mean ms of
 *                  the forward 2-D transform with rows in one phase where they fit, and
 *                  with every row split into two half-length phases (half the shared
 *                  memory per CTA, so more CTAs per SM); the faster is kept too.
 *                  Blocks until done.
 *   sbd_set_tuning picks a variant by hand (fft_split 0 or 2).
 * SBD_EINVAL for a null plan, reps < 1, acc outside {0, .., 4}, sched outside {0, 1}
 * or fft_split outside {0, 2} (acc 1 to 4 need the FP32 form, acc 3 and 4 a plan where
 * they apply; sbd_plan_info's node_binned says so).  Plans whose node step is the two-kernel
 * fallback ignore the variant.
 * ------------------------------------------------------------------------------- */
int sbd_tune(sbd_plan_t plan, int32_t reps, double* ms, void* cuda_stream);
int sbd_set_tuning(sbd_plan_t plan, int32_t acc, int32_t sched, int32_t fft_split);

/* Point-kernel work items (no counterpart in the paper): the spreading and interpolation
 * kernels take each 64 x 64 tile's records in chunks (one CTA each); crowded tiles become
 * several CTAs.  sbd_tune also times spreading plus interpolation for chunks of 128, 256,
 * 512, 1024 and 2048 records and keeps the fastest (after the node variants and the FFT
 * split).  sbd_tune_points runs that search alone (ms: host, 5 entries, mean ms per
 * spreading + interpolation, may be NULL); sbd_set_point_chunk sets a chunk by hand
 * (128 .. 2^20).  Blocking.  SBD_EINVAL for a null plan, reps < 1 or a chunk out of range. */
int sbd_tune_points(sbd_plan_t plan, int32_t reps, double* ms, void* cuda_stream);
int sbd_set_point_chunk(sbd_plan_t plan, int32_t chunk);

/* Tuning cache (no counterpart in the paper): sbd_tune keeps its choice (node variant, FFT
 * split, point chunk) per plan class (form, kernel, separate targets, uniform grid, binned
 * node kernel, float32 near field, the grid sizes, N to a half octave) and applies a class's
 * choice without timing when it meets the class again (sbd_plan_info's tuned = 2).
 * Process-wide and thread safe.
 *   sbd_tune_cache_stats   host outputs (each may be NULL): lookups that hit, missed, entries.
 *   sbd_tune_cache_save    writes the cache as a JSON object {"class": [acc, sched, split, chunk]}.
 *   sbd_tune_cache_load    merges such a file into the cache (SBD_EINVAL if unreadable or malformed).
 *   sbd_tune_cache_clear   drops every entry and zeroes the counters. */
int sbd_tune_cache_stats(int64_t* hits, int64_t* misses, int64_t* entries);
int sbd_tune_cache_save(const char* path);
int sbd_tune_cache_load(const char* path);
int sbd_tune_cache_clear(void);

/* ---------------------------------------------------------------------------------
 * sbd_plan_balanced - sbd_plan with delta_min chosen by measurement (Introduction,
 * Theorem 1, and Sec. 6: delta_min = a delta_max with a = |log eps|^(2/3) / N^(2/3 - alpha)
 * for some alpha in [0, 1/6], chosen so that the far and the close parts balance; the
 * constants of that balance depend on the machine, so it is found here by timing).
 * For each candidate alphas[i] the call builds the plan of sbd_plan with that delta_min
 * (delta_max = 2 max |z - c|, or options.delta_max when larger), tunes it (sbd_tune, 3
 * launches per variant), runs one warm-up matvec and times `reps` matvecs with nrhs
 * right-hand sides (a library-owned constant non-zero f; CUDA events on cuda_stream),
 * and keeps the fastest plan; every other plan is destroyed before the next is built,
 * so at most two plans are held at once.
 *   points, n, kernel, eps, opt   as for sbd_plan (options.max_nrhs is raised to nrhs).
 *   alphas     host, count values in [0, 1/6]; 1 <= count <= 16.
 *   nrhs       right-hand sides per timed matvec (>= 1).
 *   reps       timed matvecs per candidate (>= 1).
 *   out        receives the fastest plan (owned by the caller; free with sbd_destroy).
 *   ms         host, count entries (may be NULL): mean ms per matvec of candidate i,
 *              -1 where it could not be planned (delta_min >= delta_max, the fit could
 *              not reach eps, out of memory).
 *   chosen     host (may be NULL): index of the kept candidate.
 * Blocks until done.  SBD_EINVAL for null points/out/alphas, n < 1, count outside
 * [1, 16], an alpha outside [0, 1/6], nrhs or reps < 1, eps outside [1e-10, 0.1]; when no
 * candidate could be planned, the last candidate's error code (its message in
 * sbd_last_error_message).
 * ------------------------------------------------------------------------------- */
int sbd_plan_balanced(const double* points, int64_t n, sbd_kernel kernel, double eps, const double* alphas,
                      int32_t count, int32_t nrhs, int32_t reps, const sbd_options* opt, void* cuda_stream,
                      sbd_plan_t* out, double* ms, int32_t* chosen);

/* ---------------------------------------------------------------------------------
 * Fit cache.  The off-line fit (P search and coefficients, Sec. 3-4) depends only on
 * the kernel kind, k' (Helmholtz, Sec. 4.2), a = delta_min / scale_R, eps and fixed_P;
 * sbd_plan and sbd_offline_fit keep the last 64 distinct fits process-wide (thread
 * safe) and reuse one when these agree (a to a relative 1e-12).  The paper fits once
 * per geometry and has no counterpart; it serves repeated plans of a solve server.
 *   sbd_fit_cache_stats  host outputs (each may be NULL): lookups that hit, that
 *                        missed, entries held.  Always SBD_OK.
 *   sbd_fit_cache_clear  drops every entry and zeroes the counters.  Always SBD_OK.
 * ------------------------------------------------------------------------------- */
int sbd_fit_cache_stats(int64_t* hits, int64_t* misses, int64_t* entries);
int sbd_fit_cache_clear(void);

/* sbd_set_fit_device - where the off-line fit factors A^P when it needs its full Cholesky
 * (fit tolerances below 5e-9, e.g. eps = 1e-9; Sec. 3.2, the O(P^3) step of Sec. 6.1): the
 * matrix is then built and factored in FP64 on the current CUDA device and the factor copied
 * back.  mode 0 (default): the device when one is present and P >= 3000, else the host;
 * 1: always the host; 2: the device whenever one is present.  A device failure (no memory,
 * a CUDA error) falls back to the host.  Process-wide.  SBD_EINVAL for another mode.
 * sbd_fit_last_factorisation - host outputs (each may be NULL): the seconds of the last full
 * factorisation and where it ran (0 none yet, 1 host, 2 device).  Always SBD_OK. */
int sbd_set_fit_device(int32_t mode);
int sbd_fit_last_factorisation(double* seconds, int32_t* where);

/* sbd_y0_root - the k-th positive zero of Y0 (k >= 1) into *root (host).  For Helmholtz
 * the fit's scale k' is the first such zero >= kappa delta_max (Sec. 4.2), so a caller
 * that wants repeated fits can pick delta_max just below a zero of its choice.
 * SBD_EINVAL for k < 1 or a null pointer. */
int sbd_y0_root(int32_t k, double* root);

/* ---------------------------------------------------------------------------------
 * sbd_gmres - restarted GMRES for (shift I + scale A) x = b, A the plan's matvec: the
 * iterative solution of boundary-integral systems that motivates the fast convolution
 * (Introduction).  Arnoldi with two-pass classical Gram-Schmidt, Givens rotations.
 *   b      device, N (float64 Laplace / complex128 Helmholtz), read only.
 *   x      device, N: initial guess on entry (zero it for none), solution on return.
 *   opt    shift, scale (complex; real parts only for Laplace), tol (relative residual
 *          ||b - (shift I + scale A) x|| / ||b||), restart (Krylov dimension), max_iter.
 *   iterations, rel_residual   host outputs (may be NULL): Arnoldi steps done; the
 *          final relative residual (recomputed from b - (shift I + scale A) x when the
 *          solver stops converged, the Arnoldi estimate when it stops at max_iter).
 * Errors: SBD_EINVAL for a null plan/b/x/opt, restart < 1, max_iter < 0 or tol <= 0;
 * SBD_ECUDA from a device failure (x then holds a partial update).
 * Blocks the calling thread (one device-to-host read per Gram-Schmidt pass); runs its
 * device work on cuda_stream; allocates (restart + 2) N-vectors of workspace per call.
 * Calls for different plans may run concurrently from different host threads.
 * ------------------------------------------------------------------------------- */
typedef struct {
    double  shift_re, shift_im;
    double  scale_re, scale_im;
    double  tol;
    int32_t restart;
    int32_t max_iter;
} sbd_gmres_options;
int sbd_gmres(sbd_plan_t plan, const void* b, void* x, const sbd_gmres_options* opt, int32_t* iterations,
              double* rel_residual, void* cuda_stream);

/* ---------------------------------------------------------------------------------
 * GMRES as a resumable session (no counterpart in the paper): the iteration of sbd_gmres,
 * stopped wherever it needs a matvec of its plan, so that a caller can compute the matvecs
 * of many solves together (sbd_matvec_batched) while each solve keeps its own Krylov basis.
 *   sbd_gmres_begin    plan, b, x, opt as for sbd_gmres (x: initial guess); allocates the
 *                      workspace ((restart + 2) N-vectors) and computes ||b|| on cuda_stream,
 *                      which the session's own kernels use from then on.  *out: the session.
 *   sbd_gmres_next     1 when the session needs out = A in: the plan's plain matvec (sbd_matvec
 *                      semantics, one right-hand side; the shift and scale are the session's),
 *                      with *in and *out device vectors of the session; 0 when it has finished.
 *   sbd_gmres_advance  after the caller wrote out = A in (ordered before the session's stream,
 *                      e.g. with an event): the work up to the next matvec (Gram-Schmidt,
 *                      rotations, updates of x).  Blocks the calling thread (reads projections).
 *   sbd_gmres_end      iterations and the final relative residual (as sbd_gmres; may be NULL),
 *                      frees the session (NULL-safe).  x holds the solution.
 * Errors: as sbd_gmres.  One session is driven by one thread at a time.
 * ------------------------------------------------------------------------------- */
typedef struct sbd_gmres_session_s* sbd_gmres_session_t;
int sbd_gmres_begin(sbd_plan_t plan, const void* b, void* x, const sbd_gmres_options* opt, void* cuda_stream,
                    sbd_gmres_session_t* out);
int sbd_gmres_next(sbd_gmres_session_t session, const void** in, void** out);
int sbd_gmres_advance(sbd_gmres_session_t session);
int sbd_gmres_end(sbd_gmres_session_t session, int32_t* iterations, double* rel_residual);

/* ---------------------------------------------------------------------------------
 * Step timing of the on-line part.  sbd_profile(plan, 1) waits for the device,
 * clears the counters and starts recording a pair of CUDA events on the caller's
 * stream around every step of sbd_matvec / sbd_far / sbd_close (0 stops).
 * sbd_profile_read waits for the recorded events and returns, per step
 * (SBD_STAGE_*), the summed device time in ms and the number of timed runs into
 * host arrays of SBD_N_STAGES entries.  Not for concurrent use on one plan.
 * ------------------------------------------------------------------------------- */
#define SBD_STAGE_SUM      0   /* sum_l f_l for the xi = 0 term */
#define SBD_STAGE_SPREAD   1   /* spreading of the points onto the grid */
#define SBD_STAGE_FFT_FWD  2   /* precorrection + forward 2-D FFT */
#define SBD_STAGE_NODE     3   /* node gather, omega_hat weighting, node scatter */
#define SBD_STAGE_FFT_INV  4   /* inverse 2-D FFT + postcorrection */
#define SBD_STAGE_INTERP   5   /* interpolation at the points (+ xi = 0 term) */
#define SBD_STAGE_SPMV     6   /* close correction D f */
#define SBD_N_STAGES       7
int sbd_profile(sbd_plan_t plan, int32_t enable);
int sbd_profile_read(sbd_plan_t plan, double* ms, int64_t* count);

/* ---------------------------------------------------------------------------------
 * sbd_fft2_noalloc - sbd_fft2 without any device memory allocation.  (The paper has no
 * counterpart: this is a library service, not part of the method.)
 *
 * For callers that may not allocate device memory while they run: programs that hand
 * all device memory to their own pool at start-up, or latency-critical loops whose
 * policy forbids cudaMalloc / cudaFree (and the allocator synchronisation they may
 * imply) after initialisation.  The transform's temporary grid and its twiddle and
 * digit-reversal tables live in a fixed file-scope device array of
 * SBD_NOALLOC_FFT_MAX_BYTES + 2 * SBD_NOALLOC_FFT_MAX_SIDE * 20 bytes, which every GPU
 * that loads the library keeps until the process exits.
 *   in, out, n0, n1, sign, form, cuda_stream   as for sbd_fft2 (in and out may alias).
 *   Limits: 2 <= n0, n1 <= SBD_NOALLOC_FFT_MAX_SIDE, each a product of 2, 3 and 5, and
 *   n0 * n1 * (8 for FP32, 16 for FP64) <= SBD_NOALLOC_FFT_MAX_BYTES; larger sizes
 *   return SBD_EINVAL with the limits in sbd_last_error_message().
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * once per device, with that device current); make that first call before any stream
 * capture.  The address is kept per device ordinal for the life of the process and is
 * not looked up again after a cudaDeviceReset, so do not call this function after
 * resetting a device.  All calls share the one array and its contents persist between
 * calls, so calls that overlap on the GPU (different streams without ordering) race; the
 * function clears nothing it does not overwrite first.  Each call rebuilds the twiddle and
 * digit-reversal tables of both sides in the array (4 small launches before the 4 launches
 * of the transform), so no state carries over from one call to the next.
 * ------------------------------------------------------------------------------- */
#define SBD_NOALLOC_FFT_MAX_BYTES (4 * 1024 * 1024)
#define SBD_NOALLOC_FFT_MAX_SIDE  4096
int sbd_fft2_noalloc(const void* in, void* out, int32_t n0, int32_t n1, int32_t sign, int32_t form,
                     void* cuda_stream);

const char* sbd_error_string(int code);
const char* sbd_last_error_message(void);
const char* sbd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SBD_H */
