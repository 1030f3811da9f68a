/*
 * claire.h - C ABI of libclaire.so, a GB300 (sm_103a) implementation of the
 * semi-Lagrangian Gauss-Newton-Krylov hot path of stationary-velocity
 * diffeomorphic registration ("CLAIRE at scale", arXiv 2209.08189).
 *
 * Problem (Sec. 2.1, Eq. (1)): given a template m0 and a reference m1 on the
 * periodic grid Omega = [0, 2 pi)^3, find a stationary velocity v minimising
 *     J(v) = 1/2 ||m(1) - m1||^2 + beta_v/2 reg_v(v) + beta_w/2 reg_w(div v)
 * subject to d_t m + v . grad m = 0, m(0) = m0.  reg_v is the H1 (or H2)
 * seminorm of v and reg_w the H1 norm of w = div v (Sec. 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: N1 x N2 x N3 nodes x = (i h1, j h2, k h3), h_c = 2 pi / N_c,
 *    each N_c even and >= 8.  Scalar fields are float32 arrays of N = N1 N2 N3
 *    values in C order (index (i N2 + j) N3 + k, x3 fastest).  Vector fields
 *    are component-major: [3][N1][N2][N3].  Velocities are in physical units
 *    (radians per unit time); displacements are in grid units.
 *  - Discrete inner product: <a, b> = h1 h2 h3 sum(a b); J, the mismatch and
 *    the regularisation energy use it.
 *  - Pointers: unless an entry point says "device pointers", an array
 *    argument may be a device pointer or a host pointer (pageable or
 *    pinned); host arrays are staged through the context's workspace with
 *    copies on the context's stream.  A device array needs only float
 *    alignment: one at a 16-byte boundary (every cudaMalloc'd array) takes
 *    the kernels' 16-byte copies and vector loads, any other their 4-byte
 *    forms, with the same results.  Arrays are owned by the caller and are
 *    only read during the call, except outputs and v_inout.
 *  - Streams: all device work is queued on the context's stream (default:
 *    the legacy default stream; see claire_set_stream).  Every entry point
 *    returns after its outputs are complete and visible to the host-side
 *    caller's next operation on that stream; scalar outputs are host values.
 *  - Errors: every entry point returns a claire_status and never throws.  A
 *    negative status leaves outputs unspecified; claire_last_error() gives a
 *    one-line message.  A context is not thread-safe: use one per host thread.
 *  - Velocity screen: claire_objective, claire_gradient, claire_register,
 *    claire_transport, claire_transport_vjp, claire_detj and
 *    claire_backtrace first reduce max |v(x)| in FP64 and return
 *    CLAIRE_ENONFINITE, before any gather runs, when a component is NaN or
 *    Inf.  The gathers themselves send a tile whose displacement is
 *    non-finite or 2^20 cells or more to a global-memory path whose indices
 *    are clamped and wrapped (the result there is NaN or meaningless, never
 *    an out-of-range access).
 *  - There is no CPU fallback: without a usable CUDA device, claire_create
 *    returns CLAIRE_ECUDA.
 */
#ifndef CLAIRE_H
#define CLAIRE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct claire_ctx claire_ctx;

typedef enum {
    CLAIRE_OK = 0,
    CLAIRE_ENOTCONVERGED = 1,  /* warning: iteration cap hit; outputs hold the last iterate */
    CLAIRE_EINVAL = -1,        /* bad argument (grid, sizes, null pointer, option value) */
    CLAIRE_ENOMEM = -2,        /* device allocation failed (nothing was launched) */
    CLAIRE_ECUDA = -3,         /* CUDA runtime error (message has the CUDA error string) */
    CLAIRE_ECUFFT = -4,        /* cuFFT plan or execution error */
    CLAIRE_ENONFINITE = -5,    /* a reduction saw NaN or Inf (input or iterate) */
    CLAIRE_ELINESEARCH = -6,   /* Armijo line search found no acceptable step */
    CLAIRE_ETIMEOUT = -7,      /* wall-clock limit reached; outputs hold the last iterate */
    CLAIRE_ESTATE = -8,        /* call needs state that is not set (images, linearisation point) */
    CLAIRE_ENOTIMPL = -9,
    CLAIRE_ETOOLARGE = -10     /* size beyond the fixed maximum of claire_dot_noalloc */
} claire_status;

/* Interpolation order of the semi-Lagrangian gathers (Sec. 3, "IP kernel"). */
#define CLAIRE_INTERP_CUBIC 3   /* cubic Lagrange, nodes floor-1 .. floor+2 */
#define CLAIRE_INTERP_LINEAR 1  /* trilinear */
#define CLAIRE_INTERP_BSPLINE 4 /* cubic B-spline on the same nodes, applied to the field's spline
                                   coefficients (Sec. 3): every gathered field is prefiltered first
                                   (forward FFT, division by the sampled spline's symbol
                                   prod (2 + cos k h) / 3, inverse FFT), which needs FP32 storage and
                                   adds 3N floats + 3 half spectra of scratch on first use */

/* claire_transport flags */
#define CLAIRE_TRANSPORT_FWD 0  /* state, Eq. (1b)-(1c): m(1) from m(0) */
#define CLAIRE_TRANSPORT_ADJ 1  /* adjoint, Eq. (4): lambda(0) from lambda(1) */

/* claire_spectral ops (Sec. 2.2: "two FFTs and one Hadamard product") */
#define CLAIRE_SPECTRAL_REG 0   /* S v: first variation of the regulariser */
#define CLAIRE_SPECTRAL_INV 1   /* S^{-1} r (identity on the k = 0 mode): the preconditioner */
#define CLAIRE_SPECTRAL_K   2   /* K b = b - c u (u . b) / (a + c |u|^2): the paper's K */

typedef struct claire_opts {
    int interp;          /* CLAIRE_INTERP_CUBIC (default), CLAIRE_INTERP_LINEAR or CLAIRE_INTERP_BSPLINE */
    int reg;             /* 1 = H1 seminorm of v (default), 2 = H2 seminorm */
    double beta_w;       /* weight of the H1 norm of div v; default 1e-4 */
    int grad_form;       /* 0 = g = S v + b (default, exact gradient of J; H symmetric);
                            1 = the paper's Eq. (3) form g = beta_v A v + K b */
    double gtol;         /* stop when ||g|| / ||g0|| <= gtol; default 5e-2 (Sec. 4.2) */
    int max_gn;          /* Gauss-Newton iteration cap; default 50 */
    int max_pcg;         /* PCG iteration cap per Gauss-Newton step; default 50 */
    double pcg_rtol_max; /* forcing eta_k = min(pcg_rtol_max, sqrt(||g_k||/||g_0||)); default 0.5 */
    int pcg_fixed;       /* 1 = always run max_pcg PCG iterations (no residual exit); default 0 */
    double armijo_c1;    /* sufficient-decrease constant; default 1e-4 */
    int max_ls;          /* step halvings before CLAIRE_ELINESEARCH; default 10 */
    double wall_limit_s; /* claire_register wall-clock cap in seconds; 0 = none (default) */
    int timing;          /* 1 = time every kernel launch with CUDA events (read back lazily by
                            claire_kernel_stats); 2 = also fill claire_report.t_phase_s at the end
                            of each claire_register (one extra synchronisation) */
    int storage;         /* storage precision of the scalar fields of the solver (images, states
                            m^j and their gradients, adjoint levels, incremental fields, div v):
                            CLAIRE_STORAGE_F32 (default), _F16 or _BF16.  Arithmetic is FP32,
                            reductions FP64; velocities, displacements and the spectral/PCG
                            vectors stay FP32.  API arrays are always float32. */
    double g0_ref;       /* > 0: reference ||g0|| of the relative tolerance and of the PCG forcing in
                            claire_register, instead of the gradient norm at the initial guess; a
                            solve warm-started from a predicted velocity passes the norm of the
                            gradient at v = 0 so that it stops at the same absolute gradient as a
                            solve from zero.  Default 0 (use the initial guess's gradient). */
    int lowmem;          /* 1 = do not store the gradients grad m^j of the states: the incremental
                            sources and the gradient body compute them by FD8 where they are used
                            (3 (nt+1) N fewer stored values, about 1.3x the time of those kernels);
                            0 = store them once per linearisation (default).  Fixed at create. */
    int precond;         /* PCG preconditioner: CLAIRE_PRECOND_SPECTRAL (default, S^{-1}) or
                            CLAIRE_PRECOND_TWO_LEVEL, the paper's zero-velocity Hessian approximation
                            H0 vt = S vt + gbar (gbar . vt), gbar = sum_j w_j grad m^j at the
                            linearisation point (Sec. 2.2), inverted on a coarse grid by an inner
                            PCG, with S^{-1} on the remaining (high) modes and the identity on k = 0;
                            the outer PCG then takes the flexible (Polak-Ribiere) direction update.
                            A Gauss-Newton step whose two-level solve fails the Armijo line search is
                            solved again with S^{-1} (claire_report.pc_fallbacks).
                            Its coarse-grid buffers (about 3 fine spectra) are allocated on first use. */
    int pc_coarse;       /* fine-to-coarse ratio of the two-level grid: every N_i / pc_coarse must be
                            even and >= 4; default 2 */
    double pc_tol;       /* relative residual of the inner PCG; 0 = always run pc_maxit iterations;
                            default 1e-1 */
    int pc_maxit;        /* inner PCG iteration cap; default 50 */
    int spectral_iterate; /* 1 (default): claire_register also carries the spectrum of its iterate
                            (updated with the Fourier-space PCG solution at every accepted step) and
                            forms the regulariser S v from it.  A forward FP32 transform of v has
                            roundoff of about 1e-7 ||v|| spread over all modes, which S(k) multiplies
                            by up to beta_w (1 + |k|^2) |k|^2 (2.4e5 at 256^3, 6e7 at 1024^3); the
                            carried spectrum avoids it.  Costs 3 half spectra (3 N1 N2 (N3/2+1)
                            complex values), allocated by the first claire_register.  0: S v from the
                            transform of v, as claire_gradient always does. */
    int kernels_only;    /* 1: a context for the kernel-level entry points only (claire_interp,
                            claire_interp_fields, claire_backtrace, claire_fd8_*, claire_dot): it
                            holds the grid, the stream and a few KB of reduction scratch, no fields
                            and no FFT plans, so grids far larger than a solver workspace fit;
                            solver-level calls return CLAIRE_ESTATE.  Default 0. */
} claire_opts;

/* claire_opts.precond */
#define CLAIRE_PRECOND_SPECTRAL 0
#define CLAIRE_PRECOND_TWO_LEVEL 1

/* claire_opts.storage */
#define CLAIRE_STORAGE_F32 0
#define CLAIRE_STORAGE_F16 1
#define CLAIRE_STORAGE_BF16 2

/* Phase slots of claire_report.t_phase_s (seconds, CUDA-event timed when opts.timing = 2). */
#define CLAIRE_PHASE_BACKTRACE 0   /* RK2 characteristics, div v, div v at X+ */
#define CLAIRE_PHASE_STATE 1       /* forward solve and FD8 gradients of m^j */
#define CLAIRE_PHASE_ADJOINT 2     /* adjoint solve with gradient body */
#define CLAIRE_PHASE_INCREMENTAL 3 /* incremental state + incremental adjoint solves */
#define CLAIRE_PHASE_SPECTRAL 4    /* FFTs and spectral scaling */
#define CLAIRE_PHASE_VECTOR 5      /* PCG / line-search vector updates and reductions */
#define CLAIRE_PHASE_OBJECTIVE 6   /* line-search objective evaluations */
#define CLAIRE_PHASE_GATHER 7      /* the SL gather kernels alone (subset of 0-3, 6) */
#define CLAIRE_MAX_LOGGED_STEPS 64

typedef struct claire_report {
    int status;                 /* claire_status of the run */
    int gn_iters;               /* Gauss-Newton updates taken */
    int pcg_iters_total;        /* Hessian matvecs in all PCG solves */
    int pcg_iters[CLAIRE_MAX_LOGGED_STEPS];   /* PCG iterations per GN step */
    double alpha[CLAIRE_MAX_LOGGED_STEPS];    /* accepted step length per GN step */
    double J;                   /* objective at the returned v */
    double mismatch;            /* 1/2 ||m(1) - m1||^2 at the returned v */
    double r;                   /* relative residual ||m(1)-m1||^2 / ||m0-m1||^2 (Sec. 4.1) */
    double gnorm_rel;           /* ||g|| / ||g0|| at the returned v */
    double detj_min, detj_max;  /* extrema of det grad y at the returned v (Sec. 3, J_min) */
    double cfl;                 /* max_x |v(x)|_2 dt / min_c h_c at the returned v */
    double t_total_s;           /* wall time of the call */
    double t_phase_s[8];        /* see CLAIRE_PHASE_* */
    double gather_launches;     /* SL gather kernel launches (CLAIRE_PHASE_GATHER count) */
    double interp_points;       /* grid points x scalar fields interpolated by the gathers */
    double interp_bytes;        /* algorithmic HBM bytes of the gather kernels (each value once) */
    int pc_inner_iters_total;   /* inner PCG iterations of the two-level preconditioner (0 otherwise) */
    int pc_fallbacks;           /* Gauss-Newton steps whose two-level solve failed the line search and
                                   were solved again with the spectral preconditioner */
} claire_report;

/* Fill *opts with the defaults listed above.  Returns CLAIRE_EINVAL on NULL. */
claire_status claire_default_opts(claire_opts* opts);

/*
 * Create a context for grid[3] = {N1, N2, N3}, regularisation weight beta_v > 0
 * (Sec. 3, "beta_v") and nt >= 1 semi-Lagrangian time steps (Sec. 3, "n_t").
 * opts may be NULL for the defaults.  Allocates every device workspace up
 * front (see claire_query_workspace) and the cuFFT plans; returns
 * CLAIRE_ENOMEM before any kernel runs if the device cannot hold them.
 * *ctx receives the new context (NULL on error).
 */
claire_status claire_create(claire_ctx** ctx, const int grid[3], double beta_v, int nt,
                            const claire_opts* opts);

/* Free all device memory and plans of ctx.  NULL is accepted. */
claire_status claire_destroy(claire_ctx* ctx);

/* Queue all further work of ctx on stream (a cudaStream_t, e.g. torch's
 * current stream handle); NULL selects the legacy default stream. */
claire_status claire_set_stream(claire_ctx* ctx, void* stream);

/* Device bytes claire_create would allocate for this grid, nt and options. */
claire_status claire_query_workspace(const int grid[3], int nt, const claire_opts* opts,
                                     size_t* bytes);

/* Copy the template m0 and reference m1 (N floats each) into the context.
 * Invalidates the linearisation point. */
claire_status claire_set_images(claire_ctx* ctx, const float* m0, const float* m1);

/* Objective J(v) of Eq. (1a) and its mismatch term at v (3N floats).
 * Either output pointer may be NULL.  Does not change the linearisation point. */
claire_status claire_objective(claire_ctx* ctx, const float* v, double* J, double* mismatch);

/*
 * Reduced gradient, Eq. (3), at v (3N floats) into g (3N floats):
 *   grad_form 0: g = S v + b,  grad_form 1: g = beta_v A v + K b,
 *   b = int_0^1 lambda grad m dt (trapezoid on the nt+1 time points),
 * with the state by SL transport (Eq. (1b)) and the adjoint lambda by SL
 * transport of Eq. (4) from lambda(1) = m1 - m(1).  Makes v the
 * linearisation point of later claire_hessian_matvec calls.  J may be NULL.
 * S v is formed from an FP32 transform of v, whose roundoff S(k) amplifies
 * at high |k| (about 7e-3 of ||S v|| for a smooth v at 256^3, growing as n^4);
 * claire_register avoids that with its carried spectrum (spectral_iterate).
 * The same holds for the S vt of claire_hessian_matvec.
 */
claire_status claire_gradient(claire_ctx* ctx, const float* v, float* g, double* J);

/*
 * Gauss-Newton Hessian matvec, Eq. (6), at the last claire_gradient's v:
 *   Hvt = S vt + int_0^1 lt grad m dt   (grad_form 1: K applied to the body
 *   and beta_v A to vt), with the incremental state mt (d_t mt + v . grad mt
 *   = -vt . grad m, mt(0) = 0) and incremental adjoint lt (Eq. (4) with
 *   lt(1) = -mt(1)).  vt, Hvt: 3N floats.  CLAIRE_ESTATE without a prior
 *   claire_gradient on the current images.
 */
claire_status claire_hessian_matvec(claire_ctx* ctx, const float* vt, float* Hvt);

/* Preconditioner of the PCG solve, z = P^{-1} r (3N floats each):
 * CLAIRE_PRECOND_SPECTRAL: the spectral inverse of the regulariser (S^{-1}, or
 * (beta_v A)^{-1} for grad_form 1), identity on k = 0;
 * CLAIRE_PRECOND_TWO_LEVEL: the two-level zero-velocity preconditioner at the
 * last claire_gradient's v (CLAIRE_ESTATE without one), E H0c^{-1} R r on the
 * coarse modes |k_i| < N_i / (2 pc_coarse) other than k = 0, S^{-1} r on the
 * others, r on k = 0; H0c^{-1} is pc_maxit (or fewer, pc_tol) inner PCG
 * iterations. */
claire_status claire_precond(claire_ctx* ctx, const float* r, float* z);

/* Coarse preconditioner correction (the learned warm start's second output,
 * an extension of Sec. 2.2 "Optimization"): a pointwise weight w >= 0 of the
 * data term of the two-level preconditioner's zero-velocity operator, which
 * becomes H0c = S + gbar_c w gbar_c^T on the coarse grid (w = 1: the paper's
 * operator).  w: FP32 [Nc1][Nc2][Nc3] (device or host) on the coarse grid
 * wgrid = N / pc_coarse, copied in; negative values act as 0.  NULL clears it.
 * Used by every later two-level preconditioner set-up of this context.
 * CLAIRE_EINVAL: wgrid is not the coarse grid of the context's options (also
 * reported by the set-up if pc_coarse changes afterwards);
 * CLAIRE_ENONFINITE: w holds a non-finite value (the weight is then cleared). */
claire_status claire_set_pc_weight(claire_ctx* ctx, const float* w, const int wgrid[3]);

/* gbar = sum_j w_j grad m^j (trapezoid weights of the solves, FD8 gradients of
 * the states) at the last claire_gradient's v, the field the zero-velocity
 * operator is built from; device pointer, 3N floats.  CLAIRE_ESTATE without a
 * linearisation point. */
claire_status claire_mean_state_gradient(claire_ctx* ctx, float* gbar);

/*
 * Gauss-Newton-Krylov registration, Eq. (5): v_{k+1} = v_k + alpha_k vt_k with
 * H vt_k = -g_k solved by matrix-free PCG (forcing opts.pcg_rtol_max) and
 * alpha_k from an Armijo line search (start 1, halve).  v_inout holds the
 * initial guess (3N floats; zeros for a cold start) and receives the result.
 * rep may be NULL.  Returns CLAIRE_OK on ||g||/||g0|| <= gtol,
 * CLAIRE_ENOTCONVERGED after max_gn steps, or an error; v_inout then holds
 * the last accepted iterate.
 */
claire_status claire_register(claire_ctx* ctx, float* v_inout, claire_report* rep);

/*
 * Semi-Lagrangian transport over t in [0, 1] with nt RK2 steps by the
 * velocity v (3N floats):
 *   CLAIRE_TRANSPORT_FWD: m_out = m(1) of Eq. (1b) with m(0) = m_in;
 *   CLAIRE_TRANSPORT_ADJ: m_out = lambda(0) of Eq. (4) with lambda(1) = m_in.
 * m_in and m_out are N floats and may alias.
 */
claire_status claire_transport(claire_ctx* ctx, const float* v, const float* m_in, float* m_out,
                               int flags);

/*
 * Reverse-mode derivative of the discrete forward transport m(1) = T(v)^nt m0
 * (the same SL steps as CLAIRE_TRANSPORT_FWD: Heun characteristic X with the
 * velocity interpolated at the predictor, nt gathers; Sec. 2.2).  Given
 * gbar = dL/dm(1) (N floats) it returns the exact derivatives of the discrete
 * map (discretise-then-differentiate): gm0 = dL/dm0 (N floats) and
 * gv = dL/dv (3N floats, physical units); either output may be NULL.  The
 * scatter transposes accumulate 64-bit fixed-point integers, so results are
 * bitwise reproducible.  flags: CLAIRE_VJP_RECOMPUTE keeps only m0 and
 * recomputes m^j during the backward sweep (time-step checkpointing: 2 N
 * floats of states instead of (nt+1) N).  The first call allocates its
 * scratch ((nt+1) N floats + N 64-bit accumulators); the call invalidates the
 * linearisation point of claire_hessian_matvec.  Computes in FP32.  All
 * three interpolation orders: with cubic B-splines the interpolant gradients
 * are those of each state's (and the velocity's) spline coefficients, and
 * every scatter transpose is followed by the prefilter, whose real, even
 * symbol makes it its own transpose.
 */
#define CLAIRE_VJP_RECOMPUTE 1
claire_status claire_transport_vjp(claire_ctx* ctx, const float* v, const float* m0, const float* gbar,
                                   float* gm0, float* gv, int flags);

/*
 * Grid transfer of ncomp periodic fields (component-major, each a full grid)
 * from the grid `from` to the grid `to` (all extents even), as used to
 * register downsampled images and carry the velocity back to the base grid
 * (Sec. 4, downsampled registrations: images sampled by nearest neighbour,
 * velocity upsampled by spectral prolongation).
 *   CLAIRE_RESAMPLE_SPECTRAL: Fourier coefficients are copied between the
 *     spectra (wavenumbers at or beyond either grid's Nyquist limit are
 *     dropped, new ones are zero): band-limited interpolation / truncation.
 *   CLAIRE_RESAMPLE_NEAREST: out[j] = in[floor(j * n_from / n_to)] per axis.
 * `in` and `out` are 16-byte aligned device pointers (caller-owned, must not
 * overlap; anything else is CLAIRE_EINVAL, nothing launched); work is queued
 * on `stream`.  Needs no context.  The spectral mode keeps cuFFT
 * plans and two spectra for the last four (device, from, to) combinations
 * (freed by claire_resample_release), serialises callers on a mutex and
 * synchronises the stream before returning.  Errors: CLAIRE_EINVAL (shapes,
 * mode), CLAIRE_ENOMEM, CLAIRE_ECUFFT, CLAIRE_ECUDA, CLAIRE_ETOOLARGE (a
 * grid of 2^31 points or more).
 */
#define CLAIRE_RESAMPLE_SPECTRAL 0
#define CLAIRE_RESAMPLE_NEAREST 1
claire_status claire_resample(const float* in, const int from[3], float* out, const int to[3], int ncomp, int mode,
                              void* stream);
/* Free the plans and spectra cached by claire_resample (all devices' entries;
 * call with no claire_resample in flight). */
claire_status claire_resample_release(void);

/* Extrema of the Jacobian determinant det grad y of the deformation map of v
 * (Sec. 3, "J_min"; y = x + u with u transported by the state's SL steps,
 * F = I + FD8(u), det and extrema in FP64). */
claire_status claire_detj(claire_ctx* ctx, const float* v, double* detj_min, double* detj_max);

/* ---- kernel-level entry points (device pointers only; ctx gives grid and stream) ---- */

/* out[p] = f(x_p + d_p): f, out N floats, d 3N floats (grid units); order 3, 1 or 4
 * (CLAIRE_INTERP_BSPLINE: f is prefiltered into the context's scratch first).
 * Sec. 3 "IP kernel". */
claire_status claire_interp(claire_ctx* ctx, const float* f, const float* d, float* out, int order);

/* out[q][p] = f[q](x_p + d_p) for nf >= 1 fields sharing one displacement: f and
 * out are nf x N floats (field-major), d 3N floats; order 3 or 1 (the fields
 * are not prefiltered, so CLAIRE_INTERP_BSPLINE is rejected).  One kernel
 * reads d and forms each tile's box geometry once for all fields (Sec. 3 "IP
 * kernel" applied to several fields, as the paper's velocity components). */
claire_status claire_interp_fields(claire_ctx* ctx, const float* f, int nf, const float* d, float* out, int order);

/* Dice overlap (Sec. 4.1, measures of performance) of the label sets
 * A = {a >= 1/2} and B = {b >= 1/2}: *dice = 2 |A and B| / (|A| + |B|), 1 when
 * both are empty.  a, b: n floats (device pointers), e.g. a label's indicator
 * function carried by claire_transport and the reference label's indicator.
 * Counts are exact integers (FP64 partial sums).  Synchronises the stream. */
claire_status claire_dice(claire_ctx* ctx, const float* a, const float* b, size_t n, double* dice);

/* Number of CTAs (one per 4 x 8 x 32 tile of arrival points) of the tiled
 * gathers -- interpolation, backtrace, every SL step -- that took the
 * global-memory path because their departure box did not fit in shared
 * memory, since the last reset (reset != 0 clears it), on the current
 * device, summed over all contexts.  Synchronises the device. */
claire_status claire_gather_fallback_tiles(unsigned long long* count, int reset);

/* RK2 (Heun) characteristic displacement (Sec. 2.2) of v in grid units:
 * direction +1: X = x - dt/2 [v(x) + v(x - dt v(x))]; direction -1: X+ with +v.
 * dt = 1/nt of ctx; the velocity at the predictor point uses ctx's order. */
claire_status claire_backtrace(claire_ctx* ctx, const float* v, float* d, int direction);

/* 8th-order central FD gradient (f: N -> g: 3N) and divergence (v: 3N -> dv: N),
 * periodic (Sec. 2.2, Sec. 3 "FD kernel"). */
claire_status claire_fd8_grad(claire_ctx* ctx, const float* f, float* g);
claire_status claire_fd8_div(claire_ctx* ctx, const float* v, float* dv);

/* out = F^{-1}[M(k) F[in]] for the 3N-float vector field in (op: CLAIRE_SPECTRAL_*),
 * with the context's beta_v, beta_w and reg. */
claire_status claire_spectral(claire_ctx* ctx, const float* in, float* out, int op);

/* FP64 inner product h1 h2 h3 sum_i x_i y_i over n floats (device pointers). */
claire_status claire_dot(claire_ctx* ctx, const float* x, const float* y, size_t n, double* out);

/*
 * claire_dot_noalloc: the same FP64 inner product as claire_dot, for callers
 * that cannot allocate device memory: a process whose device memory is fully
 * reserved by another allocator, a latency-critical loop that cannot take the
 * implicit device-wide synchronisation of cudaMalloc / cudaFree, or code that
 * holds no claire context (creating one allocates all workspaces).  The paper
 * has no counterpart; this is a library convenience.
 *
 *   *out = scale * sum_{i<n} x_i y_i    (scale = h1 h2 h3 gives claire_dot)
 *
 * x, y: device pointers to n floats; out: host pointer; stream: a
 * cudaStream_t or NULL for the legacy default stream.  Allocates nothing:
 * the partial sums live in a fixed device array of 1 MiB + 256 B that every
 * GPU loading the library holds until the process exits.  n may be at most
 * 2^30 (1,073,741,824); larger n returns CLAIRE_ETOOLARGE before any launch.
 * The first call on each device looks up that array's device address (with
 * the device current); make that first call before any stream capture.
 * Calls share the array and overwrite the slots they use: calls whose work
 * overlaps on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  Synchronises `stream` before returning.
 * x and y must be memory of the current device (or managed memory): the
 * kernels run on the current device.  Returns CLAIRE_EINVAL for null or host
 * input pointers and for device memory of another GPU, CLAIRE_ECUDA on a
 * CUDA error.
 */
claire_status claire_dot_noalloc(const float* x, const float* y, size_t n, double scale,
                                 void* stream, double* out);

/* ---- instrumentation ---- */

/* Per-kernel counters of ctx since creation or the last reset: launches,
 * CUDA-event time on the context's stream (only while timing is on),
 * algorithmic HBM bytes (each value counted once) and grid points x scalar
 * fields interpolated.  name is one of sl_interp, sl_backtrace_rk2,
 * sl_adjoint_step, sl_incremental_step, sl_incremental_last, sl_pointwise,
 * fd8, spectral_scale, cufft (library transforms), reduce_f64,
 * vector_update, sl_map_step, detj_minmax. */
typedef struct claire_kernel_stat {
    char name[32];
    double launches, seconds, bytes, points;
} claire_kernel_stat;

/* Copy up to capacity entries into out; *count (may be NULL) receives the
 * number of kernel classes.  reset = 1 zeroes the counters afterwards. */
claire_status claire_kernel_stats(claire_ctx* ctx, claire_kernel_stat* out, int capacity, int* count,
                                  int reset);

/* Turn per-launch CUDA-event timing on (1) or off (0) after creation. */
claire_status claire_set_timing(claire_ctx* ctx, int on);

/* Change the regularisation weights of a live context (beta_v > 0,
 * beta_w >= 0); clears the linearisation point. */
claire_status claire_set_beta(claire_ctx* ctx, double beta_v, double beta_w);
claire_status claire_get_beta(const claire_ctx* ctx, double* beta_v, double* beta_w);

/*
 * Regularisation-parameter search and continuation (Sec. 3, "Parameter
 * identification").  Every solve is a claire_register warm-started from the
 * last accepted velocity; a solve is valid when it returns a non-negative
 * status and det grad y stays within [jmin, 1/jmin].
 *
 * Search: (i) beta_w = beta_w_max; beta_v = beta_v_max, divided by 10 after
 * every valid solve until a solve breaches the bounds (or beta_v would fall
 * below beta_v_min); then bisection (arithmetic midpoints) between the last
 * valid and the breaching beta_v until their gap is below bisect_rtol times
 * the valid one: beta_v* is the smallest valid value seen.  (ii) beta_v =
 * beta_v*; beta_w divided by 10 while the solve stays valid and beta_w >=
 * beta_w_min: beta_w* is the last valid value.
 * Continuation: beta_v = beta_v_max, /10 down to 10^ceil(log10 target_v),
 * then target_v (beta_w = beta_w_max); then beta_w /10 steps from
 * beta_w_max down to target_w; no bounds are checked.
 *
 * v_inout: initial guess in (host or device, 3N floats), velocity of the
 * last accepted solve out; the context keeps the selected (search) or target
 * (continuation) weights.  Two 3N-float device vectors are allocated for the
 * duration of the call.  Returns the status of the last accepted solve
 * (CLAIRE_ENOTCONVERGED if even beta_v_max breaches the bounds, with that
 * solve's velocity), or a negative status if a solve fails.
 */
typedef struct claire_search_opts {
    double beta_v_max;   /* default 1 */
    double beta_v_min;   /* default 1e-5 */
    double beta_w_max;   /* default 1e-5 */
    double beta_w_min;   /* default 1e-7 */
    double jmin;         /* default 0.1 (bounds [0.1, 10]) */
    double bisect_rtol;  /* default 0.1 */
    int max_solves;      /* cap on registrations; default 40 */
} claire_search_opts;

#define CLAIRE_MAX_SEARCH_SOLVES 64
typedef struct claire_search_report {
    double beta_v, beta_w;         /* selected / final weights */
    int solves;                    /* registrations run */
    double trace_beta_v[CLAIRE_MAX_SEARCH_SOLVES];
    double trace_beta_w[CLAIRE_MAX_SEARCH_SOLVES];
    double trace_detj_min[CLAIRE_MAX_SEARCH_SOLVES];
    double trace_detj_max[CLAIRE_MAX_SEARCH_SOLVES];
    int trace_valid[CLAIRE_MAX_SEARCH_SOLVES];
    int trace_gn_iters[CLAIRE_MAX_SEARCH_SOLVES];
    double t_total_s;
    claire_report last;            /* report of the accepted solve whose velocity is returned */
} claire_search_report;

claire_status claire_default_search_opts(claire_search_opts* opts);
claire_status claire_param_search(claire_ctx* ctx, float* v_inout, const claire_search_opts* opts,
                                  claire_search_report* rep);
claire_status claire_param_continuation(claire_ctx* ctx, float* v_inout, double target_beta_v,
                                        double target_beta_w, const claire_search_opts* opts,
                                        claire_search_report* rep);

/* Replace the options of an existing context (e.g. gtol, max_gn, g0_ref
 * between solves).  storage is fixed at claire_create: a different value is
 * CLAIRE_EINVAL; invalid options are CLAIRE_EINVAL and leave the context
 * unchanged.  Clears the linearisation point of claire_hessian_matvec. */
claire_status claire_set_opts(claire_ctx* ctx, const claire_opts* opts);
/* Current options of a context. */
claire_status claire_get_opts(const claire_ctx* ctx, claire_opts* opts);

/* One-line description of the last error on ctx (never NULL; "" if none). */
const char* claire_last_error(const claire_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CLAIRE_H */
