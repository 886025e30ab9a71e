/*
 * cgfill.h -- C ABI of the GB300 constrained-realization fill-in library.
 *
 * Method: Bucher & Louis, "Filling in CMB map missing data using constrained
 * Gaussian realizations" (arXiv:1109.0286), on the flat periodic sky (the
 * torus of Sect. 3).
 *
 *   Pixels split into masked M (to fill; the paper's x) and observed U (the
 *   constraints; the paper's y).  C = P + N is diagonal in Fourier space with
 *   eigenvalues P(k) (Sect. 4: the DFT is exactly unitary on the torus).
 *   One constrained realization (Sects. 2.1 and 2.3, Hoffman-Ribak):
 *       y   = F^-1 [ sqrt(P) F xi ],   xi ~ N(0,1) white noise from the seed
 *       b   = -( C^-1 z )_M,           z = d - y on U, 0 on M
 *       solve A u = b,  A = P_x C^-1 P_x          (eq. ModEq, Sect. 2.4)
 *       x_M = y_M + u,  x_U = d_U (bit for bit)
 *   by conjugate gradients (Sect. 2.4), optionally preconditioned with
 *   S = P_x C^{1/2} P_x on both sides (Sect. 2.4; run in the equivalent
 *   preconditioned form with B = S S, which exposes the true residual).
 *
 * Conventions shared by every entry point:
 *   - Grid ny x nx, row-major, periodic; either nx and ny powers of two
 *     with 32 <= nx <= 8192 and 16 <= ny <= 8192 (register-resident FFT
 *     passes), or a mixed-radix grid: nx even, nx/2 and ny products of
 *     2, 3, 5 and 7 with 8 <= nx/2 <= 4096 and 8 <= ny <= 4096 (in-place
 *     shared-memory passes of radix 2, 3, 4, 5, 7, 8; the flat-sky workloads
 *     of Sect. 3 such as 7000 x 600 = 2^3 5^3 7 x 2^3 3 5^2).
 *   - DFT: F x(k) = sum_r x(r) exp(-i k.r), F^-1 carries 1/n, n = ny*nx,
 *     k = 2 pi m / N with m in [-N/2, N/2).
 *   - P_half: host, float64, ny x (nx/2+1) row-major (the half plane of a
 *     real 2D FFT: row my in FFT order, column mx = 0..nx/2).
 *   - observed: host, uint8, ny x nx, 1 = observed (constraint), 0 = masked.
 *   - Maps passed to the compute calls are DEVICE pointers owned by the
 *     caller; their element type depends on the plan's mode (float for
 *     FILL_MODE_FP32, double otherwise).  Work is ordered on the plan's
 *     stream; the calls below return after that work has completed.
 *   - No call aborts the process: every failure is a returned status.
 *     After FILL_ECUDA the plan must be destroyed.
 */
#ifndef CGFILL_H
#define CGFILL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CGFILL_VERSION 1

typedef struct fill_plan fill_plan;

typedef enum {
  FILL_OK = 0,
  FILL_EINVAL = 1,      /* bad argument: size, spectrum, mask, pointer, non-finite data */
  FILL_ENOMEM = 2,      /* device or pinned host allocation failed */
  FILL_ENOTCONV = 3,    /* iteration limit reached before the tolerance */
  FILL_EBREAKDOWN = 4,  /* p^T A p <= 0, r^T z <= 0 or a non-finite value inside the solve */
  FILL_ETIMEOUT = 5,    /* a kernel's bounded wait for an asynchronous copy expired
                           (reported by fill_realize, fill_backward or a group call) */
  FILL_ECUDA = 6        /* CUDA runtime error (message via fill_last_error) */
} fill_status;

typedef enum {
  FILL_MODE_FP64 = 0,   /* every step in FP64 ("plain FP64 PCG") */
  FILL_MODE_FP32 = 1,   /* FP32 FFT operator and vectors, FP64-accurate inner
                           products; maps are float */
  FILL_MODE_MIXED = 2   /* high-precision draw, right-hand side and true residuals
                           in double-float arithmetic (pairs of FP32 values,
                           about 48 significant bits, run on the FP32 pipes);
                           FP32 PCG iterations with residual updates; maps double */
} fill_mode;

typedef struct {
  int mode;              /* fill_mode; default FILL_MODE_MIXED */
  int precond;           /* 0: plain CG (Sect. 3, point-source masks);
                            1: sqrt(C) split preconditioner (Sect. 2.4); default 1 */
  int batch;             /* realizations per fill_realize call (same mask and P); default 1 */
  int max_iter;          /* CG iterations per solve; default 10000 */
  int max_refine;        /* refinement steps (mixed mode, update_delta = 0); default 10 */
  int host_loops;        /* 0: each CG loop is one CUDA-graph launch (a conditional
                            WHILE node; default); 1: every kernel of the loops is
                            launched from the host, with the convergence flags read
                            back every 8 iterations (for profilers that cannot see
                            kernels inside conditional graph nodes) */
  double inner_tol;      /* relative tolerance floor of the FP32 inner solves
                            (mixed mode); default 1e-6 */
  int history_cap;       /* residual-history entries kept per realization; default 0 */
  int rows_per_cta;      /* row-pass CTA height, 0 = default schedule (the CG loop's
                            precision; the mixed mode's double-float passes keep
                            their defaults) */
  int ffts_per_cta;      /* column FFTs per CTA, 0 = default schedule (as rows_per_cta) */
  int backward;          /* 1: allocate the buffers fill_backward needs; default 0 */
  double update_delta;   /* mixed mode: one FP32 PCG with reliable updates -- the FP32
                            correction is folded into the double-float solution and
                            the residual recomputed in double-float whenever the FP32
                            residual has fallen by this factor; default 1e-2.  0:
                            restarted iterative refinement (FP32 solves to inner_tol) */
  int col_kernel;        /* column pass of the FP32 table passes (power-of-two grids):
                            0 register-fed kernel (default); 1 persistent kernel fed by
                            bulk copies (TMA) into a double-buffered shared-memory slot;
                            the same arithmetic, so the results are identical.
                            fill_autotune may switch it */
  int lanes;             /* the CG loops run the batch as this many sub-batches, each a
                            parallel branch of the loop graph (one launch per pass and
                            lane; the GPU fills one lane's gaps with another's work);
                            results are identical for any value.  0 = automatic: 2 for
                            batch >= 2 on grids of at least 2^20 pixels, else 1; at
                            most 8 */
} fill_opts;

typedef struct {
  int iters;             /* CG operator applications (all inner solves in mixed mode) */
  int refine_steps;      /* true-residual recomputations (mixed mode) */
  int status;            /* fill_status of this realization */
  int launches;          /* kernels launched by the whole call (same for every entry) */
  double rel_resid;      /* recurrence ||r|| / ||b|| at exit (last inner solve) */
  double true_rel_resid; /* ||b - A u|| / ||b|| in double-float (mixed mode), else -1 */
  double ms;             /* wall time of the whole call */
} fill_stats;

/* Fills *opts with the defaults listed above. */
void fill_opts_default(fill_opts* opts);

/*
 * fill_init -- build a plan for one grid, one spectrum P(k) and one mask.
 * Validates P (finite, > 0, and P(0,ky) = P(0,-ky), P(nx/2,ky) = P(nx/2,-ky)
 * so that C is a real symmetric operator; Sect. 4) and the mask (values 0/1),
 * builds the spectral tables 1/(nP) and sqrt(P)/n in the transposed layout of
 * the column pass, and allocates every device buffer the plan will use (the
 * compute calls allocate nothing).  stream: a cudaStream_t (NULL = legacy
 * default stream).  On success *plan owns its memory until fill_destroy.
 * Errors: FILL_EINVAL (sizes, spectrum, mask, opts), FILL_ENOMEM, FILL_ECUDA.
 */
fill_status fill_init(fill_plan** plan, int ny, int nx, const double* P_half,
                      const uint8_t* observed, const fill_opts* opts, void* stream);

/*
 * fill_realize -- `batch` constrained Gaussian realizations (Sects. 2.1-2.4).
 * d:       device, batch maps of ny*nx (float in FP32 mode, else double); the
 *          values on masked pixels are ignored.  d_stride: elements between
 *          consecutive maps (0 = one map shared by the whole batch).
 * seeds:   host, batch uint64; the seed alone fixes the white noise xi.
 * tol:     stop when ||b - A u|| <= tol ||b|| (recurrence residual in the
 *          FP32/FP64 modes; the double-float true residual in mixed mode).
 * out:     device, batch contiguous maps of ny*nx (same type as d);
 *          out_U = d_U exactly, out_M = y_M + u.
 * stats:   host array of batch entries, or NULL.
 * Data that are not finite on the observed pixels (NaN, Inf, or values so
 * large that the right-hand side overflows) give that realization the status
 * FILL_EINVAL: its solve stops before the first iteration, the call returns
 * at once, and the plan stays usable.
 * Returns the worst per-realization status -- FILL_EINVAL before
 * FILL_EBREAKDOWN before FILL_ENOTCONV (the last two leave the last iterate
 * in out) -- or FILL_EINVAL for bad arguments, or FILL_ECUDA.
 */
fill_status fill_realize(fill_plan* plan, const void* d, long long d_stride,
                         const uint64_t* seeds, double tol, void* out, fill_stats* stats);

/*
 * fill_realize_batch -- constrained realizations (Sects. 2.1-2.4) for several
 * plans in one call: masks, spectra and grid sizes may differ between plans.
 * d[i]: device, one data map shared by plan i's batch; out[i]: device, plan
 * i's batch maps; seeds: host, one per realization in plan order (plan 0's
 * batch first); stats: host, one entry per realization, or NULL.  The result
 * of each plan equals what fill_realize would give it.
 * Plans of one mode (FP32, FP64, or mixed with one update_delta > 0), one
 * precond setting and one stream run as a group (see fill_group_init): plans
 * of the same grid share every pass launch and the grid sizes run as
 * concurrent branches of one graph per CG loop.  The first call with a given
 * list of plans builds that group (device descriptors and the loop graph)
 * and caches it in plans[0]; later calls with the same list reuse it, and
 * fill_destroy(plans[0]) frees it.  Any other list (differing settings, or
 * mixed mode with restarted refinement, update_delta = 0) runs the plans one
 * after another.  Errors: as fill_realize.
 */
fill_status fill_realize_batch(fill_plan* const* plans, int count, const void* const* d,
                               const uint64_t* seeds, double tol, void* const* out,
                               fill_stats* stats);

/*
 * fill_set_spectrum -- replaces the plan's spectrum P(k) in place (for
 * band-power updates: an optimisation over the amplitudes a_b of
 * P = sum_b a_b T_b + N needs a new P at every step, Sects. 2.1, 4).  Same
 * layout and validation as fill_init's P_half (host, float64, ny x (nx/2+1),
 * finite, > 0, Hermitian-consistent); rebuilds the tables 1/(nP) and
 * sqrt(P)/n of every precision the plan holds, the relaxation level
 * max 1/P, and -- if fill_set_bands was called -- the band-gradient weights
 * at the new P.  Allocates nothing; waits for the plan's stream first.  The
 * realizations of earlier calls are not kept: fill_backward then needs a new
 * fill_realize.  Errors: FILL_EINVAL (message via fill_last_error), FILL_ECUDA.
 */
fill_status fill_set_spectrum(fill_plan* plan, const double* P_half);

/*
 * fill_ml -- maximum-likelihood fill (Sect. 2.1): x_M = -((C^-1)_MM)^-1 (C^-1)_MU d_U,
 * x_U = d_U, the mean of the constrained field (the Hoffman-Ribak
 * realization without its random part: y = 0).  Same solver, precision
 * and arguments as fill_realize without the seeds; each of the batch
 * entries fills its own data map (d_stride as in fill_realize).
 * Errors: as fill_realize.
 */
fill_status fill_ml(fill_plan* plan, const void* d, long long d_stride, double tol, void* out,
                    fill_stats* stats);

/*
 * fill_relax -- the kernel relaxation of Sect. 5 (eqs. kern:rel, Boo, Algo) on the
 * torus: writing C^-1 = a (delta - K) with a = max_k 1/P(k), the white level of the
 * precision (so that K's spectrum 1 - 1/(aP) lies in [0, 1) and K * x is a
 * weighted average), it repeats x_M <- (K * x)_M = x_M - (C^-1 x)_M / a from
 * x_M = 0, x_U = d_U, `iters` times (three passes per sweep).  Its fixed point is
 * the ML fill (eq. Boo); convergence is geometric with a rate set by the condition
 * number of C^-1, which is why the paper turns to multi-scale kernels and CG.
 * d, d_stride, out as in fill_ml; out_U = d_U exactly.  stats: iters = sweeps,
 * rel_resid = ||(C^-1 x)_M|| / ||(C^-1 x_0)_M|| before the last sweep.
 * Precision: the plan's (mixed mode: double-float).  Errors: FILL_EINVAL, FILL_ECUDA.
 */
fill_status fill_relax(fill_plan* plan, const void* d, long long d_stride, int iters, void* out,
                       fill_stats* stats);

/*
 * fill_subdivide -- the boundary layer of width delta (Sect. 6.2): the observed
 * indicator convolved with the normalised top hat of radius delta/2 on the
 * periodic grid, i.e. the fraction of the disc {dy^2 + dx^2 <= (delta/2)^2}
 * around each pixel that is observed; layer[i] = 1 for masked pixels where it
 * exceeds `threshold` (0.03 in the paper), else 0.  The fraction is an exact
 * pixel count (per-row prefix sums), and the test is
 * count * 100 > round(100 threshold) * |disc|.  No plan, no allocation.
 * observed: device, ny*nx (1 = observed); scratch: device, ny*(nx+1) int32;
 * layer: device, ny*nx uint8 (out).  Needs 2 floor(delta/2) + 1 <= ny, nx.
 * Asynchronous on `stream`.  Errors: FILL_EINVAL (message via fill_last_error),
 * FILL_ECUDA.
 */
fill_status fill_subdivide(int ny, int nx, const uint8_t* observed, double delta,
                           double threshold, int32_t* scratch, uint8_t* layer, void* stream);

/*
 * fill_set_annuli / fill_laplace_ms -- the kernel-based Laplace solver of
 * Sect. 6.3: each masked pixel is repeatedly replaced by the average of the map
 * over an annulus around it -- the mean-value property of harmonic functions --
 * taking the largest of a family of annuli that stays inside the mask, so that
 * information crosses wide holes in a number of sweeps growing like a power of
 * log(width) instead of width^2.
 * fill_set_annuli: nk annuli r_in[j]^2 < |offset|^2 <= r_out[j]^2 (the centre
 * never included; 2 r_out < nx, ny); builds their normalised transforms as
 * column-pass tables with the plan's own transforms (allocates on the first
 * call or when nk grows).  fill_laplace_ms: `iters` Jacobi sweeps from 0 on the
 * mask and d on U; cls: device, ny*nx uint8, the annulus index of every masked
 * pixel (the solver of the paper takes the largest annulus whose disc holds no
 * observed pixel, and the smallest -- which reaches the observed region -- in
 * the thin layer along the boundary); d, d_stride, out as in fill_ml (out_U =
 * d_U exactly).  stats.rel_resid = the last sweep's change over the first's
 * (L2 over the mask).  Precision: the plan's.  Errors: FILL_EINVAL (no annuli
 * set, bad radii), FILL_ENOMEM, FILL_ECUDA.
 */
fill_status fill_set_annuli(fill_plan* plan, int nk, const double* r_in, const double* r_out);
fill_status fill_laplace_ms(fill_plan* plan, const void* d, long long d_stride, int iters,
                            const uint8_t* cls, void* out, fill_stats* stats);

/*
 * fill_draw -- unconstrained realizations y = F^-1[sqrt(P) F xi(seed)] with
 * covariance C (Sect. 2.3, the draw that needs no cuts).  out: device, batch
 * maps (plan element type).  Errors: FILL_EINVAL, FILL_ECUDA.
 */
fill_status fill_draw(fill_plan* plan, const uint64_t* seeds, void* out);

/*
 * fill_apply -- one operator application on a single map, for checks of the
 * GPU operator (symmetry, parity):  which = 0: C^-1 x;  1: C^{1/2} x;
 * 2: A x = P_x C^-1 P_x x (eq. ModEq);  3: S x = P_x C^{1/2} P_x x (Sect. 2.4).
 * in, out: device maps of the plan's element type (may not alias).
 * Errors: FILL_EINVAL, FILL_ECUDA.
 */
fill_status fill_apply(fill_plan* plan, int which, const void* in, void* out);

/*
 * fill_history -- copies the residual history ||r_k||/||b||, k = 0..iters, of
 * realization `inst` of the last fill_realize into host array hist of
 * capacity cap (FP32 / FP64 modes: the CG recurrence residual per iteration;
 * mixed mode: the true residual after each residual update, k = 0 being
 * the start).  Needs opts.history_cap > 0 at fill_init; *count receives the
 * number of entries written.  Errors: FILL_EINVAL, FILL_ECUDA.
 */
fill_status fill_history(fill_plan* plan, int inst, double* hist, int cap, int* count);

/*
 * fill_lanczos -- Lanczos estimate of the extreme eigenvalues of the
 * preconditioned operator (Sect. 6.4: the condition number predicts the CG
 * convergence rate and guides the stopping rule; the tridiagonal Lanczos
 * matrix comes from the CG coefficients, cf. Golub & Van Loan) for
 * realization `inst` of the last fill_realize.  The device records the step
 * lengths alpha_j and direction updates beta_j of the first history_cap
 * iterations (FP32 / FP64 modes: the PCG; mixed mode: the FP32 PCG of the
 * last inner solve, the whole solve with reliable updates); this call builds
 *   T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},  T_{j,j+1} = sqrt(beta_j)/alpha_j
 * (k x k, k = *count) and returns its smallest and largest eigenvalues (Sturm
 * bisection on the host) in *lmin, *lmax; kappa ~ lmax / lmin.
 * alpha, beta: host arrays of capacity cap receiving alpha_j and beta_j
 * (j < min(k, cap); beta of the last iteration is 0), or NULL.  Needs
 * opts.history_cap > 0.  Errors: FILL_EINVAL, FILL_EBREAKDOWN (an alpha_j
 * <= 0 was recorded), FILL_ECUDA.
 */
fill_status fill_lanczos(fill_plan* plan, int inst, double* alpha, double* beta, int cap,
                         int* count, double* lmin, double* lmax);

/*
 * fill_time_pass -- average device time of one launch of a hot-loop pass
 * kernel over all `batch` instances, timed with CUDA events on the plan's
 * stream (`reps` launches between two events, after one warm-up launch), and
 * the algorithmic bytes of one launch (the reads and writes the pass has to
 * make: each instance's spectrum and compact vectors, plus the column table or
 * the mask words once, since the batch shares them).  pass: 0 column pass (forward column FFT, x 1/(nP), inverse FFT);
 * 1 forward row pass fused with r -= alpha q, u += alpha p; 2 forward row pass
 * fused with p = z + beta p; 3 inverse row pass fused with q = P_x(.) and
 * p^T q; 4 inverse row pass, P_x, forward row pass (middle of S S r).
 * precision: 0 FP32 kernels, 1 FP64 kernels (must exist in the plan's mode).
 * Overwrites the plan's scratch; the next fill_realize starts afresh.
 * Errors: FILL_EINVAL, FILL_ECUDA.
 */
fill_status fill_time_pass(fill_plan* plan, int pass, int precision, int reps,
                           double* ms_per_launch, double* bytes_per_launch);

/*
 * fill_set_bands -- band-power parameterisation for fill_backward:
 * P(k) = sum_b a_b T_b(k) + N with T_b(k) = 1[band(k) = b] S(k).
 * band_of_k: host int32, ny x (nx/2+1) (layout of P_half), values in
 * [0, nbands), nbands <= 64; sig_half: host float64 S(k), same layout.  The
 * derivative is taken at the plan's P.  Allocates the plan's gradient tables
 * (on the first call).  Errors: FILL_EINVAL, FILL_ENOMEM, FILL_ECUDA.
 */
fill_status fill_set_bands(fill_plan* plan, int nbands, const int32_t* band_of_k,
                           const double* sig_half);

/*
 * fill_backward -- adjoint gradients of a scalar loss L(x) through the
 * realizations of the LAST fill_realize on this plan (no other compute call
 * in between; d must be the same data).  The paper does not differentiate its
 * method; with g = dL/dx the adjoint is one more solve with the same
 * symmetric operator and preconditioner, lam = A^-1 g_M (Sect. 2.4), and
 *   dL/dd = g_U - (C^-1 lam)_U on U, 0 on M;
 *   dL/da_b = sum_k T_b(k) [ Re(conj(F h) F xi)/(2 n sqrt P)
 *                            + Re(conj(F lam) F w)/(n P^2) ]   (full k plane)
 * with h = g on M, (C^-1 lam)_U on U, w = d - y on U, u on M, and xi the
 * seed's white noise held fixed (reparameterised draw).
 * grad_x, grad_d: device, batch maps (plan element type); grad_bands: host
 * batch x nbands doubles, or NULL to skip the band gradient.  Needs
 * opts.backward = 1 (and fill_set_bands if grad_bands is given).
 * Returns like fill_realize; stats describe the adjoint solve.
 */
fill_status fill_backward(fill_plan* plan, const void* d, long long d_stride,
                          const void* grad_x, double tol, void* grad_d, double* grad_bands,
                          fill_stats* stats);

/*
 * fill_autotune -- chooses the plan's launch schedule (grid rows per CTA of
 * the row passes, column FFTs per CTA of the column pass, and which column
 * kernel) by timing every valid candidate on the device; results are cached
 * as text lines in cache_path (NULL: no cache).  Mixed-radix grids also
 * choose the radix schedule of each transform length (radix-8 stages or
 * radix 4 and 2 only; odd radices ascending or descending), timed on the
 * precision of the CG loop and applied to every precision of the plan, with
 * new tables (graphs and groups built earlier keep the tables they were
 * built with).  Results differ from the default schedule's by rounding only.
 * Call after fill_init, before fill_realize.  Errors: FILL_EINVAL (also for a
 * cached schedule that is not valid for the plan), FILL_ENOMEM, FILL_ECUDA.
 */
fill_status fill_autotune(fill_plan* plan, const char* cache_path);

/*
 * Groups: many realizations over masks and grid sizes in one call.
 * fill_group_init collects plans (all of one mode -- FILL_MODE_FP32,
 * FILL_MODE_FP64, or FILL_MODE_MIXED with one update_delta > 0 for all --,
 * same precond and stream; power-of-two or mixed-radix grids; each keeps its
 * own mask, spectrum and buffers).
 * Plans with the same grid form a size class whose instances share every pass
 * launch; the classes run concurrently as parallel branches of one captured
 * CUDA graph per CG loop (mixed mode: the reliable-update loop of
 * fill_realize, double-float draw, right-hand side and residual updates per
 * class, an update IF node per class).  autotune != 0 tunes each class's
 * schedule of the CG loop's precision (cached in cache_path if not NULL;
 * mixed-radix classes keep their plans' schedules).  The plans must outlive
 * the group.  Errors: FILL_EINVAL, FILL_ENOMEM, FILL_ECUDA.
 */
typedef struct fill_group fill_group;
fill_status fill_group_init(fill_group** group, fill_plan* const* plans, int count,
                            int autotune, const char* cache_path);

/*
 * fill_group_realize -- constrained realizations (Sects. 2.1-2.4) for every
 * plan of the group.  d[i]: device, one data map shared by plan i's batch;
 * out[i]: device, plan i's batch maps; seeds: host, one per realization in
 * plan order (plan 0's batch first); stats: host, one per realization, or
 * NULL.  Returns the worst per-realization status (ranked as in
 * fill_realize).
 */
fill_status fill_group_realize(fill_group* group, const void* const* d, const uint64_t* seeds,
                               double tol, void* const* out, fill_stats* stats);

/* Realizations per fill_group_realize call (sum of the plans' batches). */
int fill_group_size(const fill_group* group);

/* Frees the group (not its plans; NULL is allowed). */
void fill_group_destroy(fill_group* group);

/*
 * fill_apply_static -- fill_apply without a plan and without any allocation,
 * for callers that cannot allocate device memory (code that runs inside a
 * memory pool or arena it does not own, or under an allocator that forbids
 * new allocations).  The paper has no counterpart; this is a library
 * convenience.  Applies, on one FP32 map, which = 0: C^-1 x; 1: C^{1/2} x;
 * 2: P_x C^-1 P_x x; 3: P_x C^{1/2} P_x x, with the same kernels as
 * fill_apply.  All pointers are DEVICE pointers: P_half float64 ny x (nx/2+1)
 * (assumed valid as fill_init would require; not checked), observed uint8
 * ny x nx (needed for which >= 2, else ignored), in / out float ny x nx (may
 * not alias).  stream: a cudaStream_t; the call returns once the work is
 * queued.  Scratch: one 8 MiB file-scope device array per device that loads
 * the library (held until exit), which limits the grid to about 1024 x 1024
 * pixels; larger grids return FILL_EINVAL with the reason in
 * fill_last_error().  The first call on a device does a one-time set-up
 * (symbol address, kernel attributes) and should come before any stream
 * capture.  All calls share the scratch and overwrite it: calls that overlap
 * on the GPU race, so order them on one stream.  No cudaMalloc / cudaFree
 * and no allocating library routine is called.
 */
fill_status fill_apply_static(int ny, int nx, const double* P_half, const uint8_t* observed,
                              int which, const float* in, float* out, void* stream);

/* Number of masked pixels n_M of the plan's mask. */
long long fill_masked_count(const fill_plan* plan);

/* Frees every resource of the plan (NULL is allowed). */
void fill_destroy(fill_plan* plan);

/* Static description of a status code. */
const char* fill_strerror(fill_status status);

/* Text of the last CUDA error seen by this thread (empty if none). */
const char* fill_last_error(void);

/* CGFILL_VERSION of the loaded library. */
int fill_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CGFILL_H */
