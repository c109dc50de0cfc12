/*
 * mem.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * 35-moment maximal-entropy moment method (MEM), arXiv 2303.02898.
 *
 * Conventions shared by every entry point:
 *   - Statistics: the 35 orthonormal Hermite products
 *       phi_k(ubar) = He_a(ubar_x) He_b(ubar_y) He_c(ubar_z) / sqrt(a! b! c!),
 *     a + b + c <= 4 (Appendix B, orthonormal form, extended to 3D), ordered
 *     by total degree, then a descending, then b descending; k = 0 is 1.
 *   - Gauge g = (w_x, w_y, w_z, s_x, s_y, s_z), ubar = (u - w) / s per axis
 *     (Section 3.3, Eq. "Sufficient 35 ortho").
 *   - Moments M[k] = int phi_k(ubar) f(u) d^3u in the cell's gauge; M[0] = n.
 *   - Natural parameters beta[k], k >= 1, relative to the Gauss-Hermite base
 *     measure: f = n exp(-|ubar|^2/2 + sum_{k>=1} beta_k phi_k - log Z);
 *     beta[0] = n.  beta = 0 is the Maxwellian of the gauge.  This is an
 *     exact re-parameterisation of the paper's canonical form (Eq. "exp
 *     family"): subtract 1/sqrt(2) from the three (2,0,0)-type entries to get
 *     the Lebesgue-measure parameters.
 *   - Arrays are row-major float32: moments/parameters [B][35], gauges
 *     [B][6].  Pointers marked "dev" are device memory, "host" host memory.
 *     The caller owns every array it passes; the library keeps no pointer to
 *     it after the call returns (stream-ordered work may still read it until
 *     the stream reaches that point).
 *   - stream: a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Unless stated otherwise a call only enqueues work.
 *   - Return codes: MEM_OK (0) or a negative MEM_E* code; per-cell outcomes
 *     are status bits, and a failed cell never fails the call.
 */
#ifndef MEM_GB300_H
#define MEM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MEM_NP 35

/* Return codes. */
#define MEM_OK 0
#define MEM_PENDING 1
#define MEM_EINVAL (-1)
#define MEM_ENOMEM (-2)
#define MEM_ECUDA (-3)
#define MEM_EBUSY (-4)
#define MEM_ENOTFOUND (-5)

/* Per-cell status bits of mem_solve. */
#define MEM_ST_CONVERGED 1   /* Newton decrement res <= tol (Algorithm 1)      */
#define MEM_ST_STAGNATED 2   /* step size alpha <= alpha_min: also converged   */
#define MEM_ST_MAXITER 4     /* more than maxI iterations                      */
#define MEM_ST_NONFINITE 8   /* non-finite objective, gradient or Hessian      */
#define MEM_ST_LAMBDA 16     /* a lambda*I modification was needed             */
#define MEM_ST_LAMBDA_CAP 32 /* lambda retries exhausted; solve stopped        */
#define MEM_ST_BADINPUT 64   /* n <= 0 or non-finite input                     */
#define MEM_ST_FP64_OK 128   /* mixed back-end: a cell stopped by MAXITER,
                                NONFINITE or LAMBDA_CAP whose moment residual,
                                recomputed in FP64, is within 1e-5 (its beta
                                is acceptable although the step failed)       */

/* Solver back-ends. */
#define MEM_IMPL_PLAIN 0 /* separate FP32 kernels per Newton stage, host loop   */
#define MEM_IMPL_FUSED 1 /* one persistent FP32 kernel, warp per cell           */
#define MEM_IMPL_MIXED 2 /* the plain stages with the moment / Hessian
                            contraction on tcgen05 tensor cores: split TF32
                            (about FP32 accuracy) for the moments that form
                            the gradient, one TF32 product for the Hessian
                            (Newton's model only); cells whose safeguarded
                            step fails get their residual recomputed in FP64
                            (MEM_ST_FP64_OK).  quad_order 8 and 12 only.    */

/* Interface flux of the shock's finite-volume step (Section 3.3). */
#define MEM_SCHEME_LF 0   /* local Lax-Friedrichs, Eq. "The lax F"               */
#define MEM_SCHEME_LW 1   /* two-step Lax-Wendroff, Eq. "The lax W"              */
#define MEM_SCHEME_FLIC 2 /* flux-limited centred with van Leer, Eq. "The FLIC" */

typedef struct mem_ctx mem_ctx;

/* Options of Algorithm 1 (modified Newton + backtracking Armijo line search).
 * Defaults are the paper's constants (Algorithm 1; maxI = 500 as in every
 * experiment of Section 4). */
typedef struct {
    float tol;        /* res = |dbeta . grad L| / 2 <= tol stops (1e-8)      */
    int32_t maxI;     /* at most maxI + 1 passes (500)                       */
    float lambda0;    /* first multiple of the identity (1e-3)               */
    float lambda_mul; /* growth per failed Cholesky (10)                     */
    int32_t max_lambda; /* cap on lambda retries (20)                        */
    float c_armijo;   /* Armijo slope factor (5e-4)                          */
    float atol;       /* Armijo absolute slack (5e-6)                        */
    float rtol;       /* Armijo relative slack (5e-5)                        */
    int32_t maxT;     /* line-search trials s = 0..maxT (25)                 */
    float alpha_min;  /* alpha <= alpha_min stops as stagnated (1e-6)        */
    int32_t final_step; /* 0: Algorithm 1's order, the last computed direction
                           is not applied (default); 1: an extension that
                           applies it when res <= tol (moment residual of
                           the solution instead of one Newton step behind) */
    int32_t impl;     /* MEM_IMPL_PLAIN, _FUSED (default) or _MIXED          */
} mem_solve_opts;

/* Fill *o with the defaults above. */
void mem_solve_opts_default(mem_solve_opts *o);

/* Library version string and the number of entry points it exports. */
const char *mem_version(void);

/* Create a context on the current CUDA device: quadrature tables (tensor
 * Gauss-Hermite, quad_order^3 nodes fixed in the gauge frame) and the
 * statistics tables.  degree must be 4 (35 statistics); quad_order 4..16
 * (8 and 12 are the configurations of the workload).  Synchronous.  Returns
 * MEM_EINVAL on bad arguments, MEM_ECUDA / MEM_ENOMEM on CUDA failures.
 * Paper: Section 3.1, Eq. "Numerical integration" (fixed nodes and weights);
 * Appendix B (statistics). */
int mem_init(int degree, int quad_order, mem_ctx **out);

/* Create a context whose quadrature is fixed in velocity space, the rule of
 * the paper's shock computations (Section 3.1, Eq. "Numerical integration":
 * fixed nodes u_q and weights w_q; Appendix D: integration domain
 * (u_x, u_r) in [a_x, b_x] x [0, b_r], split into equal blocks, each
 * integrated by Gauss-Legendre):
 *   u_x in [ax, bx]: nbx equal blocks of ng Gauss-Legendre points;
 *   u_r in [0, br]:  nbr equal blocks of ng Gauss-Legendre points (weight
 *                    u_r), times K equispaced azimuths 2 pi k / K (exact for
 *                    the azimuthal dependence of every product of two
 *                    statistics when K >= 9).
 * A cell of gauge g sees the nodes at ubar = (u - w) / s; beta keeps its
 * meaning (relative to the gauge's Gaussian).  Unlike the Gauss-Hermite rule
 * of mem_init, whose nodes move with each cell's gauge, these nodes resolve a
 * narrow upstream beam inside a hot shocked cell, which strong shocks (Mach
 * 10) need.  (ax, bx, br) is the domain of mem_solve_gauge and mem_flux;
 * shock problems on such a context take their own domain from their
 * Rankine-Hugoniot states (mem_shock_params.na, nb, nr).  Limits: degree 4,
 * ng <= 16, K <= 64, nbx ng <= 256, nbr ng K <= 1024.  Synchronous.
 * mem_solve, mem_flux_noalloc and the plain back-end are not available on
 * such a context (MEM_EINVAL). */
int mem_init_velocity(int degree, int nbx, int nbr, int ng, int K, double ax, double bx, double br,
                      mem_ctx **out);

/* Shape (nbx, nbr, ng, K) and default domain (a_x, b_x, b_r) of a
 * velocity-space context (host arrays of 4 and 3, either may be NULL);
 * MEM_EINVAL for a Gauss-Hermite context. */
int mem_velocity_rule(const mem_ctx *ctx, int32_t *shape, double *domain);

/* Release everything the context owns (synchronises the device first). */
void mem_destroy(mem_ctx *ctx);

/* Nodes per axis and total quadrature nodes of the context. */
int mem_quad_order(const mem_ctx *ctx);

/* Moment -> parameter map: Algorithm 1 (Section 3.2) on B independent cells.
 *   M      dev [B][35] moments in each cell's own gauge, M[0] = n > 0.
 *   beta   dev [B][35] in: warm start (entries 1..34; 0 = Maxwellian),
 *                      out: solution, beta[0] = n.
 *   status dev [B] int32 MEM_ST_* bits, or NULL.
 *   iters  dev [B] int32 passes of the Newton loop, or NULL.
 *   opts   host, NULL = defaults.
 * The objective, gradient and Hessian follow Appendix C (Eq. "MLE
 * optimization goal" and its Hessian); the partition function uses the
 * log-sum-exp form of Section 3.1.  The fused back-end needs no scratch
 * memory; the plain back-end uses the context's scratch (see below) and
 * synchronises the stream once per Newton pass.  No call allocates device
 * memory.  Returns MEM_EINVAL for B < 0 or NULL arrays with B > 0.
 *
 * Context scratch: mem_init / mem_init_velocity allocate one working buffer
 * per context (chunks of 65,536 cells; about 0.5 GB at quad_order 8, 0.8 GB
 * at 12, 60 MB for a velocity-space context).  The plain back-end, mem_flux /
 * mem_flux_axisym at quad orders other than 8 and 12, and the flux of a
 * velocity-space context use it.  Such calls on one context are ordered on
 * the GPU after one another through an event the context records, whatever
 * streams they are made on (calls from several host threads are serialised
 * by the context's lock); a call made on a stream that is being captured is
 * not ordered that way, so capture none of them while other streams use the
 * same context. */
int mem_solve(mem_ctx *ctx, const float *M, float *beta, int32_t *status, int32_t *iters,
              int64_t B, const mem_solve_opts *opts, void *stream);

/* mem_solve (Algorithm 1, Section 3.2) on arrays in host memory, for a batch
 * that starts and ends on the host:
 *   M_host      host [B][35] moments (pinned memory lets the copies overlap).
 *   beta_host   host [B][35] out: solution, beta[0] = n; in: warm start when
 *               warm != 0 (warm = 0 starts every cell from beta = 0, the
 *               Maxwellian of its gauge, without reading beta_host).
 *   status_host, iters_host  host [B] int32, or NULL.
 * The batch streams through the device in chunks of 262,144 cells staged in
 * the context's scratch: while the fused kernel solves one chunk on
 * `stream`, a copy stream owned by the call brings in the next and takes out
 * the previous one.  Results equal mem_solve's bit for bit.  Asynchronous:
 * the host arrays are complete once `stream` reaches the point of the call
 * (synchronise it before reading them, and keep them alive until then).
 * The fused back-end only (opts->impl MEM_IMPL_FUSED, quad_order 8 or 12);
 * MEM_EINVAL otherwise, on a velocity-space context, for NULL M_host /
 * beta_host, or when `stream` is being captured. */
int mem_solve_host(mem_ctx *ctx, const float *M_host, float *beta_host, int32_t *status_host,
                   int32_t *iters_host, int64_t B, int warm, const mem_solve_opts *opts, void *stream);

/* The paper's own system for axisymmetric flow on a velocity-space context
 * (Appendix B: the nine statistics psi_j of (u_x, u_r) of Eq. "Sufficient
 * 35" in orthonormal form, which are orthonormal combinations v_j of the 35
 * Hermite products; Algorithm 1 over their eight natural parameters; the
 * flux and the characteristic speed of the nine-moment system, Eq. "The lax
 * F").  Per cell, in one warp:
 *   M      dev [B][35] moments; only their projections M9_j = v_j . M are
 *          read (the axisymmetric part);
 *   beta   dev [B][35] in: warm start (projected likewise), out: the
 *          solution sum_j alpha_j v_j (other entries 0), beta[0] = n;
 *   gauge  dev [B][6], axisymmetric (w_y = w_z = 0, s_y = s_z);
 *   status, iters dev [B] or NULL (MEM_ST_* bits, passes);
 *   F      dev [B][35] or NULL: the flux of the nine moments, sum_j F9_j v_j;
 *   speed  dev [B] or NULL: spectral radius of the 9 x 9 pencil, clamped to
 *          the largest |u_x| of the nodes.
 * For an axisymmetric cell this is the 35-statistic solve of mem_solve_gauge
 * in exact arithmetic.  MEM_EINVAL on a Gauss-Hermite context or bad
 * arguments.  No scratch memory. */
int mem_solve_axi(mem_ctx *ctx, const float *M, float *beta, const float *gauge, int32_t *status, int32_t *iters,
                  float *F, float *speed, int64_t B, const mem_solve_opts *opts, void *stream);

/* Relative moment residual of B cells in FP64 on the GPU,
 *   res = || E_sigma[phi](beta) - M / n ||_2 / || M / n ||_2,
 * with sigma from the context's quadrature (Section 3.1, Eq. "Numerical
 * integration moments"; the stopping quantity of the acceptance bar).
 * Gauss-Hermite contexts only.  M, beta dev [B][35]; res dev [B] double
 * (written only for evaluated cells).  mask = 0 evaluates every cell;
 * otherwise only cells with (status[c] & mask) != 0 (status dev [B],
 * required then).  If status_out (dev [B], may alias status) is not NULL,
 * an evaluated cell whose residual is <= accept gets MEM_ST_FP64_OK or-ed
 * into it.  MEM_EINVAL on bad arguments or a velocity-space context. */
int mem_residual64(mem_ctx *ctx, const float *M, const float *beta, const int32_t *status, int32_t mask,
                   double *res, int32_t *status_out, double accept, int64_t B, void *stream);

/* mem_solve for any context, with the cells' gauges gauge dev [B][6]: a
 * velocity-space rule (mem_init_velocity) places its nodes in each cell
 * through the gauge; on a Gauss-Hermite context the gauge is not read and
 * the call is mem_solve.  The velocity-space solve runs one thread block per
 * cell (Algorithm 1 in FP32, no scratch); opts->impl is not read. */
int mem_solve_gauge(mem_ctx *ctx, const float *M, float *beta, const float *gauge, int32_t *status,
                    int32_t *iters, int64_t B, const mem_solve_opts *opts, void *stream);

/* Flux and characteristic speed of B cells (Eq. "The ME equation" subeq. 3
 * and Eq. "The lax F"):
 *   F[k] = n (w_x E[phi_k] + s_x E[ubar_x phi_k])          dev [B][35]
 *   speed = max_p |lambda_p(dF/dM)|                          dev [B]
 * The eigenvalues of dF/dM are the generalised eigenvalues of
 * (E[u_x phi phi^T], E[phi phi^T]) over all 35 statistics.  beta dev [B][35]
 * (beta[0] ignored, n taken from M[0]), M dev [B][35] (only M[0] is read),
 * gauge dev [B][6].  F or speed may be NULL.  At quad_order 8 and 12 the
 * fused kernel needs no scratch; other orders and velocity-space contexts
 * use the context scratch (see mem_solve). */
int mem_flux(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F,
             float *speed, int64_t B, void *stream);

/* mem_flux for axisymmetric cells: beta and the gauge symmetric under
 * u_y -> -u_y and under u_z -> -u_z (w_y = w_z = 0, beta_abc = 0 for odd b or
 * odd c), as every cell of a one-dimensional problem is.  Then E[phi phi^T]
 * and E[u_x phi phi^T] are block-diagonal over the parity classes of (b, c)
 * -- blocks of 14 (even, even; phi_0 included), 8 (odd, even), 8 (even, odd;
 * the same spectrum as (odd, even) by y <-> z) and 5 (odd, odd) statistics --
 * and the speed is the largest over the blocks (Eq. "The lax F" restricted to
 * the invariant subspaces).  The couplings between classes, which vanish for
 * an exactly symmetric cell, are not read.  Same arguments and results as
 * mem_flux; F is computed in full.  At quad_order 8 and 12 it uses no
 * scratch; other orders take mem_flux's full pencil (and its scratch). */
int mem_flux_axisym(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F,
                    float *speed, int64_t B, void *stream);

/* mem_flux without any allocation.  The paper has no counterpart: this is a
 * service of the library for callers that cannot allocate device memory when
 * they need fluxes -- for example a caller whose allocator already owns the
 * device budget, or a latency-critical loop that cannot afford cudaMalloc's
 * implicit synchronisation.  Same arguments and results as mem_flux.
 * Working memory is a fixed 12.5 MB array inside the library image (resident
 * on every GPU that loads the library until the process exits), so:
 *   - B <= 1024 cells per call and a context with quad_order <= 12; larger
 *     requests return MEM_EINVAL without doing anything;
 *   - the current device must be the context's device (else MEM_EINVAL);
 *   - velocity-space contexts are not supported (MEM_EINVAL): their rule has
 *     no shared node tables for this path to read;
 *   - the first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture;
 *   - that address is cached per device index for the life of the process and
 *     is valid only in the device's primary context: after cudaDeviceReset
 *     (or under another context on the same device) the library image is
 *     loaded again elsewhere, so do not call this entry point again in that
 *     process;
 *   - every call uses the same array: calls whose work overlaps on the GPU
 *     (different streams, or threads without ordering) race and give wrong
 *     results.  Each call writes everything it later reads, so the contents a
 *     previous call left behind never leak into a result.
 * No cudaMalloc, cudaFree or other allocating routine is called. */
int mem_flux_noalloc(mem_ctx *ctx, const float *M, const float *beta, const float *gauge, float *F,
                     float *speed, int64_t B, void *stream);

/* Hermite gauge (Eqs. "Hermite parameters", "Hermite parameters in moments")
 * and the change of gauge of Eq. "Change gauge M F":
 *   g_out = g_H(M_in, g_in); M_out = T(g_out, g_in) M_in;
 *   beta_inout (if not NULL) is carried to the new gauge.
 * axisym = 1: the 1D-shock form (w_y = w_z = 0, s_y = s_z = s_r,
 * s_r^2 = (<u_y^2> + <u_z^2>)/2); 0: each axis separately.  All dev arrays;
 * M_out may alias M_in and g_out may alias g_in. */
int mem_gauge_hermite(mem_ctx *ctx, const float *M_in, const float *g_in, float *g_out,
                      float *M_out, float *beta_inout, int64_t B, int axisym, void *stream);

/* Change of gauge M(g_to) = T(g_to, g_from) M(g_from) for B vectors (dev). */
int mem_gauge_transform(mem_ctx *ctx, const float *g_to, const float *g_from, const float *M_in,
                        float *M_out, int64_t B, void *stream);

/* Synthetic solve targets (workload generator; not part of the paper's
 * method): the moments, in each density's own Hermite gauge, of
 * p(c) ~ exp(-|c|^2/2 + sum a_k c^k - sum b_k c^k), c = (u - v)/sqrt(T),
 * n = 1, evaluated with a gen_order^3 Gauss-Hermite rule re-centred on the
 * density.  v dev [B][3], T dev [B], a dev [B][10] (degree-3 monomials in
 * statistic order), b dev [B][6] (c_x^4, c_y^4, c_z^4, c_x^2c_y^2,
 * c_x^2c_z^2, c_y^2c_z^2).  Outputs M_out dev [B][35], g_out dev [B][6]. */
int mem_targets(mem_ctx *ctx, int gen_order, const float *v, const float *T, const float *a,
                const float *b, float *M_out, float *g_out, int64_t B, void *stream);

/* ---------------------------------------------------------------------- */
/* 1D normal shock (Algorithm 2, Appendix D). */

typedef struct mem_shock mem_shock;

typedef struct {
    double mach;       /* upstream Mach number                              */
    int32_t ncells;    /* interior cells                                    */
    double xl, xr;     /* domain [xl, xr] in upstream mean free paths       */
    double cfl;        /* dt = cfl * dx / max speed (0.5)                   */
    double Pr;         /* Prandtl number of the ES-BGK model (2/3)          */
    double gamma;      /* heat-capacity ratio for Rankine-Hugoniot (5/3)    */
    double kn;         /* upstream Knudsen number (1)                       */
    int32_t ic;        /* 0: step at x = 0 between the RH Maxwellians;
                          1: tanh blend of Appendix D, Eq. "Mx ini", with
                          thickness parameter `thickness`                  */
    int32_t impl;      /* Newton back-end, MEM_IMPL_*                       */
    int32_t graph;     /* 1: capture the time step in a CUDA graph          */
    float tol;         /* Algorithm 1 tolerance (1e-8)                      */
    int32_t maxI;      /* Algorithm 1 iteration cap (500)                   */
    double na, nb, nr; /* velocity-space rule only: the problem's domain is
                          u_x in [min(v_+ - na c_+, v_- - na c_-),
                                  max(v_- + nb c_-, v_+ + nb c_+)],
                          u_r in [0, nr max(c_-, c_+)], c = sqrt(T) of the
                          Rankine-Hugoniot states (Appendix D; 5, 5, 5)   */
    int32_t scheme;    /* interface flux, MEM_SCHEME_* (LF).  LW and FLIC
                          solve Algorithm 1 once more per interface and step:
                          the Lax-Wendroff interface moments, moved to their
                          own Hermite gauge, cold start (beta = 0 there);
                          the flux is moved to each neighbour's gauge.
                          FLIC's van Leer limiter (flic_limiter) acts on
                          the paper's nine 1D statistics (orthonormal
                          combinations of the 35 products; the other
                          directions, zero for an axisymmetric flow, keep
                          the LF flux) in the updated cell's gauge (as every
                          quantity of cell n in the paper), which conserves
                          mass exactly but momentum and energy only to the
                          limiter's gauge dependence; r = 0 where its
                          denominator is 0, and the ghost cell stands in
                          for the cell before the first one.  An interface whose solve
                          fails (non-finite, lambda cap, bad input, maxI
                          passes) takes the LF flux.                      */
    double thickness;  /* ic = 1: thickness parameter T of Eq. "Mx ini"
                          (15.7, the paper's Mach-10 start)               */
    double t_end;      /* > 0: the step that would pass simulated time t_end
                          is cut to end there, and later steps leave the
                          problem as it is (dt = 0); 0: no limit          */
    int32_t stats;     /* velocity-space rule only: 35 (default) solves the
                          35-statistic system; 9 solves the paper's own
                          nine-statistic system for axisymmetric flow
                          (Appendix B, Eq. "Sufficient 35"; mem_solve_axi)
                          in every cell and interface, with its flux and
                          its characteristic speed.  The state stays the
                          35 moments; for an axisymmetric flow both give
                          the same solution up to rounding.  Must agree
                          across a batch.                                 */
    int32_t flic_limiter; /* FLIC only.  Eq. "The FLIC" prints the limiter
                          phi_{n-1/2} without a statistic index and its
                          ratio with the moments M_i.  0 (default): one
                          van Leer phi_j per statistic of the nine, ratios
                          in the updated cell's gauge; 1: one phi per
                          interface, the smallest phi_j, ratios in the
                          interface's Hermite gauge (both sides share it:
                          conservative in every moment); 2: the density's
                          phi for all.  phi scales the nine statistics'
                          components of F^LW - F^LF.                      */
} mem_shock_params;

void mem_shock_params_default(mem_shock_params *p);

/* Condition diagnostic of Section 4 (Fig. 7: the largest condition number of
 * the moment Jacobian dM/dbeta = n H, Eq. "moments vs parameter jacob", met
 * while a shock runs) for one problem of a shock on a velocity-space
 * context: the largest, over the problem's interior cells, of the ratio of
 * the largest to the smallest Cholesky pivot of each cell's last Newton
 * factorisation in the last step (a lower bound on cond(H), or on
 * cond(H + lambda I) where the modification was needed).  Synchronises the
 * device; host output.  MEM_EINVAL on a Gauss-Hermite context or a bad
 * problem index; 0 before the first step. */
int mem_shock_condition(mem_shock *s, int problem, double *max_cond);

/* Integration domain (a_x, b_x, b_r) that a shock problem with parameters *p
 * uses on a velocity-space context (Appendix D formula, see na, nb, nr
 * above); host array of 3.  MEM_EINVAL for invalid parameters. */
int mem_shock_domain(const mem_shock_params *p, double *domain);

/* Allocate the device state of one shock problem (ncells + 2 ghost cells),
 * set the initial condition and prime the characteristic speeds.
 * Synchronous.  Returns MEM_EINVAL / MEM_ENOMEM / MEM_ECUDA. */
int mem_shock_init(mem_ctx *ctx, const mem_shock_params *p, mem_shock **out);

/* A packed batch of nprob independent shock problems (an ensemble): their
 * cells are concatenated, every step advances all of them (one launch per
 * kernel, persistent Newton kernel), each with its own dt, Knudsen and
 * Prandtl numbers and boundary states.  impl, tol and maxI must agree across
 * the batch.  mem_shock_step's steady metric is then the largest over the
 * problems; mem_shock_get returns problem 0; mem_shock_get_problem any. */
int mem_shock_init_batch(mem_ctx *ctx, const mem_shock_params *ps, int nprob, mem_shock **out);
int mem_shock_num_problems(const mem_shock *s);
int mem_shock_get_problem(mem_shock *s, int problem, float *rho, float *ux, float *T, float *sxx, float *qx,
                          double *t_out, int32_t *steps_out);

/* Advance nsteps time steps of Algorithm 2 on `stream`:
 *   dt = cfl dx / max speed of the previous transport;
 *   Collision(dt/2) -> Transport(dt) [Newton, flux, neighbour gauge
 *   transform, local Lax-Friedrichs, finite volume] -> Collision(dt/2) ->
 *   Hermite gauge and transform of M and beta.
 * If steady_metric is not NULL it receives (host, after a stream
 * synchronisation) max_n |rho^{k+1} - rho^k| / (rho_+ - rho_-) of the last
 * step; with steady_metric NULL the call does not synchronise. */
int mem_shock_step(mem_shock *s, int nsteps, double *steady_metric, void *stream);

/* Copy the state to host: any pointer may be NULL.  M_host [(N+2)][35],
 * g_host [(N+2)][6], beta_host [(N+2)][35] include the two ghost cells;
 * rho, ux, T, sxx, qx [N] are the interior profiles (number density, mean
 * x-velocity, temperature, sigma_xx = P_xx - n T, heat flux q_x), t_out the
 * simulated time.  Synchronous. */
int mem_shock_get(mem_shock *s, float *M_host, float *g_host, float *beta_host, float *rho,
                  float *ux, float *T, float *sxx, float *qx, double *t_out);

/* Device pointers of the state (for zero-copy use from the caller). */
int mem_shock_device_state(mem_shock *s, float **M, float **beta, float **g, float **speed,
                           int32_t **status, int32_t **iters);

/* Copy the interface state of Lax-Wendroff / FLIC problems (Eq. "The lax W")
 * to host, packed like the cells of the batch (NT = sum of ncells + 2 over
 * the problems): entry c is the interface between cells c - 1 and c of one
 * problem, meaningful where that problem uses LW or FLIC and c is not its
 * left ghost cell (other entries hold scratch).  MI, betaI [NT][35] and
 * gI [NT][6]: the interface moments in their own Hermite gauge and their
 * parameters; FI [NT][35]: their flux in that gauge; status, iters [NT]:
 * the last interface solve (MEM_ST_* bits, Newton passes).  Any pointer may
 * be NULL.  Synchronous.  MEM_EINVAL for a batch without LW / FLIC
 * problems. */
int mem_shock_get_interfaces(mem_shock *s, float *MI, float *betaI, float *gI, float *FI, int32_t *status,
                             int32_t *iters);

void mem_shock_free(mem_shock *s);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of shock solves with device-resident state.
 * Not part of the paper's method; a service around Algorithm 2. */

typedef struct mem_server mem_server;

typedef struct {
    int32_t status;      /* MEM_OK when done, MEM_PENDING otherwise         */
    int32_t steps;       /* time steps taken                                */
    int32_t ncells;
    int32_t steady;      /* 1 if the steady-state test was met              */
    double sim_time;     /* simulated time                                  */
    double latency_s;    /* submit -> completion, host wall clock           */
} mem_shock_result;

/* Create a server.  Admitted problems share one packed batch on the device;
 * hbm_budget_bytes bounds the device memory of resident problems and
 * max_cells their total cells (ghosts included).  A problem completes when
 * max_n |rho^{k+1} - rho^k| / (rho_+ - rho_-) < steady_tol (after at least 2
 * steps) or after max_steps steps. */
int mem_serve_create(mem_ctx *ctx, size_t hbm_budget_bytes, int32_t max_cells, double steady_tol,
                     int32_t max_steps, mem_server **out);

/* Queue a request (host only, no device work).  The server uses the fused
 * Newton back-end with the paper's defaults for every request, and the
 * statistics system (mem_shock_params.stats) of its first request for all
 * of them.  Returns MEM_OK and *req_id, MEM_EINVAL for invalid parameters or
 * another statistics system, or MEM_EBUSY when the request alone exceeds
 * the memory or cell budget. */
int mem_serve_submit(mem_server *sv, const mem_shock_params *p, uint64_t *req_id);

/* Admit queued requests that fit, run `iters` time steps of every resident
 * problem on `stream`, then retire problems that completed (profiles copied
 * to the host) and admit more.  The time step of each packed batch is
 * captured in a CUDA graph after its first step and replayed until the
 * membership changes.  Synchronises the stream. */
int mem_serve_progress(mem_server *sv, int iters, void *stream);

/* Poll a request: MEM_OK (result filled; rho/ux/T, each ncells long, copied
 * if not NULL), MEM_PENDING (queued or running), or MEM_ENOTFOUND.  A
 * finished request has res->status MEM_OK, or a negative MEM_E* code if its
 * device state was lost when a batch rebuild failed (no profiles then). */
int mem_serve_poll(mem_server *sv, uint64_t req_id, mem_shock_result *res, float *rho, float *ux,
                   float *T);

/* Queue length, resident problems and cells, completed requests. */
int mem_serve_stats(mem_server *sv, int32_t *queued, int32_t *resident, int32_t *resident_cells,
                    int32_t *completed);

void mem_serve_destroy(mem_server *sv);

/* ---------------------------------------------------------------------- */
/* Autotuner of the launch shapes (no counterpart in the paper).  The
 * persistent warp-per-cell solve kernels run one cell per warp; their launch
 * shape -- warps per block (2, 4, 8) and the resident blocks per SM --
 * changes their speed but never a result. */

#define MEM_TUNE_FUSED 0 /* the fused Gauss-Hermite solve (mem_solve, fused)    */
#define MEM_TUNE_AXI 1   /* the nine-statistic velocity-space solve             */

typedef struct {
    int32_t n;                 /* candidates timed (the default first)          */
    int32_t warps[16];         /* warps per block of candidate i                */
    int32_t blocks_per_sm[16]; /* resident-block cap of candidate i (0: none)   */
    float ms[16];              /* best time of candidate i over the repetitions */
    int32_t best;              /* index of the candidate kept                   */
    float default_ms;          /* time of the default shape (4 warps, no cap)   */
} mem_tune_report;

/* Time every candidate launch shape of `kernel` on the caller's batch (M dev
 * [B][35], start parameters beta0 dev [B][35] (not modified), gauges dev
 * [B][6] for MEM_TUNE_AXI, else NULL; opts as mem_solve, NULL = defaults),
 * reps timed runs each after one warm-up, CUDA events on `stream`; keep the
 * fastest in the context (used by every later call) and report all of them.
 * The tuner allocates a [B][35] work array for the duration of the call:
 * call it at set-up.  MEM_EINVAL for a kernel the context has no form of. */
int mem_tune(mem_ctx *ctx, int kernel, const float *M, const float *beta0, const float *gauge, int64_t B, int reps,
             const mem_solve_opts *opts, mem_tune_report *out, void *stream);

/* Set or read the launch shape of `kernel` (a stored tuning result). */
int mem_set_launch(mem_ctx *ctx, int kernel, int warps, int blocks_per_sm);
int mem_get_launch(const mem_ctx *ctx, int kernel, int32_t *warps, int32_t *blocks_per_sm);

/* The tuning table on disk, a text file of lines
 *   device-name<TAB>rule<TAB>kernel<TAB>warps<TAB>blocks_per_sm
 * keyed by the GPU's name, the context's rule ("gh8", "gh12", or
 * "vel<nbx>x<nbr>x<ng>x<K>") and the kernel (MEM_TUNE_FUSED on Gauss-Hermite
 * contexts, MEM_TUNE_AXI on velocity-space ones).  mem_tune_save writes the
 * context's current shape for its kernel, replacing the line with the same
 * key (the file is rewritten through a temporary and a rename; MEM_EINVAL if
 * it cannot be written).  mem_tune_load applies the matching line
 * (MEM_ENOTFOUND if none, MEM_EINVAL if the file cannot be read).
 * mem_init and mem_init_velocity load the table named by the environment
 * variable MEM_TUNE_TABLE, when it is set, into every new context. */
int mem_tune_save(const mem_ctx *ctx, const char *path);
int mem_tune_load(mem_ctx *ctx, const char *path);

/* ---------------------------------------------------------------------- */
/* Measurement services (no counterpart in the paper): the rates the
 * roofline fractions of the library's kernels are quoted against. */

/* One timed micro-benchmark launch on the current device (synchronous; it
 * allocates and frees a few bytes of device memory):
 *   kind 0: FP32 FMA (work = flops), 1: MUFU ex2.approx (work = exp2
 *   evaluations), 2: tcgen05.mma kind::f16 with BF16 operands, 128 x 256 x 16
 *   per instruction (work = flops), 3: tcgen05.mma kind::tf32, 128 x 256 x 8.
 * iters (1 .. 2^24) scales the work; *seconds is the launch's CUDA-event
 * time.  MEM_EINVAL on bad arguments, MEM_ECUDA on a CUDA error or when the
 * tensor cores did not signal completion within the kernel's bounded wait. */
int mem_bench_peak(int kind, int64_t iters, double *seconds, double *work);

/* D = A B^T computed by one CTA's tensor cores (tcgen05.mma, operands in
 * shared memory in the library's K-major layout, accumulator in TMEM):
 * kind 1 BF16 operands, 2 TF32 operands, FP32 accumulation.  A_host
 * [128][64], B_host [N][64], D_host [128][N] row-major float host arrays;
 * N a multiple of 16 in 16..256.  Synchronous.  A check of the operand and
 * accumulator layouts that the tensor-core kernels rely on.  kind 3: TF32
 * operands brought in by TMA tensor loads (row-major global arrays, boxes of
 * 32 columns, 128-byte swizzle) and read through swizzled descriptors, the
 * path of the mixed back-end's contraction. */
int mem_tc_selftest(int kind, int N, const float *A_host, const float *B_host, float *D_host);

#ifdef __cplusplus
}
#endif

#endif /* MEM_GB300_H */
