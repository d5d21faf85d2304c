/*
 * reg.h -- C-ABI of the GB300 spectral semi-Lagrangian Gauss-Newton-Krylov
 * image-registration library (libreg.so).
 *
 * The method: Mang, Gholami, Biros, "Distributed-memory large deformation
 * diffeomorphic 3D image registration", SC16.  Given a template image rho_T
 * and a reference image rho_R on the periodic grid [0, 2 pi)^3, find the
 * stationary velocity v minimising
 *     J[v] = 1/2 ||rho(1) - rho_R||^2 + beta/2 <v, A v>            (Eq. varopt)
 * where rho is transported by v from rho(0) = rho_T, with div v = 0 in the
 * incompressible variant.  Every call below runs on one GPU, on the stream set
 * by reg_set_stream (default: the legacy default stream).
 *
 * Conventions (all entry points):
 *  - Grid: n1 x n2 x n3 points, x_j = 2 pi i_j / n_j, n = n1 n2 n3.  Scalar
 *    fields are C-contiguous float arrays [n1][n2][n3] (x3 fastest); vector
 *    fields are structure-of-arrays [3][n1][n2][n3].  Velocities are in
 *    physical units (domain length 2 pi, unit time).
 *  - Every float* / const float* argument is CALLER-OWNED DEVICE memory of the
 *    stated size, 16-byte aligned, unless the name ends in _host.  Inputs and
 *    outputs must not overlap unless a function says so.  The library never
 *    keeps a caller pointer after a call returns.
 *  - The library owns its workspaces (allocated once in reg_create), cuFFT
 *    plans and CUDA events; all are released by reg_destroy.
 *  - Return value: a reg_status.  No entry point aborts.  On an error the
 *    message is available from reg_last_error(ctx); the context stays
 *    destroyable.  A CUDA error inside a call is reported as REG_ECUDA and
 *    the context refuses further work (REG_ECUDA) except reg_destroy.
 *  - Scalars returned through double* are HOST pointers; such calls wait for
 *    the stream to finish that value.  Calls without host outputs are
 *    asynchronous on the stream.
 *  - A context is not thread-safe; use one context per host thread / stream.
 */
#ifndef REG_H
#define REG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reg_ctx reg_ctx;

typedef enum {
    REG_OK = 0,
    REG_EINVAL = 1,       /* bad argument (size, null pointer, alignment, kind) */
    REG_ENOMEM = 2,       /* device or host allocation failed */
    REG_ECUDA = 3,        /* CUDA runtime error (context is now unusable) */
    REG_ECUFFT = 4,       /* cuFFT plan or execution failure */
    REG_ENOTREADY = 5,    /* call order: e.g. a matvec before any gradient */
    REG_ENONFINITE = 6,   /* NaN/Inf in an objective, norm or inner product */
    REG_EMAXITER = 7,     /* iteration cap reached before the tolerance */
    REG_ENOTIMPL = 8
} reg_status;

/* Regularisation operator A(k) (Eq. varopt; Eq. gradient):
 *  REG_H2    A = |k|^4, the biharmonic from ||Lap v||^2 (the paper's choice);
 *  REG_H1    A = |k|^2, -Lap from ||grad v||^2;
 *  REG_H1DIV A = |k|^2 on the Leray-projected velocity (with div v = 0 a
 *            divergence penalty vanishes, so it acts as REG_H1). */
enum { REG_H1 = 1, REG_H2 = 2, REG_H1DIV = 3 };

/* Storage precision of the images.
 *  REG_FP32        everything FP32 (reductions FP64);
 *  REG_MIXED_BF16  rho_T and rho_R stored in bfloat16 (rounded once in
 *                  reg_set_images, widened where a step reads them);
 *                  every transported field, the grad rho cache,
 *                  interpolation and FFTs in FP32; reductions, the
 *                  objective and the stopping test in FP64. */
enum { REG_FP32 = 0, REG_MIXED_BF16 = 1 };

/* ---------------------------------------------------------------- context */

/* Create a registration context for an n1 x n2 x n3 grid with nt
 * semi-Lagrangian time steps (dt = 1/nt, Sec. III-B2), regularisation weight
 * beta > 0 and operator reg_kind; incompressible != 0 enforces div v = 0 by
 * the Leray projection (Eq. gradient).  Allocates every workspace on the
 * current CUDA device.  Sizes: 4 <= n_j, n <= 2^30, 1 <= nt <= 64.
 * On success *out owns the context; on failure *out is NULL. */
int reg_create(int n1, int n2, int n3, int nt, double beta, int reg_kind,
               int incompressible, reg_ctx** out);

/* Release every resource of ctx (NULL is accepted).  Always REG_OK. */
int reg_destroy(reg_ctx* ctx);

/* Message of the last failing call on ctx ("" if none); valid until the next
 * call on ctx.  With ctx == NULL: the last failure of reg_create on this
 * thread. */
const char* reg_last_error(const reg_ctx* ctx);

/* Name of a status code. */
const char* reg_status_string(int status);

/* Set the CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream()
 * .cuda_stream) for every later call; NULL = legacy default stream. */
int reg_set_stream(reg_ctx* ctx, void* stream);

/* Storage precision, REG_FP32 (default) or REG_MIXED_BF16.  Takes effect at
 * the next reg_set_images. */
int reg_set_precision(reg_ctx* ctx, int precision);

/* Copy the template rho_T and reference rho_R ([n], device) into the context.
 * presmooth != 0 applies the spectral Gaussian of one grid cell,
 * exp(-sum_j h_j^2 k_j^2 / 2), h_j = 2 pi / n_j (Sec. III-B1).  Invalidates the
 * linearisation point. */
int reg_set_images(reg_ctx* ctx, const float* rho_T, const float* rho_R,
                   int presmooth);

/* ----------------------------------------------- objective, gradient, H */

/* J[v] (Eq. varopt) for v [3n]: one forward state solve.  *J is host. */
int reg_objective(reg_ctx* ctx, const float* v, double* J);

/* Gradient g = beta A v + P b, b = int_0^1 lam grad rho dt (Eq. gradient;
 * P -> I when compressible), for v [3n] -> g [3n]; *J (host, may be NULL)
 * receives J[v].  Makes v the linearisation point of later Hessian matvecs:
 * caches the semi-Lagrangian points of v and -v (Sec. III-C2), the state
 * history rho(t_j) and its spectral gradients.  v and g may not overlap. */
int reg_gradient(reg_ctx* ctx, const float* v, float* g, double* J);

/* Hessian matvec Hvt = beta A vt + P b~ at the last reg_gradient's v
 * (Eq. hessian): Gauss-Newton by default (without the lambda terms,
 * b~ = int lam~ grad rho dt), full Newton after reg_set_hessian.
 * vt, Hvt [3n], may not overlap.  REG_ENOTREADY before any reg_gradient. */
int reg_hessian_matvec(reg_ctx* ctx, const float* vt, float* Hvt);

/* The gradient and the Hessian matvec in the solver's own representation
 * (Sec. III-B1: every field is a trigonometric polynomial): normalised
 * half-spectrum Fourier coefficients, f_hat = F f / n with f(x) =
 * sum_k f_hat(k) exp(i k.x), stored as interleaved complex pairs
 * [3][n1][n2][n3/2 + 1][2] floats (k1, k2 in FFT order, k3 = 0 .. n3/2).
 * beta A and P act on the coefficients exactly (diagonal products), so the
 * FP32 rounding of the FFTs is not amplified by beta |k|^4 in the result as
 * it is through the physical-space calls above.  The transports run on the
 * physical field C2R(v_hat).
 * reg_gradient_spectral: g_hat = beta A v_hat + P F(b) / n (Eq. gradient),
 * *J (host, may be NULL) = J[v]; makes v the linearisation point like
 * reg_gradient.  reg_hessian_matvec_spectral: Hvt_hat = beta A vt_hat +
 * P F(b~) / n at that point (Eq. hessian; REG_ENOTREADY before a gradient).
 * Inputs and outputs may not overlap; REG_ENOMEM if the solver's vectors
 * cannot be allocated. */
int reg_gradient_spectral(reg_ctx* ctx, const float* v_hat, float* g_hat, double* J);
int reg_hessian_matvec_spectral(reg_ctx* ctx, const float* vt_hat, float* Hvt_hat);

/* Which Hessian reg_hessian_matvec(_spectral) and reg_solve apply (Eq. hessian):
 *  REG_HESS_GAUSS_NEWTON (default) drops the two terms in lam, the paper's
 *      choice for its runs (Sec. IV-A3);
 *  REG_HESS_FULL_NEWTON keeps them: the incremental adjoint carries the
 *      source div(lam v~) (Eq. inc-adj), advanced like every source term by
 *      Eq. sml-advection, and b~ = int (lam~ grad rho + lam grad rho~) dt
 *      with spectral grad rho~ on every time level.  Allocates (nt + 1) n +
 *      nt n floats for the adjoint levels of the linearisation point and
 *      the incremental-state levels (REG_ENOMEM if that fails).  Far from a
 *      minimiser this Hessian can be indefinite; PCG then stops at the
 *      negative curvature (reg_solve_stats.negative_curvature).
 * Invalidates the linearisation point (the next reg_gradient keeps the
 * adjoint levels).  REG_EINVAL on another value. */
enum { REG_HESS_GAUSS_NEWTON = 0, REG_HESS_FULL_NEWTON = 1 };
int reg_set_hessian(reg_ctx* ctx, int hessian);

/* Spectral preconditioner z = F^-1[ M(k) P(k) F r ], M = 1/(beta A(k)) for
 * k != 0 and M(0) = 1/beta (Sec. III-A: the inverse regularisation
 * operator).  r, z [3n]; r == z (in place) is allowed. */
int reg_precond_apply(reg_ctx* ctx, const float* r, float* z);

/* ------------------------------------------------------------- solver */

typedef struct {
    double gtol;          /* stop when ||g|| <= gtol ||g_0||            (1e-2) */
    int max_gn;           /* Gauss-Newton iteration cap                   (50) */
    int max_pcg;          /* PCG iterations per Newton step              (500) */
    int forcing;          /* 0: eta = min(0.5, ||g||/||g0||) (quadratic)
                             1: eta = min(0.5, sqrt(||g||/||g0||))         (0) */
    double armijo_c;      /* sufficient-decrease constant               (1e-4) */
    double armijo_shrink; /* step reduction factor                       (0.5) */
    int armijo_max;       /* line-search trials                           (10) */
    int use_graph;        /* 2: the whole PCG solve is one CUDA graph with a
                             device-side while-loop (stopping tests on the
                             GPU, one host wait per Newton step); 1: one
                             graph per PCG iteration, tests on the host;
                             0: plain launches.  2 falls back to 1 when
                             phase timing is on or the driver refuses the
                             conditional node.  The two-level
                             preconditioner's coarse PCG loops take the
                             same form                                   (2) */
    int verbose;          /* print one line per Newton iteration to stderr (0) */
    double gnorm_ref;     /* > 0: use it as ||g_0|| in the stop test and the
                             forcing term, e.g. the gradient norm at v = 0
                             when v_inout holds a prediction; < 0: use the
                             gradient norm at v = 0, from its closed form
                             P[(rho_R - rho_T) grad rho_T] (one spectral
                             gradient); 0: ||g|| at the initial guess    (0) */
    double precond_shift; /* >= 0: PCG preconditioner M = 1/(beta A + shift);
                             0 is the paper's inverse regularisation
                             operator (Sec. III-A)                       (0) */
    double beta_start;    /* > the context's beta: parameter continuation on
                             beta (Sec. III-A): Gauss-Newton solves at
                             beta_start, beta_start / beta_factor, ...
                             down to the context's beta, each from the
                             last one's velocity, every stage stopped at
                             ||g|| <= gtol ||g_0|| with ||g_0|| of the first
                             stage (at v = 0 independent of beta); 0 or
                             <= beta: one solve at the context's beta     (0) */
    double beta_factor;   /* continuation divisor per stage, > 1          (10) */
    int coarse_factor;    /* >= 2: the two-level preconditioner
                             M^-1 r = Pi_L H_c^-1 Pi_L r
                                      + (beta A)^-1 P (I - Pi_L) r
                             with H_c the Gauss-Newton Hessian on the grid
                             n_j / coarse_factor (images restricted to the
                             modes L = {|k_j| < n_j / (2 coarse_factor)},
                             linearised at the restricted v every Newton
                             step), inverted by PCG to coarse_tol; the
                             Newton steps then by flexible PCG.  Sec. I
                             names multilevel preconditioning as the
                             remedy for the beta dependence of (beta A)^-1
                             (Table 5).  Each n_j / coarse_factor must be
                             an integer >= 8.  0 or 1: off               (0) */
    double coarse_tol;    /* inner PCG relative residual tolerance       (0.2) */
    int coarse_max;       /* inner PCG iteration cap                      (12) */
    int coarse_nt;        /* semi-Lagrangian steps of the coarse Hessian,
                             1..64; 0: the context's nt. On a coarse grid
                             n/4 a point moves a quarter of the cells per
                             step: half the fine nt measured faster at the
                             same outer iteration counts (256^3, nt = 8:
                             4 instead of 8)                              (0) */
} reg_solve_opts;

typedef struct {
    int gn_iters, pcg_iters, matvecs, objective_evals, gradient_evals;
    int line_search_failed;   /* 1 if Armijo found no acceptable step */
    int negative_curvature;   /* PCG steps stopped by p.Hp <= 0 */
    double J0, J, gnorm0, gnorm, gnorm_rel, mismatch_rel;
    double ms_total;          /* wall time of the solve (host clock) */
    int stages;               /* continuation stages run (1 without) */
    int coarse_matvecs;       /* coarse-grid Hessian matvecs (two-level) */
} reg_solve_stats;

/* Set the regularisation weight beta > 0 (e.g. between the stages of a
 * hand-made continuation).  The linearisation point stays valid (the
 * transports do not depend on beta).  REG_EINVAL unless beta is finite and
 * positive. */
int reg_set_beta(reg_ctx* ctx, double beta);

/* The two-level preconditioner of reg_solve_opts.coarse_factor, applied
 * alone (normalised half-spectrum coefficients, as for
 * reg_gradient_spectral).  reg_twolevel_setup creates the coarse grid's
 * context (n_j / coarse_factor; once per factor), restricts the images to
 * it, and linearises its Gauss-Newton Hessian at the restriction of v_hat.
 * reg_twolevel_apply: z_hat = M^-1 r_hat with the inner PCG stopped at
 * ||r_c|| <= inner_tol ||r_c,0|| or after inner_max iterations
 * (inner_tol = 0: exactly inner_max unless it converges or meets negative
 * curvature); *inner_iters (may be NULL) receives the count.  REG_ENOTREADY
 * before a setup. */
int reg_twolevel_setup(reg_ctx* ctx, int coarse_factor, const float* v_hat);
/* The same with the coarse Hessian's number of time steps (0: the context's). */
int reg_twolevel_setup_nt(reg_ctx* ctx, int coarse_factor, int coarse_nt, const float* v_hat);
int reg_twolevel_apply(reg_ctx* ctx, const float* r_hat, float* z_hat, double inner_tol,
                       int inner_max, int* inner_iters);

/* Fill *opts with the defaults listed above. */
int reg_solve_opts_default(reg_solve_opts* opts);

/* Inexact Gauss-Newton-Krylov solve with Armijo line search (Sec. III-A):
 * v_inout [3n] is the initial guess on entry (zero, or a learned prediction)
 * and the solution on exit.  opts NULL = defaults; stats may be NULL.
 * Returns REG_OK when ||g|| <= gtol ||g_0||, REG_EMAXITER when max_gn was
 * reached first (v_inout then holds the last accepted iterate).  With
 * continuation (opts->beta_start) the counts of stats add up over the stages,
 * J0 is the first stage's and J, gnorm, gnorm_rel, mismatch_rel the last
 * one's; the context's beta is the target throughout and afterwards. */
int reg_solve(reg_ctx* ctx, float* v_inout, const reg_solve_opts* opts,
              reg_solve_stats* stats);

/* The same solve through HOST buffers: uploads rho_T_host, rho_R_host ([n]
 * each, host memory; pinned memory makes the copies faster) and
 * v_host_inout [3n], solves, and downloads v into v_host_inout. */
int reg_solve_host(reg_ctx* ctx, const float* rho_T_host, const float* rho_R_host,
                   int presmooth, float* v_host_inout, const reg_solve_opts* opts,
                   reg_solve_stats* stats);

/* ------------------------------------------- steps of the path, one each */

/* RK2 semi-Lagrangian points (Eq. sml-trajectory) of v [3n] and of -v, as
 * displacements X - x in GRID units: d_fwd, d_adj [3n]. */
int reg_departure(reg_ctx* ctx, const float* v, float* d_fwd, float* d_adj);

/* Tricubic Lagrange interpolation (Sec. III-C2) of nfields (1..3) scalar
 * fields field [nfields][n] at the points x + disp (disp [3n], grid units,
 * any magnitude; periodic wrap) -> out [nfields][n].  The 64 weights of a
 * point are shared by its fields. */
int reg_interp(reg_ctx* ctx, const float* field, int nfields, const float* disp,
               float* out);

/* Forward state transport (Eq. varopt:state): rho_hist [(nt+1)][n] receives
 * rho(t_0) = rho0, ..., rho(t_nt), stepping with the points d_fwd [3n]. */
int reg_state_transport(reg_ctx* ctx, const float* rho0, const float* d_fwd,
                        float* rho_hist);

/* The forward state transport of reg_state_transport, for callers that
 * cannot allocate device memory (code inside another library's callback
 * that must not touch the allocator, on a fixed memory pool that must not
 * grow, or in a loop where a possibly synchronising cudaMalloc is not
 * acceptable).  The paper
 * has no counterpart: it is a property of this library's interface only.
 * No context: grid n1 x n2 x n3 (n <= 2^22 points, else REG_EINVAL), nt
 * steps (1..64) with the points d_fwd [3n]; rho0 [n] -> rho1 [n] = rho(t_nt)
 * (only the last level; rho0 == rho1 is refused; d_fwd must not overlap
 * rho1).  Launched on `stream` (a cudaStream_t, NULL = legacy default);
 * asynchronous.  No cudaMalloc/cudaFree or allocating library call: the one
 * intermediate level lives in a fixed 16 MiB static device array that every
 * GPU loading the library keeps until exit.  The first call on a device
 * looks up that array's address (cudaGetSymbolAddress) with the device
 * current, so make the first call on each device before any stream capture;
 * a failed lookup returns REG_ECUDA, is not cached, and is retried by the
 * next call.  The tensors must be on the current device.
 * All calls share the array: calls whose GPU work overlaps (other streams,
 * other threads) race on it; serialise them.  Every element of the array is
 * written before it is read within a call.  REG_ECUDA on a launch or
 * set-up failure. */
int reg_state_transport_noalloc(int n1, int n2, int n3, int nt, const float* rho0,
                                const float* d_fwd, float* rho1, void* stream);

/* Spectral first derivatives (Sec. III-B1): grad [3n] = grad f (f [n]);
 * div [n] = div v (v [3n]).  Odd derivatives zero the Nyquist mode.  Input
 * and output must not overlap (REG_EINVAL). */
int reg_spectral_grad(reg_ctx* ctx, const float* f, float* grad);
int reg_spectral_div(reg_ctx* ctx, const float* v, float* div);

/* Leray projection pv = (I - grad Lap^-1 div) v (Eq. gradient); in place ok. */
int reg_leray(reg_ctx* ctx, const float* v, float* pv);

/* av = beta A v for the context's operator (Eq. gradient); in place ok. */
int reg_apply_regularisation(reg_ctx* ctx, const float* v, float* av);

/* Spectral Gaussian exp(-sum_j (s_j k_j)^2 / 2) of f [n] -> out [n]
 * (s_j physical units; Sec. III-B1); in place ok. */
int reg_gaussian_smooth(reg_ctx* ctx, const float* f, float* out,
                        double s1, double s2, double s3);

/* Discrete L2 inner product <a, b>_h = (2 pi)^3 / n * sum_i a_i b_i over
 * count floats (count a multiple of n: scalar or vector fields), accumulated
 * in FP64 (the Krylov inner products of Sec. III-A).  *out is host. */
int reg_inner(reg_ctx* ctx, const float* a, const float* b, size_t count,
              double* out);

/* ---------------------------------------------------- deformation check */

/* Displacement u = y(x, 1) - x of the deformation map of v [3n]: y solves
 * d_t y + v . grad y = 0, y(0) = x (Sec. II-A), so u solves
 * d_t u + v . grad u = -v, u(0) = 0, advanced by the context's nt
 * semi-Lagrangian steps with the source -v (Eq. sml-advection) on the
 * forward points of v.  u: device [3n], not overlapping v.  Overwrites the
 * context's points, so a reg_hessian_matvec needs a new reg_gradient. */
int reg_deformation(reg_ctx* ctx, const float* v, float* u);

/* det(grad y) = det(I + grad u) [n] with spectral derivatives; close to 1
 * everywhere for a divergence-free v (the incompressible check).  Needs
 * nt >= 2 (it borrows the grad rho cache, and a reg_hessian_matvec then
 * needs a new reg_gradient). */
int reg_jacobian_det(reg_ctx* ctx, const float* u, float* det);

/* ------------------------------------------------------------- tuning */

/* Tile of the interpolation kernels: each thread walks k points (a multiple
 * of 4 in 4..64, or 1 or 2 with k wy >= 4) along x1 and a block is 32 x wy
 * threads (wy in 1, 2, 4, 8, 16) over (x3, x2).  wy = 16 runs only the
 * shared-memory staged kernel (max displacement up to 3 cells; beyond that
 * the call uses wy = 8); k = 1, 2 (more warps for small grids) likewise, the
 * register-window kernel taking k = 4 then.  The default is k = 8, wy = 8.
 * Results do not depend on the tile. */
int reg_set_tile(reg_ctx* ctx, int k, int wy);
int reg_get_tile(const reg_ctx* ctx, int* k, int* wy);

/* Small grids (at most 2^18 points: the two-level preconditioner's coarse
 * grid): on = 1 runs the transports of each PCG matvec -- the
 * incremental state, the incremental adjoint with the time integral and the
 * partial sums of <p, b~> -- as ONE persistent cooperative launch with
 * grid-wide barriers between the time steps (bounded waits; a wait that
 * gives up makes <p, b~> NaN, which PCG reports as REG_ENONFINITE); on = 0
 * launches the 2 nt + 1 steps one by one (default: on a 64^3 coarse grid
 * with nt = 4 the separate launches, with the autotuned small tiles, took
 * 0.18 ms per matvec against 0.27 ms for the persistent launch).  Same
 * arithmetic up to the order of the FP32 stencil sums.  Contexts of a batch
 * use 0 (their PCG loops run side by side). */
int reg_set_persistent(reg_ctx* ctx, int on);

/* Host-side fault injection, for tests of the error paths (no GPU fault is
 * involved).  Arms one process-wide injection that fires once, at the
 * (after + 1)-th matching event, and then disarms:
 *  REG_INJECT_ALLOC       a device allocation of reg_create fails as if
 *                         cudaMalloc had: reg_create frees what it holds and
 *                         returns REG_ENOMEM with *out = NULL;
 *  REG_INJECT_CUFFT_PLAN  a cuFFT plan of reg_create fails: REG_ECUFFT;
 *  REG_INJECT_NAN_IMAGE   the next reg_set_images writes a NaN into rho_T
 *                         (in every stored copy) after its copies, so the
 *                         next objective or gradient returns REG_ENONFINITE
 *                         and the context stays usable;
 *  REG_INJECT_STAGE_TIMEOUT  the next launch of a staged interpolation
 *                         or departure-point kernel that stages its box(es)
 *                         by TMA issues no copy and waits for it at most
 *                         ~1e-4 s of SM
 *                         clock (instead of ~1 s): every block's bounded
 *                         mbarrier wait runs out, the block writes NaN for
 *                         its points (nothing is in flight), and the call
 *                         that launched it reports REG_ENONFINITE; the
 *                         context stays usable (after must be 0);
 *  REG_INJECT_NONE        disarm.
 * REG_EINVAL on an unknown kind or after < 0. */
enum { REG_INJECT_NONE = 0, REG_INJECT_ALLOC = 1, REG_INJECT_CUFFT_PLAN = 2,
       REG_INJECT_NAN_IMAGE = 3, REG_INJECT_STAGE_TIMEOUT = 4 };
int reg_debug_inject(int what, int after);

/* How the staged interpolation kernels fill their shared-memory box.
 * tma = 1 (default): one TMA tensor copy per block (cp.async.bulk.tensor,
 * completion on an mbarrier) wherever x3 is a multiple of 4 and the grid is
 * at least one box large (n3 >= 64, n2 >= wy + 3 + 2h, n1 >= k + 3 + 2h for
 * halo h); blocks at a face of the periodic domain reload the elements outside
 * the grid from their periodic images.  Elsewhere, and with tma = 0, every
 * thread issues 4-byte cp.async copies.  The departure points likewise: one
 * 4-D tensor copy of the three velocity components' boxes per block (n3 >=
 * 64, n2 >= 11 + 2h, n1 >= 7 + 2h), else the per-thread copies.  The box
 * content, and so every result, is the same either way.  REG_EINVAL unless
 * tma is 0 or 1. */
int reg_set_staging(reg_ctx* ctx, int tma);

/* Autotuner: time the interpolation kernels of the current linearisation
 * point (reg_gradient first, else REG_ENOTREADY) for a few tile shapes and
 * keep the fastest in ctx; the choice is cached per (grid, halo) for the
 * process.  *k, *wy (may be NULL) receive the chosen tile. */
int reg_autotune(reg_ctx* ctx, int* k, int* wy);

/* ------------------------------------------------------------- batch */

/* Independent registrations of image pairs of uneven sizes solved together
 * (one GPU).  Pair i has grid dims[3i..3i+2]; all share nt, beta, reg_kind,
 * incompressible and precision (REG_FP32 / REG_MIXED_BF16).  Each pair gets
 * its own context (cuFFT plans of its size) and non-blocking stream.
 * Modes (reg_batch_set_mode):
 *  REG_BATCH_ONE_GRAPH (default): the pairs take their Newton steps in
 *      lockstep.  Gradients and line searches run on host worker threads,
 *      each pair on its stream; the PCG solves of one Newton step of every
 *      pair still iterating are ONE CUDA graph, a device-controlled
 *      while-loop per pair side by side, each with its pair's scalars on the
 *      device and its own stopping test (a pair whose test is met stops
 *      while the others go on).  The graph is kept across steps and calls
 *      while the pairs' captured kernels stay the same.  Plain solver
 *      options only (no continuation, no two-level preconditioner:
 *      REG_EINVAL).
 *  REG_BATCH_THREADS: worker threads take whole solves largest first and run
 *      them concurrently, each with its own per-step PCG graph. */
enum { REG_BATCH_ONE_GRAPH = 0, REG_BATCH_THREADS = 1 };
typedef struct reg_batch reg_batch;
int reg_batch_create(int npairs, const int* dims, int nt, double beta, int reg_kind,
                     int incompressible, int precision, reg_batch** out);
int reg_batch_destroy(reg_batch* batch);
int reg_batch_set_mode(reg_batch* batch, int mode);
/* PCG graphs launched by the last reg_batch_solve in REG_BATCH_ONE_GRAPH
 * mode (one per lockstep Newton step with a pair still iterating). */
int reg_batch_graphs_launched(const reg_batch* batch, int* count);

/* Solve every pair: v_inout[i] (device, [3 n_i]) is pair i's initial guess
 * and solution, rho_T[i], rho_R[i] its images (device, [n_i]).  autotune != 0
 * runs reg_autotune on each pair first (cached per grid size).  Per pair
 * (arrays of npairs, each may be NULL): stats, latency_ms (the pair's service
 * time: from the start of its work -- the call's start in lockstep mode,
 * its dequeue in threads mode -- until its stopping test), status_out
 * (REG_OK / REG_EMAXITER / error).  Returns the first hard error, else
 * REG_OK. */
int reg_batch_solve(reg_batch* batch, float* const* v_inout, const float* const* rho_T,
                    const float* const* rho_R, int presmooth, int autotune,
                    const reg_solve_opts* opts, reg_solve_stats* stats, double* latency_ms,
                    int* status_out);

/* ------------------------------------------------- spectral resampling */

/* Trigonometric (Fourier) resampling of ncomp scalar fields from the grid
 * nin[0] x nin[1] x nin[2] to nout[0] x nout[1] x nout[2] (Sec. III-B1: fields
 * are represented by their Fourier series on the periodic grid).  The
 * coefficients with |k_j| < min(nin_j, nout_j) / 2 in every direction are
 * kept, the rest (including the Nyquist planes) are zero, so a field
 * band-limited to those modes is reproduced exactly at the new grid points.
 * in: device [ncomp][nin], out: device [ncomp][nout], not overlapping.  The
 * library caches cuFFT plans and a workspace per (sizes, ncomp) (process-wide,
 * guarded by a mutex); calls with the same sizes share that workspace, so
 * the caller orders them (one stream).  Asynchronous on `stream`. */
int reg_spectral_resample(const int* nin, const int* nout, int ncomp, const float* in,
                          float* out, void* stream);

/* ------------------------------------------ learned initial velocity */

/* A 3-D U-Net that maps the image pair (rho_T, rho_R), resampled to an R^3
 * grid, to an initial velocity [cout][R^3] for reg_solve.  No counterpart in
 * the paper, whose Gauss-Newton iteration starts from v = 0 (Sec. III-A); the
 * solve that follows is unchanged and runs to its own stopping test.
 *
 * Architecture, levels L (1..6), channels ch[0..L-1] (1..128):
 *   encoder level l:  conv3x3x3 -> ReLU -> conv3x3x3 -> ReLU = skip_l,
 *                     then 2x average pooling for l < L-1;
 *   decoder level l = L-2 .. 0: 2x nearest upsampling, concatenation
 *                     [upsampled, skip_l], conv3 -> ReLU -> conv3 -> ReLU;
 *   head: 1x1x1 conv to cout channels.  Zero padding.
 * Parameters: one flat FP32 array, per layer in the order enc0.0, enc0.1,
 * ..., enc(L-1).1, dec(L-2).0, dec(L-2).1, ..., dec0.1, head, each as the
 * weights [kz][ky][kx][cin][cout] followed by the bias [cout].
 * Arithmetic: BF16 weights and activations on the tensor cores with FP32
 * accumulation; FP32 master weights, gradients and Adam moments; FP64 loss.
 * Tensors: x is device [cin][R^3] (each channel [R][R][R], last index
 * fastest), the prediction and the target are device [cout][R^3].
 * Limits: cin, cout <= 128, R^3 <= 65535 * 64 (R <= 161). */
typedef struct reg_unet reg_unet;

/* R divisible by 2^(L-1), R >= 8; parameters zero until reg_unet_set_params. */
int reg_unet_create(int R, int levels, const int* ch, int cin, int cout, reg_unet** out);
int reg_unet_destroy(reg_unet* net);
const char* reg_unet_last_error(const reg_unet* net);
int reg_unet_set_stream(reg_unet* net, void* stream);
/* Tensor-core path of the forward 3x3x3 convolutions.  tcgen05 = 1 (default):
 * where Co is 16, 32, 64 or 128 and Ci a multiple of 8, a 128-voxel x Co tile
 * per CTA on tcgen05.mma (BF16 operands in shared memory, FP32 accumulator in
 * tensor memory); tcgen05 = 0, and every other layer and every gradient: the
 * warp-level wmma path.  Same inputs and rounding of the operands; the FP32
 * sums may differ in order.  REG_EINVAL unless tcgen05 is 0 or 1. */
int reg_unet_set_mma(reg_unet* net, int tcgen05);
int reg_unet_param_count(const reg_unet* net, size_t* count);
/* Host arrays of reg_unet_param_count floats.  set_params also zeroes the
 * Adam moments and step count.  Both wait for the stream. */
int reg_unet_set_params(reg_unet* net, const float* params_host);
int reg_unet_get_params(reg_unet* net, float* params_host);
/* y = net(x), asynchronous. */
int reg_unet_forward(reg_unet* net, const float* x, float* y);
/* Mean-squared-error loss against target (host *loss if not NULL) and its
 * gradient with respect to every parameter (host grad_host if not NULL). */
int reg_unet_gradient(reg_unet* net, const float* x, const float* target, double* loss,
                      float* grad_host);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the loss of one sample;
 * *loss (host, if not NULL) is the loss before the step. */
int reg_unet_train_step(reg_unet* net, const float* x, const float* target, float lr,
                        double* loss);

/* ------------------------------------------------------------- timing */

enum {
    REG_PH_DEPARTURE = 0,  /* semi-Lagrangian points */
    REG_PH_STATE = 1,      /* forward state steps */
    REG_PH_ADJOINT = 2,    /* adjoint steps + b accumulation */
    REG_PH_INCSTATE = 3,   /* incremental state steps */
    REG_PH_INCADJ = 4,     /* incremental adjoint steps + b~ accumulation */
    REG_PH_INTERP = 5,     /* stand-alone interpolation (reg_interp) */
    REG_PH_FFT = 6,        /* cuFFT executions */
    REG_PH_SPECTRAL = 7,   /* spectral multiplier kernels */
    REG_PH_BLAS = 8,       /* reductions and vector updates */
    REG_PH_OTHER = 9,      /* pointwise set-up kernels */
    REG_PH_DERIV = 10,     /* spectral first derivatives by 1-D FFT kernels */
    REG_NPHASES = 11
};

typedef struct {
    double ms[REG_NPHASES];         /* summed device time (CUDA events) */
    long long launches[REG_NPHASES];
    double bytes[REG_NPHASES];      /* algorithmic HBM bytes of those launches */
} reg_timing;

/* on != 0: bracket every kernel / FFT launch with CUDA events on the
 * context's stream and accumulate per phase; on == 0 stops.  Resets the
 * counters. */
int reg_set_timing(reg_ctx* ctx, int on);

/* Synchronise the stream and return the accumulated per-phase figures. */
int reg_get_timing(reg_ctx* ctx, reg_timing* out);

/* The same figures for the coarse grid of the two-level preconditioner
 * (its context follows reg_set_timing of ctx); zeros without one. */
int reg_get_coarse_timing(reg_ctx* ctx, reg_timing* out);

/* The interpolation tile (k, wy) of the two-level preconditioner's coarse
 * grid.  By default (k = wy = 0) it is autotuned (reg_autotune) each time the
 * coarse grid is linearised; a tile that reg_set_tile accepts is used as
 * given instead (for instance to keep a profiler's launch sequence that of
 * a plain run, whose autotuning the profiler's per-launch overhead would
 * distort).  REG_EINVAL for other values.  Takes effect at the next
 * linearisation. */
int reg_set_coarse_tile(reg_ctx* ctx, int k, int wy);

/* Process-wide: on = 1 (default) launches the staged interpolation steps,
 * the incremental-state start and the PCG update, direction and loop-control
 * kernels with programmatic stream serialisation, so that each may be
 * scheduled while its predecessor on the stream finishes (it waits on the
 * device for the predecessor's results before touching memory).  on = 0:
 * ordinary launches.  Same results either way.  Applies to launches and
 * graph captures made after the call; REG_EINVAL for other values. */
int reg_set_dependent_launch(int on);

/* The tile the coarse grid runs with now; 0, 0 without a coarse grid. */
int reg_get_coarse_tile(const reg_ctx* ctx, int* k, int* wy);

#ifdef __cplusplus
}
#endif

#endif /* REG_H */
