// Inexact Gauss-Newton-Krylov solve (Sec. III-A, Sec. IV-A3): PCG on
// H s = -g with the inverse-regularisation preconditioner, forcing tied to
// the relative gradient norm, Armijo backtracking on J, stop at
// ||g|| <= gtol ||g_0||.
//
// The iterate v and the Krylov vectors (g, s, r, p) are kept as normalised
// Fourier coefficients (FP32 complex, half spectrum).  The regularisation
// beta A grows like beta |k|^4 (about 2e6 at 256^3 with beta = 1e-3): applied
// to an FP32 field stored in physical space it multiplies the rounding noise
// that storage puts into every mode, and the gradient stalls at that noise
// (near 2 % of ||beta A v|| at 256^3).  On coefficients, rounding is relative
// to each coefficient and beta A, M and P are exact diagonal multiplications.
// Per PCG iteration the matvec needs p in physical space (one C2R of three
// fields) for the transports and b~ in Fourier space (one R2C); every inner
// product is taken by Parseval in FP64.  The scalars live in device memory:
// one iteration is a fixed launch sequence.  use_graph = 2 (default): the
// whole PCG solve is one CUDA graph, the iteration's launches as the body of
// a conditional while-node whose condition a one-thread kernel sets from the
// device scalars (curvature, residual, finiteness, iteration cap), so the
// host waits once per Newton step.  use_graph = 1: the iteration is a graph
// replayed by the host, which reads p.Hp and ||r|| after each one.
// use_graph = 0: plain launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <thread>
#include <utility>
#include <vector>

#include "ctx.h"

namespace reg {

static const double kTwoPi3 = 248.05021344239856;   // (2 pi)^3

// real vectors
enum { R_V = 0, R_P = 1, R_HOST = 2 };
// spectral vectors
enum { S_V = 0, S_VT = 1, S_G = 2, S_S = 3, S_R = 4, S_P = 5, S_PC = 6, S_Z = 7, S_Q = 8 };

static int finalize_to(reg_ctx* c, int t, int nb, double scale, int slot) {
    if ((long long)(t + 1) * nb > c->npartials)
        return fail(c, REG_EINVAL, "partial-sum slot out of range");
    Phase ph(c, REG_PH_BLAS, 0.0);
    REG_CK(c, launch_finalize(c->partials + (long long)t * nb, nb, scale, c->dsc + slot,
                              c->stream));
    return REG_OK;
}

// Physical-space copy of a spectral vector (C2R destroys its input, so the
// coefficients go through spec[0]).
static int to_physical(reg_ctx* c, const float2* xh, float* x) {
    REG_CK(c, cudaMemcpyAsync(c->spec[0], xh, sizeof(float2) * 3 * (size_t)c->g.nc,
                              cudaMemcpyDeviceToDevice, c->stream));
    return op_fft_c2r(c, c->spec[0], x, 3);
}

// One PCG iteration from p (p_hat, its C2R copy pc): q = beta A p + P b~(p),
// PQ = <p, q> = <p, beta A p> + <p, b~>; s += a p, r -= a q (a = RZ / PQ,
// skipped when PQ <= 0); RR = ||P r||^2, RZNEW = <r, M P r>;
// p = M P r + (RZNEW / RZ) p with <p, beta A p> for the next PQ; RZ = RZNEW.
static int pcg_iteration(reg_ctx* c) {
    const int nb = blas_blocks();
    const int proj = c->incompressible;
    float2** S = c->ss;
    float* p = c->sv[R_P];
    REG_TRY(op_fft_c2r(c, S[S_PC], p, 3));
    REG_TRY(op_matvec_transport(c, p, p, SC_PB));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    // the reductions finish inside their kernels (Fin): RR and RZNEW in the
    // update, PAP and then RZ = RZNEW in the direction
    {
        const Fin fin = finish_into(c, kTwoPi3, SC_RR, SC_RZNEW);
        Phase ph(c, REG_PH_SPECTRAL, 6.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_update(c->g, S[S_S], S[S_R], S[S_P], c->spec[1], c->dsc, SC_RZ, SC_PAP,
                                   SC_PB, SC_PQ, c->beta, c->pshift, c->kind, proj, c->partials,
                                   nb, c->stream, &fin));
    }
    {
        const Fin fin = finish_into(c, kTwoPi3, SC_PAP, 0, SC_RZNEW, SC_RZ);
        Phase ph(c, REG_PH_SPECTRAL, 4.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_direction(c->g, S[S_R], S[S_P], S[S_PC], c->dsc, SC_RZNEW, SC_RZ, 0,
                                      c->beta, c->pshift, c->kind, proj, c->partials, nb,
                                      c->stream, &fin));
    }
    return REG_OK;
}

struct PcgResult { int iters; bool neg_curv; bool converged; };

enum { PCG_RUN = 0, PCG_CONVERGED = 1, PCG_NEGCURV = 2, PCG_NONFINITE = 3, PCG_MAXIT = 4 };

__global__ void k_pcg_setup(double* dsc, double tol2, int max_it) {
    dsc[SC_IT] = 0.0;
    dsc[SC_FLAG] = PCG_RUN;
    dsc[SC_TOL2] = tol2;
    dsc[SC_MAXIT] = max_it;
}

// The stopping tests of one PCG iteration, in the host loop's order; a zero
// condition ends the graph's while-loop.  The cap max_it bounds the loop.
__global__ void k_pcg_control(double* dsc, cudaGraphConditionalHandle h) {
    pdl_wait();
    const double it = dsc[SC_IT] + 1.0;
    dsc[SC_IT] = it;
    const double pq = dsc[SC_PQ], rr = dsc[SC_RR];
    int flag = PCG_RUN;
    if (!isfinite(pq) || !isfinite(rr)) flag = PCG_NONFINITE;
    else if (pq <= 0.0) flag = PCG_NEGCURV;
    else if (rr <= dsc[SC_TOL2]) flag = PCG_CONVERGED;
    else if (it >= dsc[SC_MAXIT]) flag = PCG_MAXIT;
    dsc[SC_FLAG] = flag;
    cudaGraphSetConditional(h, flag == PCG_RUN ? 1u : 0u);
}

// Add c's PCG loop to `graph` with no dependencies: a while-node whose body
// is one PCG iteration and its stopping test (k_pcg_control), captured on the
// context's capture stream.  false when the driver does not take it.
static bool add_pcg_loop(reg_ctx* c, cudaGraph_t graph) {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return false;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) != cudaSuccess) return false;
    cudaGraph_t body = p.conditional.phGraph_out[0];
    cudaStream_t user = c->stream;
    bool ok = bind_stream(c, c->capture_stream) == REG_OK;
    if (ok && cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        int s = pcg_iteration(c);
        if (s == REG_OK) {
            if (launch_dependent(k_pcg_control, dim3(1), dim3(1), 0, c->stream, c->dsc, h) !=
                cudaSuccess)
                s = REG_ECUDA;
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &captured);
        ok = s == REG_OK && e == cudaSuccess;
    } else {
        ok = false;
    }
    if (bind_stream(c, user) != REG_OK) ok = false;
    return ok;
}

// The PCG loop as one executable graph (a while-node around the iteration),
// or nullptr (with the context's error state untouched) when the driver does
// not take it.
static cudaGraphExec_t build_pcg_loop(reg_ctx* c) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess && add_pcg_loop(c, graph);
    if (ok && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        exec = nullptr;
        ok = false;
    }
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        c->dead = false;   // a refused capture is not a device fault
        c->err.clear();
    }
    return exec;
}

// r = -g, s = 0, p = M P r and the initial scalars; res->converged when the
// initial residual already meets *tol (rel_tol > 0: *tol becomes
// rel_tol ||P r_0||).
static int pcg_prologue(reg_ctx* c, double* tol, int verbose, PcgResult* res,
                        double rel_tol = 0.0) {
    const int nb = blas_blocks();
    float2** S = c->ss;
    res->iters = 0;
    res->neg_curv = false;
    res->converged = false;
    {
        Phase ph(c, REG_PH_SPECTRAL, 5.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_init(c->g, S[S_G], S[S_R], S[S_S], S[S_P], S[S_PC], c->beta,
                                 c->pshift, c->kind, c->incompressible, c->partials, nb,
                                 c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_RR));
    REG_TRY(finalize_to(c, 1, nb, kTwoPi3, SC_RZ));
    REG_TRY(finalize_to(c, 2, nb, kTwoPi3, SC_PAP));
    REG_TRY(read_scalars(c, SC_RZ, 13));
    if (rel_tol > 0.0) *tol = rel_tol * std::sqrt(c->hsc[SC_RR]);
    if (verbose > 1)
        fprintf(stderr, "  pcg 0  rr %.6e  rz %.6e  pap %.6e  tol %.6e\n", c->hsc[SC_RR],
                c->hsc[SC_RZ], c->hsc[SC_PAP], *tol);
    if (std::sqrt(c->hsc[SC_RR]) <= *tol) res->converged = true;
    return REG_OK;
}

// After a device-controlled PCG loop ran on c->stream: its count and exit
// flag (waits for the stream); on negative curvature in the first iteration
// the step becomes the preconditioned steepest-descent direction.
static int pcg_loop_result(reg_ctx* c, PcgResult* res) {
    REG_TRY(read_scalars(c, 0, SC_MAXIT + 1));
    res->iters = (int)c->hsc[SC_IT];
    const int flag = (int)c->hsc[SC_FLAG];
    if (flag == PCG_NONFINITE) return fail(c, REG_ENONFINITE, "non-finite value in PCG");
    res->converged = flag == PCG_CONVERGED;
    if (flag == PCG_NEGCURV) {
        res->neg_curv = true;
        if (res->iters == 1) {
            float2** S = c->ss;
            REG_CK(c, launch_sp_direction(c->g, S[S_R], S[S_S], nullptr, c->dsc, SC_ZERO, SC_RZ, 1,
                                          c->beta, c->pshift, c->kind, c->incompressible,
                                          c->partials, blas_blocks(), c->stream));
        }
    }
    return REG_OK;
}

// rel_tol > 0: the tolerance is rel_tol ||P r_0|| instead of tol.
static int pcg_solve(reg_ctx* c, double tol, int max_it, int use_graph, int verbose,
                     PcgResult* res, double rel_tol = 0.0) {
    const int nb = blas_blocks();
    const int proj = c->incompressible;
    float2** S = c->ss;
    REG_TRY(pcg_prologue(c, &tol, verbose, res, rel_tol));
    if (res->converged) return REG_OK;

    if (use_graph >= 2 && !c->timing && verbose <= 1) {
        // reuse the captured loop while its kernels and launch shapes are
        // unchanged (they depend on the halos and the tile only)
        const int key[5] = {c->halo_fwd, c->halo_adj, c->tile.k, c->tile.wy, c->hessian};
        if (c->pcg_exec && (memcmp(key, c->pcg_key, sizeof key) != 0 ||
                            c->pcg_key_shift != c->pshift || c->pcg_key_beta != c->beta)) {
            cudaGraphExecDestroy(c->pcg_exec);
            c->pcg_exec = nullptr;
        }
        if (!c->pcg_exec) {
            c->pcg_exec = build_pcg_loop(c);
            memcpy(c->pcg_key, key, sizeof key);
            c->pcg_key_shift = c->pshift;
            c->pcg_key_beta = c->beta;
        }
        cudaGraphExec_t loop = c->pcg_exec;
        if (loop) {
            k_pcg_setup<<<1, 1, 0, c->stream>>>(c->dsc, tol * tol, max_it);
            cudaError_t e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaGraphLaunch(loop, c->stream);
            if (e != cudaSuccess) return fail_cuda(c, e, "PCG loop launch", __LINE__);
            return pcg_loop_result(c, res);
        }
    }

    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    if (use_graph) {
        // The legacy default stream cannot be captured: capture on the
        // context's own capture stream and replay on the caller's stream.
        // With timing on, the phase events are captured too and read back
        // after every replay.
        cudaStream_t user = c->stream;
        REG_TRY(bind_stream(c, c->capture_stream));
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            c->capturing = true;
            const int s = pcg_iteration(c);
            c->capturing = false;
            const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
            if (s != REG_OK || e != cudaSuccess ||
                cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                graph = nullptr;
                exec = nullptr;
                release_graph_timing(c);
                c->dead = false;   // a failed capture is not a device fault
                c->err.clear();
            }
        } else {
            cudaGetLastError();
        }
        REG_TRY(bind_stream(c, user));
    }
    int status = REG_OK;
    for (int it = 1; it <= max_it; ++it) {
        if (exec) {
            const cudaError_t e = cudaGraphLaunch(exec, c->stream);
            if (e != cudaSuccess) { status = fail_cuda(c, e, "cudaGraphLaunch", __LINE__); break; }
        } else {
            status = pcg_iteration(c);
            if (status != REG_OK) break;
        }
        status = read_scalars(c, SC_PQ, 2);    // PQ, RR (synchronises the stream)
        if (status != REG_OK) break;
        if (exec && c->timing) {
            status = harvest_graph_timing(c);
            if (status != REG_OK) break;
        }
        res->iters = it;
        const double pq = c->hsc[SC_PQ], rr = c->hsc[SC_RR];
        if (verbose > 1) {
            read_scalars(c, SC_RZ, 10);
            fprintf(stderr, "  pcg %d  pq %.6e  rr %.6e  rz %.6e  pap %.6e  pb %.6e\n", it, pq, rr,
                    c->hsc[SC_RZ], c->hsc[SC_PAP], c->hsc[SC_PB]);
        }
        if (!std::isfinite(pq) || !std::isfinite(rr)) {
            status = fail(c, REG_ENONFINITE, "non-finite value in PCG");
            break;
        }
        if (pq <= 0.0) {
            res->neg_curv = true;
            if (it == 1) {
                // first direction: the preconditioned steepest-descent step
                // s = M P r (r is still -g: the update was skipped)
                const cudaError_t e = launch_sp_direction(c->g, S[S_R], S[S_S], nullptr, c->dsc,
                                                          SC_ZERO, SC_RZ, 1, c->beta, c->pshift,
                                                          c->kind, proj, c->partials, nb,
                                                          c->stream);
                if (e != cudaSuccess) status = fail_cuda(c, e, "launch_sp_direction", __LINE__);
            }
            break;
        }
        if (std::sqrt(rr) <= tol) { res->converged = true; break; }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    release_graph_timing(c);
    return status;
}

// ------------------------------------------------ two-level preconditioner
// M^-1 r = Pi_L H_c^-1 Pi_L r + (beta A)^-1 P (I - Pi_L) r: H_c is the
// Gauss-Newton Hessian on the coarse grid n_j / factor (the images restricted
// to the modes L = {|k_j| < n_j / (2 factor)}, linearised at the restriction
// of v), inverted by the coarse context's own device-controlled PCG to a
// relative tolerance; the modes outside L get the inverse regularisation
// operator.  Normalised coefficients of the modes in L are the same numbers
// on both grids, so restriction and prolongation are copies.

static int child_fail(reg_ctx* c, int s) {
    if (s != REG_OK && c->coarse && !c->coarse->err.empty())
        fail(c, s, "coarse grid: " + c->coarse->err);
    if (s == REG_ECUDA) c->dead = true;
    return s;
}

// Create (or keep) the coarse context and give it the restricted images.
static int twolevel_setup(reg_ctx* c, int factor, int coarse_nt) {
    const Dims& g = c->g;
    if (factor < 2 || g.n1 % factor || g.n2 % factor || g.n3 % factor ||
        g.n1 / factor < 8 || g.n2 / factor < 8 || g.n3 / factor < 8)
        return fail(c, REG_EINVAL, "coarse factor: >= 2, dividing every n_j, n_j / factor >= 8");
    if (coarse_nt < 0 || coarse_nt > 64) return fail(c, REG_EINVAL, "coarse_nt must be 0..64");
    const int nt = coarse_nt > 0 ? coarse_nt : c->nt;
    if (!c->have_images) return fail(c, REG_ENOTREADY, "reg_set_images first");
    if (c->coarse && (c->coarse_factor != factor || c->coarse->nt != nt)) {
        reg_destroy(c->coarse);
        c->coarse = nullptr;
    }
    if (!c->coarse) {
        reg_ctx* k = nullptr;
        const int s = reg_create(g.n1 / factor, g.n2 / factor, g.n3 / factor, nt, c->beta,
                                 c->kind, c->incompressible, &k);
        if (s != REG_OK) return fail(c, s, std::string("coarse grid: ") + reg_last_error(nullptr));
        c->coarse = k;
        c->coarse_factor = factor;
        c->coarse_img_version = -1;
    }
    reg_ctx* k = c->coarse;
    if (k->timing != c->timing) REG_TRY(child_fail(c, reg_set_timing(k, c->timing ? 1 : 0)));
    REG_TRY(child_fail(c, bind_stream(k, c->stream)));
    REG_TRY(child_fail(c, ensure_solver(k)));
    k->beta = c->beta;
    k->pshift = 0.0;
    k->hessian = REG_HESS_GAUSS_NEWTON;
    if (c->coarse_img_version != c->img_version) {
        const int nin[3] = {g.n1, g.n2, g.n3}, nout[3] = {k->g.n1, k->g.n2, k->g.n3};
        int s = reg_spectral_resample(nin, nout, 1, c->rho_T, k->rho_T, c->stream);
        if (s == REG_OK) s = reg_spectral_resample(nin, nout, 1, c->rho_R, k->rho_R, c->stream);
        if (s != REG_OK) return fail(c, s, "coarse grid: image restriction failed");
        REG_TRY(child_fail(c, reg_set_images(k, k->rho_T, k->rho_R, 0)));
        c->coarse_img_version = c->img_version;
    }
    return REG_OK;
}

// Linearise the coarse Hessian at the restriction of the fine v_hat.
static int twolevel_linearize(reg_ctx* c, const float2* v_hat) {
    reg_ctx* k = c->coarse;
    {
        Phase ph(c, REG_PH_SPECTRAL, 24.0 * 2.0 * (double)k->g.nc);
        REG_CK(c, launch_sp_restrict(c->g, k->g, v_hat, k->ss[S_V], 1.f, c->stream));
    }
    float* vc = k->sv[R_V];
    REG_TRY(child_fail(c, to_physical(k, k->ss[S_V], vc)));
    REG_TRY(child_fail(c, op_linearize(k, vc, false, k->ss[S_V])));
    // the coarse grid's launches are small: its own tile, set by
    // reg_set_coarse_tile or autotuned (cached per grid and halo)
    if (c->coarse_tile_k > 0) return child_fail(c, reg_set_tile(k, c->coarse_tile_k, c->coarse_tile_wy));
    return child_fail(c, reg_autotune(k, nullptr, nullptr));
}

// z_hat = M^-1 r_hat and dsc[slot] = <r, z>; *inner = coarse PCG iterations.
// use_graph: the coarse PCG loop's form (as reg_solve_opts.use_graph).
static int twolevel_apply(reg_ctx* c, const float2* r_hat, float2* z_hat, double tol_rel,
                          int max_it, int slot, int* inner, int use_graph = 2) {
    reg_ctx* k = c->coarse;
    const int nb = blas_blocks();
    {
        Phase ph(c, REG_PH_SPECTRAL, 24.0 * 2.0 * (double)k->g.nc);
        REG_CK(c, launch_sp_restrict(c->g, k->g, r_hat, k->ss[S_G], -1.f, c->stream));
    }
    PcgResult pr;
    // the coarse PCG solves H_c s = -g_c = Pi_L r
    const int s = pcg_solve(k, 0.0, max_it, use_graph, 0, &pr, tol_rel > 0.0 ? tol_rel : 1e-30);
    if (s != REG_OK) return child_fail(c, s);
    if (inner) *inner = pr.iters;
    {
        Phase ph(c, REG_PH_SPECTRAL, 24.0 * 3.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_twolevel(c->g, k->g, r_hat, k->ss[S_S], z_hat, c->beta, 0.0, c->kind,
                                     c->incompressible, c->partials, nb, c->stream));
    }
    return finalize_to(c, 0, nb, kTwoPi3, slot);
}

// Flexible PCG on H s = -g (Sec. III-A with the two-level preconditioner):
// the direction p_{k+1} = z_{k+1} + b p_k with b = -alpha <z_{k+1}, H p_k> /
// <r_k, z_k>, H-conjugate to the last direction however M^-1 varies.
// Host-driven (it reads the scalars every iteration); the same stopping
// tests as pcg_solve.
static int pcg_solve_twolevel(reg_ctx* c, double tol, int max_it, double ctol, int cmax,
                              int use_graph, PcgResult* res, int* coarse_iters) {
    const int nb = blas_blocks();
    const int proj = c->incompressible;
    float2** S = c->ss;
    res->iters = 0;
    res->neg_curv = false;
    res->converged = false;
    // r = -g, s = 0 (p, pc are overwritten below)
    {
        Phase ph(c, REG_PH_SPECTRAL, 5.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_init(c->g, S[S_G], S[S_R], S[S_S], S[S_P], S[S_PC], c->beta, 0.0,
                                 c->kind, proj, c->partials, nb, c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_RR));
    REG_TRY(read_scalars(c, SC_RR, 1));
    if (std::sqrt(c->hsc[SC_RR]) <= tol) { res->converged = true; return REG_OK; }
    int it_in = 0;
    REG_TRY(twolevel_apply(c, S[S_R], S[S_Z], ctol, cmax, SC_RZ, &it_in, use_graph));
    *coarse_iters += it_in;
    // p = z, and spec[0] = p: the inverse transform destroys its input, so
    // it always works on spec[0], which the direction update refreshes
    REG_CK(c, cudaMemcpyAsync(S[S_P], S[S_Z], sizeof(float2) * 3 * (size_t)c->g.nc,
                              cudaMemcpyDeviceToDevice, c->stream));
    REG_CK(c, cudaMemcpyAsync(c->spec[0], S[S_Z], sizeof(float2) * 3 * (size_t)c->g.nc,
                              cudaMemcpyDeviceToDevice, c->stream));
    for (int it = 1; it <= max_it; ++it) {
        // q = H p on the coefficients
        REG_TRY(op_fft_c2r(c, c->spec[0], c->sv[R_P], 3));
        REG_TRY(op_matvec_transport(c, c->sv[R_P], nullptr, 0));
        REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
        {
            Phase ph(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
            REG_CK(c, launch_sp_gradient(c->g, S[S_P], c->spec[1], S[S_Q], c->beta, c->kind, proj,
                                         c->partials, nb, c->stream));
        }
        {
            Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
            REG_CK(c, launch_sp_dot(c->g, S[S_P], S[S_Q], c->partials, nb, c->stream));
        }
        REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_PQ));
        REG_TRY(read_scalars(c, SC_RZ, 2));   // RZ, PQ
        res->iters = it;
        const double rz = c->hsc[SC_RZ], pq = c->hsc[SC_PQ];
        if (!std::isfinite(pq) || !std::isfinite(rz))
            return fail(c, REG_ENONFINITE, "non-finite value in PCG");
        if (pq <= 0.0) {
            res->neg_curv = true;
            if (it == 1)   // first direction: s = p = M^-1 r
                REG_CK(c, cudaMemcpyAsync(S[S_S], S[S_P], sizeof(float2) * 3 * (size_t)c->g.nc,
                                          cudaMemcpyDeviceToDevice, c->stream));
            break;
        }
        const float alpha = (float)(rz / pq);
        {
            Phase ph(c, REG_PH_SPECTRAL, 6.0 * 24.0 * (double)c->g.nc);
            REG_CK(c, launch_sp_fcg_update(c->g, S[S_S], S[S_R], S[S_P], S[S_Q], alpha,
                                           c->partials, nb, c->stream));
        }
        REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_RR));
        REG_TRY(read_scalars(c, SC_RR, 1));
        if (!std::isfinite(c->hsc[SC_RR])) return fail(c, REG_ENONFINITE, "non-finite residual");
        if (std::sqrt(c->hsc[SC_RR]) <= tol) { res->converged = true; break; }
        if (it == max_it) break;
        REG_TRY(twolevel_apply(c, S[S_R], S[S_Z], ctol, cmax, SC_RZNEW, &it_in, use_graph));
        *coarse_iters += it_in;
        {
            Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
            REG_CK(c, launch_sp_dot(c->g, S[S_Z], S[S_Q], c->partials, nb, c->stream));
        }
        REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_TMP));
        // RZNEW and TMP in one wait (slots SC_TMP .. SC_RZNEW)
        static_assert(SC_TMP < SC_RZNEW, "scalar slots");
        REG_TRY(read_scalars(c, SC_TMP, SC_RZNEW - SC_TMP + 1));
        const float bk = (float)(-(double)alpha * c->hsc[SC_TMP] / rz);
        {
            Phase ph(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
            REG_CK(c, launch_sp_axpy(c->g, S[S_P], c->spec[0], S[S_Z], S[S_P], bk, c->kind, 0,
                                     c->partials, nb, c->stream));
        }
        REG_CK(c, cudaMemcpyAsync(c->dsc + SC_RZ, c->dsc + SC_RZNEW, sizeof(double),
                                  cudaMemcpyDeviceToDevice, c->stream));
    }
    return REG_OK;
}

static int ensure_flexible(reg_ctx* c) {
    if (c->ss[S_Q]) return REG_OK;
    if (cudaMalloc(&c->ss[S_Q], sizeof(float2) * 3 * (size_t)c->g.nc) != cudaSuccess) {
        cudaGetLastError();
        c->ss[S_Q] = nullptr;
        return fail(c, REG_ENOMEM, "cannot allocate the flexible PCG vector");
    }
    return REG_OK;
}

// g_hat = beta A v_hat + P b_hat at the spectral iterate; J and ||g||.
// after_trial: the accepted line-search trial point is v; its physical copy,
// points and state history are still in place.
static int evaluate_gradient(reg_ctx* c, double* J, double* gnorm, bool after_trial = false) {
    const int nb = blas_blocks();
    float2** S = c->ss;
    float* v = c->sv[R_V];
    if (!after_trial) REG_TRY(to_physical(c, S[S_V], v));
    REG_TRY(op_linearize(c, v, after_trial, S[S_V]));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    {
        Phase ph(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_gradient(c->g, S[S_V], c->spec[1], S[S_G], c->beta, c->kind,
                                     c->incompressible, c->partials, nb, c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_GG));
    REG_TRY(finalize_to(c, 1, nb, 0.5 * c->beta * kTwoPi3, SC_JREG));
    REG_TRY(read_scalars(c, SC_JMIS, 9));
    *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
    *gnorm = std::sqrt(c->hsc[SC_GG]);
    if (!std::isfinite(*J) || !std::isfinite(*gnorm))
        return fail(c, REG_ENONFINITE, "non-finite objective or gradient");
    return REG_OK;
}

// J at v_hat + alpha s_hat (into S_VT): points and forward state solve of the
// trial, kept in the linearisation buffers for the gradient that follows an
// accepted step.
static int evaluate_trial(reg_ctx* c, double alpha, double* J) {
    const int nb = blas_blocks();
    float2** S = c->ss;
    {
        Phase ph(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_axpy(c->g, S[S_VT], c->spec[0], S[S_V], S[S_S], (float)alpha, c->kind, 0,
                                 c->partials, nb, c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, 0.5 * c->beta * kTwoPi3, SC_JREG));
    float* v = c->sv[R_V];
    REG_TRY(op_fft_c2r(c, c->spec[0], v, 3));
    REG_TRY(op_trial_state(c, v));
    REG_TRY(read_scalars(c, SC_JMIS, 2));
    *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
    return REG_OK;
}

// ||g(0)||: at v = 0 the transport is the identity, so rho(t) = rho(t_0),
// lam(t) = rho_R - rho(t_0) and b = (rho_R - rho(t_0)) grad rho(t_0)
// (trapezoid weights sum to 1); g(0) = P b (Eq. gradient).  One spectral
// gradient instead of a linearisation; equal to the gradient at v = 0 up to
// FP32 rounding.  Clobbers the linearisation buffers and S_G.
static int gradient_norm_at_zero(reg_ctx* c, double* g0) {
    const long long n = c->g.n;
    const int nb = blas_blocks();
    float2** S = c->ss;
    c->have_lin = false;
    float* r0 = c->rho_hist;   // rho(t_0) as the state solve starts from it
    if (c->precision == REG_MIXED_BF16 && c->img_bf) {
        Phase p(c, REG_PH_OTHER, 6.0 * n);
        REG_CK(c, launch_from_bf16(c->img_bf, r0, n, c->stream));
    } else {
        REG_CK(c, cudaMemcpyAsync(r0, c->rho_T, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                  c->stream));
    }
    {
        Phase p(c, REG_PH_OTHER, 12.0 * n);
        REG_CK(c, launch_axpby_out(c->tmp3, c->rho_R, r0, 1.f, -1.f, n, c->stream));
    }
    REG_TRY(op_grad(c, r0, c->grad_hist));
    c->grad0_valid = true;   // level 0 of the cache: grad rho(t_0)
    {
        Phase p(c, REG_PH_OTHER, 28.0 * n);
        REG_CK(c, launch_mul_fields(c->tmp3, c->grad_hist, c->bacc, n, c->stream));
    }
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    {
        Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_normalise(c->g, c->spec[1], S[S_G], c->incompressible, c->stream));
    }
    {
        Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_dot(c->g, S[S_G], S[S_G], c->partials, nb, c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_GG));
    REG_TRY(read_scalars(c, SC_GG, 1));
    *g0 = std::sqrt(c->hsc[SC_GG]);
    return REG_OK;
}

// The Gauss-Newton loop in steps, so that the batch driver can interleave the
// pairs of a batch: begin (initial gradient), per Newton step the PCG
// tolerance, the PCG solve, then the line search and the new gradient, end.
struct SolveState {
    std::chrono::steady_clock::time_point t0;
    double m0 = 0, g0 = 0, J = 0, gn = 0, jmis = 0;
    int k = 0;
    int status = REG_EMAXITER;
    bool done = false;
};

static int solve_begin(reg_ctx* c, float* v_io, const reg_solve_opts* o, reg_solve_stats* st,
                       SolveState* S) {
    S->t0 = std::chrono::steady_clock::now();
    const long long n = c->g.n;
    float2** V = c->ss;
    // v_hat = F v / n (projected when incompressible)
    REG_TRY(op_fft_r2c(c, v_io, c->spec[0], 3));
    {
        Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_normalise(c->g, c->spec[0], V[S_V], c->incompressible, c->stream));
    }
    // ||rho_T - rho_R|| for the relative mismatch
    REG_CK(c, launch_axpby_out(c->tmp3, c->rho_T, c->rho_R, 1.f, -1.f, n, c->stream));
    REG_TRY(op_inner(c, c->tmp3, c->tmp3, n, SC_TMP));
    REG_TRY(read_scalars(c, SC_TMP, 1));
    S->m0 = std::sqrt(c->hsc[SC_TMP]);
    double gz = 0.0;
    if (o->gnorm_ref < 0.0) REG_TRY(gradient_norm_at_zero(c, &gz));
    REG_TRY(evaluate_gradient(c, &S->J, &S->gn));
    st->gradient_evals++;
    // the stop test and the forcing term are relative to ||g_0||: the
    // gradient at the initial guess, or a reference norm (the caller's, or
    // the gradient at v = 0 when the guess is a prediction)
    S->g0 = o->gnorm_ref > 0.0 ? o->gnorm_ref : (o->gnorm_ref < 0.0 ? gz : S->gn);
    st->J0 = S->J;
    st->gnorm0 = S->g0;
    S->jmis = c->hsc[SC_JMIS];
    return REG_OK;
}

// True when another Newton step is due; *tol = eta ||g|| (quadratic or
// square-root forcing).  Marks the solve done (converged or at max_gn).
static bool solve_step_due(const reg_solve_opts* o, SolveState* S, double* tol) {
    if (S->done) return false;
    if (S->gn <= o->gtol * S->g0 || S->g0 == 0.0) {
        S->status = REG_OK;
        S->done = true;
        return false;
    }
    if (S->k >= o->max_gn) {
        S->done = true;
        return false;
    }
    const double ratio = S->gn / S->g0;
    const double eta = std::fmin(0.5, o->forcing == 1 ? std::sqrt(ratio) : ratio);
    *tol = eta * S->gn;
    return true;
}

// After the PCG solve of step S->k: Armijo line search along s, the gradient
// at the accepted point.
static int solve_step_finish(reg_ctx* c, const reg_solve_opts* o, reg_solve_stats* st,
                             SolveState* S, const PcgResult& pr) {
    const int nb = blas_blocks();
    float2** V = c->ss;
    st->pcg_iters += pr.iters;
    st->matvecs += pr.iters;
    st->negative_curvature += pr.neg_curv ? 1 : 0;
    {
        Phase ph(c, REG_PH_SPECTRAL, 2.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_dot(c->g, V[S_G], V[S_S], c->partials, nb, c->stream));
    }
    REG_TRY(finalize_to(c, 0, nb, kTwoPi3, SC_GS));
    REG_TRY(read_scalars(c, SC_GS, 1));
    const double slope = c->hsc[SC_GS];
    double alpha = 1.0, Jt = S->J;
    bool accepted = false;
    for (int m = 0; m < o->armijo_max; ++m) {
        REG_TRY(evaluate_trial(c, alpha, &Jt));
        st->objective_evals++;
        if (std::isfinite(Jt) && Jt <= S->J + o->armijo_c * alpha * slope) {
            accepted = true;
            break;
        }
        alpha *= o->armijo_shrink;
    }
    if (!accepted) {
        st->line_search_failed = 1;
        S->status = REG_EMAXITER;
        S->done = true;
        return REG_OK;
    }
    std::swap(V[S_V], V[S_VT]);
    REG_TRY(evaluate_gradient(c, &S->J, &S->gn, true));
    S->jmis = c->hsc[SC_JMIS];
    st->gradient_evals++;
    S->k++;
    st->gn_iters = S->k;
    if (o->verbose)
        fprintf(stderr, "GN %3d  J %.6e  |g|/|g0| %.3e  pcg %3d  alpha %.3g%s\n", S->k, S->J,
                S->gn / S->g0, pr.iters, alpha, pr.neg_curv ? "  (negative curvature)" : "");
    return REG_OK;
}

static int solve_end(reg_ctx* c, float* v_io, const reg_solve_opts* o, reg_solve_stats* st,
                     SolveState* S) {
    if (S->status == REG_EMAXITER && (S->gn <= o->gtol * S->g0 || S->g0 == 0.0))
        S->status = REG_OK;
    REG_TRY(to_physical(c, c->ss[S_V], v_io));
    st->J = S->J;
    st->gnorm = S->gn;
    st->gnorm_rel = S->g0 > 0 ? S->gn / S->g0 : 0.0;
    st->mismatch_rel = S->m0 > 0 ? std::sqrt(2.0 * S->jmis) / S->m0 : 0.0;
    REG_CK(c, cudaStreamSynchronize(c->stream));
    st->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                             S->t0)
                       .count();
    if (S->status == REG_EMAXITER) fail(c, REG_EMAXITER, "Gauss-Newton stopped before gtol");
    return S->status;
}

static int solve_impl(reg_ctx* c, float* v_io, const reg_solve_opts* o, reg_solve_stats* st) {
    SolveState S;
    REG_TRY(solve_begin(c, v_io, o, st, &S));
    double tol = 0.0;
    while (solve_step_due(o, &S, &tol)) {
        PcgResult pr;
        if (o->coarse_factor >= 2) {
            REG_TRY(twolevel_linearize(c, c->ss[S_V]));
            REG_TRY(pcg_solve_twolevel(c, tol, o->max_pcg, o->coarse_tol, o->coarse_max,
                                       o->use_graph, &pr, &st->coarse_matvecs));
        } else {
            REG_TRY(pcg_solve(c, tol, o->max_pcg, o->use_graph, o->verbose, &pr));
        }
        REG_TRY(solve_step_finish(c, o, st, &S, pr));
    }
    return solve_end(c, v_io, o, st, &S);
}

// ------------------------------------------------------------ batches
// Independent pairs advanced in lockstep Newton steps: the gradients and line
// searches of the active pairs run on host worker threads (each pair on its
// own stream), and the PCG solves of one Newton step of every active pair are
// ONE CUDA graph: a while-node per pair, side by side, each running that
// pair's iterations until its own device-side stopping test.

static void parallel_for(const std::vector<int>& items, int workers, int dev,
                         const std::function<void(int)>& fn) {
    if (items.empty()) return;
    std::atomic<size_t> next(0);
    auto run = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const size_t q = next.fetch_add(1);
            if (q >= items.size()) break;
            fn(items[q]);
        }
    };
    const int nw = std::max(1, std::min<int>(workers, (int)items.size()));
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(run);
    run();
    for (auto& t : pool) t.join();
}

int batch_solve_graph(const std::vector<reg_ctx*>& ctx, float* const* v_io,
                      const float* const* rho_T, const float* const* rho_R, int presmooth,
                      int autotune, const reg_solve_opts* opts, reg_solve_stats* stats,
                      double* latency_ms, int* status_out, int workers, cudaStream_t launch,
                      BatchGraphCache* cache, int* graphs_launched) {
    const int np = (int)ctx.size();
    reg_solve_opts o;
    reg_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.beta_start > 0.0 || o.coarse_factor >= 2 || o.max_gn < 0 || o.max_pcg < 1 ||
        o.armijo_max < 1 || !(o.armijo_shrink > 0.0 && o.armijo_shrink < 1.0) ||
        !(o.gtol >= 0.0) || !(o.precond_shift >= 0.0) || !std::isfinite(o.gnorm_ref))
        return REG_EINVAL;   // the batch graph runs the plain solver options
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return REG_ECUDA;
    std::vector<SolveState> S(np);
    std::vector<reg_solve_stats> st(np);
    std::vector<int> status(np, REG_OK), need(np, 0);
    std::vector<PcgResult> pr(np);
    std::vector<double> tol(np, 0.0), lat(np, 0.0);
    std::vector<cudaEvent_t> ev(np, nullptr);
    cudaEvent_t done_ev = nullptr;
    for (int i = 0; i < np; ++i) memset(&st[i], 0, sizeof(reg_solve_stats));
    for (int i = 0; i < np; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) return REG_ECUDA;
    if (cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming) != cudaSuccess) return REG_ECUDA;
    const auto t0 = std::chrono::steady_clock::now();
    auto ms_since = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    };
    // the pair is finished: velocity out, statistics, latency
    auto finish = [&](int i) {
        reg_ctx* c = ctx[i];
        const int s = status[i] != REG_OK ? status[i] : solve_end(c, v_io[i], &o, &st[i], &S[i]);
        status[i] = s;
        st[i].stages = 1;
        lat[i] = ms_since();
    };
    std::vector<int> all(np);
    for (int i = 0; i < np; ++i) all[i] = i;
    parallel_for(all, workers, dev, [&](int i) {
        reg_ctx* c = ctx[i];
        int s = reg_set_images(c, rho_T[i], rho_R[i], presmooth);
        if (s == REG_OK) s = ensure_solver(c);
        if (s == REG_OK && autotune) {
            s = reg_gradient(c, v_io[i], c->sv[3], nullptr);
            if (s == REG_OK) s = reg_autotune(c, nullptr, nullptr);
        }
        c->pshift = o.precond_shift;
        if (s == REG_OK) s = solve_begin(c, v_io[i], &o, &st[i], &S[i]);
        if (s != REG_OK) {
            status[i] = s;
            S[i].done = true;
            lat[i] = ms_since();
        }
    });
    int launched = 0;
    for (;;) {
        // Newton step due?  PCG prologue (r = -g, p = M P r, first scalars)
        std::vector<int> active;
        for (int i = 0; i < np; ++i)
            if (!S[i].done || status[i] == REG_OK) active.push_back(i);
        std::vector<int> stepping;
        for (int i : active) {
            if (status[i] != REG_OK) continue;
            if (solve_step_due(&o, &S[i], &tol[i])) stepping.push_back(i);
        }
        // pairs that stopped this round: finish them
        std::vector<int> stopped;
        for (int i : active)
            if (status[i] == REG_OK && S[i].done && lat[i] == 0.0) stopped.push_back(i);
        parallel_for(stopped, workers, dev, finish);
        if (stepping.empty()) break;
        parallel_for(stepping, workers, dev, [&](int i) {
            reg_ctx* c = ctx[i];
            int s = pcg_prologue(c, &tol[i], 0, &pr[i]);
            need[i] = 0;
            if (s == REG_OK && !pr[i].converged) {
                k_pcg_setup<<<1, 1, 0, c->stream>>>(c->dsc, tol[i] * tol[i], o.max_pcg);
                cudaError_t e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaEventRecord(ev[i], c->stream);
                if (e != cudaSuccess) s = fail_cuda(c, e, "batch PCG set-up", __LINE__);
                need[i] = 1;
            }
            if (s != REG_OK) {
                status[i] = s;
                need[i] = 0;
            }
        });
        std::vector<int> loops;
        for (int i : stepping)
            if (need[i]) loops.push_back(i);
        if (!loops.empty()) {
            // one graph with every pair's PCG loop, rebuilt when a pair's
            // captured kernels change (halos, tile, Hessian, beta, shift)
            std::vector<double> key;
            for (int i : loops) {
                const reg_ctx* c = ctx[i];
                key.insert(key.end(), {(double)i, (double)c->halo_fwd, (double)c->halo_adj,
                                       (double)c->tile.k, (double)c->tile.wy, (double)c->hessian,
                                       c->beta, c->pshift});
            }
            if (cache->exec && cache->key != key) {
                cudaGraphExecDestroy(cache->exec);
                cache->exec = nullptr;
            }
            if (!cache->exec) {
                cudaGraph_t graph = nullptr;
                bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
                for (int i : loops) ok = ok && add_pcg_loop(ctx[i], graph);
                if (ok && cudaGraphInstantiate(&cache->exec, graph, 0) != cudaSuccess) {
                    cache->exec = nullptr;
                    ok = false;
                }
                if (graph) cudaGraphDestroy(graph);
                if (!ok) {
                    cudaGetLastError();
                    for (int i : loops) status[i] = REG_ECUDA;
                    break;
                }
                cache->key = key;
            }
            bool ok = true;
            for (int i : loops) ok = ok && cudaStreamWaitEvent(launch, ev[i], 0) == cudaSuccess;
            ok = ok && cudaGraphLaunch(cache->exec, launch) == cudaSuccess &&
                 cudaEventRecord(done_ev, launch) == cudaSuccess;
            for (int i : loops) ok = ok && cudaStreamWaitEvent(ctx[i]->stream, done_ev, 0) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                for (int i : loops) status[i] = REG_ECUDA;
                break;
            }
            ++launched;
        }
        parallel_for(stepping, workers, dev, [&](int i) {
            if (status[i] != REG_OK) return;
            reg_ctx* c = ctx[i];
            int s = need[i] ? pcg_loop_result(c, &pr[i]) : REG_OK;
            if (s == REG_OK) s = solve_step_finish(c, &o, &st[i], &S[i], pr[i]);
            if (s != REG_OK) status[i] = s;
        });
        for (int i : stepping)
            if (status[i] != REG_OK && lat[i] == 0.0) {
                S[i].done = true;
                lat[i] = ms_since();
            }
    }
    int first_err = REG_OK;
    for (int i = 0; i < np; ++i) {
        if (lat[i] == 0.0) lat[i] = ms_since();
        if (stats) stats[i] = st[i];
        if (latency_ms) latency_ms[i] = lat[i];
        if (status_out) status_out[i] = status[i];
        if (status[i] != REG_OK && status[i] != REG_EMAXITER && first_err == REG_OK)
            first_err = status[i];
    }
    for (auto e : ev) if (e) cudaEventDestroy(e);
    if (done_ev) cudaEventDestroy(done_ev);
    if (graphs_launched) *graphs_launched = launched;
    return first_err;
}

}  // namespace reg

using namespace reg;

extern "C" {

int reg_solve_opts_default(reg_solve_opts* o) {
    if (!o) return REG_EINVAL;
    o->gtol = 1e-2;
    o->max_gn = 50;
    o->max_pcg = 500;
    o->forcing = 0;
    o->armijo_c = 1e-4;
    o->armijo_shrink = 0.5;
    o->armijo_max = 10;
    o->use_graph = 2;
    o->verbose = 0;
    o->gnorm_ref = 0.0;
    o->precond_shift = 0.0;
    o->beta_start = 0.0;
    o->beta_factor = 10.0;
    o->coarse_factor = 0;
    o->coarse_tol = 0.2;
    o->coarse_max = 12;
    o->coarse_nt = 0;
    return REG_OK;
}

int reg_twolevel_setup_nt(reg_ctx* c, int coarse_factor, int coarse_nt, const float* v_hat) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!v_hat || ((uintptr_t)v_hat & 15u)) return fail(c, REG_EINVAL, "bad v_hat");
    REG_TRY(ensure_solver(c));
    REG_TRY(twolevel_setup(c, coarse_factor, coarse_nt));
    return twolevel_linearize(c, reinterpret_cast<const float2*>(v_hat));
}

int reg_twolevel_setup(reg_ctx* c, int coarse_factor, const float* v_hat) {
    return reg_twolevel_setup_nt(c, coarse_factor, 0, v_hat);
}

int reg_twolevel_apply(reg_ctx* c, const float* r_hat, float* z_hat, double inner_tol,
                       int inner_max, int* inner_iters) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!r_hat || !z_hat || ((uintptr_t)r_hat & 15u) || ((uintptr_t)z_hat & 15u) ||
        r_hat == z_hat)
        return fail(c, REG_EINVAL, "r_hat / z_hat: null, unaligned or overlapping");
    if (!(inner_tol >= 0.0) || inner_max < 1) return fail(c, REG_EINVAL, "bad inner options");
    if (!c->coarse || !c->coarse->have_lin)
        return fail(c, REG_ENOTREADY, "reg_twolevel_setup first");
    c->coarse->beta = c->beta;
    int it = 0;
    REG_TRY(twolevel_apply(c, reinterpret_cast<const float2*>(r_hat),
                           reinterpret_cast<float2*>(z_hat), inner_tol, inner_max, SC_TMP, &it));
    if (inner_iters) *inner_iters = it;
    return REG_OK;
}

int reg_set_beta(reg_ctx* c, double beta) {
    if (!c) return REG_EINVAL;
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(c, REG_EINVAL, "beta must be > 0");
    c->beta = beta;
    return REG_OK;
}

int reg_solve(reg_ctx* c, float* v_inout, const reg_solve_opts* opts, reg_solve_stats* stats) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!v_inout || ((uintptr_t)v_inout & 15u)) return fail(c, REG_EINVAL, "bad v_inout");
    if (!c->have_images) return fail(c, REG_ENOTREADY, "reg_set_images first");
    reg_solve_opts o;
    reg_solve_opts_default(&o);
    if (opts) o = *opts;
    if (!(o.gtol >= 0.0) || !std::isfinite(o.gnorm_ref) || !(o.precond_shift >= 0.0) ||
        o.max_gn < 0 || o.max_pcg < 1 || o.armijo_max < 1 ||
        !(o.armijo_shrink > 0.0 && o.armijo_shrink < 1.0))
        return fail(c, REG_EINVAL, "bad solver options");
    if (!(o.beta_start >= 0.0) || !std::isfinite(o.beta_start) || !(o.beta_factor > 1.0) ||
        !std::isfinite(o.beta_factor))
        return fail(c, REG_EINVAL, "bad continuation options");
    if (o.coarse_factor != 0 && o.coarse_factor != 1) {
        if (!(o.coarse_tol >= 0.0) || o.coarse_max < 1)
            return fail(c, REG_EINVAL, "bad coarse-grid options");
    }
    REG_TRY(ensure_solver(c));
    if (o.coarse_factor >= 2) {
        REG_TRY(ensure_flexible(c));
        REG_TRY(twolevel_setup(c, o.coarse_factor, o.coarse_nt));
    } else {
        o.coarse_factor = 0;
    }
    c->pshift = o.precond_shift;
    reg_solve_stats local;
    memset(&local, 0, sizeof local);
    if (!(o.beta_start > c->beta * (1.0 + 1e-12))) {
        const int s = solve_impl(c, v_inout, &o, &local);
        local.stages = 1;
        if (stats) *stats = local;
        return s;
    }
    // continuation: beta_start, beta_start / factor, ... down to the target
    const auto t0 = std::chrono::steady_clock::now();
    const double target = c->beta;
    double b = o.beta_start;
    int s = REG_OK;
    bool last = false;
    for (int stage = 0; !last; ++stage) {
        last = !(b > target * (1.0 + 1e-12));
        c->beta = last ? target : b;
        if (c->coarse) c->coarse->beta = c->beta;
        reg_solve_stats st;
        memset(&st, 0, sizeof st);
        s = solve_impl(c, v_inout, &o, &st);
        if (stage == 0) {
            local.J0 = st.J0;
            // later stages stop at the first stage's ||g_0||
            if (o.gnorm_ref == 0.0 || o.gnorm_ref < 0.0) o.gnorm_ref = st.gnorm0;
        }
        local.gn_iters += st.gn_iters;
        local.pcg_iters += st.pcg_iters;
        local.matvecs += st.matvecs;
        local.objective_evals += st.objective_evals;
        local.gradient_evals += st.gradient_evals;
        local.line_search_failed |= st.line_search_failed;
        local.negative_curvature += st.negative_curvature;
        local.coarse_matvecs += st.coarse_matvecs;
        local.gnorm0 = st.gnorm0;
        local.J = st.J;
        local.gnorm = st.gnorm;
        local.gnorm_rel = st.gnorm_rel;
        local.mismatch_rel = st.mismatch_rel;
        local.stages = stage + 1;
        if (s != REG_OK && s != REG_EMAXITER) break;
        b /= o.beta_factor;
    }
    c->beta = target;
    if (c->coarse) c->coarse->beta = target;
    local.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = local;
    return s;
}

int reg_gradient_spectral(reg_ctx* c, const float* v_hat, float* g_hat, double* J) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!v_hat || !g_hat || ((uintptr_t)v_hat & 15u) || ((uintptr_t)g_hat & 15u))
        return fail(c, REG_EINVAL, "v_hat / g_hat: null or not 16-byte aligned");
    if (v_hat == g_hat) return fail(c, REG_EINVAL, "v_hat and g_hat overlap");
    if (!c->have_images) return fail(c, REG_ENOTREADY, "reg_set_images first");
    REG_TRY(ensure_solver(c));
    const int nb = blas_blocks();
    const float2* vh = reinterpret_cast<const float2*>(v_hat);
    float* v = c->sv[R_V];
    REG_TRY(to_physical(c, vh, v));
    REG_TRY(op_linearize(c, v, false, vh));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    {
        Phase ph(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
        REG_CK(c, launch_sp_gradient(c->g, vh, c->spec[1], reinterpret_cast<float2*>(g_hat),
                                     c->beta, c->kind, c->incompressible, c->partials, nb,
                                     c->stream));
    }
    REG_TRY(finalize_to(c, 1, nb, 0.5 * c->beta * kTwoPi3, SC_JREG));
    if (J) {
        REG_TRY(read_scalars(c, SC_JMIS, 2));
        *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
        if (!std::isfinite(*J)) return fail(c, REG_ENONFINITE, "objective is not finite");
    }
    return REG_OK;
}

int reg_hessian_matvec_spectral(reg_ctx* c, const float* vt_hat, float* Hvt_hat) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!vt_hat || !Hvt_hat || ((uintptr_t)vt_hat & 15u) || ((uintptr_t)Hvt_hat & 15u))
        return fail(c, REG_EINVAL, "vt_hat / Hvt_hat: null or not 16-byte aligned");
    if (vt_hat == Hvt_hat) return fail(c, REG_EINVAL, "vt_hat and Hvt_hat overlap");
    if (!c->have_lin) return fail(c, REG_ENOTREADY, "reg_gradient must come first");
    REG_TRY(ensure_solver(c));
    const int nb = blas_blocks();
    const float2* ph = reinterpret_cast<const float2*>(vt_hat);
    float* p = c->sv[R_P];
    REG_TRY(to_physical(c, ph, p));
    REG_TRY(op_matvec_transport(c, p, nullptr, 0));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    Phase pq(c, REG_PH_SPECTRAL, 3.0 * 24.0 * (double)c->g.nc);
    REG_CK(c, launch_sp_gradient(c->g, ph, c->spec[1], reinterpret_cast<float2*>(Hvt_hat),
                                 c->beta, c->kind, c->incompressible, c->partials, nb,
                                 c->stream));
    return REG_OK;
}

int reg_solve_host(reg_ctx* c, const float* rho_T_host, const float* rho_R_host, int presmooth,
                   float* v_host_inout, const reg_solve_opts* opts, reg_solve_stats* stats) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!rho_T_host || !rho_R_host || !v_host_inout)
        return fail(c, REG_EINVAL, "null host pointer");
    REG_TRY(ensure_solver(c));
    const size_t n = (size_t)c->g.n;
    REG_CK(c, cudaMemcpyAsync(c->rho_T, rho_T_host, sizeof(float) * n, cudaMemcpyHostToDevice,
                              c->stream));
    REG_CK(c, cudaMemcpyAsync(c->rho_R, rho_R_host, sizeof(float) * n, cudaMemcpyHostToDevice,
                              c->stream));
    REG_TRY(reg_set_images(c, c->rho_T, c->rho_R, presmooth));
    float* v = c->sv[R_HOST];
    REG_CK(c, cudaMemcpyAsync(v, v_host_inout, sizeof(float) * 3 * n, cudaMemcpyHostToDevice,
                              c->stream));
    const int s = reg_solve(c, v, opts, stats);
    if (s != REG_OK && s != REG_EMAXITER) return s;
    REG_CK(c, cudaMemcpyAsync(v_host_inout, v, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost,
                              c->stream));
    REG_CK(c, cudaStreamSynchronize(c->stream));
    return s;
}

}  // extern "C"
