// Inexact Gauss-Newton-Krylov solve (Sec. III-A, Sec. IV-A3): PCG on
// H s = -g with the spectral preconditioner, forcing tied to the relative
// gradient norm, Armijo backtracking on J, stop at ||g|| <= gtol ||g_0||.
//
// The PCG recurrence keeps its scalars (r.z, p.Hp, r.r) in device memory and
// the update kernels read alpha and beta from there, so one PCG iteration is
// a fixed sequence of launches with no host round trip; the host reads r.r
// and p.Hp once per iteration (after the speculative preconditioner and
// direction update) for the stopping and curvature tests.  With
// use_graph = 1 that sequence is captured once into a CUDA graph and
// replayed, one launch per iteration.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "ctx.h"

namespace reg {

static const double kTwoPi3 = 248.05021344239856;   // (2 pi)^3

enum { V_G = 0, V_S = 1, V_R = 2, V_Z = 3, V_P = 4, V_Q = 5, V_TRIAL = 6, V_SPARE = 7 };

// One PCG iteration from p: q = H p; PQ = <p, q>; s += a p, r -= a q (a = RZ/PQ,
// skipped when PQ <= 0); RR = <r, r>; z = M r; RZNEW = <r, z>;
// p = z + (RZNEW/RZ) p; RZ = RZNEW.
static int pcg_iteration(reg_ctx* c) {
    const long long cnt = 3LL * c->g.n;
    float** v = c->sv;
    REG_TRY(op_matvec(c, v[V_P], v[V_Q]));
    REG_TRY(op_inner(c, v[V_P], v[V_Q], cnt, SC_PQ));
    const int nb = blas_blocks();
    REG_CK(c, launch_pcg_update(v[V_S], v[V_R], v[V_P], v[V_Q], c->dsc, SC_RZ, SC_PQ, cnt,
                                c->partials, nb, c->stream));
    REG_CK(c, launch_finalize(c->partials, nb, kTwoPi3 / c->g.n, c->dsc + SC_RR, c->stream));
    REG_TRY(op_precond(c, v[V_R], v[V_Z]));
    REG_TRY(op_inner(c, v[V_R], v[V_Z], cnt, SC_RZNEW));
    REG_CK(c, launch_pcg_direction(v[V_P], v[V_Z], c->dsc, SC_RZNEW, SC_RZ, cnt, c->stream));
    REG_CK(c, cudaMemcpyAsync(c->dsc + SC_RZ, c->dsc + SC_RZNEW, sizeof(double),
                              cudaMemcpyDeviceToDevice, c->stream));
    return REG_OK;
}

struct PcgResult { int iters; bool neg_curv; bool converged; };

static int pcg_solve(reg_ctx* c, double tol, int max_it, bool use_graph, PcgResult* res) {
    const long long cnt = 3LL * c->g.n;
    float** v = c->sv;
    res->iters = 0;
    res->neg_curv = false;
    res->converged = false;
    // s = 0, r = -g, z = M r, p = z
    REG_CK(c, cudaMemsetAsync(v[V_S], 0, sizeof(float) * cnt, c->stream));
    REG_CK(c, launch_axpby_out(v[V_R], v[V_G], v[V_G], -1.f, 0.f, cnt, c->stream));
    REG_TRY(op_precond(c, v[V_R], v[V_Z]));
    REG_CK(c, cudaMemcpyAsync(v[V_P], v[V_Z], sizeof(float) * cnt, cudaMemcpyDeviceToDevice,
                              c->stream));
    REG_TRY(op_inner(c, v[V_R], v[V_Z], cnt, SC_RZ));
    REG_TRY(op_inner(c, v[V_R], v[V_R], cnt, SC_RR));
    REG_TRY(read_scalars(c, SC_RR, 1));
    if (std::sqrt(c->hsc[SC_RR]) <= tol) { res->converged = true; return REG_OK; }

    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    if (use_graph && !c->timing) {
        // The legacy default stream cannot be captured: capture on the
        // context's own capture stream and replay on the caller's stream.
        cudaStream_t user = c->stream;
        REG_TRY(bind_stream(c, c->capture_stream));
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int s = pcg_iteration(c);
            const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
            if (s != REG_OK || e != cudaSuccess ||
                cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                cudaGetLastError();
                if (graph) cudaGraphDestroy(graph);
                graph = nullptr;
                exec = nullptr;
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
        status = read_scalars(c, SC_PQ, 2);    // PQ, RR
        if (status != REG_OK) break;
        res->iters = it;
        const double pq = c->hsc[SC_PQ], rr = c->hsc[SC_RR];
        if (!std::isfinite(pq) || !std::isfinite(rr)) {
            status = fail(c, REG_ENONFINITE, "non-finite value in PCG");
            break;
        }
        if (pq <= 0.0) {
            res->neg_curv = true;
            if (it == 1) {
                // first direction: the preconditioned steepest-descent step
                status = op_precond(c, v[V_R], v[V_S]);
            }
            break;
        }
        if (std::sqrt(rr) <= tol) { res->converged = true; break; }
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return status;
}

static int evaluate_gradient(reg_ctx* c, const float* v, float* g, double* J, double* gnorm) {
    REG_TRY(op_gradient(c, v, g, SC_J));
    REG_TRY(op_inner(c, g, g, 3LL * c->g.n, SC_GG));
    REG_TRY(read_scalars(c, SC_JMIS, 9));
    *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
    *gnorm = std::sqrt(c->hsc[SC_GG]);
    if (!std::isfinite(*J) || !std::isfinite(*gnorm))
        return fail(c, REG_ENONFINITE, "non-finite objective or gradient");
    return REG_OK;
}

static int solve_impl(reg_ctx* c, float* v, const reg_solve_opts* o, reg_solve_stats* st) {
    const auto t0 = std::chrono::steady_clock::now();
    const long long n = c->g.n, cnt = 3 * n;
    float** w = c->sv;
    if (c->incompressible) REG_TRY(op_leray(c, v, v));
    // ||rho_T - rho_R|| for the relative mismatch
    REG_CK(c, launch_axpby_out(c->tmp3, c->rho_T, c->rho_R, 1.f, -1.f, n, c->stream));
    REG_TRY(op_inner(c, c->tmp3, c->tmp3, n, SC_TMP));
    REG_TRY(read_scalars(c, SC_TMP, 1));
    const double m0 = std::sqrt(c->hsc[SC_TMP]);

    double J, gn;
    REG_TRY(evaluate_gradient(c, v, w[V_G], &J, &gn));
    st->gradient_evals++;
    const double g0 = gn;
    st->J0 = J;
    st->gnorm0 = g0;
    int status = REG_EMAXITER;
    for (int k = 0; k < o->max_gn; ++k) {
        if (gn <= o->gtol * g0 || g0 == 0.0) { status = REG_OK; break; }
        const double ratio = gn / g0;
        const double eta = std::fmin(0.5, o->forcing == 1 ? std::sqrt(ratio) : ratio);
        PcgResult pr;
        REG_TRY(pcg_solve(c, eta * gn, o->max_pcg, o->use_graph != 0, &pr));
        st->pcg_iters += pr.iters;
        st->matvecs += pr.iters;
        st->negative_curvature += pr.neg_curv ? 1 : 0;
        REG_TRY(op_inner(c, w[V_G], w[V_S], cnt, SC_GS));
        REG_TRY(read_scalars(c, SC_GS, 1));
        const double slope = c->hsc[SC_GS];
        double alpha = 1.0, Jt = J;
        bool accepted = false;
        for (int m = 0; m < o->armijo_max; ++m) {
            REG_CK(c, launch_axpby_out(w[V_TRIAL], v, w[V_S], 1.f, (float)alpha, cnt, c->stream));
            REG_TRY(op_objective(c, w[V_TRIAL], SC_J));
            REG_TRY(read_scalars(c, SC_JMIS, 2));
            st->objective_evals++;
            Jt = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
            if (std::isfinite(Jt) && Jt <= J + o->armijo_c * alpha * slope) {
                accepted = true;
                break;
            }
            alpha *= o->armijo_shrink;
        }
        if (!accepted) {
            st->line_search_failed = 1;
            status = REG_EMAXITER;
            break;
        }
        REG_CK(c, cudaMemcpyAsync(v, w[V_TRIAL], sizeof(float) * cnt, cudaMemcpyDeviceToDevice,
                                  c->stream));
        REG_TRY(evaluate_gradient(c, v, w[V_G], &J, &gn));
        st->gradient_evals++;
        st->gn_iters = k + 1;
        if (o->verbose)
            fprintf(stderr, "GN %3d  J %.6e  |g|/|g0| %.3e  pcg %3d  alpha %.3g%s\n", k + 1, J,
                    gn / g0, pr.iters, alpha, pr.neg_curv ? "  (negative curvature)" : "");
    }
    if (status == REG_EMAXITER && (gn <= o->gtol * g0 || g0 == 0.0)) status = REG_OK;
    st->J = J;
    st->gnorm = gn;
    st->gnorm_rel = g0 > 0 ? gn / g0 : 0.0;
    st->mismatch_rel = m0 > 0 ? std::sqrt(2.0 * c->hsc[SC_JMIS]) / m0 : 0.0;
    REG_CK(c, cudaStreamSynchronize(c->stream));
    st->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (status == REG_EMAXITER) fail(c, REG_EMAXITER, "Gauss-Newton stopped before gtol");
    return status;
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
    o->use_graph = 1;
    o->verbose = 0;
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
    if (!(o.gtol >= 0.0) || o.max_gn < 0 || o.max_pcg < 1 || o.armijo_max < 1 ||
        !(o.armijo_shrink > 0.0 && o.armijo_shrink < 1.0))
        return fail(c, REG_EINVAL, "bad solver options");
    REG_TRY(ensure_solver(c));
    reg_solve_stats local;
    memset(&local, 0, sizeof local);
    const int s = solve_impl(c, v_inout, &o, &local);
    if (stats) *stats = local;
    return s;
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
    float* v = c->sv[V_SPARE];
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
