// Context management, timing, the internal operations of the hot path and
// their C-ABI entry points.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>

#include "ctx.h"

namespace reg {

static thread_local std::string g_create_error;

static const double kTwoPi = 6.283185307179586476925286766559;

int fail(reg_ctx* c, int status, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return status;
}

int fail_cuda(reg_ctx* c, cudaError_t e, const char* what, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s [ctx.cu:%d]", (int)e,
             cudaGetErrorString(e), what, line);
    if (c) c->dead = true;
    return fail(c, REG_ECUDA, buf);
}

static int fail_fft(reg_ctx* c, cufftResult r, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "cuFFT error %d in %s", (int)r, what);
    return fail(c, REG_ECUFFT, buf);
}

// ----------------------------------------------------------------- timing

void phase_begin(reg_ctx* c, cudaEvent_t* ev) {
    *ev = nullptr;
    if (!c->timing) return;
    if (c->free_events.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->free_events.push_back(e);
    }
    *ev = c->free_events.back();
    c->free_events.pop_back();
    // inside a stream capture an ordinary record only orders streams; an
    // external record becomes an event node that fires on every replay
    if (c->capturing) cudaEventRecordWithFlags(*ev, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(*ev, c->stream);
}

void phase_end(reg_ctx* c, int phase, cudaEvent_t ev, double bytes) {
    if (!c->timing || !ev) return;
    if (c->free_events.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { c->free_events.push_back(ev); return; }
        c->free_events.push_back(e);
    }
    cudaEvent_t b = c->free_events.back();
    c->free_events.pop_back();
    if (c->capturing) cudaEventRecordWithFlags(b, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(b, c->stream);
    if (c->capturing) {
        c->graph_pairs.push_back({phase, ev, b, bytes});
        return;
    }
    c->pending.push_back({phase, ev, b, bytes});
    // keep the number of outstanding event pairs bounded
    if (c->pending.size() > 4096) {
        cudaEventSynchronize(b);
        for (auto& p : c->pending) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p.a, p.b);
            c->acc.ms[p.phase] += ms;
            c->acc.launches[p.phase] += 1;
            c->acc.bytes[p.phase] += p.bytes;
            c->free_events.push_back(p.a);
            c->free_events.push_back(p.b);
        }
        c->pending.clear();
    }
}

int harvest_graph_timing(reg_ctx* c) {
    for (auto& p : c->graph_pairs) {
        float ms = 0.f;
        REG_CK(c, cudaEventElapsedTime(&ms, p.a, p.b));
        c->acc.ms[p.phase] += ms;
        c->acc.launches[p.phase] += 1;
        c->acc.bytes[p.phase] += p.bytes;
    }
    return REG_OK;
}

void release_graph_timing(reg_ctx* c) {
    for (auto& p : c->graph_pairs) {
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->graph_pairs.clear();
}

// ------------------------------------------------------------- operations

int op_departure(reg_ctx* c, const float* v, float* d_fwd, float* d_adj, bool* maxed) {
    // the predictor's displacement dt v_j n_j / (2 pi) (grid units) is below
    // max |v| dt max_j n_j / (2 pi): its ceiling is the staged kernel's halo
    const int nmax = std::max(c->g.n1, std::max(c->g.n2, c->g.n3));
    int halo = 0;
    REG_TRY(op_halo(c, v, &halo, (float)(nmax / (c->nt * 6.283185307179586))));
    Phase p(c, REG_PH_DEPARTURE, (double)c->g.n * (d_adj ? 36.0 : 24.0));
    REG_CK(c, launch_departure(c->g, tile_with(c, halo), v, (float)(1.0 / c->nt), d_fwd, d_adj,
                               c->stream, maxed ? c->dabs : nullptr, maxed));
    return REG_OK;
}

// ceil(max |d|) from the bits of a float maximum (as op_halo).
static int halo_of(reg_ctx* c, unsigned int bits, int* halo) {
    float m;
    memcpy(&m, &bits, sizeof m);
    if (!std::isfinite(m)) return fail(c, REG_ENONFINITE, "non-finite displacement");
    *halo = m < 1e6f ? (int)std::ceil(m) : 1000000;
    return REG_OK;
}

int op_fft_r2c(reg_ctx* c, const float* in, float2* out, int ncomp) {
    Phase p(c, REG_PH_FFT, (double)ncomp * (4.0 * c->g.n + 8.0 * c->g.nc));
    cufftHandle h = ncomp == 3 ? c->r2c3 : c->r2c1;
    cufftResult r = cufftExecR2C(h, const_cast<cufftReal*>(in), reinterpret_cast<cufftComplex*>(out));
    if (r != CUFFT_SUCCESS) return fail_fft(c, r, "cufftExecR2C");
    return REG_OK;
}

int op_fft_c2r(reg_ctx* c, float2* in, float* out, int ncomp) {
    Phase p(c, REG_PH_FFT, (double)ncomp * (4.0 * c->g.n + 8.0 * c->g.nc));
    cufftHandle h = ncomp == 3 ? c->c2r3 : c->c2r1;
    cufftResult r = cufftExecC2R(h, reinterpret_cast<cufftComplex*>(in), out);
    if (r != CUFFT_SUCCESS) return fail_fft(c, r, "cufftExecC2R");
    return REG_OK;
}

int op_spectral(reg_ctx* c, SpecOp op, const SpecArgs& a, int nfields) {
    Phase p(c, REG_PH_SPECTRAL, 8.0 * nfields * c->g.nc);
    REG_CK(c, launch_spectral(c->g, op, a, c->stream));
    return REG_OK;
}

static SpecArgs spec_args(reg_ctx* c) {
    SpecArgs a;
    memset(&a, 0, sizeof a);
    a.beta = c->beta;
    a.kind = c->kind;
    a.project = c->incompressible;
    return a;
}

int op_grad(reg_ctx* c, const float* f, float* out3) {
    if (deriv_supported(c->g, f, out3)) {
        // one-dimensional transforms per axis: one read and one write each,
        // the three axes in one launch where the grid is cubic
        const long long n = c->g.n;
        const Dims& g = c->g;
        if (g.n1 == g.n2 && g.n1 == g.n3 && g.n1 >= 32 && g.n1 <= 256) {
            Phase p(c, REG_PH_DERIV, 24.0 * n);
            REG_CK(c, launch_grad(g, f, out3, c->stream));
            return REG_OK;
        }
        for (int ax = 0; ax < 3; ++ax) {
            Phase p(c, REG_PH_DERIV, 8.0 * n);
            REG_CK(c, launch_deriv(c->g, ax, f, out3 + ax * n, 0, c->stream));
        }
        return REG_OK;
    }
    REG_TRY(op_fft_r2c(c, f, c->spec[0], 1));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[1];
    REG_TRY(op_spectral(c, SPEC_GRAD, a, 4));
    return op_fft_c2r(c, c->spec[1], out3, 3);
}

int op_div(reg_ctx* c, const float* v3, float* out) {
    if (deriv_supported(c->g, v3, out)) {
        const long long n = c->g.n;
        for (int ax = 0; ax < 3; ++ax) {
            Phase p(c, REG_PH_DERIV, (ax ? 12.0 : 8.0) * n);
            REG_CK(c, launch_deriv(c->g, ax, v3 + ax * n, out, ax ? 1 : 0, c->stream));
        }
        return REG_OK;
    }
    REG_TRY(op_fft_r2c(c, v3, c->spec[0], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[1];
    REG_TRY(op_spectral(c, SPEC_DIV, a, 4));
    return op_fft_c2r(c, c->spec[1], out, 1);
}

int op_leray(reg_ctx* c, const float* v, float* out) {
    REG_TRY(op_fft_r2c(c, v, c->spec[0], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[0];
    REG_TRY(op_spectral(c, SPEC_LERAY, a, 6));
    return op_fft_c2r(c, c->spec[0], out, 3);
}

// dsc[slot] = (2 pi)^3 / n * <a, b>
int op_inner(reg_ctx* c, const float* a, const float* b, long long count, int slot) {
    const int nb = blas_blocks();
    {
        Phase p(c, REG_PH_BLAS, 8.0 * count);
        REG_CK(c, launch_dot_partials(a, b, count, c->partials, nb, c->stream));
    }
    Phase p(c, REG_PH_BLAS, 0.0);
    REG_CK(c, launch_finalize(c->partials, nb, kTwoPi * kTwoPi * kTwoPi / c->g.n,
                              c->dsc + slot, c->stream));
    return REG_OK;
}

int bind_stream(reg_ctx* c, cudaStream_t s) {
    c->stream = s;
    cufftHandle hs[4] = {c->r2c1, c->c2r1, c->r2c3, c->c2r3};
    for (int i = 0; i < 4; ++i) {
        cufftResult r = cufftSetStream(hs[i], s);
        if (r != CUFFT_SUCCESS) return fail_fft(c, r, "cufftSetStream");
    }
    return REG_OK;
}

int read_scalars(reg_ctx* c, int first, int count) {
    REG_CK(c, cudaMemcpyAsync(c->hsc + first, c->dsc + first, sizeof(double) * count,
                              cudaMemcpyDeviceToHost, c->stream));
    REG_CK(c, cudaStreamSynchronize(c->stream));
    return REG_OK;
}

int op_halo(reg_ctx* c, const float* d, int* halo, float scale) {
    REG_CK(c, launch_absmax(d, 3LL * c->g.n, c->dabs, c->stream));
    unsigned int bits = 0;
    REG_CK(c, cudaMemcpyAsync(&bits, c->dabs, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
    REG_CK(c, cudaStreamSynchronize(c->stream));
    float m;
    memcpy(&m, &bits, sizeof m);
    m *= scale;
    if (!std::isfinite(m)) return fail(c, REG_ENONFINITE, "non-finite displacement");
    *halo = m < 1e6f ? (int)std::ceil(m) : 1000000;
    return REG_OK;
}

// The configured tile with a halo; when its staged box does not fit in shared
// memory, halve k (down to 4) before falling back to the register window.
Tile tile_with(const reg_ctx* c, int halo) {
    Tile t = c->tile;
    t.halo = halo;
    // 16-row blocks exist only as the fixed-halo staged kernel (halo <= 3)
    if (t.wy == 16 && halo > 3) t.wy = 8;
    while (!tile_staged(t) && t.k > 4) t.k = ((t.k / 2) + 3) & ~3;
    if (!tile_staged(t)) {   // register-window kernel, configured tile
        t = c->tile;
        t.halo = halo;
        if (t.wy == 16) t.wy = 8;
        if (t.k < 4) t.k = 4;   // it marches in groups of four points
    }
    return t;
}

static const float* grad_level(reg_ctx* c, int j) {
    return c->grad_hist ? c->grad_hist + (long long)j * 3 * c->g.n : nullptr;
}


// Forward state solve (Eq. varopt:state).  keep_hist: all levels in hist
// [(nt+1) n]; otherwise hist holds two ping-pong levels.  The last step
// writes lam(1) = rho_R - rho(1) to lam_out (if not null) and the mismatch
// 1/2 ||rho(1) - rho_R||^2_h to dsc[SC_JMIS].
static int state_solve(reg_ctx* c, const float* d_fwd, int halo, float* hist, bool keep_hist,
                       float* lam_out) {
    const Dims& g = c->g;
    const long long n = g.n;
    const int nt = c->nt;
    if (c->precision == REG_MIXED_BF16 && c->img_bf) {
        Phase p(c, REG_PH_OTHER, 6.0 * n);
        REG_CK(c, launch_from_bf16(c->img_bf, hist, n, c->stream));
    } else {
        REG_CK(c, cudaMemcpyAsync(hist, c->rho_T, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                  c->stream));
    }
    int nb = 0;
    for (int j = 0; j < nt; ++j) {
        const float* in = keep_hist ? hist + j * n : hist + (j & 1) * n;
        float* out = keep_hist ? hist + (j + 1) * n : hist + ((j + 1) & 1) * n;
        const bool fin = (j == nt - 1);
        double bytes = 20.0 * n;
        if (fin) bytes += (lam_out ? 8.0 : 4.0) * n;
        Phase p(c, REG_PH_STATE, bytes);
        REG_CK(c, launch_state_step(g, tile_with(c, halo), in, d_fwd, out,
                                    fin ? c->rho_R : nullptr,
                                    fin ? lam_out : nullptr, c->partials, c->npartials, &nb,
                                    c->stream));
    }
    Phase p(c, REG_PH_BLAS, 0.0);
    REG_CK(c, launch_finalize(c->partials, nb, 0.5 * kTwoPi * kTwoPi * kTwoPi / n,
                              c->dsc + SC_JMIS, c->stream));
    return REG_OK;
}

// dsc[SC_JREG] = beta/2 <v, A v>_h from the spectrum of v (3 fields).
static int reg_energy(reg_ctx* c, const float2* vhat) {
    const int nb = blas_blocks();
    {
        Phase p(c, REG_PH_SPECTRAL, 24.0 * c->g.nc);
        REG_CK(c, launch_spec_energy(c->g, vhat, c->kind, c->partials, nb, c->stream));
    }
    const double n = c->g.n;
    Phase p(c, REG_PH_BLAS, 0.0);
    REG_CK(c, launch_finalize(c->partials, nb, 0.5 * c->beta * kTwoPi * kTwoPi * kTwoPi / (n * n),
                              c->dsc + SC_JREG, c->stream));
    return REG_OK;
}

int op_mismatch(reg_ctx* c, const float* v) {
    // scratch only: the linearisation point stays intact
    REG_TRY(op_departure(c, v, c->tmp3, nullptr));
    int halo;
    REG_TRY(op_halo(c, c->tmp3, &halo));
    float* ping = reinterpret_cast<float*>(c->buf[0]);   // 2n floats: two levels
    return state_solve(c, c->tmp3, halo, ping, false, nullptr);
}

int op_objective(reg_ctx* c, const float* v, int slot_J) {
    (void)slot_J;
    REG_TRY(op_mismatch(c, v));
    REG_TRY(op_fft_r2c(c, v, c->spec[0], 3));
    return reg_energy(c, c->spec[0]);
}

// Adjoint (or incremental adjoint) solve from levels[nt] = lam(1), fused
// with the trapezoid time integral of Eq. gradient / Eq. inc-control: every
// tau-step stores lam_j (except the last, unless keep_all) and accumulates
// b = sum_j w_j lam_j grad rho_j into out at its output points; with dotp,
// dsc[slot] = <dotp, b>_h.  src_vt (full Newton incremental adjoint,
// Eq. inc-adj): the equation carries the known source s_j = div(lam_j v~)
// with lam_j the adjoint levels of the linearisation point (lam_lin); each
// step then adds dt/2 (1 + dt dv) I[s_{j+1}](X) + dt/2 s_j(x).
Fin finish_into(reg_ctx* c, double scale, int slot0, int slot1, int copy_from, int copy_to) {
    Fin f;
    f.count = c->gsync + 2;
    f.sc = c->dsc;
    f.scale = scale;
    f.out[0] = slot0;
    f.out[1] = slot1;
    f.out[2] = 0;
    f.copy_from = copy_from;
    f.copy_to = copy_to;
    return f;
}

static int adjoint_solve(reg_ctx* c, int phase, float* levels, bool keep_all,
                         const float* src_vt, float* out, const float* dotp, int slot) {
    const long long n = c->g.n;
    const int nt = c->nt;
    const bool comp = !c->incompressible;
    const float dt = 1.f / (float)nt;
    float* sbuf[2] = {reinterpret_cast<float*>(c->buf[0]),
                      reinterpret_cast<float*>(c->buf[0]) + n};
    float* add = reinterpret_cast<float*>(c->buf[1]);
    // s_j = div(lam_j v~) into sbuf[j & 1]
    auto source_level = [&](int j) -> int {
        {
            Phase p(c, phase, 28.0 * n);
            REG_CK(c, launch_mul_fields(c->lam_lin + j * n, src_vt, c->tmp3, n, c->stream));
        }
        return op_div(c, c->tmp3, sbuf[j & 1]);
    };
    if (src_vt) REG_TRY(source_level(nt));
    int nb = 0;
    for (int j = nt - 1; j >= 0; --j) {
        const bool first = (j == nt - 1), last = (j == 0);
        const float w = last ? 0.5f * dt : dt;
        if (src_vt) {
            REG_TRY(source_level(j));
            Phase p(c, phase, (comp ? 24.0 : 20.0) * n);
            REG_CK(c, launch_source_step(c->g, tile_with(c, c->halo_adj), sbuf[(j + 1) & 1],
                                         c->d_adj, comp ? c->divv : nullptr, sbuf[j & 1], dt, add,
                                         c->stream));
        }
        // X 12, lam 4, c 4, lam_j 4 (not after the last step); grad_j 12; b
        // written 12 and read 12 (first step: lam(1) 4 and grad rho(1) 12
        // instead); dotp 12; the source part 4
        const bool store = !last || keep_all;
        double bytes = (comp ? 20.0 : 16.0) + (store ? 4.0 : 0.0) + 24.0 +
                       (first ? 16.0 : 12.0) + (last && dotp ? 12.0 : 0.0) +
                       (src_vt ? 4.0 : 0.0);
        // the last step finishes <dotp, b> into dsc[slot] itself
        const Fin fin = finish_into(c, kTwoPi * kTwoPi * kTwoPi / n, slot);
        Phase p(c, phase, bytes * n);
        REG_CK(c, launch_adjoint_acc(c->g, tile_with(c, c->halo_adj), levels + (j + 1) * n,
                                     c->d_adj, comp ? c->coef : nullptr,
                                     store ? levels + j * n : nullptr, grad_level(c, j), w,
                                     out, first ? levels + nt * n : nullptr,
                                     first ? grad_level(c, nt) : nullptr, 0.5f * dt,
                                     last ? dotp : nullptr, c->partials, c->npartials, &nb,
                                     c->stream, src_vt ? add : nullptr, &fin));
    }
    return REG_OK;
}

// The points of v and -v, their halos and the state history of v (with
// lam(1) and the mismatch) in the linearisation buffers.
static int state_of(reg_ctx* c, const float* v) {
    // the tensor-copy departure kernel leaves both fields' maxima in dabs:
    // one wait for the two halos instead of two reductions and two waits
    bool maxed = false;
    REG_TRY(op_departure(c, v, c->d_fwd, c->d_adj, &maxed));
    if (maxed) {
        unsigned int bits[2] = {0u, 0u};
        REG_CK(c, cudaMemcpyAsync(bits, c->dabs, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
        REG_CK(c, cudaStreamSynchronize(c->stream));
        REG_TRY(halo_of(c, bits[0], &c->halo_fwd));
        REG_TRY(halo_of(c, bits[1], &c->halo_adj));
    } else {
        REG_TRY(op_halo(c, c->d_fwd, &c->halo_fwd));
        REG_TRY(op_halo(c, c->d_adj, &c->halo_adj));
    }
    return state_solve(c, c->d_fwd, c->halo_fwd, c->rho_hist, true,
                       c->lam_hist + (long long)c->nt * c->g.n);
}

int op_trial_state(reg_ctx* c, const float* v) {
    c->have_lin = false;
    return state_of(c, v);
}

int op_linearize(reg_ctx* c, const float* v, bool state_ready, const float2* v_hat) {
    const Dims& g = c->g;
    const long long n = g.n;
    const int nt = c->nt;
    const bool comp = !c->incompressible;
    c->have_lin = false;
    // points, halos, state history, lam(1) = rho_R - rho(1) and the mismatch
    if (!state_ready) REG_TRY(state_of(c, v));
    if (comp) {
        if (v_hat && !deriv_supported(g, v, c->divv)) {
            SpecArgs a = spec_args(c);
            a.in_a = v_hat;
            a.out = c->spec[1];
            a.normalised = 1;
            REG_TRY(op_spectral(c, SPEC_DIV, a, 4));
            REG_TRY(op_fft_c2r(c, c->spec[1], c->divv, 1));
        } else {
            REG_TRY(op_div(c, v, c->divv));
        }
        Phase p(c, REG_PH_ADJOINT, 20.0 * n);
        REG_CK(c, launch_adjoint_coef(g, tile_with(c, c->halo_adj), c->divv, c->d_adj,
                                      (float)(1.0 / nt), c->coef, c->stream));
    }
    // spectral gradients of every level (cached for the matvecs); level 0 is
    // rho_T whatever v is, so its gradient is kept across linearisations
    for (int j = c->grad0_valid ? 1 : 0; j <= nt; ++j) {
        float* gj = c->grad_hist + (long long)j * 3 * n;
        REG_TRY(op_grad(c, c->rho_hist + j * n, gj));
    }
    c->grad0_valid = true;
    if (c->hessian == REG_HESS_FULL_NEWTON) {
        // the full Newton matvec needs every adjoint level of this point
        REG_CK(c, cudaMemcpyAsync(c->lam_lin + nt * n, c->lam_hist + nt * n, sizeof(float) * n,
                                  cudaMemcpyDeviceToDevice, c->stream));
        REG_TRY(adjoint_solve(c, REG_PH_ADJOINT, c->lam_lin, true, nullptr, c->bacc, nullptr, 0));
    } else {
        REG_TRY(adjoint_solve(c, REG_PH_ADJOINT, c->lam_hist, false, nullptr, c->bacc, nullptr,
                              0));
    }
    c->have_lin = true;
    return REG_OK;
}

int op_gradient(reg_ctx* c, const float* v, float* gout, int slot_J) {
    (void)slot_J;
    REG_TRY(op_linearize(c, v));
    c->have_lin = false;
    // g = beta A v + P b
    REG_TRY(op_fft_r2c(c, v, c->spec[0], 3));
    REG_TRY(reg_energy(c, c->spec[0]));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.in_b = c->spec[1];
    a.out = c->spec[1];
    REG_TRY(op_spectral(c, SPEC_ASSEMBLE, a, 9));
    REG_TRY(op_fft_c2r(c, c->spec[1], gout, 3));
    c->have_lin = true;
    return REG_OK;
}

int op_matvec_transport(reg_ctx* c, const float* vt, const float* dotp, int slot) {
    const Dims& g = c->g;
    const long long n = g.n;
    const int nt = c->nt;
    const float dt = (float)(1.0 / nt);
    const double gb = 12.0;
    const bool full = c->hessian == REG_HESS_FULL_NEWTON;
    // Gauss-Newton: the carried incremental state u_j in two ping-pong
    // levels; full Newton: every level u_0 .. u_{nt-1} (for grad rho~_j)
    float* u[2] = {reinterpret_cast<float*>(c->buf[0]), reinterpret_cast<float*>(c->buf[1])};
    auto level = [&](int j) { return full ? c->rt_hist + j * n : u[j & 1]; };
    // small grids (the two-level preconditioner's coarse grid): the whole
    // sequence in one persistent launch, where its sum <dotp, b~> is read
    if (!full && dotp && c->persistent && n <= (1LL << 18)) {
        int nb = 0;
        cudaError_t e;
        {
            Phase p(c, REG_PH_INCADJ, (16.0 + gb + nt * (32.0 + gb) + nt * 60.0 + 12.0) * n);
            e = launch_matvec_persistent(g, c->halo_fwd, c->halo_adj, nt, dt, vt, c->grad_hist,
                                         c->d_fwd, c->d_adj,
                                         c->incompressible ? nullptr : c->coef, u[0], u[1],
                                         c->lam_hist, c->bacc, dotp, c->partials, c->npartials,
                                         c->gsync, reinterpret_cast<int*>(c->gsync + 1), &nb,
                                         c->stream);
        }
        if (e == cudaSuccess) {
            Phase p(c, REG_PH_BLAS, 0.0);
            REG_CK(c, launch_finalize(c->partials, nb, kTwoPi * kTwoPi * kTwoPi / n,
                                      c->dsc + slot, c->stream));
            return REG_OK;
        }
        // not for this launch (halo > 3) or refused: the steps one by one
        cudaGetLastError();
        if (e != cudaErrorNotSupported) c->persistent = false;
    }
    {
        Phase p(c, REG_PH_INCSTATE, (16.0 + gb) * n);
        REG_CK(c, launch_incstate_init(g, vt, grad_level(c, 0), dt, level(0), c->stream));
    }
    for (int j = 0; j < nt; ++j) {
        const bool fin = (j == nt - 1);
        Phase p(c, REG_PH_INCSTATE, (32.0 + gb) * n);
        REG_CK(c, launch_incstate_step(g, tile_with(c, c->halo_fwd), level(j), c->d_fwd, vt,
                                       grad_level(c, j + 1), dt, fin ? 1 : 0,
                                       fin ? c->lam_hist + nt * n : level(j + 1), c->stream));
    }
    if (!full) return adjoint_solve(c, REG_PH_INCADJ, c->lam_hist, false, nullptr, c->bacc, dotp,
                                    slot);
    // full Newton (Eq. inc-adj with div(lam v~); b~ += int lam grad rho~ dt)
    REG_TRY(adjoint_solve(c, REG_PH_INCADJ, c->lam_hist, false, vt, c->bacc, nullptr, 0));
    float* rt = reinterpret_cast<float*>(c->buf[0]);
    for (int j = 1; j <= nt; ++j) {
        const float w = (j == nt) ? 0.5f * dt : dt;
        const float* f = rt;
        float wj = w;
        if (j < nt) {
            Phase p(c, REG_PH_INCADJ, 20.0 * n);
            REG_CK(c, launch_inc_state_level(g, level(j), vt, grad_level(c, j), dt, rt,
                                             c->stream));
        } else {
            f = c->lam_hist + nt * n;   // rho~(1) = -lam~(1)
            wj = -w;
        }
        REG_TRY(op_grad(c, f, c->tmp3));
        Phase p(c, REG_PH_INCADJ, 28.0 * n);
        REG_CK(c, launch_acc_scaled_grad(g, c->lam_lin + j * n, c->tmp3, wj, c->bacc, c->stream));
    }
    if (dotp) REG_TRY(op_inner(c, dotp, c->bacc, 3 * n, slot));
    return REG_OK;
}

int op_matvec(reg_ctx* c, const float* vt, float* out) {
    REG_TRY(op_matvec_transport(c, vt, nullptr, 0));
    REG_TRY(op_fft_r2c(c, vt, c->spec[0], 3));
    REG_TRY(op_fft_r2c(c, c->bacc, c->spec[1], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.in_b = c->spec[1];
    a.out = c->spec[1];
    REG_TRY(op_spectral(c, SPEC_ASSEMBLE, a, 9));
    return op_fft_c2r(c, c->spec[1], out, 3);
}

int op_precond(reg_ctx* c, const float* r, float* z) {
    REG_TRY(op_fft_r2c(c, r, c->spec[0], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[0];
    REG_TRY(op_spectral(c, SPEC_PRECOND, a, 6));
    return op_fft_c2r(c, c->spec[0], z, 3);
}

int ensure_solver(reg_ctx* c) {
    if (c->have_solver) return REG_OK;
    const size_t rb = sizeof(float) * 3 * (size_t)c->g.n;
    const size_t sb = sizeof(float2) * 3 * (size_t)c->g.nc;
    bool ok = true;
    for (int i = 0; i < 4 && ok; ++i) ok = cudaMalloc(&c->sv[i], rb) == cudaSuccess;
    for (int i = 0; i < 8 && ok; ++i) ok = cudaMalloc(&c->ss[i], sb) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (int i = 0; i < 4; ++i) { if (c->sv[i]) cudaFree(c->sv[i]); c->sv[i] = nullptr; }
        for (int i = 0; i < 8; ++i) { if (c->ss[i]) cudaFree(c->ss[i]); c->ss[i] = nullptr; }
        return fail(c, REG_ENOMEM, "cannot allocate solver vectors");
    }
    c->have_solver = true;
    return REG_OK;
}

}  // namespace reg

// ====================================================================== C-ABI

using namespace reg;

#define CHECK_CTX(c)                                                         \
    do {                                                                     \
        if (!(c)) return REG_EINVAL;                                         \
        if ((c)->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error"); \
    } while (0)

#define CHECK_PTR(c, p)                                                      \
    do {                                                                     \
        if (!(p)) return fail(c, REG_EINVAL, "null pointer: " #p);           \
        if (((uintptr_t)(p)) & 15u) return fail(c, REG_EINVAL, "pointer not 16-byte aligned: " #p); \
    } while (0)

static void free_ctx(reg_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int i = 0; i < 4; ++i)
        if (c->plans[i]) cufftDestroy(i == 0 ? c->r2c1 : i == 1 ? c->c2r1 : i == 2 ? c->r2c3 : c->c2r3);
    void* ptrs[] = {c->rho_T, c->rho_R, c->img_bf, c->d_fwd, c->d_adj, c->divv, c->rho_hist,
                    c->grad_hist, c->lam_hist, c->coef, c->buf[0], c->buf[1],
                    c->bacc, c->tmp3, c->spec[0], c->spec[1], c->partials, c->dsc, c->dabs,
                    c->gsync, c->lam_lin, c->rt_hist};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < 4; ++i)
        if (c->sv[i]) cudaFree(c->sv[i]);
    for (int i = 0; i < 9; ++i)
        if (c->ss[i]) cudaFree(c->ss[i]);
    if (c->coarse) free_ctx(c->coarse);
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    for (auto& p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto& p : c->graph_pairs) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : c->free_events) cudaEventDestroy(e);
    delete c;
}

// Host-side fault injection (reg_debug_inject): the armed kind fires at its
// (after + 1)-th event and disarms.
static std::atomic<int> g_inject_what{REG_INJECT_NONE};
static std::atomic<int> g_inject_left{0};

static bool inject_fires(int what) {
    if (g_inject_what.load() != what) return false;
    if (g_inject_left.fetch_sub(1) > 0) return false;
    g_inject_what.store(REG_INJECT_NONE);
    return true;
}

static int alloc_grad_hist(reg_ctx* c) {
    const size_t cnt = (size_t)(c->nt + 1) * 3 * c->g.n;
    if (c->grad_hist) { cudaFree(c->grad_hist); c->grad_hist = nullptr; }
    const cudaError_t e = cudaMalloc(&c->grad_hist, cnt * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, REG_ENOMEM, "cannot allocate the grad rho cache");
    }
    return REG_OK;
}

extern "C" {

int reg_create(int n1, int n2, int n3, int nt, double beta, int reg_kind, int incompressible,
               reg_ctx** out) {
    if (!out) return fail(nullptr, REG_EINVAL, "out is NULL");
    *out = nullptr;
    if (n1 < 4 || n2 < 4 || n3 < 4)
        return fail(nullptr, REG_EINVAL, "grid sizes must be >= 4");
    if ((long long)n1 * n2 * n3 > (1LL << 30))
        return fail(nullptr, REG_EINVAL, "grid larger than 2^30 points");
    if (nt < 1 || nt > 64) return fail(nullptr, REG_EINVAL, "nt must be in [1, 64]");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(nullptr, REG_EINVAL, "beta must be > 0");
    if (reg_kind != REG_H1 && reg_kind != REG_H2 && reg_kind != REG_H1DIV)
        return fail(nullptr, REG_EINVAL, "unknown reg_kind");
    reg_ctx* c = new (std::nothrow) reg_ctx();
    if (!c) return fail(nullptr, REG_ENOMEM, "host allocation failed");
    c->g = make_dims(n1, n2, n3);
    c->nt = nt;
    c->beta = beta;
    c->kind = reg_kind;
    c->incompressible = incompressible ? 1 : 0;
    c->precision = REG_FP32;
    c->stream = nullptr;
    const long long n = c->g.n;
    const long long nc = c->g.nc;
    c->tile.k = 8;
    c->tile.wy = 8;
    c->halo_fwd = c->halo_adj = -1;
    c->persistent = false;
    // partial sums: the largest marching grid (k = 4, wy = 1), or up to
    // kMaxSlots partial-sum slots of the BLAS / spectral grid
    c->npartials = march_blocks(c->g, Tile{4, 1});
    if (c->npartials < kMaxSlots * blas_blocks()) c->npartials = kMaxSlots * blas_blocks();
    struct A { void** p; size_t bytes; } allocs[] = {
        {(void**)&c->rho_T, sizeof(float) * n},
        {(void**)&c->rho_R, sizeof(float) * n},
        {(void**)&c->d_fwd, sizeof(float) * 3 * n},
        {(void**)&c->d_adj, sizeof(float) * 3 * n},
        {(void**)&c->divv, sizeof(float) * n},
        {(void**)&c->rho_hist, sizeof(float) * (nt + 1) * n},
        {(void**)&c->lam_hist, sizeof(float) * (nt + 1) * n},
        {(void**)&c->coef, sizeof(float) * n},
        {(void**)&c->buf[0], sizeof(float2) * n},
        {(void**)&c->buf[1], sizeof(float2) * n},
        {(void**)&c->bacc, sizeof(float) * 3 * n},
        {(void**)&c->tmp3, sizeof(float) * 3 * n},
        {(void**)&c->spec[0], sizeof(float2) * 3 * nc},
        {(void**)&c->spec[1], sizeof(float2) * 3 * nc},
        {(void**)&c->partials, sizeof(double) * c->npartials},
        {(void**)&c->dsc, sizeof(double) * 32},
        {(void**)&c->dabs, sizeof(unsigned int) * 4},
        {(void**)&c->gsync, sizeof(unsigned int) * 4},
    };
    for (auto& a : allocs) {
        if (inject_fires(REG_INJECT_ALLOC) || cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return fail(nullptr, REG_ENOMEM, "device allocation failed in reg_create");
        }
    }
    if (cudaMallocHost(&c->hsc, sizeof(double) * 32) != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return fail(nullptr, REG_ENOMEM, "pinned host allocation failed");
    }
    if (alloc_grad_hist(c) != REG_OK) {
        free_ctx(c);
        return fail(nullptr, REG_ENOMEM, "cannot allocate the grad rho cache");
    }
    cudaMemset(c->dsc, 0, sizeof(double) * 32);
    cudaMemset(c->gsync, 0, sizeof(unsigned int) * 4);   // barrier, error flag, finish ticket
    int dims[3] = {n1, n2, n3};
    cufftResult r;
    r = inject_fires(REG_INJECT_CUFFT_PLAN)
                ? CUFFT_ALLOC_FAILED
                : cufftPlanMany(&c->r2c1, 3, dims, nullptr, 1, (int)n, nullptr, 1, (int)nc, CUFFT_R2C, 1);
    c->plans[0] = (r == CUFFT_SUCCESS);
    if (r == CUFFT_SUCCESS) {
        r = inject_fires(REG_INJECT_CUFFT_PLAN)
                ? CUFFT_ALLOC_FAILED
                : cufftPlanMany(&c->c2r1, 3, dims, nullptr, 1, (int)nc, nullptr, 1, (int)n, CUFFT_C2R, 1);
        c->plans[1] = (r == CUFFT_SUCCESS);
    }
    if (r == CUFFT_SUCCESS) {
        r = inject_fires(REG_INJECT_CUFFT_PLAN)
                ? CUFFT_ALLOC_FAILED
                : cufftPlanMany(&c->r2c3, 3, dims, nullptr, 1, (int)n, nullptr, 1, (int)nc, CUFFT_R2C, 3);
        c->plans[2] = (r == CUFFT_SUCCESS);
    }
    if (r == CUFFT_SUCCESS) {
        r = inject_fires(REG_INJECT_CUFFT_PLAN)
                ? CUFFT_ALLOC_FAILED
                : cufftPlanMany(&c->c2r3, 3, dims, nullptr, 1, (int)nc, nullptr, 1, (int)n, CUFFT_C2R, 3);
        c->plans[3] = (r == CUFFT_SUCCESS);
    }
    if (r != CUFFT_SUCCESS) {
        free_ctx(c);
        char buf[128];
        snprintf(buf, sizeof buf, "cufftPlanMany failed (%d)", (int)r);
        return fail(nullptr, REG_ECUFFT, buf);
    }
    if (cudaStreamCreate(&c->capture_stream) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_ctx(c);
        return fail(nullptr, REG_ECUDA, "CUDA error during reg_create");
    }
    *out = c;
    return REG_OK;
}

int reg_destroy(reg_ctx* c) {
    free_ctx(c);
    return REG_OK;
}

const char* reg_last_error(const reg_ctx* c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

const char* reg_status_string(int s) {
    switch (s) {
    case REG_OK: return "REG_OK";
    case REG_EINVAL: return "REG_EINVAL";
    case REG_ENOMEM: return "REG_ENOMEM";
    case REG_ECUDA: return "REG_ECUDA";
    case REG_ECUFFT: return "REG_ECUFFT";
    case REG_ENOTREADY: return "REG_ENOTREADY";
    case REG_ENONFINITE: return "REG_ENONFINITE";
    case REG_EMAXITER: return "REG_EMAXITER";
    case REG_ENOTIMPL: return "REG_ENOTIMPL";
    default: return "unknown status";
    }
}

int reg_set_stream(reg_ctx* c, void* stream) {
    CHECK_CTX(c);
    return bind_stream(c, (cudaStream_t)stream);
}

int reg_set_precision(reg_ctx* c, int precision) {
    CHECK_CTX(c);
    if (precision != REG_FP32 && precision != REG_MIXED_BF16)
        return fail(c, REG_EINVAL, "unknown precision");
    if (precision == c->precision) return REG_OK;
    REG_CK(c, cudaStreamSynchronize(c->stream));
    c->precision = precision;
    c->have_lin = false;
    c->grad0_valid = false;
    c->have_images = false;
    if (precision == REG_MIXED_BF16 && !c->img_bf) {
        if (cudaMalloc(&c->img_bf, sizeof(__nv_bfloat16) * 2 * c->g.n) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, REG_ENOMEM, "cannot allocate bf16 images");
        }
    }
    return REG_OK;
}

int reg_set_persistent(reg_ctx* c, int on) {
    CHECK_CTX(c);
    if (on != 0 && on != 1) return fail(c, REG_EINVAL, "persistent: 0 or 1");
    c->persistent = on != 0;
    if (c->pcg_exec) {   // the captured PCG loop holds the other launch sequence
        cudaGraphExecDestroy(c->pcg_exec);
        c->pcg_exec = nullptr;
    }
    return REG_OK;
}

int reg_set_hessian(reg_ctx* c, int hessian) {
    CHECK_CTX(c);
    if (hessian != REG_HESS_GAUSS_NEWTON && hessian != REG_HESS_FULL_NEWTON)
        return fail(c, REG_EINVAL, "hessian must be REG_HESS_GAUSS_NEWTON or REG_HESS_FULL_NEWTON");
    if (hessian == c->hessian) return REG_OK;
    REG_CK(c, cudaStreamSynchronize(c->stream));
    if (hessian == REG_HESS_FULL_NEWTON && !c->lam_lin) {
        const size_t n = (size_t)c->g.n;
        if (cudaMalloc(&c->lam_lin, sizeof(float) * (c->nt + 1) * n) != cudaSuccess ||
            cudaMalloc(&c->rt_hist, sizeof(float) * c->nt * n) != cudaSuccess) {
            cudaGetLastError();
            if (c->lam_lin) cudaFree(c->lam_lin);
            if (c->rt_hist) cudaFree(c->rt_hist);
            c->lam_lin = c->rt_hist = nullptr;
            return fail(c, REG_ENOMEM, "cannot allocate the full Newton levels");
        }
    }
    c->hessian = hessian;
    c->have_lin = false;   // the adjoint levels are kept only by the next gradient
    return REG_OK;
}

int reg_set_images(reg_ctx* c, const float* rho_T, const float* rho_R, int presmooth) {
    CHECK_CTX(c);
    CHECK_PTR(c, rho_T);
    CHECK_PTR(c, rho_R);
    const long long n = c->g.n;
    c->have_lin = false;
    c->grad0_valid = false;
    c->img_version++;
    if (rho_T != c->rho_T)
        REG_CK(c, cudaMemcpyAsync(c->rho_T, rho_T, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                  c->stream));
    if (rho_R != c->rho_R)
        REG_CK(c, cudaMemcpyAsync(c->rho_R, rho_R, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                  c->stream));
    if (presmooth) {
        const double h1 = kTwoPi / c->g.n1, h2 = kTwoPi / c->g.n2, h3 = kTwoPi / c->g.n3;
        for (int k = 0; k < 2; ++k) {
            float* f = k == 0 ? c->rho_T : c->rho_R;
            REG_TRY(op_fft_r2c(c, f, c->spec[0], 1));
            SpecArgs a = spec_args(c);
            a.in_a = c->spec[0];
            a.out = c->spec[0];
            a.s1 = (float)h1; a.s2 = (float)h2; a.s3 = (float)h3;
            REG_TRY(op_spectral(c, SPEC_GAUSS, a, 2));
            REG_TRY(op_fft_c2r(c, c->spec[0], f, 1));
        }
    }
    if (c->precision == REG_MIXED_BF16) {
        // images are kept in bfloat16: round both, and use the rounded values
        REG_CK(c, launch_to_bf16(c->rho_T, c->img_bf, n, c->stream));
        REG_CK(c, launch_to_bf16(c->rho_R, c->img_bf + n, n, c->stream));
        REG_CK(c, launch_from_bf16(c->img_bf + n, c->rho_R, n, c->stream));
    }
    if (inject_fires(REG_INJECT_NAN_IMAGE)) {
        // all-ones bits: a NaN in FP32 and in bfloat16
        REG_CK(c, cudaMemsetAsync(c->rho_T, 0xFF, sizeof(float), c->stream));
        if (c->img_bf) REG_CK(c, cudaMemsetAsync(c->img_bf, 0xFF, sizeof(__nv_bfloat16), c->stream));
    }
    c->have_images = true;
    return REG_OK;
}

int reg_objective(reg_ctx* c, const float* v, double* J) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    if (!J) return fail(c, REG_EINVAL, "J is NULL");
    if (!c->have_images) return fail(c, REG_ENOTREADY, "reg_set_images first");
    REG_TRY(op_objective(c, v, SC_J));
    REG_TRY(read_scalars(c, SC_JMIS, 2));
    *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
    if (!std::isfinite(*J)) return fail(c, REG_ENONFINITE, "objective is not finite");
    return REG_OK;
}

int reg_gradient(reg_ctx* c, const float* v, float* g, double* J) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, g);
    if (v == g) return fail(c, REG_EINVAL, "v and g overlap");
    if (!c->have_images) return fail(c, REG_ENOTREADY, "reg_set_images first");
    REG_TRY(op_gradient(c, v, g, SC_J));
    if (J) {
        REG_TRY(read_scalars(c, SC_JMIS, 2));
        *J = c->hsc[SC_JMIS] + c->hsc[SC_JREG];
        if (!std::isfinite(*J)) return fail(c, REG_ENONFINITE, "objective is not finite");
    }
    return REG_OK;
}

int reg_hessian_matvec(reg_ctx* c, const float* vt, float* Hvt) {
    CHECK_CTX(c);
    CHECK_PTR(c, vt);
    CHECK_PTR(c, Hvt);
    if (vt == Hvt) return fail(c, REG_EINVAL, "vt and Hvt overlap");
    if (!c->have_lin) return fail(c, REG_ENOTREADY, "reg_gradient must come first");
    return op_matvec(c, vt, Hvt);
}

int reg_precond_apply(reg_ctx* c, const float* r, float* z) {
    CHECK_CTX(c);
    CHECK_PTR(c, r);
    CHECK_PTR(c, z);
    return op_precond(c, r, z);
}

int reg_departure(reg_ctx* c, const float* v, float* d_fwd, float* d_adj) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, d_fwd);
    CHECK_PTR(c, d_adj);
    return op_departure(c, v, d_fwd, d_adj);
}

int reg_deformation(reg_ctx* c, const float* v, float* u) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, u);
    if (u == v) return fail(c, REG_EINVAL, "v and u overlap");
    const long long n = c->g.n;
    c->have_lin = false;   // d_fwd / d_adj are overwritten
    REG_TRY(op_departure(c, v, c->d_fwd, c->d_adj));
    // ping-pong between u and tmp3 so that the last step writes u
    float* bufs[2] = {u, c->tmp3};
    const int nt = c->nt;
    float* first_in = bufs[nt % 2];
    REG_CK(c, cudaMemsetAsync(first_in, 0, sizeof(float) * 3 * n, c->stream));
    for (int j = 0; j < nt; ++j) {
        const float* in = bufs[(nt - j) % 2];
        float* out = bufs[(nt - 1 - j) % 2];
        Phase p(c, REG_PH_OTHER, 12.0 * 3 * n);
        REG_CK(c, launch_deformation_step(c->g, in, v, c->d_fwd, (float)(1.0 / nt), out,
                                          c->stream));
    }
    return REG_OK;
}

int reg_jacobian_det(reg_ctx* c, const float* u, float* det) {
    CHECK_CTX(c);
    CHECK_PTR(c, u);
    CHECK_PTR(c, det);
    if (c->nt < 2) return fail(c, REG_ENOTIMPL, "reg_jacobian_det needs nt >= 2 (scratch space)");
    const long long n = c->g.n;
    c->have_lin = false;   // the grad rho cache holds the derivatives
    c->grad0_valid = false;
    float* gu = c->grad_hist;   // (nt + 1) 3n >= 9n floats
    for (int comp = 0; comp < 3; ++comp) REG_TRY(op_grad(c, u + comp * n, gu + comp * 3 * n));
    Phase p(c, REG_PH_OTHER, 40.0 * n);
    REG_CK(c, launch_jacobian_det(gu, det, n, c->stream));
    return REG_OK;
}

int reg_interp(reg_ctx* c, const float* field, int nfields, const float* disp, float* out) {
    CHECK_CTX(c);
    CHECK_PTR(c, field);
    CHECK_PTR(c, disp);
    CHECK_PTR(c, out);
    if (nfields < 1 || nfields > 3) return fail(c, REG_EINVAL, "nfields must be 1..3");
    const long long n = c->g.n;
    int halo;
    REG_TRY(op_halo(c, disp, &halo));
    for (int k = 0; k < nfields; ++k) {
        Phase p(c, REG_PH_INTERP, 20.0 * n);
        REG_CK(c, launch_interp(c->g, tile_with(c, halo), field + k * n, disp, out + k * n,
                                c->stream));
    }
    return REG_OK;
}

int reg_state_transport(reg_ctx* c, const float* rho0, const float* d_fwd, float* rho_hist) {
    CHECK_CTX(c);
    CHECK_PTR(c, rho0);
    CHECK_PTR(c, d_fwd);
    CHECK_PTR(c, rho_hist);
    const long long n = c->g.n;
    int halo;
    REG_TRY(op_halo(c, d_fwd, &halo));
    REG_CK(c, cudaMemcpyAsync(rho_hist, rho0, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                              c->stream));
    for (int j = 0; j < c->nt; ++j) {
        Phase p(c, REG_PH_STATE, 20.0 * n);
        REG_CK(c, launch_state_step(c->g, tile_with(c, halo), rho_hist + j * n, d_fwd,
                                    rho_hist + (j + 1) * n, nullptr, nullptr, nullptr, 0, nullptr,
                                    c->stream));
    }
    return REG_OK;
}

// [a, a + na) and [b, b + nb) share an element.
static bool ranges_overlap(const float* a, long long na, const float* b, long long nb) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(a), b0 = reinterpret_cast<uintptr_t>(b);
    return a0 < b0 + sizeof(float) * nb && b0 < a0 + sizeof(float) * na;
}

int reg_spectral_grad(reg_ctx* c, const float* f, float* grad) {
    CHECK_CTX(c);
    CHECK_PTR(c, f);
    CHECK_PTR(c, grad);
    if (ranges_overlap(f, c->g.n, grad, 3LL * c->g.n))
        return fail(c, REG_EINVAL, "f and grad overlap");
    return op_grad(c, f, grad);
}

int reg_spectral_div(reg_ctx* c, const float* v, float* div) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, div);
    if (ranges_overlap(v, 3LL * c->g.n, div, c->g.n))
        return fail(c, REG_EINVAL, "v and div overlap");
    return op_div(c, v, div);
}

int reg_leray(reg_ctx* c, const float* v, float* pv) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, pv);
    return op_leray(c, v, pv);
}

int reg_apply_regularisation(reg_ctx* c, const float* v, float* av) {
    CHECK_CTX(c);
    CHECK_PTR(c, v);
    CHECK_PTR(c, av);
    REG_TRY(op_fft_r2c(c, v, c->spec[0], 3));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[0];
    REG_TRY(op_spectral(c, SPEC_REG, a, 6));
    return op_fft_c2r(c, c->spec[0], av, 3);
}

int reg_gaussian_smooth(reg_ctx* c, const float* f, float* out, double s1, double s2, double s3) {
    CHECK_CTX(c);
    CHECK_PTR(c, f);
    CHECK_PTR(c, out);
    REG_TRY(op_fft_r2c(c, f, c->spec[0], 1));
    SpecArgs a = spec_args(c);
    a.in_a = c->spec[0];
    a.out = c->spec[0];
    a.s1 = (float)s1; a.s2 = (float)s2; a.s3 = (float)s3;
    REG_TRY(op_spectral(c, SPEC_GAUSS, a, 2));
    return op_fft_c2r(c, c->spec[0], out, 1);
}

int reg_inner(reg_ctx* c, const float* a, const float* b, size_t count, double* out) {
    CHECK_CTX(c);
    CHECK_PTR(c, a);
    CHECK_PTR(c, b);
    if (!out) return fail(c, REG_EINVAL, "out is NULL");
    if (count == 0 || count % (size_t)c->g.n)
        return fail(c, REG_EINVAL, "count must be a positive multiple of n");
    REG_TRY(op_inner(c, a, b, (long long)count, SC_INNER));
    REG_TRY(read_scalars(c, SC_INNER, 1));
    *out = c->hsc[SC_INNER];
    if (!std::isfinite(*out)) return fail(c, REG_ENONFINITE, "inner product is not finite");
    return REG_OK;
}

int reg_set_tile(reg_ctx* c, int k, int wy) {
    CHECK_CTX(c);
    const bool kok = (k == 1 || k == 2) ? wy * k >= 4 : (k >= 4 && k <= 64 && !(k & 3));
    if (!kok || !(wy == 1 || wy == 2 || wy == 4 || wy == 8 || wy == 16))
        return fail(c, REG_EINVAL,
                    "tile: k in {1, 2} (with k wy >= 4) or a multiple of 4 in [4, 64]; "
                    "wy in {1,2,4,8,16}");
    c->tile.k = k;
    c->tile.wy = wy;
    return REG_OK;
}

int reg_debug_inject(int what, int after) {
    if (what < REG_INJECT_NONE || what > REG_INJECT_STAGE_TIMEOUT || after < 0) return REG_EINVAL;
    if (what == REG_INJECT_STAGE_TIMEOUT) {
        if (after != 0) return REG_EINVAL;
        arm_stage_timeout(1);
        return REG_OK;
    }
    if (what == REG_INJECT_NONE) arm_stage_timeout(0);
    g_inject_what.store(REG_INJECT_NONE);
    g_inject_left.store(after);
    g_inject_what.store(what);
    return REG_OK;
}

int reg_set_staging(reg_ctx* c, int tma) {
    CHECK_CTX(c);
    if (tma != 0 && tma != 1) return fail(c, REG_EINVAL, "staging: tma must be 0 or 1");
    c->tile.tma = tma;
    return REG_OK;
}

int reg_get_tile(const reg_ctx* c, int* k, int* wy) {
    if (!c || !k || !wy) return REG_EINVAL;
    *k = c->tile.k;
    *wy = c->tile.wy;
    return REG_OK;
}

int reg_set_timing(reg_ctx* c, int on) {
    CHECK_CTX(c);
    if (c->coarse) REG_TRY(reg_set_timing(c->coarse, on));
    REG_CK(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->pending.clear();
    memset(&c->acc, 0, sizeof c->acc);
    c->timing = on != 0;
    return REG_OK;
}

int reg_get_timing(reg_ctx* c, reg_timing* out) {
    CHECK_CTX(c);
    if (!out) return fail(c, REG_EINVAL, "out is NULL");
    REG_CK(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        float ms = 0.f;
        REG_CK(c, cudaEventElapsedTime(&ms, p.a, p.b));
        c->acc.ms[p.phase] += ms;
        c->acc.launches[p.phase] += 1;
        c->acc.bytes[p.phase] += p.bytes;
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->pending.clear();
    *out = c->acc;
    return REG_OK;
}

int reg_get_coarse_timing(reg_ctx* c, reg_timing* out) {
    CHECK_CTX(c);
    if (!out) return fail(c, REG_EINVAL, "out is NULL");
    if (!c->coarse) {
        memset(out, 0, sizeof *out);
        return REG_OK;
    }
    const int s = reg_get_timing(c->coarse, out);
    if (s != REG_OK) return fail(c, s, "coarse grid: " + c->coarse->err);
    return REG_OK;
}

int reg_set_dependent_launch(int on) {
    if (on != 0 && on != 1) return REG_EINVAL;
    set_dependent_launch(on != 0);
    return REG_OK;
}

int reg_set_coarse_tile(reg_ctx* c, int k, int wy) {
    CHECK_CTX(c);
    if (k == 0 && wy == 0) {
        c->coarse_tile_k = c->coarse_tile_wy = 0;
        return REG_OK;
    }
    const bool kok = (k == 1 || k == 2) ? wy * k >= 4 : (k >= 4 && k <= 64 && !(k & 3));
    if (!kok || !(wy == 1 || wy == 2 || wy == 4 || wy == 8 || wy == 16))
        return fail(c, REG_EINVAL, "coarse tile: 0, 0 or a tile reg_set_tile accepts");
    c->coarse_tile_k = k;
    c->coarse_tile_wy = wy;
    return REG_OK;
}

int reg_get_coarse_tile(const reg_ctx* c, int* k, int* wy) {
    if (!c || !k || !wy) return REG_EINVAL;
    *k = c->coarse ? c->coarse->tile.k : 0;
    *wy = c->coarse ? c->coarse->tile.wy : 0;
    return REG_OK;
}

}  // extern "C"
