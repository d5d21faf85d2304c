// Fused spectral multipliers on the half spectrum (Sec. III-B1): gradient,
// divergence, regularisation beta A, Leray projection P, the gradient /
// Hessian assembly beta A v + P b, the inverse-regularisation preconditioner
// and the Gaussian filter.  Each is one pass over the coefficients between a
// cuFFT R2C and C2R; every output is scaled by 1/n so that C2R(R2C(f)) = f.
//
// Wavenumbers: k_j in FFT order along x1 and x2 (0..n/2-1, -n/2..-1), 0..n3/2
// along x3.  Odd derivatives use k' (Nyquist entry set to 0); even operators
// use the full k; P uses k' and is the identity where k' = 0.
#include "common.cuh"
#include "reg.h"

namespace reg {

namespace {

constexpr int kThreads = 256;

struct Wave {
    float k1, k2, k3;      // full wavenumbers
    float p1, p2, p3;      // odd-derivative wavenumbers k'
    float herm;            // Hermitian weight of this half-spectrum entry
};

__device__ __forceinline__ Wave wave(const Dims& g, int idx) {
    const int i3 = idx % g.m3;
    const int r = idx / g.m3;
    const int i2 = r % g.n2;
    const int i1 = r / g.n2;
    Wave w;
    const int k1 = (i1 < (g.n1 + 1) / 2) ? i1 : i1 - g.n1;
    const int k2 = (i2 < (g.n2 + 1) / 2) ? i2 : i2 - g.n2;
    const int k3 = i3;
    w.k1 = (float)k1; w.k2 = (float)k2; w.k3 = (float)k3;
    w.p1 = ((g.n1 & 1) == 0 && 2 * i1 == g.n1) ? 0.f : w.k1;
    w.p2 = ((g.n2 & 1) == 0 && 2 * i2 == g.n2) ? 0.f : w.k2;
    const bool nyq3 = ((g.n3 & 1) == 0 && 2 * i3 == g.n3);
    w.p3 = nyq3 ? 0.f : w.k3;
    w.herm = (i3 == 0 || nyq3) ? 1.f : 2.f;
    return w;
}

__device__ __forceinline__ float reg_symbol(const Wave& w, int kind) {
    const float s = w.k1 * w.k1 + w.k2 * w.k2 + w.k3 * w.k3;
    return kind == REG_H2 ? s * s : s;
}

__device__ __forceinline__ float2 cmul_i(float k, float2 a) {   // i k a
    return make_float2(-k * a.y, k * a.x);
}

__device__ __forceinline__ void leray3(const Wave& w, float2& a, float2& b, float2& c) {
    const float kk = w.p1 * w.p1 + w.p2 * w.p2 + w.p3 * w.p3;
    if (kk > 0.f) {
        const float inv = 1.f / kk;
        const float dx = (w.p1 * a.x + w.p2 * b.x + w.p3 * c.x) * inv;
        const float dy = (w.p1 * a.y + w.p2 * b.y + w.p3 * c.y) * inv;
        a.x -= w.p1 * dx; a.y -= w.p1 * dy;
        b.x -= w.p2 * dx; b.y -= w.p2 * dy;
        c.x -= w.p3 * dx; c.y -= w.p3 * dy;
    }
}

__device__ __forceinline__ float2 scale2(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__global__ void __launch_bounds__(kThreads)
k_spectral(Dims g, int op, SpecArgs a, float inv_n) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.nc) return;
    const long long nc = g.nc;
    const Wave w = wave(g, idx);
    switch (op) {
    case SPEC_GRAD: {
        const float2 f = scale2(a.in_a[idx], inv_n);
        a.out[idx] = cmul_i(w.p1, f);
        a.out[nc + idx] = cmul_i(w.p2, f);
        a.out[2 * nc + idx] = cmul_i(w.p3, f);
        break;
    }
    case SPEC_DIV: {
        const float2 x = a.in_a[idx], y = a.in_a[nc + idx], z = a.in_a[2 * nc + idx];
        const float re = -(w.p1 * x.y + w.p2 * y.y + w.p3 * z.y);
        const float im = w.p1 * x.x + w.p2 * y.x + w.p3 * z.x;
        const float sc = a.normalised ? 1.f : inv_n;
        a.out[idx] = make_float2(re * sc, im * sc);
        break;
    }
    case SPEC_ASSEMBLE:
    case SPEC_LERAY:
    case SPEC_REG:
    case SPEC_PRECOND: {
        float2 o0 = make_float2(0.f, 0.f), o1 = o0, o2 = o0;
        if (op == SPEC_ASSEMBLE) {
            if (a.in_b) {
                o0 = a.in_b[idx]; o1 = a.in_b[nc + idx]; o2 = a.in_b[2 * nc + idx];
                if (a.project) leray3(w, o0, o1, o2);
            }
            if (a.in_a) {
                const float s = (float)a.beta * reg_symbol(w, a.kind);
                const float2 v0 = a.in_a[idx], v1 = a.in_a[nc + idx], v2 = a.in_a[2 * nc + idx];
                o0.x = fmaf(s, v0.x, o0.x); o0.y = fmaf(s, v0.y, o0.y);
                o1.x = fmaf(s, v1.x, o1.x); o1.y = fmaf(s, v1.y, o1.y);
                o2.x = fmaf(s, v2.x, o2.x); o2.y = fmaf(s, v2.y, o2.y);
            }
        } else {
            o0 = a.in_a[idx]; o1 = a.in_a[nc + idx]; o2 = a.in_a[2 * nc + idx];
            if (op == SPEC_LERAY || (op == SPEC_PRECOND && a.project)) leray3(w, o0, o1, o2);
            if (op == SPEC_REG) {
                const float s = (float)a.beta * reg_symbol(w, a.kind);
                o0 = scale2(o0, s); o1 = scale2(o1, s); o2 = scale2(o2, s);
            } else if (op == SPEC_PRECOND) {
                const float A = reg_symbol(w, a.kind);
                const float m = A > 0.f ? 1.f / ((float)a.beta * A) : 1.f / (float)a.beta;
                o0 = scale2(o0, m); o1 = scale2(o1, m); o2 = scale2(o2, m);
            }
        }
        a.out[idx] = scale2(o0, inv_n);
        a.out[nc + idx] = scale2(o1, inv_n);
        a.out[2 * nc + idx] = scale2(o2, inv_n);
        break;
    }
    case SPEC_GAUSS: {
        const float e = a.s1 * a.s1 * w.k1 * w.k1 + a.s2 * a.s2 * w.k2 * w.k2 +
                        a.s3 * a.s3 * w.k3 * w.k3;
        a.out[idx] = scale2(a.in_a[idx], expf(-0.5f * e) * inv_n);
        break;
    }
    default:
        break;
    }
}

__global__ void __launch_bounds__(kThreads)
k_spec_energy(Dims g, const float2* __restrict__ v, int kind, double* partials) {
    const long long nc = g.nc;
    double acc = 0.0;
    for (int idx = blockIdx.x * kThreads + threadIdx.x; idx < g.nc;
         idx += gridDim.x * kThreads) {
        const Wave w = wave(g, idx);
        const float A = reg_symbol(w, kind) * w.herm;
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 x = v[c * nc + idx];
            s = fmaf(x.x, x.x, s);
            s = fmaf(x.y, x.y, s);
        }
        acc += (double)(A * s);
    }
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (wid == 0) {
        acc = lane < kThreads / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) partials[blockIdx.x] = acc;
    }
}

// ------------------------------------------------ spectral Krylov vectors
// The solver keeps v, g, s, r, p as normalised half-spectrum coefficients
// (C2R gives the field itself): 3 components x nc entries.  Inner products
// <a, b>_h = (2 pi)^3 sum_k herm(k) Re(conj(a_k) b_k) (Parseval).  Each kernel
// writes per-block FP64 partials, slot t at partials[t * gridDim.x + block].

// Spectral preconditioner 1 / (beta A + shift) (shift 0: the inverse
// regularisation operator, with 1 / beta at k = 0).
__device__ __forceinline__ float mprec(float A, float beta, float shift) {
    return A > 0.f ? 1.f / fmaf(beta, A, shift) : 1.f / (beta + shift);
}

// herm |(a, b, c)|^2 of one coefficient: the products in FP32 (one rounding
// of an FP32 value's square, relative 6e-8), the sums over the spectrum in
// FP64 by the callers.  GB300 runs FP64 arithmetic at a small fraction of
// FP32, and a per-coefficient FP64 product chain was a measurable part of
// these bandwidth-bound kernels.
__device__ __forceinline__ float herm_sq(const Wave& w, float2 a, float2 b, float2 c) {
    float s = a.x * a.x;
    s = fmaf(a.y, a.y, s);
    s = fmaf(b.x, b.x, s);
    s = fmaf(b.y, b.y, s);
    s = fmaf(c.x, c.x, s);
    s = fmaf(c.y, c.y, s);
    return w.herm * s;
}

template <int NS>
__device__ __forceinline__ void store_partials(double (&acc)[NS], double* partials) {
    __shared__ double red[NS][kThreads / 32];
#pragma unroll
    for (int t = 0; t < NS; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int t = 0; t < NS; ++t) red[t][wid] = acc[t];
    __syncthreads();
    if (threadIdx.x < NS) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += red[threadIdx.x][i];
        partials[threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

#define SPEC_LOOP for (int idx = blockIdx.x * kThreads + threadIdx.x; idx < g.nc; \
                       idx += gridDim.x * kThreads)

// r = -g, s = 0, z = M P r, p = pc = z; partials: |P r|^2, M |P r|^2, beta A |p|^2.
__global__ void __launch_bounds__(kThreads)
k_sp_init(Dims g, const float2* __restrict__ gh, float2* __restrict__ r, float2* __restrict__ s,
          float2* __restrict__ p, float2* __restrict__ pc, float beta, float shift, int kind,
          int project,
          double* partials) {
    const long long nc = g.nc;
    double acc[3] = {0.0, 0.0, 0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float2 a = gh[idx], b = gh[nc + idx], c = gh[2 * nc + idx];
        a = scale2(a, -1.f); b = scale2(b, -1.f); c = scale2(c, -1.f);
        r[idx] = a; r[nc + idx] = b; r[2 * nc + idx] = c;
        const float2 zero = make_float2(0.f, 0.f);
        s[idx] = zero; s[nc + idx] = zero; s[2 * nc + idx] = zero;
        if (project) leray3(w, a, b, c);
        const float A = reg_symbol(w, kind);
        const float m = mprec(A, beta, shift);
        const float e = herm_sq(w, a, b, c);
        acc[0] += e;
        acc[1] += (double)(m * e);
        acc[2] += (double)(beta * A * m * m * e);
        a = scale2(a, m); b = scale2(b, m); c = scale2(c, m);
        p[idx] = a; p[nc + idx] = b; p[2 * nc + idx] = c;
        pc[idx] = a; pc[nc + idx] = b; pc[2 * nc + idx] = c;
    }
    store_partials<3>(acc, partials);
}

// PQ = sc[ipap] + sc[ipb] (written to sc_out[ipq] by block 0), alpha = RZ / PQ
// (0 if PQ <= 0); q = beta A p + P B / n; s += alpha p; r -= alpha q;
// partials: |P r|^2, M |P r|^2.
__global__ void __launch_bounds__(kThreads)
k_sp_update(Dims g, float2* __restrict__ s, float2* __restrict__ r, const float2* __restrict__ p,
            const float2* __restrict__ B, double* sc, int irz, int ipap, int ipb, int ipq,
            float beta, float shift, int kind, int project, float inv_n, double* partials,
            Fin fin) {
    pdl_wait();
    pdl_trigger();
    const long long nc = g.nc;
    const double pq = sc[ipap] + sc[ipb];
    const float alpha = pq > 0.0 ? (float)(sc[irz] / pq) : 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) sc[ipq] = pq;
    double acc[2] = {0.0, 0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        const float A = reg_symbol(w, kind);
        const float bA = beta * A;
        float2 b0 = scale2(B[idx], inv_n), b1 = scale2(B[nc + idx], inv_n),
               b2 = scale2(B[2 * nc + idx], inv_n);
        if (project) leray3(w, b0, b1, b2);
        float2 rr[3], pp[3];
        const float2 bb[3] = {b0, b1, b2};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            pp[k] = p[k * nc + idx];
            float2 sv = s[k * nc + idx];
            sv.x = fmaf(alpha, pp[k].x, sv.x);
            sv.y = fmaf(alpha, pp[k].y, sv.y);
            s[k * nc + idx] = sv;
            const float2 q = make_float2(fmaf(bA, pp[k].x, bb[k].x), fmaf(bA, pp[k].y, bb[k].y));
            rr[k] = r[k * nc + idx];
            rr[k].x = fmaf(-alpha, q.x, rr[k].x);
            rr[k].y = fmaf(-alpha, q.y, rr[k].y);
            r[k * nc + idx] = rr[k];
        }
        if (project) leray3(w, rr[0], rr[1], rr[2]);
        const float e = herm_sq(w, rr[0], rr[1], rr[2]);
        acc[0] += e;
        acc[1] += (double)(mprec(A, beta, shift) * e);
    }
    store_partials<2>(acc, partials);
    if (fin.count) finish_partials<2>(partials, gridDim.x, fin);
}

// b = sc[irznew] / sc[irz] (0 with zero_beta); p = M P r + b p; pc = p (or, with
// to_s, s = M P r only); partials: beta A |p|^2.
__global__ void __launch_bounds__(kThreads)
k_sp_direction(Dims g, const float2* __restrict__ r, float2* __restrict__ p,
               float2* __restrict__ pc, const double* sc, int irznew, int irz,
               int zero_beta, float beta, float shift, int kind, int project, double* partials,
               Fin fin) {
    pdl_wait();
    pdl_trigger();
    const long long nc = g.nc;
    const double den = sc[irz];
    const float bk = (zero_beta || den == 0.0) ? 0.f : (float)(sc[irznew] / den);
    double acc[1] = {0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float2 a = r[idx], b = r[nc + idx], c = r[2 * nc + idx];
        if (project) leray3(w, a, b, c);
        const float A = reg_symbol(w, kind);
        const float m = mprec(A, beta, shift);
        float2 z[3] = {scale2(a, m), scale2(b, m), scale2(c, m)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float2 pv = zero_beta ? make_float2(0.f, 0.f) : p[k * nc + idx];
            pv.x = fmaf(bk, pv.x, z[k].x);
            pv.y = fmaf(bk, pv.y, z[k].y);
            p[k * nc + idx] = pv;
            if (pc) pc[k * nc + idx] = pv;
            z[k] = pv;
        }
        acc[0] += (double)(beta * A * herm_sq(w, z[0], z[1], z[2]));
    }
    store_partials<1>(acc, partials);
    if (fin.count) finish_partials<1>(partials, gridDim.x, fin);
}

// g = beta A v + P B / n; partials: |g|^2, A |v|^2.
__global__ void __launch_bounds__(kThreads)
k_sp_gradient(Dims g, const float2* __restrict__ v, const float2* __restrict__ B,
              float2* __restrict__ gout, float beta, int kind, int project, float inv_n,
              double* partials) {
    const long long nc = g.nc;
    double acc[2] = {0.0, 0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        const float A = reg_symbol(w, kind);
        float2 b0 = scale2(B[idx], inv_n), b1 = scale2(B[nc + idx], inv_n),
               b2 = scale2(B[2 * nc + idx], inv_n);
        if (project) leray3(w, b0, b1, b2);
        const float2 v0 = v[idx], v1 = v[nc + idx], v2 = v[2 * nc + idx];
        const float bA = beta * A;
        const float2 g0 = make_float2(fmaf(bA, v0.x, b0.x), fmaf(bA, v0.y, b0.y));
        const float2 g1 = make_float2(fmaf(bA, v1.x, b1.x), fmaf(bA, v1.y, b1.y));
        const float2 g2 = make_float2(fmaf(bA, v2.x, b2.x), fmaf(bA, v2.y, b2.y));
        gout[idx] = g0; gout[nc + idx] = g1; gout[2 * nc + idx] = g2;
        acc[0] += herm_sq(w, g0, g1, g2);
        acc[1] += (double)(A * herm_sq(w, v0, v1, v2));
    }
    store_partials<2>(acc, partials);
}

// out = x + a y (y may be null), copy = out (may be null), optional Leray
// projection; partials: A |out|^2.
__global__ void __launch_bounds__(kThreads)
k_sp_axpy(Dims g, float2* __restrict__ out, float2* __restrict__ copy, const float2* x,
          const float2* __restrict__ y, float a, int kind, int project, double* partials) {
    const long long nc = g.nc;
    double acc[1] = {0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float2 o[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = x[k * nc + idx];
            if (y) {
                const float2 yv = y[k * nc + idx];
                o[k].x = fmaf(a, yv.x, o[k].x);
                o[k].y = fmaf(a, yv.y, o[k].y);
            }
        }
        if (project) leray3(w, o[0], o[1], o[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            out[k * nc + idx] = o[k];
            if (copy) copy[k * nc + idx] = o[k];
        }
        acc[0] += (double)(reg_symbol(w, kind) * herm_sq(w, o[0], o[1], o[2]));
    }
    store_partials<1>(acc, partials);
}

// partials: sum herm Re(conj(a) b) over the 3 components.
__global__ void __launch_bounds__(kThreads)
k_sp_dot(Dims g, const float2* __restrict__ a, const float2* __restrict__ b, double* partials) {
    const long long nc = g.nc;
    double acc[1] = {0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float2 x = a[k * nc + idx], y = b[k * nc + idx];
            s = fmaf(x.x, y.x, s);
            s = fmaf(x.y, y.y, s);
        }
        acc[0] += (double)(w.herm * s);
    }
    store_partials<1>(acc, partials);
}

// Flexible PCG step: s += a p, r -= a q, partials: herm |r|^2 -- the two
// updates and the residual norm of k_sp_axpy and k_sp_dot in one pass (the
// same operations, so the same values).
__global__ void __launch_bounds__(kThreads)
k_sp_fcg_update(Dims g, float2* __restrict__ s, float2* __restrict__ r,
                const float2* __restrict__ p, const float2* __restrict__ q, float a,
                double* partials) {
    const long long nc = g.nc;
    double acc[1] = {0.0};
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float sum = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float2 sv = s[k * nc + idx];
            const float2 pv = p[k * nc + idx];
            sv.x = fmaf(a, pv.x, sv.x);
            sv.y = fmaf(a, pv.y, sv.y);
            s[k * nc + idx] = sv;
            float2 rv = r[k * nc + idx];
            const float2 qv = q[k * nc + idx];
            rv.x = fmaf(-a, qv.x, rv.x);
            rv.y = fmaf(-a, qv.y, rv.y);
            r[k * nc + idx] = rv;
            sum = fmaf(rv.x, rv.x, sum);
            sum = fmaf(rv.y, rv.y, sum);
        }
        acc[0] += (double)(w.herm * sum);
    }
    store_partials<1>(acc, partials);
}

// out = in / n (normalise a raw R2C spectrum), optional Leray projection.
__global__ void __launch_bounds__(kThreads)
k_sp_normalise(Dims g, const float2* in, float2* out, int project, float inv_n) {
    const long long nc = g.nc;
    SPEC_LOOP {
        const Wave w = wave(g, idx);
        float2 a = scale2(in[idx], inv_n), b = scale2(in[nc + idx], inv_n),
               c = scale2(in[2 * nc + idx], inv_n);
        if (project) leray3(w, a, b, c);
        out[idx] = a; out[nc + idx] = b; out[2 * nc + idx] = c;
    }
}

// Two-level preconditioner (coarse grid gc of the fine grid gf): the modes
// L = {|k_j| < nc_j / 2} are the same normalised coefficients on both grids.
__device__ __forceinline__ int fft_k(int i, int n) { return 2 * i < n ? i : i - n; }

// out (coarse) = scale * in (fine) on L, 0 on the coarse Nyquist planes.
__global__ void __launch_bounds__(kThreads)
k_sp_restrict(Dims gf, Dims gc, const float2* __restrict__ in, float2* __restrict__ out,
              float scale) {
    const long long ncf = gf.nc, ncc = gc.nc;
    for (int idx = blockIdx.x * kThreads + threadIdx.x; idx < gc.nc; idx += gridDim.x * kThreads) {
        const int i3 = idx % gc.m3;
        const int r = idx / gc.m3;
        const int i2 = r % gc.n2, i1 = r / gc.n2;
        const int k1 = fft_k(i1, gc.n1), k2 = fft_k(i2, gc.n2);
        const bool keep = 2 * abs(k1) < gc.n1 && 2 * abs(k2) < gc.n2 && 2 * i3 < gc.n3;
        const int f1 = k1 >= 0 ? k1 : k1 + gf.n1, f2 = k2 >= 0 ? k2 : k2 + gf.n2;
        const long long fi = ((long long)f1 * gf.n2 + f2) * gf.m3 + i3;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            out[c * ncc + idx] = keep ? scale2(in[c * ncf + fi], scale) : make_float2(0.f, 0.f);
    }
}

// z = y (coarse) on L, M P r elsewhere; partials: <r, z>.
__global__ void __launch_bounds__(kThreads)
k_sp_twolevel(Dims gf, Dims gc, const float2* __restrict__ r, const float2* __restrict__ y,
              float2* __restrict__ z, float beta, float shift, int kind, int project,
              double* partials) {
    const long long ncf = gf.nc, ncc = gc.nc;
    double acc[1] = {0.0};
    for (int idx = blockIdx.x * kThreads + threadIdx.x; idx < gf.nc; idx += gridDim.x * kThreads) {
        const Wave w = wave(gf, idx);
        const int k1 = (int)w.k1, k2 = (int)w.k2, k3 = (int)w.k3;
        float2 rr[3] = {r[idx], r[ncf + idx], r[2 * ncf + idx]};
        float2 zz[3];
        if (2 * abs(k1) < gc.n1 && 2 * abs(k2) < gc.n2 && 2 * k3 < gc.n3) {
            const int c1 = k1 >= 0 ? k1 : k1 + gc.n1, c2 = k2 >= 0 ? k2 : k2 + gc.n2;
            const long long ci = ((long long)c1 * gc.n2 + c2) * gc.m3 + k3;
#pragma unroll
            for (int c = 0; c < 3; ++c) zz[c] = y[c * ncc + ci];
        } else {
            zz[0] = rr[0]; zz[1] = rr[1]; zz[2] = rr[2];
            if (project) leray3(w, zz[0], zz[1], zz[2]);
            const float m = mprec(reg_symbol(w, kind), beta, shift);
#pragma unroll
            for (int c = 0; c < 3; ++c) zz[c] = scale2(zz[c], m);
        }
        float sdot = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            z[c * ncf + idx] = zz[c];
            sdot = fmaf(rr[c].x, zz[c].x, sdot);
            sdot = fmaf(rr[c].y, zz[c].y, sdot);
        }
        acc[0] += (double)(w.herm * sdot);
    }
    store_partials<1>(acc, partials);
}

}  // namespace

cudaError_t launch_sp_init(const Dims& g, const float2* gh, float2* r, float2* s, float2* p,
                           float2* pc, double beta, double shift, int kind, int project,
                           double* partials, int nblk, cudaStream_t st) {
    k_sp_init<<<nblk, kThreads, 0, st>>>(g, gh, r, s, p, pc, (float)beta, (float)shift, kind,
                                         project, partials);
    return cudaGetLastError();
}

cudaError_t launch_sp_update(const Dims& g, float2* s, float2* r, const float2* p,
                             const float2* B, double* sc, int irz, int ipap, int ipb, int ipq,
                             double beta, double shift, int kind, int project,
                             double* partials, int nblk, cudaStream_t st, const Fin* fin) {
    const Fin f = fin ? *fin : Fin{};
    return launch_dependent(k_sp_update, dim3(nblk), dim3(kThreads), 0, st, g, s, r, p, B, sc,
                            irz, ipap, ipb, ipq, (float)beta, (float)shift, kind, project,
                            1.0f / (float)g.n, partials, f);
}

cudaError_t launch_sp_direction(const Dims& g, const float2* r, float2* p, float2* pc,
                                const double* sc, int irznew, int irz, int zero_beta,
                                double beta, double shift, int kind, int project,
                                double* partials, int nblk, cudaStream_t st,
                                const Fin* fin) {
    const Fin f = fin ? *fin : Fin{};
    return launch_dependent(k_sp_direction, dim3(nblk), dim3(kThreads), 0, st, g, r, p, pc, sc,
                            irznew, irz, zero_beta, (float)beta, (float)shift, kind, project,
                            partials, f);
}

cudaError_t launch_sp_gradient(const Dims& g, const float2* v, const float2* B, float2* gout,
                               double beta, int kind, int project, double* partials, int nblk,
                               cudaStream_t st) {
    k_sp_gradient<<<nblk, kThreads, 0, st>>>(g, v, B, gout, (float)beta, kind, project,
                                             1.0f / (float)g.n, partials);
    return cudaGetLastError();
}

cudaError_t launch_sp_axpy(const Dims& g, float2* out, float2* copy, const float2* x,
                           const float2* y, float a, int kind, int project, double* partials,
                           int nblk, cudaStream_t st) {
    k_sp_axpy<<<nblk, kThreads, 0, st>>>(g, out, copy, x, y, a, kind, project, partials);
    return cudaGetLastError();
}

cudaError_t launch_sp_fcg_update(const Dims& g, float2* s, float2* r, const float2* p,
                                 const float2* q, float a, double* partials, int nblk,
                                 cudaStream_t st) {
    k_sp_fcg_update<<<nblk, kThreads, 0, st>>>(g, s, r, p, q, a, partials);
    return cudaGetLastError();
}

cudaError_t launch_sp_dot(const Dims& g, const float2* a, const float2* b, double* partials,
                          int nblk, cudaStream_t st) {
    k_sp_dot<<<nblk, kThreads, 0, st>>>(g, a, b, partials);
    return cudaGetLastError();
}

cudaError_t launch_sp_normalise(const Dims& g, const float2* in, float2* out, int project,
                                cudaStream_t st) {
    const int nb = (g.nc + kThreads - 1) / kThreads;
    k_sp_normalise<<<nb < 152 * 8 ? nb : 152 * 8, kThreads, 0, st>>>(g, in, out, project,
                                                                     1.0f / (float)g.n);
    return cudaGetLastError();
}

cudaError_t launch_sp_restrict(const Dims& gf, const Dims& gc, const float2* in, float2* out,
                               float scale, cudaStream_t st) {
    const int nb = (gc.nc + kThreads - 1) / kThreads;
    k_sp_restrict<<<nb < 152 * 8 ? nb : 152 * 8, kThreads, 0, st>>>(gf, gc, in, out, scale);
    return cudaGetLastError();
}

cudaError_t launch_sp_twolevel(const Dims& gf, const Dims& gc, const float2* r, const float2* y,
                               float2* z, double beta, double shift, int kind, int project,
                               double* partials, int nblk, cudaStream_t st) {
    k_sp_twolevel<<<nblk, kThreads, 0, st>>>(gf, gc, r, y, z, (float)beta, (float)shift, kind,
                                             project, partials);
    return cudaGetLastError();
}

cudaError_t launch_spectral(const Dims& g, SpecOp op, const SpecArgs& a, cudaStream_t st) {
    const int nb = (g.nc + kThreads - 1) / kThreads;
    k_spectral<<<nb, kThreads, 0, st>>>(g, (int)op, a, 1.0f / (float)g.n);
    return cudaGetLastError();
}

cudaError_t launch_spec_energy(const Dims& g, const float2* v, int kind, double* partials,
                               int nblk, cudaStream_t st) {
    k_spec_energy<<<nblk, kThreads, 0, st>>>(g, v, kind, partials);
    return cudaGetLastError();
}

}  // namespace reg
