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
        a.out[idx] = make_float2(re * inv_n, im * inv_n);
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
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float2 x = v[c * nc + idx];
            s += (double)x.x * x.x + (double)x.y * x.y;
        }
        acc += (double)A * s;
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

}  // namespace

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
