// Shared device helpers and the internal launcher interface of libreg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cufft.h>
#include <stdint.h>

namespace reg {

// Grid geometry.  n <= 2^30 so a point index fits in int; component offsets
// (c * n) use long long.
struct Dims {
    int n1, n2, n3;
    int n23;          // n2 * n3
    int n;            // n1 * n2 * n3
    int m3;           // n3 / 2 + 1 (half spectrum along x3)
    int nc;           // n1 * n2 * m3 complex coefficients per field
};

inline Dims make_dims(int n1, int n2, int n3) {
    Dims d;
    d.n1 = n1; d.n2 = n2; d.n3 = n3;
    d.n23 = n2 * n3;
    d.n = n1 * n2 * n3;
    d.m3 = n3 / 2 + 1;
    d.nc = n1 * n2 * d.m3;
    return d;
}

// ------------------------------------------------------------ device side

// i mod n for any int i (n > 0).
__device__ __forceinline__ int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Cubic Lagrange basis on the nodes -1, 0, 1, 2 at t in [0, 1].
__device__ __forceinline__ void lagrange4(float t, float w[4]) {
    const float tp1 = t + 1.f, tm1 = t - 1.f, tm2 = t - 2.f;
    const float a = t * tm1;            // t (t-1)
    const float b = tp1 * tm2;          // (t+1)(t-2)
    w[0] = -a * tm2 * (1.f / 6.f);
    w[1] = b * tm1 * 0.5f;
    w[2] = -b * t * 0.5f;
    w[3] = a * tp1 * (1.f / 6.f);
}

// The 4 x 4 x 4 stencil of the point i + d (grid units): wrapped element
// offsets per axis and the Lagrange weights.
struct Stencil {
    int o1[4], o2[4], o3[4];
    float w1[4], w2[4], w3[4];
};

__device__ __forceinline__ void axis_stencil(int i, float d, int n, int stride,
                                             int o[4], float w[4]) {
    const float fl = floorf(d);
    lagrange4(d - fl, w);
    int b = wrap(i + (int)fl - 1, n);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        o[a] = b * stride;
        b = (b + 1 == n) ? 0 : b + 1;
    }
}

__device__ __forceinline__ void make_stencil(Stencil& s, const Dims& g, int i1, int i2,
                                             int i3, float d1, float d2, float d3) {
    axis_stencil(i1, d1, g.n1, g.n23, s.o1, s.w1);
    axis_stencil(i2, d2, g.n2, g.n3, s.o2, s.w2);
    axis_stencil(i3, d3, g.n3, 1, s.o3, s.w3);
}

// sum_{abc} w1 w2 w3 f[...] for one scalar field.
__device__ __forceinline__ float gather1(const Stencil& s, const float* __restrict__ f) {
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float acc2 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float* row = f + s.o1[a] + s.o2[b];
            float r = s.w3[0] * __ldg(row + s.o3[0]);
            r = fmaf(s.w3[1], __ldg(row + s.o3[1]), r);
            r = fmaf(s.w3[2], __ldg(row + s.o3[2]), r);
            r = fmaf(s.w3[3], __ldg(row + s.o3[3]), r);
            acc2 = fmaf(s.w2[b], r, acc2);
        }
        acc = fmaf(s.w1[a], acc2, acc);
    }
    return acc;
}

// Interleaved pair (x, y): returns (sum w x, sum w y).
__device__ __forceinline__ float2 gather2(const Stencil& s, const float2* __restrict__ f) {
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float bx = 0.f, by = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float2* row = f + s.o1[a] + s.o2[b];
            float rx = 0.f, ry = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 v = __ldg(row + s.o3[c]);
                rx = fmaf(s.w3[c], v.x, rx);
                ry = fmaf(s.w3[c], v.y, ry);
            }
            bx = fmaf(s.w2[b], rx, bx);
            by = fmaf(s.w2[b], ry, by);
        }
        ax = fmaf(s.w1[a], bx, ax);
        ay = fmaf(s.w1[a], by, ay);
    }
    return make_float2(ax, ay);
}

// Interleaved pair (x, y): returns (sum w x, sum w x*y) -- the transported
// field and its product with a grid factor (lam and lam * div v).
__device__ __forceinline__ float2 gather2_prod(const Stencil& s, const float2* __restrict__ f) {
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float bx = 0.f, by = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float2* row = f + s.o1[a] + s.o2[b];
            float rx = 0.f, ry = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float2 v = __ldg(row + s.o3[c]);
                rx = fmaf(s.w3[c], v.x, rx);
                ry = fmaf(s.w3[c], v.x * v.y, ry);
            }
            bx = fmaf(s.w2[b], rx, bx);
            by = fmaf(s.w2[b], ry, by);
        }
        ax = fmaf(s.w1[a], bx, ax);
        ay = fmaf(s.w1[a], by, ay);
    }
    return make_float2(ax, ay);
}

// Decompose a point index into (i1, i2, i3).
__device__ __forceinline__ void unflatten(const Dims& g, int idx, int& i1, int& i2, int& i3) {
    i1 = idx / g.n23;
    const int r = idx - i1 * g.n23;
    i2 = r / g.n3;
    i3 = r - i2 * g.n3;
}

// ------------------------------------------------------------ launchers

// transport.cu
cudaError_t launch_departure(const Dims& g, const float* v, float dt, float* d_fwd,
                             float* d_adj, cudaStream_t st);
cudaError_t launch_interp(const Dims& g, const float* field, int nfields, const float* disp,
                          float* out, cudaStream_t st);
// rho_out = I[rho_in](x + d).  With rho_R != nullptr (final step) also writes
// the adjoint initial value lam = rho_R - rho_out into lam_out (float2 with
// divv when divv != nullptr, plain float otherwise; lam_out may be nullptr)
// and per-block FP64 partial sums of (rho_out - rho_R)^2 into partials.
cudaError_t launch_state_step(const Dims& g, const float* rho_in, const float* d,
                              float* rho_out, const float* rho_R, const float* divv,
                              void* lam_out, double* partials, int nblk_partials,
                              cudaStream_t st);
// Adjoint / incremental adjoint tau-step with b accumulation.
struct AdjointStepArgs {
    const void* lam_in;        // float2 (lam, divv) if compressible else float
    void* lam_out;
    const float* d;            // semi-Lagrangian points of -v, [3n]
    const float* grad_j;       // grad rho(t_j), [3n]  (fp32 or bf16, see below)
    const float* grad_j1;      // grad rho(t_{j+1}) (first step only)
    const __nv_bfloat16* grad_j_bf;
    const __nv_bfloat16* grad_j1_bf;
    float* b;                  // [3n] accumulator
    float w_j, w_j1, dt;
    int compressible, first;
};
cudaError_t launch_adjoint_step(const Dims& g, const AdjointStepArgs& a, cudaStream_t st);
// Incremental state step: in = (rho~_j, f_j) float2; writes (rho~_{j+1}, f_{j+1})
// or, when final, the incremental-adjoint initial value -rho~_nt (float2 with
// divv when compressible, else float) into out.
struct IncStateStepArgs {
    const float2* in;
    void* out;
    const float* d;            // semi-Lagrangian points of v
    const float* vt;           // [3n]
    const float* grad_j1;      // grad rho(t_{j+1}) [3n]
    const __nv_bfloat16* grad_j1_bf;
    const float* divv;         // final step, compressible only
    float dt;
    int final_step, compressible;
};
cudaError_t launch_incstate_step(const Dims& g, const IncStateStepArgs& a, cudaStream_t st);
// out = (0, -vt . grad rho(t_0)).
cudaError_t launch_incstate_init(const Dims& g, const float* vt, const float* grad0,
                                 const __nv_bfloat16* grad0_bf, float2* out,
                                 cudaStream_t st);
// Pack (lam, divv): out[i] = (lam[i], divv[i]).
cudaError_t launch_pack2(const Dims& g, const float* lam, const float* divv, float2* out,
                         cudaStream_t st);
// Deformation displacement step: u_{j+1} = I[u_j](X) + dt/2 (I[-v](X) - v(x)).
cudaError_t launch_deformation_step(const Dims& g, const float* u_in, const float* v,
                                    const float* d, float dt, float* u_out,
                                    cudaStream_t st);
// float -> bfloat16 copy (count elements).
cudaError_t launch_to_bf16(const float* in, __nv_bfloat16* out, long long count,
                           cudaStream_t st);
cudaError_t launch_from_bf16(const __nv_bfloat16* in, float* out, long long count,
                             cudaStream_t st);

// spectral.cu -- multipliers on the half spectrum (cufftComplex = float2).
// All scale by 1/n (the unnormalised inverse FFT).
enum SpecOp {
    SPEC_GRAD = 0,      // out[3] = i k' in[1]
    SPEC_DIV = 1,       // out[1] = i k' . in[3]
    SPEC_ASSEMBLE = 2,  // out[3] = beta A in_a[3] + (P) in_b[3]   (in_a or in_b may be null)
    SPEC_PRECOND = 3,   // out[3] = M (P) in[3]
    SPEC_GAUSS = 4,     // out[1] = G in[1]
    SPEC_LERAY = 5,     // out[3] = P in[3]
    SPEC_REG = 6        // out[3] = beta A in[3]
};
struct SpecArgs {
    const float2* in_a;
    const float2* in_b;
    float2* out;
    double beta;
    int kind;           // REG_H1 / REG_H2 / REG_H1DIV
    int project;        // apply P
    float s1, s2, s3;   // Gaussian widths
};
cudaError_t launch_spectral(const Dims& g, SpecOp op, const SpecArgs& a, cudaStream_t st);
// Per-block FP64 partials of sum_k weight(k) A(k) |V(k)|^2 over 3 fields
// (Hermitian weights on the half spectrum).
cudaError_t launch_spec_energy(const Dims& g, const float2* v, int kind, double* partials,
                               int nblk, cudaStream_t st);

// blas.cu
int blas_blocks();   // number of partial-sum blocks used by reductions
cudaError_t launch_dot_partials(const float* a, const float* b, long long count,
                                double* partials, int nblk, cudaStream_t st);
// result[0] = scale * sum(partials[0..nblk)); also flags non-finite values.
cudaError_t launch_finalize(const double* partials, int nblk, double scale, double* result,
                            cudaStream_t st);
// PCG pieces; scalars live in device memory (sc[]), see solver.
cudaError_t launch_axpy(float* y, const float* x, float alpha, long long count,
                        cudaStream_t st);           // y += alpha x
cudaError_t launch_axpby_out(float* out, const float* x, const float* y, float a, float b,
                             long long count, cudaStream_t st);   // out = a x + b y
// x += alpha p; r -= alpha q; partials of r.r   (alpha = sc[ia] / sc[ib])
cudaError_t launch_pcg_update(float* x, float* r, const float* p, const float* q,
                              const double* sc, int ia, int ib, long long count,
                              double* partials, int nblk, cudaStream_t st);
// p = z + beta p, beta = sc[ia] / sc[ib]
cudaError_t launch_pcg_direction(float* p, const float* z, const double* sc, int ia, int ib,
                                 long long count, cudaStream_t st);
cudaError_t launch_scale(float* y, float alpha, long long count, cudaStream_t st);

}  // namespace reg
