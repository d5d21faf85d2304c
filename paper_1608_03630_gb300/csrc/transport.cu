// Semi-Lagrangian kernels: RK2 points, tricubic interpolation and the fused
// transport steps of the state, adjoint, incremental state and incremental
// adjoint equations (Sec. III-B2, Sec. III-C2, Algorithm 2).
//
// One thread per output grid point, x3 fastest across a warp so the reads of
// the per-point inputs (displacements, grid fields) are coalesced; the 64
// stencil values come through the read-only cache.
#include "common.cuh"

namespace reg {

namespace {

constexpr int kThreads = 256;

inline int nblocks(long long n) { return (int)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ float ld(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, long long i) {
    return __bfloat162float(p[i]);
}

// Eq. (sml-trajectory) for v and -v.  dtoh_j = dt / h_j converts velocity to
// grid units per step.
__global__ void __launch_bounds__(kThreads)
k_departure(Dims g, const float* __restrict__ v, float dth1, float dth2, float dth3,
            float* __restrict__ d_fwd, float* __restrict__ d_adj) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    int i1, i2, i3;
    unflatten(g, idx, i1, i2, i3);
    const long long n = g.n;
    const float u1 = v[idx] * dth1, u2 = v[n + idx] * dth2, u3 = v[2 * n + idx] * dth3;
    const float* v1 = v;
    const float* v2 = v + n;
    const float* v3 = v + 2 * n;
    Stencil s;
    // forward: X* = x - dt v(x)
    make_stencil(s, g, i1, i2, i3, -u1, -u2, -u3);
    float a1 = gather1(s, v1) * dth1, a2 = gather1(s, v2) * dth2, a3 = gather1(s, v3) * dth3;
    d_fwd[idx] = -0.5f * (u1 + a1);
    d_fwd[n + idx] = -0.5f * (u2 + a2);
    d_fwd[2 * n + idx] = -0.5f * (u3 + a3);
    if (d_adj == nullptr) return;
    // adjoint (velocity -v): X* = x + dt v(x), X = x + dt/2 (v(x) + v(X*))
    make_stencil(s, g, i1, i2, i3, u1, u2, u3);
    a1 = gather1(s, v1) * dth1; a2 = gather1(s, v2) * dth2; a3 = gather1(s, v3) * dth3;
    d_adj[idx] = 0.5f * (u1 + a1);
    d_adj[n + idx] = 0.5f * (u2 + a2);
    d_adj[2 * n + idx] = 0.5f * (u3 + a3);
}

__global__ void __launch_bounds__(kThreads)
k_interp(Dims g, const float* __restrict__ f, int nf, const float* __restrict__ d,
         float* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    int i1, i2, i3;
    unflatten(g, idx, i1, i2, i3);
    const long long n = g.n;
    Stencil s;
    make_stencil(s, g, i1, i2, i3, d[idx], d[n + idx], d[2 * n + idx]);
    for (int c = 0; c < nf; ++c) out[c * n + idx] = gather1(s, f + c * n);
}

// Block reduction of a double into partials[blockIdx.x].
__device__ __forceinline__ void block_sum_to(double v, double* partials) {
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < kThreads / 32 ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) partials[blockIdx.x] = v;
    }
}

// State step; the final step also forms lam(1) = rho_R - rho(1) and the
// mismatch partial sums (Eq. varopt, Eq. adjoint).
template <bool FINAL>
__global__ void __launch_bounds__(kThreads)
k_state_step(Dims g, const float* __restrict__ rin, const float* __restrict__ d,
             float* __restrict__ rout, const float* __restrict__ rho_R,
             const float* __restrict__ divv, void* __restrict__ lam_out,
             double* __restrict__ partials) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    double e2 = 0.0;
    if (idx < g.n) {
        int i1, i2, i3;
        unflatten(g, idx, i1, i2, i3);
        const long long n = g.n;
        Stencil s;
        make_stencil(s, g, i1, i2, i3, d[idx], d[n + idx], d[2 * n + idx]);
        const float r = gather1(s, rin);
        rout[idx] = r;
        if (FINAL) {
            const float lam = rho_R[idx] - r;
            e2 = (double)lam * (double)lam;
            if (lam_out) {
                if (divv) reinterpret_cast<float2*>(lam_out)[idx] = make_float2(lam, divv[idx]);
                else reinterpret_cast<float*>(lam_out)[idx] = lam;
            }
        }
    }
    if (FINAL) block_sum_to(e2, partials);
}

// Adjoint tau-step (Eq. adjoint, Eq. sml-advection), with b += w lam grad rho.
// Compressible: lam_in holds (lam, div v); source f = lam div v,
//   nu0 = I[lam](X), f0 = I[lam div v](X), nu* = nu0 + dt f0,
//   lam_new = nu0 + dt/2 (f0 + nu* div v(x)).
// Divergence free: lam_new = I[lam](X).
template <bool COMP, bool FIRST, typename GT>
__global__ void __launch_bounds__(kThreads)
k_adjoint_step(Dims g, const void* __restrict__ lam_in_, void* __restrict__ lam_out_,
               const float* __restrict__ d, const GT* __restrict__ gj,
               const GT* __restrict__ gj1, float* __restrict__ b, float w_j, float w_j1,
               float dt) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    int i1, i2, i3;
    unflatten(g, idx, i1, i2, i3);
    const long long n = g.n;
    Stencil s;
    make_stencil(s, g, i1, i2, i3, d[idx], d[n + idx], d[2 * n + idx]);
    float lam_new, lam_old;
    if (COMP) {
        const float2* lin = reinterpret_cast<const float2*>(lam_in_);
        const float2 own = lin[idx];
        const float2 nf = gather2_prod(s, lin);
        const float nu_star = fmaf(dt, nf.y, nf.x);
        lam_new = fmaf(0.5f * dt, nf.y + nu_star * own.y, nf.x);
        lam_old = own.x;
        reinterpret_cast<float2*>(lam_out_)[idx] = make_float2(lam_new, own.y);
    } else {
        const float* lin = reinterpret_cast<const float*>(lam_in_);
        lam_new = gather1(s, lin);
        lam_old = FIRST ? lin[idx] : 0.f;
        reinterpret_cast<float*>(lam_out_)[idx] = lam_new;
    }
    const float c = w_j * lam_new;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float acc = c * ld(gj, k * n + idx);
        if (FIRST) acc = fmaf(w_j1 * lam_old, ld(gj1, k * n + idx), acc);
        else acc += b[k * n + idx];
        b[k * n + idx] = acc;
    }
}

// Incremental state step (Eq. inc-state, Algorithm 2):
// rho~_{j+1} = I[rho~_j](X) + dt/2 (I[f_j](X) + f_{j+1}(x)), f = -v~ . grad rho.
template <bool FINAL, bool COMP, typename GT>
__global__ void __launch_bounds__(kThreads)
k_incstate_step(Dims g, const float2* __restrict__ in, void* __restrict__ out_,
                const float* __restrict__ d, const float* __restrict__ vt,
                const GT* __restrict__ gj1, const float* __restrict__ divv, float dt) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    int i1, i2, i3;
    unflatten(g, idx, i1, i2, i3);
    const long long n = g.n;
    Stencil s;
    make_stencil(s, g, i1, i2, i3, d[idx], d[n + idx], d[2 * n + idx]);
    const float2 nf = gather2(s, in);
    const float f1 = -(vt[idx] * ld(gj1, idx) + vt[n + idx] * ld(gj1, n + idx) +
                       vt[2 * n + idx] * ld(gj1, 2 * n + idx));
    const float r = fmaf(0.5f * dt, nf.y + f1, nf.x);
    if (!FINAL) {
        reinterpret_cast<float2*>(out_)[idx] = make_float2(r, f1);
    } else if (COMP) {
        reinterpret_cast<float2*>(out_)[idx] = make_float2(-r, divv[idx]);
    } else {
        reinterpret_cast<float*>(out_)[idx] = -r;
    }
}

template <typename GT>
__global__ void __launch_bounds__(kThreads)
k_incstate_init(Dims g, const float* __restrict__ vt, const GT* __restrict__ g0,
                float2* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    const long long n = g.n;
    const float f0 = -(vt[idx] * ld(g0, idx) + vt[n + idx] * ld(g0, n + idx) +
                       vt[2 * n + idx] * ld(g0, 2 * n + idx));
    out[idx] = make_float2(0.f, f0);
}

__global__ void k_pack2(int n, const float* __restrict__ a, const float* __restrict__ b,
                        float2* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx < n) out[idx] = make_float2(a[idx], b[idx]);
}

__global__ void __launch_bounds__(kThreads)
k_deformation_step(Dims g, const float* __restrict__ u_in, const float* __restrict__ v,
                   const float* __restrict__ d, float dt, float* __restrict__ u_out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    int i1, i2, i3;
    unflatten(g, idx, i1, i2, i3);
    const long long n = g.n;
    Stencil s;
    make_stencil(s, g, i1, i2, i3, d[idx], d[n + idx], d[2 * n + idx]);
    for (int c = 0; c < 3; ++c) {
        const float nu0 = gather1(s, u_in + c * n);
        const float f0 = -gather1(s, v + c * n);
        u_out[c * n + idx] = fmaf(0.5f * dt, f0 - v[c * n + idx], nu0);
    }
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          long long count) {
    long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long stride = (long long)gridDim.x * kThreads;
    for (; i < count; i += stride) out[i] = __float2bfloat16(in[i]);
}

__global__ void k_from_bf16(const __nv_bfloat16* __restrict__ in, float* __restrict__ out,
                            long long count) {
    long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long stride = (long long)gridDim.x * kThreads;
    for (; i < count; i += stride) out[i] = __bfloat162float(in[i]);
}

}  // namespace

cudaError_t launch_departure(const Dims& g, const float* v, float dt, float* d_fwd,
                             float* d_adj, cudaStream_t st) {
    const float two_pi = 6.283185307179586f;
    k_departure<<<nblocks(g.n), kThreads, 0, st>>>(
        g, v, dt * g.n1 / two_pi, dt * g.n2 / two_pi, dt * g.n3 / two_pi, d_fwd, d_adj);
    return cudaGetLastError();
}

cudaError_t launch_interp(const Dims& g, const float* field, int nfields, const float* disp,
                          float* out, cudaStream_t st) {
    k_interp<<<nblocks(g.n), kThreads, 0, st>>>(g, field, nfields, disp, out);
    return cudaGetLastError();
}

cudaError_t launch_state_step(const Dims& g, const float* rho_in, const float* d,
                              float* rho_out, const float* rho_R, const float* divv,
                              void* lam_out, double* partials, int nblk_partials,
                              cudaStream_t st) {
    const int nb = nblocks(g.n);
    if (rho_R) {
        if (nb > nblk_partials) return cudaErrorInvalidValue;
        k_state_step<true><<<nb, kThreads, 0, st>>>(g, rho_in, d, rho_out, rho_R, divv,
                                                    lam_out, partials);
    } else {
        k_state_step<false><<<nb, kThreads, 0, st>>>(g, rho_in, d, rho_out, nullptr,
                                                     nullptr, nullptr, nullptr);
    }
    return cudaGetLastError();
}

template <typename GT>
static void adjoint_dispatch(const Dims& g, const AdjointStepArgs& a, const GT* gj,
                             const GT* gj1, cudaStream_t st) {
    const int nb = nblocks(g.n);
    if (a.compressible) {
        if (a.first)
            k_adjoint_step<true, true, GT><<<nb, kThreads, 0, st>>>(
                g, a.lam_in, a.lam_out, a.d, gj, gj1, a.b, a.w_j, a.w_j1, a.dt);
        else
            k_adjoint_step<true, false, GT><<<nb, kThreads, 0, st>>>(
                g, a.lam_in, a.lam_out, a.d, gj, gj1, a.b, a.w_j, a.w_j1, a.dt);
    } else {
        if (a.first)
            k_adjoint_step<false, true, GT><<<nb, kThreads, 0, st>>>(
                g, a.lam_in, a.lam_out, a.d, gj, gj1, a.b, a.w_j, a.w_j1, a.dt);
        else
            k_adjoint_step<false, false, GT><<<nb, kThreads, 0, st>>>(
                g, a.lam_in, a.lam_out, a.d, gj, gj1, a.b, a.w_j, a.w_j1, a.dt);
    }
}

cudaError_t launch_adjoint_step(const Dims& g, const AdjointStepArgs& a, cudaStream_t st) {
    if (a.grad_j_bf) adjoint_dispatch(g, a, a.grad_j_bf, a.grad_j1_bf, st);
    else adjoint_dispatch(g, a, a.grad_j, a.grad_j1, st);
    return cudaGetLastError();
}

template <typename GT>
static void incstate_dispatch(const Dims& g, const IncStateStepArgs& a, const GT* gj1,
                              cudaStream_t st) {
    const int nb = nblocks(g.n);
    if (!a.final_step)
        k_incstate_step<false, false, GT><<<nb, kThreads, 0, st>>>(g, a.in, a.out, a.d, a.vt,
                                                                   gj1, a.divv, a.dt);
    else if (a.compressible)
        k_incstate_step<true, true, GT><<<nb, kThreads, 0, st>>>(g, a.in, a.out, a.d, a.vt,
                                                                 gj1, a.divv, a.dt);
    else
        k_incstate_step<true, false, GT><<<nb, kThreads, 0, st>>>(g, a.in, a.out, a.d, a.vt,
                                                                  gj1, a.divv, a.dt);
}

cudaError_t launch_incstate_step(const Dims& g, const IncStateStepArgs& a, cudaStream_t st) {
    if (a.grad_j1_bf) incstate_dispatch(g, a, a.grad_j1_bf, st);
    else incstate_dispatch(g, a, a.grad_j1, st);
    return cudaGetLastError();
}

cudaError_t launch_incstate_init(const Dims& g, const float* vt, const float* grad0,
                                 const __nv_bfloat16* grad0_bf, float2* out,
                                 cudaStream_t st) {
    if (grad0_bf)
        k_incstate_init<<<nblocks(g.n), kThreads, 0, st>>>(g, vt, grad0_bf, out);
    else
        k_incstate_init<<<nblocks(g.n), kThreads, 0, st>>>(g, vt, grad0, out);
    return cudaGetLastError();
}

cudaError_t launch_pack2(const Dims& g, const float* lam, const float* divv, float2* out,
                         cudaStream_t st) {
    k_pack2<<<nblocks(g.n), kThreads, 0, st>>>(g.n, lam, divv, out);
    return cudaGetLastError();
}

cudaError_t launch_deformation_step(const Dims& g, const float* u_in, const float* v,
                                    const float* d, float dt, float* u_out,
                                    cudaStream_t st) {
    k_deformation_step<<<nblocks(g.n), kThreads, 0, st>>>(g, u_in, v, d, dt, u_out);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float* in, __nv_bfloat16* out, long long count,
                           cudaStream_t st) {
    int nb = (int)((count + kThreads - 1) / kThreads);
    if (nb > 152 * 16) nb = 152 * 16;
    k_to_bf16<<<nb, kThreads, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

cudaError_t launch_from_bf16(const __nv_bfloat16* in, float* out, long long count,
                             cudaStream_t st) {
    int nb = (int)((count + kThreads - 1) / kThreads);
    if (nb > 152 * 16) nb = 152 * 16;
    k_from_bf16<<<nb, kThreads, 0, st>>>(in, out, count);
    return cudaGetLastError();
}

}  // namespace reg
