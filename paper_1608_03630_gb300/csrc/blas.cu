// Krylov vector kernels (Sec. III-A): FP64-accumulated inner products with
// warp-shuffle block reductions, and the fused PCG updates.  Scalars that the
// PCG recurrence needs (alpha, beta) are read from device memory, so an
// iteration can be captured in a CUDA graph without host round trips.
#include "common.cuh"

namespace reg {

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 152 * 4;   // partial-sum blocks (4 per SM)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_store(double v, double* partials) {
    __shared__ double red[kThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < kThreads / 32 ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) partials[blockIdx.x] = v;
    }
}

// Grid-stride dot product; float4 body when count % 4 == 0 (pointers are
// 16-byte aligned by contract).
__global__ void __launch_bounds__(kThreads)
k_dot(const float* __restrict__ a, const float* __restrict__ b, long long count,
      double* partials) {
    double acc = 0.0;
    const long long tid = (long long)blockIdx.x * kThreads + threadIdx.x;
    const long long stride = (long long)gridDim.x * kThreads;
    if ((count & 3) == 0) {
        const float4* a4 = reinterpret_cast<const float4*>(a);
        const float4* b4 = reinterpret_cast<const float4*>(b);
        const long long n4 = count >> 2;
        for (long long i = tid; i < n4; i += stride) {
            const float4 x = __ldg(a4 + i), y = __ldg(b4 + i);
            acc += (double)x.x * y.x + (double)x.y * y.y + (double)x.z * y.z +
                   (double)x.w * y.w;
        }
    } else {
        for (long long i = tid; i < count; i += stride) acc += (double)a[i] * b[i];
    }
    block_store(acc, partials);
}

// Single block: result = scale * sum(partials).
__global__ void __launch_bounds__(kThreads)
k_finalize(const double* __restrict__ partials, int nblk, double scale, double* result) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) acc += partials[i];
    __shared__ double red[kThreads / 32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
        result[0] = s * scale;
    }
}

__global__ void k_axpy(float* __restrict__ y, const float* __restrict__ x, float alpha,
                       long long count) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride)
        y[i] = fmaf(alpha, x[i], y[i]);
}

__global__ void k_axpby_out(float* __restrict__ out, const float* __restrict__ x,
                            const float* __restrict__ y, float a, float b, long long count) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride)
        out[i] = fmaf(a, x[i], b * y[i]);
}

__global__ void k_scale(float* __restrict__ y, float alpha, long long count) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride)
        y[i] *= alpha;
}

// x += alpha p; r -= alpha q; partials of r.r.  alpha = sc[ia] / sc[ib].
__global__ void __launch_bounds__(kThreads)
k_pcg_update(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
             const float* __restrict__ q, const double* __restrict__ sc, int ia, int ib,
             long long count, double* partials) {
    // a non-positive curvature p.Hp leaves the iterate unchanged (the host
    // then stops the Krylov solve)
    const double den = sc[ib];
    const float alpha = den > 0.0 ? (float)(sc[ia] / den) : 0.f;
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * kThreads;
    const long long tid = (long long)blockIdx.x * kThreads + threadIdx.x;
    if ((count & 3) == 0) {
        float4* x4 = reinterpret_cast<float4*>(x);
        float4* r4 = reinterpret_cast<float4*>(r);
        const float4* p4 = reinterpret_cast<const float4*>(p);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        for (long long i = tid; i < (count >> 2); i += stride) {
            float4 xv = x4[i], rv = r4[i];
            const float4 pv = p4[i], qv = q4[i];
            xv.x = fmaf(alpha, pv.x, xv.x); xv.y = fmaf(alpha, pv.y, xv.y);
            xv.z = fmaf(alpha, pv.z, xv.z); xv.w = fmaf(alpha, pv.w, xv.w);
            rv.x = fmaf(-alpha, qv.x, rv.x); rv.y = fmaf(-alpha, qv.y, rv.y);
            rv.z = fmaf(-alpha, qv.z, rv.z); rv.w = fmaf(-alpha, qv.w, rv.w);
            x4[i] = xv; r4[i] = rv;
            acc += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z +
                   (double)rv.w * rv.w;
        }
    } else {
        for (long long i = tid; i < count; i += stride) {
            x[i] = fmaf(alpha, p[i], x[i]);
            const float rv = fmaf(-alpha, q[i], r[i]);
            r[i] = rv;
            acc += (double)rv * rv;
        }
    }
    block_store(acc, partials);
}

// p = z + beta p, beta = sc[ia] / sc[ib].
__global__ void k_pcg_direction(float* __restrict__ p, const float* __restrict__ z,
                                const double* __restrict__ sc, int ia, int ib, long long count) {
    const double den = sc[ib];
    const float beta = den != 0.0 ? (float)(sc[ia] / den) : 0.f;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride)
        p[i] = fmaf(beta, p[i], z[i]);
}

inline int grid_for(long long count) {
    long long nb = (count + kThreads - 1) / kThreads;
    if (nb > 152 * 16) nb = 152 * 16;
    return (int)(nb < 1 ? 1 : nb);
}

}  // namespace

int blas_blocks() { return kBlocks; }

cudaError_t launch_dot_partials(const float* a, const float* b, long long count,
                                double* partials, int nblk, cudaStream_t st) {
    k_dot<<<nblk, kThreads, 0, st>>>(a, b, count, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partials, int nblk, double scale, double* result,
                            cudaStream_t st) {
    k_finalize<<<1, kThreads, 0, st>>>(partials, nblk, scale, result);
    return cudaGetLastError();
}

cudaError_t launch_axpy(float* y, const float* x, float alpha, long long count,
                        cudaStream_t st) {
    k_axpy<<<grid_for(count), kThreads, 0, st>>>(y, x, alpha, count);
    return cudaGetLastError();
}

cudaError_t launch_axpby_out(float* out, const float* x, const float* y, float a, float b,
                             long long count, cudaStream_t st) {
    k_axpby_out<<<grid_for(count), kThreads, 0, st>>>(out, x, y, a, b, count);
    return cudaGetLastError();
}

cudaError_t launch_scale(float* y, float alpha, long long count, cudaStream_t st) {
    k_scale<<<grid_for(count), kThreads, 0, st>>>(y, alpha, count);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(float* x, float* r, const float* p, const float* q,
                              const double* sc, int ia, int ib, long long count,
                              double* partials, int nblk, cudaStream_t st) {
    k_pcg_update<<<nblk, kThreads, 0, st>>>(x, r, p, q, sc, ia, ib, count, partials);
    return cudaGetLastError();
}

cudaError_t launch_pcg_direction(float* p, const float* z, const double* sc, int ia, int ib,
                                 long long count, cudaStream_t st) {
    k_pcg_direction<<<grid_for(count), kThreads, 0, st>>>(p, z, sc, ia, ib, count);
    return cudaGetLastError();
}

}  // namespace reg
