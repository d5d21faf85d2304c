// Physical-space vector kernels (Sec. III-A): FP64-accumulated inner products
// with warp-shuffle block reductions, their finalisation into device scalars
// (so a launch sequence can be captured in a CUDA graph without host round
// trips), and simple vector updates.
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

// det(I + grad u) at every point, gu[(3 c + j) n + i] = d_j u_c
__global__ void k_jacobian_det(const float* __restrict__ gu, float* __restrict__ det,
                               long long n) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        float m[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < 3; ++j) m[c][j] = gu[(3 * c + j) * n + i] + (c == j ? 1.f : 0.f);
        det[i] = m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
                 m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
                 m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
    }
}

// out[c n + i] = s[i] v[c n + i], c = 0, 1, 2
__global__ void k_mul_fields(const float* __restrict__ s, const float* __restrict__ v,
                             float* __restrict__ out, long long n) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const float a = s[i];
        out[i] = a * v[i];
        out[n + i] = a * v[n + i];
        out[2 * n + i] = a * v[2 * n + i];
    }
}

__global__ void k_scale(float* __restrict__ y, float alpha, long long count) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count; i += stride)
        y[i] *= alpha;
}

// result[k] = scale * sum(partials[k * stride .. k * stride + nblk)), one block per k.
__global__ void __launch_bounds__(kThreads)
k_finalize_multi(const double* __restrict__ partials, int nblk, int stride, double scale,
                 double* result) {
    const double* p = partials + (long long)blockIdx.x * stride;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += kThreads) acc += p[i];
    __shared__ double red[kThreads / 32];
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
        result[blockIdx.x] = s * scale;
    }
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

cudaError_t launch_jacobian_det(const float* gu, float* det, long long n, cudaStream_t st) {
    k_jacobian_det<<<grid_for(n), kThreads, 0, st>>>(gu, det, n);
    return cudaGetLastError();
}

cudaError_t launch_mul_fields(const float* s, const float* v, float* out, long long n,
                              cudaStream_t st) {
    k_mul_fields<<<grid_for(n), kThreads, 0, st>>>(s, v, out, n);
    return cudaGetLastError();
}

cudaError_t launch_scale(float* y, float alpha, long long count, cudaStream_t st) {
    k_scale<<<grid_for(count), kThreads, 0, st>>>(y, alpha, count);
    return cudaGetLastError();
}

cudaError_t launch_finalize_multi(const double* partials, int nblk, int stride, int count,
                                  double scale, double* result, cudaStream_t st) {
    k_finalize_multi<<<count, kThreads, 0, st>>>(partials, nblk, stride, scale, result);
    return cudaGetLastError();
}

}  // namespace reg
