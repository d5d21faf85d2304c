// Kernels of the 3-D U-Net that predicts the initial velocity: convolutions
// as implicit GEMMs on the BF16 tensor cores (FP32 accumulation), and the
// element-wise layers (ReLU, 2x average pooling, 2x nearest upsampling,
// concatenation copies, mean-squared-error loss, Adam).
//
// Activations are channels-last [V][C] (V = D H W voxels, z slowest).  A
// convolution of kernel size ks (3 or 1, zero padding ks/2) with weights
// w[k][ci][co] (k = dz ks^2 + dy ks + dx) is the GEMM
//   forward      Y[v][co]  = sum_{k,ci} X[v + o_k][ci] w[k][ci][co]
//   data grad    dX[v][ci] = sum_{k,co} dY[v - o_k][co] w[k][ci][co]
//   weight grad  dW[k ci][co] = sum_v X[v + o_k][ci] dY[v][co]
// with the gathered operand built tile by tile in shared memory.
#include <mma.h>

#include "common.cuh"
#include "unet.h"

namespace reg {
namespace unet {

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int LDA = BK + 8;    // row-major A tile [BM][LDA]
constexpr int LDAT = BM + 8;   // k-major A tile [BK][LDAT]
constexpr int LDB = BN + 8;    // B tile [BK][LDB]
constexpr int LDC = BN + 4;    // C tile [BM][LDC] (float)

struct Vox {
    int z, y, x;
};

__device__ __forceinline__ Vox vox(const ConvGeom& g, int v) {
    Vox r;
    r.x = v % g.W;
    const int t = v / g.W;
    r.y = t % g.H;
    r.z = t / g.H;
    return r;
}

// voxel v shifted by kernel offset k (sign +1 forward, -1 for the data
// gradient), or -1 outside the volume (zero padding)
__device__ __forceinline__ int shifted(const ConvGeom& g, const Vox& p, int k, int sign) {
    const int ks = g.ks, pad = ks / 2;
    const int dz = k / (ks * ks), dy = (k / ks) % ks, dx = k % ks;
    const int z = p.z + sign * (dz - pad), y = p.y + sign * (dy - pad), x = p.x + sign * (dx - pad);
    if (z < 0 || y < 0 || x < 0 || z >= g.D || y >= g.H || x >= g.W) return -1;
    return (z * g.H + y) * g.W + x;
}

template <int MODE>
__global__ void __launch_bounds__(128)
k_igemm(IgemmArgs a) {
    __shared__ __align__(32) bf16 As[BM * LDA > BK * LDAT ? BM * LDA : BK * LDAT];
    __shared__ __align__(32) bf16 Bs[BK * LDB];
    __shared__ __align__(32) float Cs[BM * LDC];
    const ConvGeom& g = a.g;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KS3 = g.ks * g.ks * g.ks;
    int M, N, K, kbeg, kend;
    if (MODE == MODE_FWD) { M = g.V; N = g.Co; K = KS3 * g.Ci; }
    else if (MODE == MODE_BWD_DATA) { M = g.V; N = g.Ci; K = KS3 * g.Co; }
    else { M = KS3 * g.Ci; N = g.Co; K = g.V; }
    if (MODE == MODE_BWD_WEIGHT) {
        kbeg = blockIdx.z * a.kchunk;
        kend = min(K, kbeg + a.kchunk);
    } else {
        kbeg = 0;
        kend = K;
    }
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.f);
    const int wm = warp >> 1, wn = warp & 1;
    const bf16 zero = __float2bfloat16(0.f);

    for (int kt = kbeg; kt < kend; kt += BK) {
        // ---- A tile
        if (MODE != MODE_BWD_WEIGHT) {
            // thread: row r = tid / 2, 16 consecutive k starting at (tid & 1) * 16
            const int r = tid >> 1, kk0 = (tid & 1) * 16;
            const int m = m0 + r;
            const int C = (MODE == MODE_FWD) ? g.Ci : g.Co;
            const bf16* src = a.A_src;
            bf16* dst = As + r * LDA + kk0;
            if (m < M) {
                const Vox p = vox(g, m);
                int k = kt + kk0;
                int off = k / C, c = k - off * C;
                int nb = (k < kend) ? shifted(g, p, off, MODE == MODE_FWD ? 1 : -1) : -1;
#pragma unroll 4
                for (int e = 0; e < 16; ++e) {
                    dst[e] = (k < kend && nb >= 0) ? src[(long long)nb * C + c] : zero;
                    ++k;
                    if (++c == C) {
                        c = 0;
                        ++off;
                        nb = (k < kend) ? shifted(g, p, off, MODE == MODE_FWD ? 1 : -1) : -1;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) dst[e] = zero;
            }
        } else {
            // k-major: thread: voxel row kk = tid / 4, 16 consecutive m from (tid & 3) * 16
            const int kk = tid >> 2, mm0 = (tid & 3) * 16;
            const int v = kt + kk;
            bf16* dst = As + kk * LDAT + mm0;
            if (v < kend) {
                const Vox p = vox(g, v);
                int m = m0 + mm0;
                int off = m / g.Ci, c = m - off * g.Ci;
                int nb = (m < M) ? shifted(g, p, off, 1) : -1;
#pragma unroll 4
                for (int e = 0; e < 16; ++e) {
                    dst[e] = (m < M && nb >= 0) ? a.A_src[(long long)nb * g.Ci + c] : zero;
                    ++m;
                    if (++c == g.Ci) {
                        c = 0;
                        ++off;
                        nb = (m < M) ? shifted(g, p, off, 1) : -1;
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) dst[e] = zero;
            }
        }
        // ---- B tile: row kk = tid / 4, 16 consecutive n from (tid & 3) * 16
        {
            const int kk = tid >> 2, nn0 = (tid & 3) * 16;
            const int k = kt + kk;
            bf16* dst = Bs + kk * LDB + nn0;
            const bool ok = k < kend;
            const bf16* row = a.B_src + (long long)k * N;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int n = n0 + nn0 + e;
                dst[e] = (ok && n < N) ? row[n] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfr[2];
#pragma unroll
            for (int j = 0; j < 2; ++j)
                wmma::load_matrix_sync(bfr[j], Bs + ks * LDB + wn * 32 + j * 16, LDB);
            if (MODE != MODE_BWD_WEIGHT) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> afr[2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    wmma::load_matrix_sync(afr[i], As + (wm * 32 + i * 16) * LDA + ks, LDA);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], afr[i], bfr[j], acc[i][j]);
            } else {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> afr[2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    wmma::load_matrix_sync(afr[i], As + ks * LDAT + wm * 32 + i * 16, LDAT);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], afr[i], bfr[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    // ---- epilogue through shared memory
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
            wmma::store_matrix_sync(Cs + (wm * 32 + i * 16) * LDC + wn * 32 + j * 16, acc[i][j], LDC,
                                    wmma::mem_row_major);
    __syncthreads();
    for (int e = tid; e < BM * BN; e += 128) {
        const int r = e / BN, cidx = e - r * BN;
        const int m = m0 + r, n = n0 + cidx;
        if (m >= M || n >= N) continue;
        float val = Cs[r * LDC + cidx];
        if (MODE == MODE_FWD) {
            if (a.bias) val += a.bias[n];
            if (a.relu) val = fmaxf(val, 0.f);
            const long long o = (long long)m * a.out_stride + a.out_off + n;
            if (a.out_f) a.out_f[o] = val;
            else a.out_bf[o] = __float2bfloat16(val);
        } else if (MODE == MODE_BWD_DATA) {
            a.dX[(long long)m * a.out_stride + a.out_off + n] = val;
        } else {
            atomicAdd(a.dW + (long long)m * N + n, val);
        }
    }
}

}  // namespace

cudaError_t launch_igemm(int mode, const IgemmArgs& a, cudaStream_t st) {
    const ConvGeom& g = a.g;
    const int KS3 = g.ks * g.ks * g.ks;
    if (mode == MODE_FWD) {
        dim3 grid((g.Co + BN - 1) / BN, (g.V + BM - 1) / BM);
        k_igemm<MODE_FWD><<<grid, 128, 0, st>>>(a);
    } else if (mode == MODE_BWD_DATA) {
        dim3 grid((g.Ci + BN - 1) / BN, (g.V + BM - 1) / BM);
        k_igemm<MODE_BWD_DATA><<<grid, 128, 0, st>>>(a);
    } else {
        const int M = KS3 * g.Ci;
        dim3 grid((g.Co + BN - 1) / BN, (M + BM - 1) / BM, (g.V + a.kchunk - 1) / a.kchunk);
        k_igemm<MODE_BWD_WEIGHT><<<grid, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace unet
}  // namespace reg
