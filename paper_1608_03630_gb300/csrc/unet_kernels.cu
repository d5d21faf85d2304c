// Convolutions of the 3-D U-Net that predicts the initial velocity, as
// implicit GEMMs on the BF16 tensor cores (wmma m16n16k16, FP32
// accumulation).  The element-wise layers are in unet.cu.
//
// Activations are channels-last [V][C] (V = D H W voxels, z slowest).  A
// convolution of kernel size ks (3 or 1, zero padding ks/2) with weights
// w[k][ci][co] (k = dz ks^2 + dy ks + dx) is the GEMM
//   forward      Y[v][co]  = sum_{k,ci} X[v + o_k][ci] w[k][ci][co]
//   data grad    dX[v][ci] = sum_{k,co} dY[v - o_k][co] w[k][ci][co]
//   weight grad  dW[k ci][co] = sum_v X[v + o_k][ci] dY[v][co]
// with the gathered operand built tile by tile in shared memory.  With
// channel counts that are multiples of 16, a run of 16 gathered elements is
// one neighbour's 16 consecutive channels: two 16-byte loads.  The block
// shape follows N (c_out, or c_in for the data gradient) so that layers of
// 16 or 32 channels do not waste three quarters or half of every MMA.
#include <mma.h>

#include "common.cuh"
#include "unet.h"

namespace reg {
namespace unet {

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int BK = 32;

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

// E consecutive bf16 from src (16-byte aligned when vec) into dst, or zeros
template <int E>
__device__ __forceinline__ void copy_run(bf16* dst, const bf16* src, bool vec) {
    static_assert(E % 4 == 0, "runs of 4, 8 or 16");
    if (vec && E >= 8) {
#pragma unroll
        for (int e = 0; e < E; e += 8)
            *reinterpret_cast<uint4*>(dst + e) = __ldg(reinterpret_cast<const uint4*>(src + e));
    } else if (vec) {
        *reinterpret_cast<uint2*>(dst) = __ldg(reinterpret_cast<const uint2*>(src));
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) dst[e] = src[e];
    }
}

template <int E>
__device__ __forceinline__ void zero_run(bf16* dst) {
#pragma unroll
    for (int e = 0; e < E; e += 4) *reinterpret_cast<uint2*>(dst + e) = make_uint2(0u, 0u);
}

// Gathered run of E operand elements j0 .. j0+E-1 along the gathered index
// j = offset * C + channel of voxel p (rows beyond `jend` are zero).  With
// C % E == 0 and j0 % E == 0 the run lies in one neighbour: one vector copy.
template <int E>
__device__ __forceinline__ void gather_run(bf16* dst, const bf16* src, const ConvGeom& g,
                                           const Vox& p, int j0, int jend, int C, int sign,
                                           bool vec) {
    if (vec) {
        const int off = j0 / C, c = j0 - off * C;
        const int nb = j0 < jend ? shifted(g, p, off, sign) : -1;
        if (nb >= 0) copy_run<E>(dst, src + (long long)nb * C + c, true);
        else zero_run<E>(dst);
        return;
    }
    const bf16 zero = __float2bfloat16(0.f);
    int j = j0;
    int off = j / C, c = j - off * C;
    int nb = j < jend ? shifted(g, p, off, sign) : -1;
#pragma unroll 4
    for (int e = 0; e < E; ++e) {
        dst[e] = (j < jend && nb >= 0) ? src[(long long)nb * C + c] : zero;
        ++j;
        if (++c == C) {
            c = 0;
            ++off;
            nb = j < jend ? shifted(g, p, off, sign) : -1;
        }
    }
}

// Implicit GEMM C[M][N] = A[M][K] B[K][N] on 4 warps in a WM x WN grid, warp
// tile 32 x (BN / WN), BM = 32 WM.  MODE selects which operand is gathered.
template <int MODE, int WM, int WN, int BN>
__global__ void __launch_bounds__(128)
k_igemm(IgemmArgs a) {
    constexpr int BM = 32 * WM;
    constexpr int WTN = BN / WN;          // warp tile columns (16 or 32)
    constexpr int FN = WTN / 16;          // accumulator fragments per warp row
    constexpr int LDA = BK + 8;           // row-major A tile [BM][LDA]
    constexpr int LDAT = BM + 8;          // k-major A tile [BK][LDAT]
    constexpr int LDB = BN + 8;           // B tile [BK][LDB]
    constexpr int LDC = BN + 4;           // C tile [BM][LDC] (float)
    constexpr int ASZ = BM * LDA > BK * LDAT ? BM * LDA : BK * LDAT;
    __shared__ __align__(32) bf16 As[ASZ];
    __shared__ __align__(32) bf16 Bs[BK * LDB];
    __shared__ __align__(32) float Cs[BM * LDC];
    const ConvGeom& g = a.g;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KS3 = g.ks * g.ks * g.ks;
    int M, N, K, kbeg, kend, CA;
    if (MODE == MODE_FWD) { M = g.V; N = g.Co; K = KS3 * g.Ci; CA = g.Ci; }
    else if (MODE == MODE_BWD_DATA) { M = g.V; N = g.Ci; K = KS3 * g.Co; CA = g.Co; }
    else { M = KS3 * g.Ci; N = g.Co; K = g.V; CA = g.Ci; }
    if (MODE == MODE_BWD_WEIGHT) {
        kbeg = blockIdx.z * a.kchunk;
        kend = min(K, kbeg + a.kchunk);
    } else {
        kbeg = 0;
        kend = K;
    }
    // runs along the gathered index are one vector copy when they stay in
    // one neighbour's channels; B rows when N is a multiple of the run
    constexpr int EA = (MODE == MODE_BWD_WEIGHT) ? BM / 4 : BK * BM / 128;
    constexpr int EB = BN / 4;
    const bool vecA = (CA % 16 == 0) && (((unsigned long long)a.A_src & 15) == 0);
    const bool vecB = (N % EB == 0) && (((unsigned long long)a.B_src & 15) == 0);
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][FN];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < FN; ++j) wmma::fill_fragment(acc[i][j], 0.f);
    const int wm = warp / WN, wn = warp % WN;

    // per-thread fixed coordinates of the A rows (FWD / BWD_DATA: the
    // thread's voxel row does not change along k)
    const int sign = (MODE == MODE_BWD_DATA) ? -1 : 1;
    int arow = 0, ak0 = 0;
    Vox ap = {0, 0, 0};
    bool arow_ok = false;
    if (MODE != MODE_BWD_WEIGHT) {
        constexpr int TPR = 128 / BM;     // threads per A row (2 or 1)
        arow = tid / TPR;
        ak0 = (tid % TPR) * EA;
        arow_ok = m0 + arow < M;
        if (arow_ok) ap = vox(g, m0 + arow);
    }

    for (int kt = kbeg; kt < kend; kt += BK) {
        // ---- A tile
        if (MODE != MODE_BWD_WEIGHT) {
            bf16* dst = As + arow * LDA + ak0;
            if (arow_ok) {
#pragma unroll
                for (int e = 0; e < EA; e += 16)
                    gather_run<16>(dst + e, a.A_src, g, ap, kt + ak0 + e, kend, CA, sign, vecA);
            } else {
#pragma unroll
                for (int e = 0; e < EA; e += 16) zero_run<16>(dst + e);
            }
        } else {
            // k-major: voxel row kk = tid / 4, EA consecutive m from (tid & 3) EA
            const int kk = tid >> 2, mm0 = (tid & 3) * EA;
            const int v = kt + kk;
            bf16* dst = As + kk * LDAT + mm0;
            if (v < kend) {
                const Vox p = vox(g, v);
#pragma unroll
                for (int e = 0; e < EA; e += 16)
                    gather_run<16>(dst + e, a.A_src, g, p, m0 + mm0 + e, M, CA, 1, vecA);
            } else {
#pragma unroll
                for (int e = 0; e < EA; e += 16) zero_run<16>(dst + e);
            }
        }
        // ---- B tile: row kk = tid / 4, EB consecutive n from (tid & 3) EB
        {
            const int kk = tid >> 2, nn0 = (tid & 3) * EB;
            const int k = kt + kk;
            bf16* dst = Bs + kk * LDB + nn0;
            const int n = n0 + nn0;
            if (k < kend && n + EB <= N) {
                copy_run<EB>(dst, a.B_src + (long long)k * N + n, vecB);
            } else if (k < kend && n < N) {
                const bf16* row = a.B_src + (long long)k * N;
#pragma unroll
                for (int e = 0; e < EB; ++e)
                    dst[e] = (n + e < N) ? row[n + e] : __float2bfloat16(0.f);
            } else {
                zero_run<EB>(dst);
            }
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < BK; ks += 16) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bfr[FN];
#pragma unroll
            for (int j = 0; j < FN; ++j)
                wmma::load_matrix_sync(bfr[j], Bs + ks * LDB + wn * WTN + j * 16, LDB);
            if (MODE != MODE_BWD_WEIGHT) {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> afr[2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    wmma::load_matrix_sync(afr[i], As + (wm * 32 + i * 16) * LDA + ks, LDA);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < FN; ++j) wmma::mma_sync(acc[i][j], afr[i], bfr[j], acc[i][j]);
            } else {
                wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> afr[2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    wmma::load_matrix_sync(afr[i], As + ks * LDAT + wm * 32 + i * 16, LDAT);
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < FN; ++j) wmma::mma_sync(acc[i][j], afr[i], bfr[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
    // ---- epilogue through shared memory
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < FN; ++j)
            wmma::store_matrix_sync(Cs + (wm * 32 + i * 16) * LDC + wn * WTN + j * 16, acc[i][j],
                                    LDC, wmma::mem_row_major);
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

template <int MODE, int WM, int WN, int BN>
void launch_shape(const IgemmArgs& a, int M, int N, int zdim, cudaStream_t st) {
    constexpr int BM = 32 * WM;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, zdim);
    k_igemm<MODE, WM, WN, BN><<<grid, 128, 0, st>>>(a);
}

// Block shape by the GEMM's N: 64 x 64 (2 x 2 warps) for N > 32, else
// 128 x 32 or 128 x 16 (4 x 1 warps) so narrow layers waste no MMA columns.
template <int MODE>
void launch_mode(const IgemmArgs& a, int M, int N, int zdim, cudaStream_t st) {
    if (N > 32) launch_shape<MODE, 2, 2, 64>(a, M, N, zdim, st);
    else if (N > 16) launch_shape<MODE, 4, 1, 32>(a, M, N, zdim, st);
    else launch_shape<MODE, 4, 1, 16>(a, M, N, zdim, st);
}

}  // namespace

cudaError_t launch_igemm(int mode, const IgemmArgs& a, cudaStream_t st) {
    const ConvGeom& g = a.g;
    const int KS3 = g.ks * g.ks * g.ks;
    if (mode == MODE_FWD) {
        launch_mode<MODE_FWD>(a, g.V, g.Co, 1, st);
    } else if (mode == MODE_BWD_DATA) {
        launch_mode<MODE_BWD_DATA>(a, g.V, g.Ci, 1, st);
    } else {
        launch_mode<MODE_BWD_WEIGHT>(a, KS3 * g.Ci, g.Co, (g.V + a.kchunk - 1) / a.kchunk, st);
    }
    return cudaGetLastError();
}

}  // namespace unet
}  // namespace reg
