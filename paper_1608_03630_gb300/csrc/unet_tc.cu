// Forward 3x3x3 convolutions of the U-Net on the 5th-generation tensor cores
// (tcgen05): the implicit GEMM Y[v][co] = sum_{k,ci} X[v + o_k][ci] w[k][ci][co]
// with a 128-voxel x Co tile per CTA, the FP32 accumulator in tensor memory
// (TMEM), BF16 operands staged in shared memory in the canonical K-major
// layout without swizzle, and one thread issuing the MMAs.
//
// Shared-memory operand layout (A = gathered activations [128][32] and B =
// weights [Co][32] per K chunk of 32): "core matrices" of 8 rows x 16 bytes;
// core matrix (row group r, K group q) at byte (4 r + q) * 128, row i of it at
// + 16 i.  In the matrix descriptor the K-direction core-matrix stride
// (leading byte offset) is 128 B and the row-group stride (stride byte
// offset) 512 B; one MMA (K = 16) reads K groups 2s and 2s + 1 from the chunk
// base + 256 s.
//
// Pipeline: three stages.  Every thread copies its part of chunk q + 2 with
// 16-byte cp.async copies (8 consecutive channels of one neighbour, zero
// filled outside the volume) while the tensor core works on chunk q; when a
// chunk has landed, the threads fence it for the tensor core (async proxy)
// and synchronise, and thread 0 issues its two MMAs and commits them to the
// stage's mbarrier, which the threads wait on (bounded, about a second)
// before they refill that stage.  Epilogue: warp w reads TMEM lanes 32w ..
// 32w + 31 (its voxels) with tcgen05.ld, adds the bias, applies ReLU, and
// stores BF16 channels-last rows with 16-byte stores -- or, for the data
// gradient of a layer (the forward convolution of dY with the mirrored
// weights), stores the FP32 sums as they are.
#include <cstdint>

#include "common.cuh"
#include "unet.h"

namespace reg {
namespace unet {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TBM = 128;    // voxels per CTA (MMA M)
constexpr int TBK = 32;     // K elements per chunk (two MMAs of K = 16)
constexpr int kStages = 3;  // chunks in flight
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n"
            "  .reg .pred p;\n"
            "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "  selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// Matrix descriptor: start address, K-direction (leading) and row-group
// (stride) core-matrix offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((su32(p) & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  setp.ne.b32 p, %4, 0;\n"
        "  tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            su32(b))
        : "memory");
}

__device__ __forceinline__ void ld_tmem16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// byte offset of element group (row, K group) in a staged operand: core
// matrix (row / 8, kg) of a chunk with TBK / 8 K groups, row row % 8 of it
__device__ __forceinline__ int core_off(int row, int kg) {
    return (((row >> 3) * (TBK / 8)) + kg) * 128 + (row & 7) * 16;
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
// (src is then not read, but stays a valid address)
__device__ __forceinline__ void cp16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(dst)), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}

__device__ __forceinline__ int nbr(const ConvGeom& g, int z, int y, int x, int k) {
    const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || yy < 0 || xx < 0 || zz >= g.D || yy >= g.H || xx >= g.W) return -1;
    return (zz * g.H + yy) * g.W + xx;
}

template <int BN>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(IgemmArgs a) {
    constexpr int A_BYTES = TBM * TBK * 2;
    constexpr int B_BYTES = BN * TBK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;   // a multiple of 1024
    constexpr int TCOLS = BN < 32 ? 32 : BN;   // TMEM columns: a power of two >= 32
    constexpr int KG = TBK / 8;                // K groups per chunk
    constexpr int SBO = 128 * KG;              // row-group stride of the staged operands
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kStages * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kStages * STAGE + 8 * kStages);
    const ConvGeom& g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * TBM;
    const int Ci = g.Ci, K = 27 * Ci;
    const int nq = (K + TBK - 1) / TBK;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         su32(tslot)),
                     "r"(TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kStages; ++i) bar_init(&bar[i]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;

    // the thread's A row: voxel m0 + tid
    const int m = m0 + tid;
    const bool row_ok = m < g.V;
    int pz = 0, py = 0, px = 0;
    if (row_ok) {
        px = m % g.W;
        py = (m / g.W) % g.H;
        pz = m / (g.W * g.H);
    }
    const bf16* X = a.A_src;
    const bf16* Wt = a.Bt_src;   // [27][Co][Ci]
    constexpr uint32_t idesc = instr_desc(BN);

    // Chunks are issued in order 0, 1, 2, ..., so the gathered index
    // j = k Ci + c of every 16-byte piece advances without divisions: the A
    // pieces of a row are consecutive (8 channels each; Ci is a multiple of
    // 8), and each B piece of the thread moves by one chunk (TBK) per issue.
    int a_k = 0, a_c = 0;
    int a_nb = row_ok ? nbr(g, pz, py, px, 0) : -1;
    constexpr int NPB = (BN * KG + 127) / 128;
    int b_k[NPB], b_c[NPB];
#pragma unroll
    for (int i = 0; i < NPB; ++i) {
        const int j = ((tid + 128 * i) / BN) * 8;
        b_k[i] = j / Ci;
        b_c[i] = j - b_k[i] * Ci;
    }
    // chunk q into stage q % kStages: A row tid (KG groups of 8 channels of
    // one neighbour), B rows n (consecutive threads, consecutive n)
    auto issue = [&](int q) {
        uint8_t* As = smem + (q % kStages) * STAGE;
        uint8_t* Bs = As + A_BYTES;
#pragma unroll
        for (int kg = 0; kg < KG; ++kg) {
            const bf16* src = X;
            uint32_t bytes = 0;
            if (a_k < 27 && a_nb >= 0) {
                src = X + (long long)a_nb * Ci + a_c;
                bytes = 16;
            }
            cp16(As + core_off(tid, kg), src, bytes);
            a_c += 8;
            if (a_c == Ci) {
                a_c = 0;
                ++a_k;
                a_nb = (row_ok && a_k < 27) ? nbr(g, pz, py, px, a_k) : -1;
            }
        }
#pragma unroll
        for (int i = 0; i < NPB; ++i) {
            const int e = tid + 128 * i;
            if (e < BN * KG) {
                const int n = e % BN, kg = e / BN;
                const bf16* src = Wt;
                uint32_t bytes = 0;
                if (b_k[i] < 27) {
                    src = Wt + ((long long)b_k[i] * BN + n) * Ci + b_c[i];
                    bytes = 16;
                }
                cp16(Bs + core_off(n, kg), src, bytes);
                b_c[i] += TBK;
                while (b_c[i] >= Ci) {
                    b_c[i] -= Ci;
                    ++b_k[i];
                }
            }
        }
    };

    // prologue: chunks 0 .. kStages - 2 in flight, one commit group each
#pragma unroll
    for (int q = 0; q < kStages - 1; ++q) {
        if (q < nq) issue(q);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    bool ok = true;
    for (int q = 0; q < nq; ++q) {
        const int s = q % kStages;
        // this thread's copies of chunk q have landed (kStages - 2 newer
        // groups may still be in flight); make them visible to the tensor
        // core, then wait for every thread's
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            uint8_t* As = smem + s * STAGE;
            uint8_t* Bs = As + A_BYTES;
#pragma unroll
            for (int ks = 0; ks < TBK / 16; ++ks)
                mma_bf16(tmem, smem_desc(As + ks * 256, 128, SBO),
                         smem_desc(Bs + ks * 256, 128, SBO), idesc, (q > 0 || ks > 0) ? 1u : 0u);
            mma_commit(&bar[s]);
        }
        // refill the stage of chunk q - 1 with chunk q + kStages - 1 once the
        // MMAs of chunk q - 1 have read it
        const int qn = q + kStages - 1;
        if (qn < nq) {
            if (q >= 1) ok = bar_wait(&bar[(q - 1) % kStages], ((q - 1) / kStages) & 1) && ok;
            issue(qn);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // the last commit covers every MMA of the CTA
    ok = bar_wait(&bar[(nq - 1) % kStages], ((nq - 1) / kStages) & 1) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    // epilogue: TMEM lane = voxel row, column = output channel
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
        float v[16];
        ld_tmem16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
        if (row_ok && a.out_f) {
            // FP32 output, no bias or activation (the data gradient)
            float4* dst = reinterpret_cast<float4*>(a.out_f + (long long)m * a.out_stride +
                                                    a.out_off + c0);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float4 q = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                if (!ok) q.x = q.y = q.z = q.w = __int_as_float(0x7fffffff);
                dst[i] = q;
            }
        } else if (row_ok) {
            uint32_t w[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float lo = v[2 * i], hi = v[2 * i + 1];
                if (a.bias) {
                    lo += a.bias[c0 + 2 * i];
                    hi += a.bias[c0 + 2 * i + 1];
                }
                if (a.relu) {
                    lo = fmaxf(lo, 0.f);
                    hi = fmaxf(hi, 0.f);
                }
                if (!ok) lo = hi = __int_as_float(0x7fffffff);
                const __nv_bfloat162 p2 = __floats2bfloat162_rn(lo, hi);
                w[i] = *reinterpret_cast<const uint32_t*>(&p2);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.out_bf + (long long)m * a.out_stride +
                                                  a.out_off + c0);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(TCOLS)
                     : "memory");
}

template <int BN>
cudaError_t launch_bn(const IgemmArgs& a, cudaStream_t st) {
    constexpr int STAGE = TBM * TBK * 2 + BN * TBK * 2;
    // stages, barriers + TMEM slot, alignment slack
    const int smem = kStages * STAGE + 8 * kStages + 16 + 1024;
    // set once per process (thread-safe static initialisation)
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_conv_fwd_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (attr != cudaSuccess) return attr;
    const int grid = (a.g.V + TBM - 1) / TBM;
    k_conv_fwd_tc<BN><<<grid, 128, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool conv_fwd_tc_ok(const IgemmArgs& a) {
    const ConvGeom& g = a.g;
    const bool n_ok = g.Co == 16 || g.Co == 32 || g.Co == 64 || g.Co == 128;
    // exactly one output: BF16 (bias, ReLU) or FP32 (plain sums)
    const bool one_out = (a.out_bf != nullptr) != (a.out_f != nullptr);
    const uintptr_t al = reinterpret_cast<uintptr_t>(a.A_src) |
                         reinterpret_cast<uintptr_t>(a.Bt_src) |
                         reinterpret_cast<uintptr_t>(a.out_bf) |
                         reinterpret_cast<uintptr_t>(a.out_f);
    return g.ks == 3 && n_ok && g.Ci % 8 == 0 && g.Ci > 0 && a.Bt_src && one_out &&
           (!a.out_f || (!a.bias && !a.relu)) && (al & 15) == 0 && a.out_stride % 8 == 0 &&
           a.out_off % 8 == 0 && g.V > 0;
}

cudaError_t launch_conv_fwd_tc(const IgemmArgs& a, cudaStream_t st) {
    switch (a.g.Co) {
        case 16: return launch_bn<16>(a, st);
        case 32: return launch_bn<32>(a, st);
        case 64: return launch_bn<64>(a, st);
        case 128: return launch_bn<128>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace unet
}  // namespace reg
