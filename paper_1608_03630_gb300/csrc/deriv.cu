// Spectral first derivatives along one axis (Sec. III-B1) by one-dimensional
// FFTs in shared memory.
//
// The derivative d_j f = F^-1[ i k'_j F f ] needs only the transform along
// axis j: the multiplier i k'_j depends on k_j alone, so the transforms along
// the other two axes cancel (F^-1 = F_j^-1 F_other^-1 and F_other^-1 F_other
// = I).  Each block loads 32 real lines of length N along the axis, packs
// them in pairs as 16 complex lines z = a + i b, runs a forward FFT, scales
// coefficient k by i k' / N (k' = k in FFT order with the Nyquist entry set
// to 0, as every odd derivative of the library), runs the inverse FFT and
// writes Re z = d_j a and Im z = d_j b: the multiplier maps the spectrum of a
// real line to the spectrum of a real line, so the two stay apart.  One read
// and one write of the field per derivative.
//
// Lines of 32..256 points use a register-blocked four-step transform
// (below); lines of 16 and 512 points a Stockham FFT in shared memory.  On
// cubic grids of 32..256 points a side the three derivatives of a gradient
// run as one launch (k_grad_r), the blocks of the three axes side by side.
// Stockham: natural order in and out, radix 4 with one radix-2 stage when
// log2 N is odd, each stage in place in one shared buffer (every thread
// reads its butterflies' inputs into registers, the block synchronises, then
// it writes their outputs); twiddles exp(-2 pi i m / N) from a table the
// block fills with sincospif.  Lines along x3 are rows (contiguous; the
// four-step kernel loads its elements of them straight into registers);
// lines along x1 or x2 are 32 neighbouring x3 columns, staged through shared
// memory in 16-byte row segments.
#include <cstdint>
#include <mutex>

#include "common.cuh"

namespace reg {

namespace {

constexpr int kLines = 16;      // complex lines per block (32 real lines)
constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// One Stockham stage of radix R over the kLines lines of buf, in place: every
// thread first reads the inputs of all its butterflies into registers, the
// block synchronises, then every thread writes its outputs (line stride S
// complex).  Ns: length of the sub-transforms already done.  inverse:
// conjugate twiddles and butterflies.
template <int N, int R, int S>
__device__ __forceinline__ void stockham_stage(float2* buf, const float2* __restrict__ tw,
                                               int Ns, bool inverse) {
    constexpr int B = N / R;                        // butterflies per line
    constexpr int PER = (kLines * B + kThreads - 1) / kThreads;   // per thread
    float2 v[PER][R];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int w = threadIdx.x + q * kThreads;
        if (w >= kLines * B) break;
        const int line = w / B, j = w - line * B;
        const float2* src = buf + line * S;
        const int k = j % Ns;
        // twiddle angle -2 pi k r / (Ns R) = table index k r N / (Ns R)
        const int step = k * (N / (Ns * R));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 x = src[j + r * B];
            if (r > 0) {
                const float2 t = tw[(step * r) & (N - 1)];
                x = cmul(x, inverse ? conj2(t) : t);
            }
            v[q][r] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int w = threadIdx.x + q * kThreads;
        if (w >= kLines * B) break;
        const int line = w / B, j = w - line * B;
        float2* dst = buf + line * S;
        const int k = j % Ns;
        float2* u = v[q];
        if (R == 2) {
            const float2 a = u[0], b = u[1];
            u[0] = make_float2(a.x + b.x, a.y + b.y);
            u[1] = make_float2(a.x - b.x, a.y - b.y);
        } else {
            // radix-4 DFT: (a + c) +- (b + d), (a - c) -+ i (b - d) (forward)
            const float2 a = u[0], b = u[1], c = u[2], d = u[3];
            const float2 s0 = make_float2(a.x + c.x, a.y + c.y);
            const float2 s1 = make_float2(a.x - c.x, a.y - c.y);
            const float2 s2 = make_float2(b.x + d.x, b.y + d.y);
            const float2 s3 = make_float2(b.x - d.x, b.y - d.y);
            // -i s3 (forward) or +i s3 (inverse)
            const float2 t3 = inverse ? make_float2(-s3.y, s3.x) : make_float2(s3.y, -s3.x);
            u[0] = make_float2(s0.x + s2.x, s0.y + s2.y);
            u[2] = make_float2(s0.x - s2.x, s0.y - s2.y);
            u[1] = make_float2(s1.x + t3.x, s1.y + t3.y);
            u[3] = make_float2(s1.x - t3.x, s1.y - t3.y);
        }
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * Ns] = u[r];
    }
    __syncthreads();
}

// Full transform of the kLines lines of buf, in place.
template <int N, int S>
__device__ __forceinline__ void fft_lines(float2* buf, const float2* tw, bool inverse) {
    int Ns = 1;
    while (Ns * 4 <= N) {
        stockham_stage<N, 4, S>(buf, tw, Ns, inverse);
        Ns *= 4;
    }
    if (Ns < N) stockham_stage<N, 2, S>(buf, tw, Ns, inverse);
}

// AXIS 2: lines are rows (i1, i2) of length N = n3, 32 consecutive rows per
// block.  AXIS 0 / 1: lines run along x1 / x2 through 32 consecutive x3
// columns; blockIdx.x picks the 32-column group and the fixed coordinate.
// accumulate: out += d f instead of out = d f.
template <int N, int AXIS>
__global__ void __launch_bounds__(kThreads)
k_deriv(Dims g, const float* __restrict__ f, float* __restrict__ out, int accumulate) {
    constexpr int S = N + 1;                      // padded line stride (complex)
    extern __shared__ float2 sm[];
    float2* bufA = sm;
    float2* tw = sm + kLines * S;
    for (int m = threadIdx.x; m < N; m += kThreads) {
        float s, c;
        sincospif(-2.0f * (float)m / (float)N, &s, &c);
        tw[m] = make_float2(c, s);
    }
    // element (line l of 32, position a) -> global index
    long long base;
    long long lstride, astride;   // between real lines, between positions
    if (AXIS == 2) {
        base = (long long)blockIdx.x * 32 * N;
        lstride = N;
        astride = 1;
    } else {
        const int groups = g.n3 / 32;
        const int fixed = blockIdx.x / groups, col0 = (blockIdx.x - fixed * groups) * 32;
        lstride = 1;
        if (AXIS == 1) {          // fixed i1, lines along i2
            base = (long long)fixed * g.n23 + col0;
            astride = g.n3;
        } else {                  // fixed i2, lines along i1
            base = (long long)fixed * g.n3 + col0;
            astride = g.n23;
        }
    }
    // load: consecutive threads take consecutive elements of the fast index
    float* bufAf = reinterpret_cast<float*>(bufA);
    for (int e = threadIdx.x; e < 32 * N; e += kThreads) {
        int l, a;
        if (AXIS == 2) { l = e / N; a = e - l * N; }
        else { a = e >> 5; l = e & 31; }
        bufAf[2 * ((l >> 1) * S + a) + (l & 1)] = __ldg(f + base + l * lstride + a * astride);
    }
    __syncthreads();
    fft_lines<N, S>(bufA, tw, false);
    float2* z = bufA;
    // i k' / N, k' = k in FFT order, Nyquist 0
    const float inv_n = 1.0f / (float)N;
    for (int e = threadIdx.x; e < kLines * N; e += kThreads) {
        const int l = e / N, k = e - l * N;
        const float kk = (2 * k < N) ? (float)k : (2 * k == N ? 0.f : (float)(k - N));
        const float2 v = z[l * S + k];
        z[l * S + k] = make_float2(-kk * inv_n * v.y, kk * inv_n * v.x);
    }
    __syncthreads();
    fft_lines<N, S>(z, tw, true);
    const float* zf = reinterpret_cast<const float*>(z);
    for (int e = threadIdx.x; e < 32 * N; e += kThreads) {
        int l, a;
        if (AXIS == 2) { l = e / N; a = e - l * N; }
        else { a = e >> 5; l = e & 31; }
        const long long gi = base + l * lstride + a * astride;
        const float d = zf[2 * ((l >> 1) * S + a) + (l & 1)];
        out[gi] = accumulate ? out[gi] + d : d;
    }
}

// ------------------------------------------ register-blocked four-step FFT
// N = N1 N2 (N1 >= N2, both powers of two, N1 <= 16): a line is held by N2
// threads, thread t owning x[t + N2 m] (m < N1).  Forward: a DFT of size N1
// over m in registers, the twiddle exp(-2 pi i t q / N), a transpose through
// shared memory, and thread s computes, for each q = s + N2 j, the DFT of
// size N2 over t; it then owns X[q + N1 r] = X[s + N2 (j + (N1 / N2) r)]: the
// same stride-N2 ownership as the input, so the inverse transform runs the
// same steps on it and returns y[s + N2 m] to thread s.  Two transposes per
// derivative instead of a shared-memory pass per radix stage.

// exp(-2 pi i k / 16), k < 8 (the roots of the register DFTs, sizes <= 16)
__device__ __forceinline__ float2 root16(int k) {
    switch (k) {
    case 0: return make_float2(1.f, 0.f);
    case 1: return make_float2(0.92387953251128674f, -0.38268343236508977f);
    case 2: return make_float2(0.70710678118654752f, -0.70710678118654752f);
    case 3: return make_float2(0.38268343236508977f, -0.92387953251128674f);
    case 4: return make_float2(0.f, -1.f);
    case 5: return make_float2(-0.38268343236508977f, -0.92387953251128674f);
    case 6: return make_float2(-0.70710678118654752f, -0.70710678118654752f);
    default: return make_float2(-0.92387953251128674f, -0.38268343236508977f);
    }
}

__host__ __device__ constexpr int bitrev(int i, int L) {
    int r = 0;
    for (int b = 1; b < L; b <<= 1) {
        r = (r << 1) | (i & 1);
        i >>= 1;
    }
    return r;
}

// Bit-reversal permutation of a register array, every index a compile-time
// constant (so the array stays in registers).
template <int L, int I = 0>
__device__ __forceinline__ void bitrev_swap(float2 (&v)[L]) {
    if constexpr (I < L) {
        constexpr int J = bitrev(I, L);
        if constexpr (I < J) {
            const float2 t = v[I];
            v[I] = v[J];
            v[J] = t;
        }
        bitrev_swap<L, I + 1>(v);
    }
}

// One radix-2 stage (butterflies of span LEN) of the in-register DFT.
template <int L, int LEN>
__device__ __forceinline__ void dft_stage(float2 (&v)[L], bool inverse) {
#pragma unroll
    for (int i = 0; i < L; i += LEN) {
#pragma unroll
        for (int k = 0; k < LEN / 2; ++k) {
            float2 w = root16(k * (16 / LEN));
            if (inverse) w.y = -w.y;
            const float2 a = v[i + k];
            const float2 b = cmul(v[i + k + LEN / 2], w);
            v[i + k] = make_float2(a.x + b.x, a.y + b.y);
            v[i + k + LEN / 2] = make_float2(a.x - b.x, a.y - b.y);
        }
    }
    if constexpr (2 * LEN <= L) dft_stage<L, 2 * LEN>(v, inverse);
}

// In-register DFT of size L (radix 2, decimation in time), forward or
// inverse (conjugate roots); natural order in and out, every register index
// a compile-time constant.
template <int L>
__device__ __forceinline__ void dft_reg(float2 (&v)[L], bool inverse) {
    bitrev_swap<L>(v);
    dft_stage<L, 2>(v, inverse);
}

// One four-step transform of the block's 16 lines held in registers
// (ownership as above); T: shared transpose buffer [16][N1][N2 + 1].
template <int N1, int N2>
__device__ __forceinline__ void fourstep(float2 (&v)[N1], float2* T, const float2* tw, int line,
                                         int t, bool inverse) {
    constexpr int N = N1 * N2;
    constexpr int TS = N2 + 1;
    dft_reg<N1>(v, inverse);
#pragma unroll
    for (int q = 0; q < N1; ++q) {
        float2 w = tw[(t * q) & (N - 1)];
        if (inverse) w.y = -w.y;
        v[q] = cmul(v[q], w);
    }
    float2* Tl = T + line * N1 * TS;
#pragma unroll
    for (int q = 0; q < N1; ++q) Tl[q * TS + t] = v[q];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N1 / N2; ++j) {
        float2 c[N2];
#pragma unroll
        for (int u = 0; u < N2; ++u) c[u] = Tl[(t + N2 * j) * TS + u];
        dft_reg<N2>(c, inverse);
        // thread t now owns X[t + N2 (j + (N1 / N2) r)], r < N2
#pragma unroll
        for (int r = 0; r < N2; ++r) v[j + (N1 / N2) * r] = c[r];
    }
    __syncthreads();
}

// Column tile (lines along x1 or x2: RL = 2 LC neighbouring x3 columns) <->
// shared complex lines, in 16-byte global accesses with every load of a
// thread issued before its first shared-memory store (the bytes in flight
// per SM are what bounds a streaming kernel).  Complex line c of the block
// holds real lines 2c (Re) and 2c + 1 (Im) at stride S.  A unit is (position,
// 4 neighbouring real lines): one float4 of a row, stored as two complex
// values.  (Rows along x3 need no staging: the kernel loads them straight
// into registers.)
template <int N, int LC, int TH>
struct TileRegs {   // one thread's share of a block tile, between load and store
    static constexpr int G = LC / 2;        // float4 units per position
    static constexpr int U = G * N;
    static_assert(U % TH == 0, "units per thread");
    float4 x[U / TH];
};

template <int N, int LC, int TH>
__device__ __forceinline__ void tile_fetch(TileRegs<N, LC, TH>& r, const float* __restrict__ f,
                                           long long base, long long astride) {
    constexpr int G = TileRegs<N, LC, TH>::G;
#pragma unroll
    for (int q = 0; q < TileRegs<N, LC, TH>::U / TH; ++q) {
        const int u = threadIdx.x + q * TH;
        const int a = u / G, l4 = 4 * (u % G);
        r.x[q] = __ldg(reinterpret_cast<const float4*>(f + base + l4 + a * astride));
    }
}

template <int N, int LC, int S, int TH>
__device__ __forceinline__ void tile_put(float2* buf, const TileRegs<N, LC, TH>& r) {
    constexpr int G = TileRegs<N, LC, TH>::G;
#pragma unroll
    for (int q = 0; q < TileRegs<N, LC, TH>::U / TH; ++q) {
        const int u = threadIdx.x + q * TH;
        const int a = u / G, c = 2 * (u % G);
        buf[c * S + a] = make_float2(r.x[q].x, r.x[q].y);
        buf[(c + 1) * S + a] = make_float2(r.x[q].z, r.x[q].w);
    }
}

template <int N, int LC, int S, int TH>
__device__ __forceinline__ void tile_store(const float2* buf, float* __restrict__ out,
                                           long long base, long long astride, int accumulate) {
    constexpr int G = LC / 2;
#pragma unroll
    for (int q = 0; q < G * N / TH; ++q) {
        const int u = threadIdx.x + q * TH;
        const int a = u / G, c = 2 * (u % G);
        const float2 z0 = buf[c * S + a], z1 = buf[(c + 1) * S + a];
        float4 w = make_float4(z0.x, z0.y, z1.x, z1.y);
        float4* d = reinterpret_cast<float4*>(out + base + 4 * (u % G) + a * astride);
        if (accumulate) {
            const float4 p = *d;
            w.x += p.x; w.y += p.y; w.z += p.z; w.w += p.w;
        }
        *d = w;
    }
}

// Complex lines per block of the four-step kernel (2 LC real lines: rows
// along x3, or neighbouring x3 columns along x1 / x2).  With MINB = 3 blocks
// an SM (48 / LC) the 256-point kernel keeps 80 registers; 8 or 32 lines,
// and 2 or 4 blocks an SM, measured slower on the column axes at 256^3.
constexpr int kDerivLines = 16;

// The lines of block `blk` of one axis (the block's whole work; sm: its
// dynamic shared memory).
template <int N1, int N2, int AXIS, int LC>
__device__ __forceinline__ void deriv_lines(const Dims& g, const float* __restrict__ f,
                                            float* __restrict__ out, int accumulate, int blk,
                                            float2* sm) {
    constexpr int N = N1 * N2;
    constexpr int S = N + 1;                       // load buffer line stride
    constexpr int TH = LC * N2;                    // threads
    constexpr int RL = 2 * LC;                     // real lines per block
    float2* buf = sm;                              // max(LC S, LC N1 (N2 + 1)) complex
    float2* tw = sm + (LC * S > LC * N1 * (N2 + 1) ? LC * S : LC * N1 * (N2 + 1));
    for (int m = threadIdx.x; m < N; m += TH) {
        float sn, cs;
        sincospif(-2.0f * (float)m / (float)N, &sn, &cs);
        tw[m] = make_float2(cs, sn);
    }
    long long base, astride;
    if (AXIS == 2) {
        base = (long long)blk * RL * N;
        astride = 1;
    } else {
        const int groups = g.n3 / RL;
        const int fixed = blk / groups, col0 = (blk - fixed * groups) * RL;
        if (AXIS == 1) { base = (long long)fixed * g.n23 + col0; astride = g.n3; }
        else { base = (long long)fixed * g.n3 + col0; astride = g.n23; }
    }
    const int line = threadIdx.x / N2, t = threadIdx.x - line * N2;
    float2 v[N1];
    if constexpr (AXIS == 2) {
        // rows are contiguous: each thread loads its stride-N2 elements of
        // the two real rows of its complex line straight into registers
        // (a warp reads 64-byte row segments); no staging pass
        const float* r0 = f + base + (long long)(2 * line) * N + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = make_float2(__ldg(r0 + N2 * m), __ldg(r0 + N + N2 * m));
        __syncthreads();                           // the twiddle table
    } else {
        TileRegs<N, LC, TH> r;
        tile_fetch<N, LC, TH>(r, f, base, astride);
        tile_put<N, LC, S, TH>(buf, r);
        __syncthreads();
#pragma unroll
        for (int m = 0; m < N1; ++m) v[m] = buf[line * S + t + N2 * m];
        __syncthreads();                           // buf becomes the transpose buffer
    }
    fourstep<N1, N2>(v, buf, tw, line, t, false);
    // i k' / N at k = t + N2 m (Nyquist 0)
    const float inv_n = 1.0f / (float)N;
#pragma unroll
    for (int m = 0; m < N1; ++m) {
        const int k = t + N2 * m;
        const float kk = (2 * k < N) ? (float)k : (2 * k == N ? 0.f : (float)(k - N));
        v[m] = make_float2(-kk * inv_n * v[m].y, kk * inv_n * v[m].x);
    }
    fourstep<N1, N2>(v, buf, tw, line, t, true);
    if constexpr (AXIS == 2) {
        float* o0 = out + base + (long long)(2 * line) * N + t;
#pragma unroll
        for (int m = 0; m < N1; ++m) {
            float re = v[m].x, im = v[m].y;
            if (accumulate) {
                re += o0[N2 * m];
                im += o0[N + N2 * m];
            }
            o0[N2 * m] = re;
            o0[N + N2 * m] = im;
        }
    } else {
#pragma unroll
        for (int m = 0; m < N1; ++m) buf[line * S + t + N2 * m] = v[m];
        __syncthreads();
        tile_store<N, LC, S, TH>(buf, out, base, astride, accumulate);
    }
}

template <int N1, int N2, int AXIS, int LC, int MINB = 48 / LC>
__global__ void __launch_bounds__(LC * N2, MINB)
k_deriv_r(Dims g, const float* __restrict__ f, float* __restrict__ out, int accumulate) {
    extern __shared__ float2 sm[];
    deriv_lines<N1, N2, AXIS, LC>(g, f, out, accumulate, blockIdx.x, sm);
}

// The three derivatives of a gradient in one launch (cubic grids: every axis
// has N^2 / (2 LC) blocks, the same count): blocks [0, per) take x1,
// [per, 2 per) x2, [2 per, 3 per) x3, so the launch has one tail instead of
// three and the field's second and third reads can come from L2.
template <int N1, int N2, int LC, int MINB = 48 / LC>
__global__ void __launch_bounds__(LC * N2, MINB)
k_grad_r(Dims g, const float* __restrict__ f, float* __restrict__ out3, int per) {
    extern __shared__ float2 sm[];
    const int ax = blockIdx.x / per, blk = blockIdx.x - ax * per;
    float* out = out3 + (long long)ax * g.n;
    if (ax == 0) deriv_lines<N1, N2, 0, LC>(g, f, out, 0, blk, sm);
    else if (ax == 1) deriv_lines<N1, N2, 1, LC>(g, f, out, 0, blk, sm);
    else deriv_lines<N1, N2, 2, LC>(g, f, out, 0, blk, sm);
}

template <int N1, int N2, int AXIS>
cudaError_t run_deriv_r(const Dims& g, const float* f, float* out, int accumulate,
                        cudaStream_t st) {
    constexpr int LC = kDerivLines;
    constexpr int N = N1 * N2;
    const int bufc = LC * (N + 1) > LC * N1 * (N2 + 1) ? LC * (N + 1) : LC * N1 * (N2 + 1);
    const size_t smem = sizeof(float2) * (bufc + N);
    if (smem > 48 * 1024) {
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [&] {
            attr = cudaFuncSetAttribute(k_deriv_r<N1, N2, AXIS, LC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (attr != cudaSuccess) return attr;
    }
    int blocks;
    if (AXIS == 2) blocks = g.n1 * g.n2 / (2 * LC);
    else blocks = (AXIS == 1 ? g.n1 : g.n2) * (g.n3 / (2 * LC));
    k_deriv_r<N1, N2, AXIS, LC><<<blocks, LC * N2, smem, st>>>(g, f, out, accumulate);
    return cudaGetLastError();
}

template <int N1, int N2>
cudaError_t run_grad_r(const Dims& g, const float* f, float* out3, cudaStream_t st) {
    constexpr int LC = kDerivLines;
    constexpr int N = N1 * N2;
    const int bufc = LC * (N + 1) > LC * N1 * (N2 + 1) ? LC * (N + 1) : LC * N1 * (N2 + 1);
    const size_t smem = sizeof(float2) * (bufc + N);
    if (smem > 48 * 1024) {
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [&] {
            attr = cudaFuncSetAttribute(k_grad_r<N1, N2, LC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (attr != cudaSuccess) return attr;
    }
    const int per = N * N / (2 * LC);              // blocks per axis (n1 = n2 = n3 = N)
    k_grad_r<N1, N2, LC><<<3 * per, LC * N2, smem, st>>>(g, f, out3, per);
    return cudaGetLastError();
}

template <int N, int AXIS>
cudaError_t run_deriv(const Dims& g, const float* f, float* out, int accumulate, cudaStream_t st) {
    const size_t smem = sizeof(float2) * (kLines * (N + 1) + N);
    if (smem > 48 * 1024) {
        // once per kernel instantiation (thread-safe)
        static std::once_flag once;
        static cudaError_t attr = cudaSuccess;
        std::call_once(once, [&] {
            attr = cudaFuncSetAttribute(k_deriv<N, AXIS>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        });
        if (attr != cudaSuccess) return attr;
    }
    int blocks;
    if (AXIS == 2) blocks = g.n1 * g.n2 / 32;
    else blocks = (AXIS == 1 ? g.n1 : g.n2) * (g.n3 / 32);
    k_deriv<N, AXIS><<<blocks, kThreads, smem, st>>>(g, f, out, accumulate);
    return cudaGetLastError();
}

template <int AXIS>
cudaError_t dispatch(const Dims& g, int N, const float* f, float* out, int acc, cudaStream_t st) {
    switch (N) {
    case 16: return run_deriv<16, AXIS>(g, f, out, acc, st);
    case 32: return run_deriv_r<8, 4, AXIS>(g, f, out, acc, st);
    case 64: return run_deriv_r<8, 8, AXIS>(g, f, out, acc, st);
    case 128: return run_deriv_r<16, 8, AXIS>(g, f, out, acc, st);
    case 256: return run_deriv_r<16, 16, AXIS>(g, f, out, acc, st);
    case 512: return run_deriv<512, AXIS>(g, f, out, acc, st);
    default: return cudaErrorNotSupported;
    }
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace

bool deriv_supported(const Dims& g, const void* f, const void* out) {
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(out)) & 15;
    return mis == 0 && pow2_in(g.n1, 16, 512) && pow2_in(g.n2, 16, 512) &&
           pow2_in(g.n3, 32, 512);
}

cudaError_t launch_grad(const Dims& g, const float* f, float* out3, cudaStream_t st) {
    if (!deriv_supported(g, f, out3) || g.n1 != g.n2 || g.n1 != g.n3)
        return cudaErrorNotSupported;
    switch (g.n1) {
    case 32: return run_grad_r<8, 4>(g, f, out3, st);
    case 64: return run_grad_r<8, 8>(g, f, out3, st);
    case 128: return run_grad_r<16, 8>(g, f, out3, st);
    case 256: return run_grad_r<16, 16>(g, f, out3, st);
    default: return cudaErrorNotSupported;
    }
}

cudaError_t launch_deriv(const Dims& g, int axis, const float* f, float* out, int accumulate,
                         cudaStream_t st) {
    if (!deriv_supported(g, f, out)) return cudaErrorNotSupported;
    if (axis == 0) return dispatch<0>(g, g.n1, f, out, accumulate, st);
    if (axis == 1) return dispatch<1>(g, g.n2, f, out, accumulate, st);
    return dispatch<2>(g, g.n3, f, out, accumulate, st);
}

}  // namespace reg
