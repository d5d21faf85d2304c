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
// FFT: Stockham autosort (natural order in and out), radix 4 with one
// radix-2 stage when log2 N is odd, each stage in place in one shared buffer
// (every thread reads its butterflies' inputs into registers, the block
// synchronises, then it writes their outputs); twiddles exp(-2 pi i m / N)
// from a table the block fills with sincospif.  Lines along x3 are rows (contiguous); lines along x1 or x2
// are 32 neighbouring x3 columns, so every global access is a coalesced
// 128-byte row segment.
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
    case 32: return run_deriv<32, AXIS>(g, f, out, acc, st);
    case 64: return run_deriv<64, AXIS>(g, f, out, acc, st);
    case 128: return run_deriv<128, AXIS>(g, f, out, acc, st);
    case 256: return run_deriv<256, AXIS>(g, f, out, acc, st);
    case 512: return run_deriv<512, AXIS>(g, f, out, acc, st);
    default: return cudaErrorNotSupported;
    }
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace

bool deriv_supported(const Dims& g) {
    return pow2_in(g.n1, 16, 512) && pow2_in(g.n2, 16, 512) && pow2_in(g.n3, 32, 512);
}

cudaError_t launch_deriv(const Dims& g, int axis, const float* f, float* out, int accumulate,
                         cudaStream_t st) {
    if (!deriv_supported(g)) return cudaErrorNotSupported;
    if (axis == 0) return dispatch<0>(g, g.n1, f, out, accumulate, st);
    if (axis == 1) return dispatch<1>(g, g.n2, f, out, accumulate, st);
    return dispatch<2>(g, g.n3, f, out, accumulate, st);
}

}  // namespace reg
