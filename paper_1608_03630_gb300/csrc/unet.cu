// The 3-D U-Net of the learned initial velocity: network state, element-wise
// kernels, forward / backward / Adam, and its C-ABI entry points.
//
// Architecture (levels L, channels ch[0..L-1]): encoder level l = conv3 ->
// ReLU -> conv3 -> ReLU (the skip), then 2x average pooling (l < L-1);
// decoder level l = L-2 .. 0: 2x nearest upsampling, concatenation with the
// skip, conv3 -> ReLU -> conv3 -> ReLU; head conv1 to cout channels.  BF16
// weights and activations, FP32 accumulation, FP32 master weights, gradients
// and Adam moments, FP64 loss.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "reg.h"
#include "unet.h"

using reg::unet::ConvGeom;
using reg::unet::IgemmArgs;
typedef __nv_bfloat16 bf16;

struct UConv {
    int ci, co, ks;
    size_t woff, boff;   // offsets of w [ks^3 ci][co] and b [co] in the flat parameters
};

struct reg_unet {
    int R, L, cin, cout;
    int ch[8];
    cudaStream_t stream;
    std::string err;
    std::vector<UConv> layers;   // enc l.0, enc l.1 (l = 0..L-1), dec l.0, dec l.1 (l = L-2..0), head
    size_t np;
    float *p, *grad, *m, *v;     // FP32 parameters, gradients, Adam moments
    bf16 *wbf, *wtbf;            // bf16 weights [k][ci][co] and transposed [k][co][ci]
    bf16* wmbf;                  // bf16 weights with mirrored offsets [K-1-k][ci][co]
    int tc;                      // forward 3x3x3 convolutions on tcgen05 where they fit (1)
                                 // or on the wmma path (0)
    long long step;
    // activations (bf16, channels last)
    bf16* xin;
    std::vector<bf16*> a0, a1, pool, cat, d0, d1;
    float* y;                    // head output [V0][cout]
    float *g1, *g2, *gcat;       // FP32 gradient scratch
    std::vector<float*> gskip;
    bf16* gb;                    // bf16 gradient operand
    float* yt;                   // packed target [V0][cout]
    double* dpart;               // loss partials
    double* hloss;               // pinned
};

namespace {

constexpr int kT = 256;

__host__ __device__ inline long long vol(int r) { return (long long)r * r * r; }

int ufail(reg_unet* u, int s, const char* msg) {
    if (u) u->err = msg;
    return s;
}

#define U_CK(u, call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return ufail(u, REG_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

#define U_TRY(call)                \
    do {                           \
        int s_ = (call);           \
        if (s_ != REG_OK) return s_; \
    } while (0)

inline int grid_of(long long n) {
    long long b = (n + kT - 1) / kT;
    if (b > 152 * 32) b = 152 * 32;
    return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- kernels

// SoA [c][V] fp32 -> channels-last [V][c] bf16
__global__ void k_pack(const float* __restrict__ x, bf16* __restrict__ out, int C, long long V) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < V * C;
         i += (long long)gridDim.x * kT) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        out[i] = __float2bfloat16(x[c * V + v]);
    }
}

// channels-last [V][c] fp32 -> SoA [c][V] fp32 (or the reverse with dir = 1)
__global__ void k_transpose_f32(const float* __restrict__ in, float* __restrict__ out, int C,
                                long long V, int to_soa) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < V * C;
         i += (long long)gridDim.x * kT) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        if (to_soa) out[c * V + v] = in[i];
        else out[i] = in[c * V + v];
    }
}

// 2x average pooling, channels last.
__global__ void k_pool(const bf16* __restrict__ in, bf16* __restrict__ out, int R, int C) {
    const int r = R / 2;
    const long long n = vol(r) * C;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const int c = (int)(i % C);
        long long v = i / C;
        const int x = (int)(v % r), y = (int)((v / r) % r), z = (int)(v / ((long long)r * r));
        float s = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const long long src = (((long long)(2 * z + (d >> 2)) * R + 2 * y + ((d >> 1) & 1)) * R +
                                   2 * x + (d & 1)) * C + c;
            s += __bfloat162float(in[src]);
        }
        out[i] = __float2bfloat16(0.125f * s);
    }
}

// gradient of pooling: out[fine] = g[coarse] / 8 (+ add[fine] if add)
__global__ void k_pool_bwd(const float* __restrict__ g, const float* __restrict__ add,
                           float* __restrict__ out, int R, int C) {
    const long long n = vol(R) * C;
    const int r = R / 2;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const int c = (int)(i % C);
        const long long v = i / C;
        const int x = (int)(v % R), y = (int)((v / R) % R), z = (int)(v / ((long long)R * R));
        const long long src = (((long long)(z / 2) * r + y / 2) * r + x / 2) * C + c;
        out[i] = 0.125f * g[src] + (add ? add[i] : 0.f);
    }
}

// nearest 2x upsampling of in [r^3][C] into cat [R^3][Ctot] channels [0, C)
__global__ void k_up(const bf16* __restrict__ in, bf16* __restrict__ cat, int R, int C, int Ctot) {
    const long long n = vol(R) * C;
    const int r = R / 2;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const int c = (int)(i % C);
        const long long v = i / C;
        const int x = (int)(v % R), y = (int)((v / R) % R), z = (int)(v / ((long long)R * R));
        cat[v * Ctot + c] = in[(((long long)(z / 2) * r + y / 2) * r + x / 2) * C + c];
    }
}

// gradient of upsampling: out[coarse][c] = sum of gcat[fine][c] over the 8 children
__global__ void k_up_bwd(const float* __restrict__ gcat, float* __restrict__ out, int R, int C,
                         int Ctot) {
    const int r = R / 2;
    const long long n = vol(r) * C;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const int c = (int)(i % C);
        const long long v = i / C;
        const int x = (int)(v % r), y = (int)((v / r) % r), z = (int)(v / ((long long)r * r));
        float s = 0.f;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const long long f = ((long long)(2 * z + (d >> 2)) * R + 2 * y + ((d >> 1) & 1)) * R +
                                2 * x + (d & 1);
            s += gcat[f * Ctot + c];
        }
        out[i] = s;
    }
}

// copy channels: dst[v][off + c] = src[v][c] (bf16), or the fp32 reverse
__global__ void k_copy_to_cat(const bf16* __restrict__ src, bf16* __restrict__ cat, long long V,
                              int C, int Ctot, int off) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < V * C;
         i += (long long)gridDim.x * kT) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        cat[v * Ctot + off + c] = src[i];
    }
}

__global__ void k_copy_from_cat(const float* __restrict__ gcat, float* __restrict__ dst,
                                long long V, int C, int Ctot, int off) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < V * C;
         i += (long long)gridDim.x * kT) {
        const long long v = i / C;
        const int c = (int)(i - v * C);
        dst[i] = gcat[v * Ctot + off + c];
    }
}

// ReLU gradient through the post-activation `act` (null: identity), bf16
// result for the GEMMs, and the bias gradient db[c] += sum_v d[v][c].  Thread
// t < (kT / C) C of a block owns channel t % C and walks voxels with stride
// (kT / C) x blocks, so the bias sum is thread-local until one shared-memory
// and one global atomic per thread.
__global__ void __launch_bounds__(kT)
k_act_bwd(const float* __restrict__ g, const bf16* __restrict__ act, bf16* __restrict__ out,
          float* __restrict__ db, long long V, int C) {
    __shared__ float sdb[128];
    for (int c = threadIdx.x; c < C; c += kT) sdb[c] = 0.f;
    __syncthreads();
    const int lanes = kT / C;
    if (threadIdx.x < lanes * C) {
        const int c = threadIdx.x % C;
        float acc = 0.f;
        for (long long v = (long long)blockIdx.x * lanes + threadIdx.x / C; v < V;
             v += (long long)gridDim.x * lanes) {
            const long long i = v * C + c;
            float d = g[i];
            if (act && __bfloat162float(act[i]) <= 0.f) d = 0.f;
            out[i] = __float2bfloat16(d);
            acc += d;
        }
        atomicAdd(&sdb[c], acc);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += kT) atomicAdd(&db[c], sdb[c]);
}

// mean squared error: dy = 2 (y - t) / N and FP64 partial sums of (y - t)^2
__global__ void __launch_bounds__(kT)
k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
      long long N, double* __restrict__ part) {
    double acc = 0.0;
    const float sc = 2.f / (float)N;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < N;
         i += (long long)gridDim.x * kT) {
        const float r = y[i] - t[i];
        acc += (double)r * r;
        dy[i] = sc * r;
    }
    __shared__ double red[kT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kT / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// bf16 copies of one layer's weights: w [k][ci][co] and wt [k][co][ci]
// BF16 copies of one layer's weights w [K][ci][co]: wb (same layout), wt
// [K][co][ci] (transposed) and wm [K][ci][co] with the kernel offsets
// mirrored (k -> K - 1 - k): the data gradient dX = sum_k dY(v - o_k) w_k^T is
// the forward convolution of dY with wm, whose K-major B operand for output
// channel ci is wm[k][ci][.].
__global__ void k_wconvert(const float* __restrict__ w, bf16* __restrict__ wb,
                           bf16* __restrict__ wt, bf16* __restrict__ wm, int K, int ci,
                           int co) {
    const long long n = (long long)K * ci * co;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n;
         i += (long long)gridDim.x * kT) {
        const int o = (int)(i % co);
        const long long t = i / co;
        const int c = (int)(t % ci);
        const long long k = t / ci;
        const bf16 b = __float2bfloat16(w[i]);
        wb[i] = b;
        wt[(k * co + o) * ci + c] = b;
        wm[((K - 1 - k) * ci + c) * co + o] = b;
    }
}

__global__ void k_finalize_sum(const double* part, int nb, double scale, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 32) s += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = s * scale;
}

// ---------------------------------------------------------------- layers

int conv_fwd(reg_unet* u, const UConv& L, int R, const bf16* x, bf16* out_bf, float* out_f,
             int out_stride, int out_off, int relu) {
    IgemmArgs a;
    memset(&a, 0, sizeof a);
    a.g = ConvGeom{R, R, R, (int)vol(R), L.ci, L.co, L.ks};
    a.A_src = x;
    a.B_src = u->wbf + L.woff;
    a.out_bf = out_bf;
    a.out_f = out_f;
    a.out_stride = out_stride;
    a.out_off = out_off;
    a.bias = u->p + L.boff;
    a.relu = relu;
    a.Bt_src = u->wtbf + L.woff;
    if (u->tc && reg::unet::conv_fwd_tc_ok(a))
        U_CK(u, reg::unet::launch_conv_fwd_tc(a, u->stream));
    else
        U_CK(u, reg::unet::launch_igemm(reg::unet::MODE_FWD, a, u->stream));
    return REG_OK;
}

// Backward of one conv given d (bf16 gradient wrt its output, after the
// activation): dW, and dX into dx (fp32 [V][dx_stride] at channel offset 0)
// when dx is not null.
int conv_bwd(reg_unet* u, const UConv& L, int R, const bf16* x, const bf16* d, float* dx) {
    IgemmArgs a;
    memset(&a, 0, sizeof a);
    a.g = ConvGeom{R, R, R, (int)vol(R), L.ci, L.co, L.ks};
    a.A_src = x;
    a.B_src = d;
    a.dW = u->grad + L.woff;
    a.kchunk = 2048;
    U_CK(u, reg::unet::launch_igemm(reg::unet::MODE_BWD_WEIGHT, a, u->stream));
    if (dx) {
        // on tcgen05: the forward convolution of dY (Ci' = co input channels)
        // with the mirrored weights to Co' = ci output channels, FP32 out
        IgemmArgs t;
        memset(&t, 0, sizeof t);
        t.g = ConvGeom{R, R, R, (int)vol(R), L.co, L.ci, L.ks};
        t.A_src = d;
        t.Bt_src = u->wmbf + L.woff;
        t.out_f = dx;
        t.out_stride = L.ci;
        t.out_off = 0;
        if (u->tc && reg::unet::conv_fwd_tc_ok(t)) {
            U_CK(u, reg::unet::launch_conv_fwd_tc(t, u->stream));
            return REG_OK;
        }
        IgemmArgs b;
        memset(&b, 0, sizeof b);
        b.g = a.g;
        b.A_src = d;
        b.B_src = u->wtbf + L.woff;
        b.dX = dx;
        b.out_stride = L.ci;
        b.out_off = 0;
        U_CK(u, reg::unet::launch_igemm(reg::unet::MODE_BWD_DATA, b, u->stream));
    }
    return REG_OK;
}

int act_bwd(reg_unet* u, const float* g, const bf16* act, const UConv& L, int R) {
    const long long n = vol(R) * L.co;
    k_act_bwd<<<grid_of(n), kT, 0, u->stream>>>(g, act, u->gb, u->grad + L.boff, vol(R), L.co);
    U_CK(u, cudaGetLastError());
    return REG_OK;
}

int convert_weights(reg_unet* u) {
    for (const auto& L : u->layers) {
        const int K = L.ks * L.ks * L.ks;
        k_wconvert<<<grid_of((long long)K * L.ci * L.co), kT, 0, u->stream>>>(
            u->p + L.woff, u->wbf + L.woff, u->wtbf + L.woff, u->wmbf + L.woff, K, L.ci, L.co);
        U_CK(u, cudaGetLastError());
    }
    return REG_OK;
}

int forward(reg_unet* u, const float* x_soa) {
    const int L = u->L;
    k_pack<<<grid_of(vol(u->R) * u->cin), kT, 0, u->stream>>>(x_soa, u->xin, u->cin, vol(u->R));
    U_CK(u, cudaGetLastError());
    const bf16* h = u->xin;
    int li = 0;
    for (int l = 0; l < L; ++l) {
        const int R = u->R >> l, C = u->ch[l];
        U_TRY(conv_fwd(u, u->layers[li++], R, h, u->a0[l], nullptr, C, 0, 1));
        U_TRY(conv_fwd(u, u->layers[li++], R, u->a0[l], u->a1[l], nullptr, C, 0, 1));
        if (l < L - 1) {
            k_pool<<<grid_of(vol(R / 2) * C), kT, 0, u->stream>>>(u->a1[l], u->pool[l], R, C);
            U_CK(u, cudaGetLastError());
            h = u->pool[l];
        } else {
            h = u->a1[l];
        }
    }
    for (int l = L - 2; l >= 0; --l) {
        const int R = u->R >> l, Cu = u->ch[l + 1], Cs = u->ch[l], Ct = Cu + Cs;
        k_up<<<grid_of(vol(R) * Cu), kT, 0, u->stream>>>(h, u->cat[l], R, Cu, Ct);
        U_CK(u, cudaGetLastError());
        k_copy_to_cat<<<grid_of(vol(R) * Cs), kT, 0, u->stream>>>(u->a1[l], u->cat[l], vol(R), Cs,
                                                                 Ct, Cu);
        U_CK(u, cudaGetLastError());
        U_TRY(conv_fwd(u, u->layers[li++], R, u->cat[l], u->d0[l], nullptr, Cs, 0, 1));
        U_TRY(conv_fwd(u, u->layers[li++], R, u->d0[l], u->d1[l], nullptr, Cs, 0, 1));
        h = u->d1[l];
    }
    return conv_fwd(u, u->layers[li], u->R, h, nullptr, u->y, u->cout, 0, 0);
}

// Backward from the FP32 gradient dy [V0][cout] in g1; accumulates u->grad.
int backward(reg_unet* u) {
    const int L = u->L;
    const int nl = (int)u->layers.size();
    // head (no activation)
    const bf16* hin = L > 1 ? u->d1[0] : u->a1[0];
    U_TRY(act_bwd(u, u->g1, nullptr, u->layers[nl - 1], u->R));
    U_TRY(conv_bwd(u, u->layers[nl - 1], u->R, hin, u->gb, u->g2));
    float* g = u->g2;       // gradient wrt the current activation
    float* spare = u->g1;
    int li = nl - 2;        // layers in reverse: dec 0.1, dec 0.0, dec 1.1, ...
    for (int l = 0; l <= L - 2; ++l) {
        const int R = u->R >> l, Cu = u->ch[l + 1], Cs = u->ch[l], Ct = Cu + Cs;
        const UConv& c1 = u->layers[li--];   // dec l.1
        const UConv& c0 = u->layers[li--];   // dec l.0
        U_TRY(act_bwd(u, g, u->d1[l], c1, R));
        U_TRY(conv_bwd(u, c1, R, u->d0[l], u->gb, spare));
        U_TRY(act_bwd(u, spare, u->d0[l], c0, R));
        U_TRY(conv_bwd(u, c0, R, u->cat[l], u->gb, u->gcat));
        k_copy_from_cat<<<grid_of(vol(R) * Cs), kT, 0, u->stream>>>(u->gcat, u->gskip[l], vol(R),
                                                                   Cs, Ct, Cu);
        U_CK(u, cudaGetLastError());
        k_up_bwd<<<grid_of(vol(R / 2) * Cu), kT, 0, u->stream>>>(u->gcat, g, R, Cu, Ct);
        U_CK(u, cudaGetLastError());
    }
    // layers of the encoder, in reverse order: enc (L-1).1, enc (L-1).0, ...
    li = 2 * L - 1;
    for (int l = L - 1; l >= 0; --l) {
        const int R = u->R >> l;
        const UConv& c1 = u->layers[li--];
        const UConv& c0 = u->layers[li--];
        U_TRY(act_bwd(u, g, u->a1[l], c1, R));
        U_TRY(conv_bwd(u, c1, R, u->a0[l], u->gb, spare));
        U_TRY(act_bwd(u, spare, u->a0[l], c0, R));
        const bf16* xin = l > 0 ? u->pool[l - 1] : u->xin;
        U_TRY(conv_bwd(u, c0, R, xin, u->gb, l > 0 ? spare : nullptr));
        if (l > 0) {
            // spare = gradient wrt pool[l-1] (level l-1 resolution / 2)
            const int Rf = u->R >> (l - 1), C = u->ch[l - 1];
            k_pool_bwd<<<grid_of(vol(Rf) * C), kT, 0, u->stream>>>(spare, u->gskip[l - 1], g, Rf, C);
            U_CK(u, cudaGetLastError());
        }
    }
    return REG_OK;
}

int loss_and_grad(reg_unet* u, const float* x, const float* t_soa, double* loss) {
    U_TRY(forward(u, x));
    const long long V = vol(u->R);
    k_transpose_f32<<<grid_of(V * u->cout), kT, 0, u->stream>>>(t_soa, u->yt, u->cout, V, 0);
    U_CK(u, cudaGetLastError());
    const int nb = 152 * 4;
    k_mse<<<nb, kT, 0, u->stream>>>(u->y, u->yt, u->g1, V * u->cout, u->dpart);
    U_CK(u, cudaGetLastError());
    k_finalize_sum<<<1, 32, 0, u->stream>>>(u->dpart, nb, 1.0 / (double)(V * u->cout),
                                            u->dpart + nb);
    U_CK(u, cudaGetLastError());
    U_CK(u, cudaMemsetAsync(u->grad, 0, sizeof(float) * u->np, u->stream));
    U_TRY(backward(u));
    if (loss) {
        U_CK(u, cudaMemcpyAsync(u->hloss, u->dpart + nb, sizeof(double), cudaMemcpyDeviceToHost,
                                u->stream));
        U_CK(u, cudaStreamSynchronize(u->stream));
        *loss = u->hloss[0];
    }
    return REG_OK;
}

void free_unet(reg_unet* u) {
    if (!u) return;
    if (u->stream) cudaStreamSynchronize(u->stream);
    std::vector<void*> ptrs = {u->p, u->grad, u->m, u->v, u->wbf, u->wtbf, u->wmbf, u->xin, u->y,
                               u->g1, u->g2, u->gcat, u->gb, u->yt, u->dpart};
    for (auto* vec : {&u->a0, &u->a1, &u->pool, &u->cat, &u->d0, &u->d1})
        for (auto q : *vec) ptrs.push_back(q);
    for (auto q : u->gskip) ptrs.push_back(q);
    for (void* q : ptrs)
        if (q) cudaFree(q);
    if (u->hloss) cudaFreeHost(u->hloss);
    delete u;
}

}  // namespace

extern "C" {

int reg_unet_create(int res, int levels, const int* ch, int cin, int cout, reg_unet** out) {
    if (!out) return REG_EINVAL;
    *out = nullptr;
    if (levels < 1 || levels > 6 || !ch || cin < 1 || cout < 1 || cin > 128 || cout > 128 ||
        res < 8)
        return REG_EINVAL;
    if (res % (1 << (levels - 1))) return REG_EINVAL;
    for (int l = 0; l < levels; ++l)
        if (ch[l] < 1 || ch[l] > 128) return REG_EINVAL;
    // voxel tiles of the GEMMs index grid.y (at most 65535 tiles of 64)
    if (vol(res) > 65535LL * 64) return REG_EINVAL;
    reg_unet* u = new (std::nothrow) reg_unet();
    if (!u) return REG_ENOMEM;
    u->R = res;
    u->L = levels;
    u->tc = 1;
    u->cin = cin;
    u->cout = cout;
    for (int l = 0; l < levels; ++l) u->ch[l] = ch[l];
    size_t off = 0;
    auto add = [&](int ci, int co, int ks) {
        UConv c{ci, co, ks, off, 0};
        off += (size_t)ks * ks * ks * ci * co;
        c.boff = off;
        off += co;
        u->layers.push_back(c);
    };
    int prev = cin;
    for (int l = 0; l < levels; ++l) {
        add(prev, ch[l], 3);
        add(ch[l], ch[l], 3);
        prev = ch[l];
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(ch[l + 1] + ch[l], ch[l], 3);
        add(ch[l], ch[l], 3);
    }
    add(ch[0], cout, 1);
    u->np = off;
    bool ok = true;
    auto dalloc = [&](void** q, size_t bytes) {
        if (ok && cudaMalloc(q, bytes) != cudaSuccess) { cudaGetLastError(); ok = false; }
    };
    dalloc((void**)&u->p, sizeof(float) * off);
    dalloc((void**)&u->grad, sizeof(float) * off);
    dalloc((void**)&u->m, sizeof(float) * off);
    dalloc((void**)&u->v, sizeof(float) * off);
    dalloc((void**)&u->wbf, sizeof(bf16) * off);
    dalloc((void**)&u->wtbf, sizeof(bf16) * off);
    dalloc((void**)&u->wmbf, sizeof(bf16) * off);
    const long long V0 = vol(res);
    dalloc((void**)&u->xin, sizeof(bf16) * V0 * cin);
    dalloc((void**)&u->y, sizeof(float) * V0 * cout);
    dalloc((void**)&u->yt, sizeof(float) * V0 * cout);
    long long gmax = V0 * (cout > cin ? cout : cin);
    u->a0.assign(levels, nullptr);
    u->a1.assign(levels, nullptr);
    u->pool.assign(levels, nullptr);
    u->cat.assign(levels, nullptr);
    u->d0.assign(levels, nullptr);
    u->d1.assign(levels, nullptr);
    u->gskip.assign(levels, nullptr);
    for (int l = 0; l < levels; ++l) {
        const long long V = vol(res >> l);
        dalloc((void**)&u->a0[l], sizeof(bf16) * V * ch[l]);
        dalloc((void**)&u->a1[l], sizeof(bf16) * V * ch[l]);
        gmax = std::max(gmax, V * ch[l]);
        if (l < levels - 1) {
            dalloc((void**)&u->pool[l], sizeof(bf16) * (V / 8) * ch[l]);
            dalloc((void**)&u->cat[l], sizeof(bf16) * V * (ch[l] + ch[l + 1]));
            dalloc((void**)&u->d0[l], sizeof(bf16) * V * ch[l]);
            dalloc((void**)&u->d1[l], sizeof(bf16) * V * ch[l]);
            dalloc((void**)&u->gskip[l], sizeof(float) * V * ch[l]);
            gmax = std::max(gmax, V * (ch[l] + ch[l + 1]));
        }
    }
    dalloc((void**)&u->g1, sizeof(float) * gmax);
    dalloc((void**)&u->g2, sizeof(float) * gmax);
    dalloc((void**)&u->gcat, sizeof(float) * gmax);
    dalloc((void**)&u->gb, sizeof(bf16) * gmax);
    dalloc((void**)&u->dpart, sizeof(double) * (152 * 4 + 1));
    if (ok && cudaMallocHost(&u->hloss, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ok = false;
    }
    if (!ok) {
        free_unet(u);
        return REG_ENOMEM;
    }
    cudaMemset(u->p, 0, sizeof(float) * off);
    cudaMemset(u->m, 0, sizeof(float) * off);
    cudaMemset(u->v, 0, sizeof(float) * off);
    *out = u;
    return REG_OK;
}

int reg_unet_destroy(reg_unet* u) {
    free_unet(u);
    return REG_OK;
}

const char* reg_unet_last_error(const reg_unet* u) { return u ? u->err.c_str() : ""; }

int reg_unet_set_stream(reg_unet* u, void* stream) {
    if (!u) return REG_EINVAL;
    u->stream = (cudaStream_t)stream;
    return REG_OK;
}

int reg_unet_set_mma(reg_unet* u, int tcgen05) {
    if (!u || (tcgen05 != 0 && tcgen05 != 1)) return REG_EINVAL;
    u->tc = tcgen05;
    return REG_OK;
}

int reg_unet_param_count(const reg_unet* u, size_t* count) {
    if (!u || !count) return REG_EINVAL;
    *count = u->np;
    return REG_OK;
}

int reg_unet_set_params(reg_unet* u, const float* host) {
    if (!u || !host) return REG_EINVAL;
    U_CK(u, cudaMemcpyAsync(u->p, host, sizeof(float) * u->np, cudaMemcpyHostToDevice, u->stream));
    U_CK(u, cudaMemsetAsync(u->m, 0, sizeof(float) * u->np, u->stream));
    U_CK(u, cudaMemsetAsync(u->v, 0, sizeof(float) * u->np, u->stream));
    u->step = 0;
    U_TRY(convert_weights(u));
    U_CK(u, cudaStreamSynchronize(u->stream));
    return REG_OK;
}

int reg_unet_get_params(reg_unet* u, float* host) {
    if (!u || !host) return REG_EINVAL;
    U_CK(u, cudaMemcpyAsync(host, u->p, sizeof(float) * u->np, cudaMemcpyDeviceToHost, u->stream));
    U_CK(u, cudaStreamSynchronize(u->stream));
    return REG_OK;
}

int reg_unet_forward(reg_unet* u, const float* x, float* y) {
    if (!u || !x || !y) return REG_EINVAL;
    U_TRY(forward(u, x));
    const long long V = vol(u->R);
    k_transpose_f32<<<grid_of(V * u->cout), kT, 0, u->stream>>>(u->y, y, u->cout, V, 1);
    U_CK(u, cudaGetLastError());
    return REG_OK;
}

int reg_unet_gradient(reg_unet* u, const float* x, const float* target, double* loss,
                      float* grad_host) {
    if (!u || !x || !target) return REG_EINVAL;
    U_TRY(loss_and_grad(u, x, target, loss));
    if (grad_host) {
        U_CK(u, cudaMemcpyAsync(grad_host, u->grad, sizeof(float) * u->np,
                                cudaMemcpyDeviceToHost, u->stream));
        U_CK(u, cudaStreamSynchronize(u->stream));
    }
    return REG_OK;
}

int reg_unet_train_step(reg_unet* u, const float* x, const float* target, float lr,
                        double* loss) {
    if (!u || !x || !target || !(lr > 0.f)) return REG_EINVAL;
    U_TRY(loss_and_grad(u, x, target, loss));
    u->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, (float)u->step));
    const float c2 = 1.f / (1.f - std::pow(b2, (float)u->step));
    k_adam<<<grid_of((long long)u->np), kT, 0, u->stream>>>(u->p, u->grad, u->m, u->v,
                                                            (long long)u->np, lr, b1, b2, 1e-8f,
                                                            c1, c2);
    U_CK(u, cudaGetLastError());
    return convert_weights(u);
}

}  // extern "C"
