// Semi-Lagrangian kernels (Sec. III-B2, Sec. III-C2, Algorithm 2): RK2
// points, tricubic Lagrange interpolation and the fused transport steps of
// the state, adjoint, incremental state and incremental adjoint.
//
// Every transport step gathers ONE scalar field at the semi-Lagrangian
// points:
//   state            rho_{j+1} = I[rho_j](X)
//   (inc.) adjoint   lam_j = c(x) I[lam_{j+1}](X)        (source lam div v)
//   inc. state       u_{j+1} = I[u_j](X) + dt f_{j+1}(x),  u = rho~ + dt/2 f
// (the last two are exact rearrangements of Eq. (sml-advection), see the
// launchers).  The gather runs in x1-marching kernels: a block is 32 lanes
// along x3 (coalesced per-point reads and writes) by wy rows along x2, and
// each thread walks k consecutive points along x1.  The 4 x 4 x 4 stencil
// values stay in registers as four x1-planes of 4 x 4; when the next point's
// stencil is the current one shifted by one plane along x1 (same x2/x3 base),
// only the new plane (16 values) is loaded and the other 48 are reused.  The
// plane slots rotate with a period of four unrolled steps, so every register
// index is static.
#include <atomic>
#include <climits>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda.h>            // CUtensorMap and its enums (no driver library link:
#include <cudaTypedefs.h>    // the encoder is fetched through the runtime)

#include "common.cuh"

namespace reg {

namespace {

constexpr int kThreads = 256;

inline int nblocks(long long n) { return (int)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ float ld(const float* p, long long i) { return __ldg(p + i); }

// ------------------------------------------------------ plain gather kernels

// Eq. (sml-trajectory) for v and -v.  dth_j = dt / h_j converts a velocity
// to grid units per step.
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
    // forward: X* = x - dt v(x), X = x - dt/2 (v(x) + v(X*))
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

// ---------------------------------------------------- x1-marching kernels

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) {
        s = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// i mod n for i in [-n, 2n) with two compares; any other i through wrap().
__device__ __forceinline__ int wrap_near(int i, int n) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) i = wrap(i, n);
    return i;
}

struct Window {
    float w[4][16];   // four x1-planes of 4 (x2) x 4 (x3) stencil values
    int off;          // wrapped x2 base * n3 + wrapped x3 base (interior stencils)
    int o2[4], o3[4]; // per-node offsets, for stencils that wrap in x2 or x3
    bool interior;    // no wrap in x2 and x3: rows are off + b n3, columns + c
    int cp, cb2, cb3; // unwrapped plane of node -1, x2 and x3 bases of the cache
};

template <int SLOT>
__device__ __forceinline__ void load_plane(Window& W, const float* __restrict__ f,
                                           const Dims& g, int plane) {
    const float* base = f + (long long)wrap_near(plane, g.n1) * g.n23;
    if (W.interior) {
        const float* q = base + W.off;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float* row = q + b * g.n3;
#pragma unroll
            for (int c = 0; c < 4; ++c) W.w[SLOT][b * 4 + c] = __ldg(row + c);
        }
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) W.w[SLOT][b * 4 + c] = __ldg(base + W.o2[b] + W.o3[c]);
    }
}

// One marching step at rotation R: interpolate f at the point (i1, i2, i3) +
// (d1, d2, d3) using and updating the window.
template <int R>
__device__ __forceinline__ float march_interp(Window& W, const float* __restrict__ f,
                                              const Dims& g, int i1, int i2, int i3, float d1,
                                              float d2, float d3) {
    const float fl1 = floorf(d1), fl2 = floorf(d2), fl3 = floorf(d3);
    float w1[4], w2[4], w3[4];
    lagrange4(d1 - fl1, w1);
    lagrange4(d2 - fl2, w2);
    lagrange4(d3 - fl3, w3);
    const int p = i1 + (int)fl1 - 1;
    const int b2 = i2 + (int)fl2 - 1;
    const int b3 = i3 + (int)fl3 - 1;
    if (!(b2 == W.cb2 && b3 == W.cb3 && p == W.cp + 1)) {
        const int q2 = wrap_near(b2, g.n2), q3 = wrap_near(b3, g.n3);
        W.interior = (q2 <= g.n2 - 4) && (q3 <= g.n3 - 4);
        W.off = q2 * g.n3 + q3;
        if (!W.interior) {
            int r2 = q2, r3 = q3;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                W.o2[a] = r2 * g.n3;
                W.o3[a] = r3;
                r2 = (r2 + 1 == g.n2) ? 0 : r2 + 1;
                r3 = (r3 + 1 == g.n3) ? 0 : r3 + 1;
            }
        }
        W.cb2 = b2;
        W.cb3 = b3;
        load_plane<(R + 0) & 3>(W, f, g, p);
        load_plane<(R + 1) & 3>(W, f, g, p + 1);
        load_plane<(R + 2) & 3>(W, f, g, p + 2);
    }
    W.cp = p;
    load_plane<(R + 3) & 3>(W, f, g, p + 3);
    float val = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float* pl = W.w[(R + a) & 3];
        float r = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float s = w3[0] * pl[b * 4 + 0];
            s = fmaf(w3[1], pl[b * 4 + 1], s);
            s = fmaf(w3[2], pl[b * 4 + 2], s);
            s = fmaf(w3[3], pl[b * 4 + 3], s);
            r = fmaf(w2[b], s, r);
        }
        val = fmaf(w1[a], r, val);
    }
    return val;
}

// Epilogues: pre(idx) loads the per-point inputs that do not depend on the
// gather (issued four points ahead of use), post(idx, val, pre, acc)
// finishes the point, done(acc) runs once per thread after the march (all
// threads of the block, for reductions).

struct EpiStore {            // out = val
    static constexpr bool kPreFixed = true;
    float* out;
    struct Pre {};
    __device__ Pre pre(int) const { return {}; }
    __device__ void post(int idx, float val, const Pre&, double&) const { out[idx] = val; }
    __device__ void done(double) const {}
};

struct EpiStateFinal {       // out = val; lam = rho_R - val; sum (val - rho_R)^2
    static constexpr bool kPreFixed = true;
    float* out;
    const float* rho_R;
    float* lam;              // may be null
    double* partials;
    struct Pre { float r; };
    __device__ Pre pre(int idx) const { return {__ldg(rho_R + idx)}; }
    __device__ void post(int idx, float val, const Pre& p, double& acc) const {
        out[idx] = val;
        const float l = p.r - val;
        if (lam) lam[idx] = l;
        acc += (double)(l * l);
    }
    __device__ void done(double acc) const {
        const double s = block_sum(acc);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
    }
};

// Adjoint step fused with the time integral b = sum_j w_j lam_j grad rho_j
// (trapezoid rule): lam_j = c(x) val is stored for the next step (out may be
// null after the last one) and b at the output point gains w lam_j grad_j.
// init (first step): b starts from w_first lam_first grad_first at the point
// (the level the solve starts from) instead of its stored value.  dotp (last
// step): per-block FP64 partial sums of <dotp, b>.  kAdd: lam_j = c(x) val +
// add(x), the known-source part of the step (full Newton incremental
// adjoint); a separate instantiation, so the Gauss-Newton path loads nothing
// more.
template <bool kAdd>
struct EpiAdjAccT {
    static constexpr bool kPreFixed = false;   // b: the previous step's output
    float* out;
    const float* c;          // may be null (c = 1)
    const float* grad;       // grad rho_j [3n]
    float* b;                // [3n], read and written at the output point
    long long n;
    float w;
    const float* lam_first;  // init only (else null)
    const float* grad_first;
    float w_first;
    const float* dotp;       // last step only (else null)
    double* partials;
    const float* add;        // kAdd only: [n] added to lam_j
    Fin fin;                 // last step: finish <dotp, b> in the launch (count may be null)
    struct Pre { float c, g0, g1, g2, b0, b1, b2, a; };
    __device__ Pre pre(int idx) const {
        Pre p;
        p.c = c ? __ldg(c + idx) : 1.f;
        p.g0 = ld(grad, idx);
        p.g1 = ld(grad, n + idx);
        p.g2 = ld(grad, 2 * n + idx);
        // b and lam(1) are written by earlier steps (in the persistent
        // small-grid kernel, earlier in the same launch): L2-coherent loads
        if (lam_first) {
            const float l = w_first * __ldcg(lam_first + idx);
            p.b0 = l * ld(grad_first, idx);
            p.b1 = l * ld(grad_first, n + idx);
            p.b2 = l * ld(grad_first, 2 * n + idx);
        } else {
            p.b0 = __ldcg(b + idx);
            p.b1 = __ldcg(b + n + idx);
            p.b2 = __ldcg(b + 2 * n + idx);
        }
        p.a = kAdd ? __ldg(add + idx) : 0.f;
        return p;
    }
    __device__ void post(int idx, float val, const Pre& p, double& acc) const {
        const float lam = kAdd ? fmaf(p.c, val, p.a) : p.c * val;
        if (out) out[idx] = lam;
        const float l = w * lam;
        const float b0 = fmaf(l, p.g0, p.b0), b1 = fmaf(l, p.g1, p.b1), b2 = fmaf(l, p.g2, p.b2);
        b[idx] = b0;
        b[n + idx] = b1;
        b[2 * n + idx] = b2;
        if (dotp)
            acc += (double)fmaf(dotp[idx], b0, fmaf(dotp[n + idx], b1, dotp[2 * n + idx] * b2));
    }
    __device__ void done(double acc) const {
        if (!dotp) return;   // uniform over the grid
        const double s = block_sum(acc);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
        if (fin.count) finish_partials<1>(partials, gridDim.x * gridDim.y * gridDim.z, fin);
    }
};
using EpiAdjAcc = EpiAdjAccT<false>;

// Known-source part of an adjoint tau-step (Eq. sml-advection with a source
// s(x, t) that does not depend on the transported field): the step reaches
// lam_new = c(x) I[lam_old](X) + dt/2 (1 + dt dv(x)) I[s_old](X) + dt/2 s_new(x)
// (dv = div v; 0 when divergence free).  This epilogue writes the last two
// terms, val = I[s_old](X).
struct EpiSrcAdd {
    static constexpr bool kPreFixed = false;   // s_new: written just before
    float* out;
    const float* divv;       // may be null
    const float* s_new;
    float dt;
    struct Pre { float dv, s; };
    __device__ Pre pre(int idx) const {
        return {divv ? __ldg(divv + idx) : 0.f, __ldg(s_new + idx)};
    }
    __device__ void post(int idx, float val, const Pre& p, double&) const {
        const float h = 0.5f * dt;
        out[idx] = fmaf(h * fmaf(dt, p.dv, 1.f), val, h * p.s);
    }
    __device__ void done(double) const {}
};

struct EpiCoef {             // c = 1 + dt/2 (dX + dv + dt dX dv), val = dX
    static constexpr bool kPreFixed = false;   // div v: written just before
    float* out;
    const float* divv;
    float dt;
    struct Pre { float dv; };
    __device__ Pre pre(int idx) const { return {__ldg(divv + idx)}; }
    __device__ void post(int idx, float val, const Pre& p, double&) const {
        // explicit fused operations: the same rounding at every inlined
        // call site of the point routine (the compiler's contraction choices
        // may differ between sites)
        out[idx] = fmaf(0.5f * dt, fmaf(dt * val, p.dv, val + p.dv), 1.f);
    }
    __device__ void done(double) const {}
};

struct EpiIncState {         // u_{j+1} = val + dt f_{j+1}; final: lam~ = -(val + dt/2 f_nt)
    static constexpr bool kPreFixed = true;    // v~, grad rho_{j+1}: not the previous step's
    float* out;
    const float* vt;
    const float* gj1;
    long long n;
    float dt;
    int final_step;
    struct Pre { float v0, v1, v2, g0, g1, g2; };
    __device__ Pre pre(int idx) const {
        return {__ldg(vt + idx), __ldg(vt + n + idx), __ldg(vt + 2 * n + idx),
                ld(gj1, idx), ld(gj1, n + idx), ld(gj1, 2 * n + idx)};
    }
    __device__ void post(int idx, float val, const Pre& p, double&) const {
        // explicit fused operations (see EpiCoef)
        const float f = -fmaf(p.v2, p.g2, fmaf(p.v1, p.g1, p.v0 * p.g0));
        out[idx] = final_step ? -fmaf(0.5f * dt, f, val) : fmaf(dt, f, val);
    }
    __device__ void done(double) const {}
};

// Per-point inputs of one marching point, loaded ahead of use.
template <class Epi>
struct Ahead {
    float d1, d2, d3;
    typename Epi::Pre pre;
};

template <class Epi>
__device__ __forceinline__ void fetch(Ahead<Epi>& a, const float* __restrict__ d, const Dims& g,
                                      const Epi& epi, int i1, int i2, int i3) {
    const long long n = g.n;
    const int idx = (i1 * g.n2 + i2) * g.n3 + i3;
    a.d1 = __ldg(d + idx);
    a.d2 = __ldg(d + n + idx);
    a.d3 = __ldg(d + 2 * n + idx);
    a.pre = epi.pre(idx);
}

// Point k = k0 + R of the thread's column: use the inputs fetched two points
// earlier into slot R & 1, refill it with point k + 2, interpolate, finish.
template <int R, class Epi>
__device__ __forceinline__ void march_point(Window& W, Ahead<Epi> (&ah)[2],
                                            const float* __restrict__ f,
                                            const float* __restrict__ d, const Dims& g,
                                            const Epi& epi, int i1b, int k0, int kend, int i2,
                                            int i3, double& acc) {
    const int k = k0 + R;
    if (k >= kend) return;
    const Ahead<Epi> cur = ah[R & 1];
    if (k + 2 < kend) fetch(ah[R & 1], d, g, epi, i1b + k + 2, i2, i3);
    const int i1 = i1b + k;
    const int idx = (i1 * g.n2 + i2) * g.n3 + i3;
    const float val = march_interp<R>(W, f, g, i1, i2, i3, cur.d1, cur.d2, cur.d3);
    epi.post(idx, val, cur.pre, acc);
}

template <class Epi>
__global__ void __launch_bounds__(256)
k_march(Dims g, int K, const float* __restrict__ f, const float* __restrict__ d, Epi epi) {
    const int i3 = blockIdx.x * 32 + threadIdx.x;
    const int i2 = blockIdx.y * blockDim.y + threadIdx.y;
    const int i1b = blockIdx.z * K;
    double acc = 0.0;
    if (i3 < g.n3 && i2 < g.n2) {
        const int kend = min(K, g.n1 - i1b);
        Window W;
        W.cp = INT_MIN / 2;
        W.cb2 = INT_MIN / 2;
        W.cb3 = INT_MIN / 2;
        W.interior = false;
        W.off = 0;
        Ahead<Epi> ah[2];
        if (0 < kend) fetch(ah[0], d, g, epi, i1b + 0, i2, i3);
        if (1 < kend) fetch(ah[1], d, g, epi, i1b + 1, i2, i3);
        for (int k0 = 0; k0 < kend; k0 += 4) {
            march_point<0>(W, ah, f, d, g, epi, i1b, k0, kend, i2, i3, acc);
            march_point<1>(W, ah, f, d, g, epi, i1b, k0, kend, i2, i3, acc);
            march_point<2>(W, ah, f, d, g, epi, i1b, k0, kend, i2, i3, acc);
            march_point<3>(W, ah, f, d, g, epi, i1b, k0, kend, i2, i3, acc);
        }
    }
    epi.done(acc);
}

dim3 march_grid(const Dims& g, Tile t);

// 4-byte asynchronous global -> shared copy (sm_80+ cp.async): the staging
// loads of a whole box are all in flight before the block waits for them.
__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Tensor-memory-accelerator staging: one cp.async.bulk.tensor copy brings a
// whole 3-D box from global to shared memory, and an mbarrier counts its
// bytes in (complete_tx).
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of the barrier for at most ~1 s of SM clock; false
// when it gave up (the copy never completed).
constexpr long long kStageWaitCycles = 2000000000LL;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  long long limit = kStageWaitCycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Host-armed test of the bounded wait (reg_debug_inject with
// REG_INJECT_STAGE_TIMEOUT): the next launch of the staged kernel that
// stages by TMA issues no copy, so its mbarrier phase never completes, and
// waits only kInjectWaitCycles before giving up.  No copy is in flight when
// its blocks exit.
constexpr long long kInjectWaitCycles = 200000LL;
std::atomic<int> g_inject_stage{0};

// Box of the 3-D tensor map at element coordinates (x3, x2, x1) = (x, y, z);
// x * 4 bytes must be a multiple of 16.  Coordinates outside the grid read
// zeros.
__device__ __forceinline__ void tma_load_box(float* dst, const CUtensorMap* map, uint64_t* bar,
                                             int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Box of a 4-D tensor map at element coordinates (x3, x2, x1, component).
__device__ __forceinline__ void tma_load_box4(float* dst, const CUtensorMap* map, uint64_t* bar,
                                              int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
        "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------- shared-memory staged kernel
// The block's output tile is 32 (x3) x wy (x2) x k (x1) points.  With every
// |floor(d)| <= H, the stencils of the tile lie in the box of
// (k + 3 + 2H) x (wy + 3 + 2H) x (35 + 2H) grid values around it; the block
// stages that box in shared memory with coalesced loads (periodic wrap at
// load time), then each point gathers its 64 values from shared memory:
// consecutive lanes read consecutive words, so the gathers are conflict free
// and no lane diverges.  A point outside the box (the bound was too small)
// falls back to a global gather.

template <class Epi>
__device__ __forceinline__ void tile_point(const float* __restrict__ box, int E1, int E2, int E3,
                                           int P3, int o1, int o2, int o3, const Epi& epi,
                                           const float* __restrict__ f, const Dims& g, int i1,
                                           int i2, int i3, float d1, float d2, float d3,
                                           const typename Epi::Pre& pre, double& acc) {
    const float fl1 = floorf(d1), fl2 = floorf(d2), fl3 = floorf(d3);
    float w1[4], w2[4], w3[4];
    lagrange4(d1 - fl1, w1);
    lagrange4(d2 - fl2, w2);
    lagrange4(d3 - fl3, w3);
    const int l1 = i1 + (int)fl1 - 1 - o1;
    const int l2 = i2 + (int)fl2 - 1 - o2;
    const int l3 = i3 + (int)fl3 - 1 - o3;
    const int idx = (i1 * g.n2 + i2) * g.n3 + i3;
    float val = 0.f;
    if (l1 >= 0 && l2 >= 0 && l3 >= 0 && l1 <= E1 - 4 && l2 <= E2 - 4 && l3 <= E3 - 4) {
        const float* base = box + (l1 * E2 + l2) * P3 + l3;
        const int E23 = E2 * P3;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            float r = 0.f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float* row = base + a * E23 + b * P3;
                float s = w3[0] * row[0];
                s = fmaf(w3[1], row[1], s);
                s = fmaf(w3[2], row[2], s);
                s = fmaf(w3[3], row[3], s);
                r = fmaf(w2[b], s, r);
            }
            val = fmaf(w1[a], r, val);
        }
    } else {
        Stencil s;
        make_stencil(s, g, i1, i2, i3, d1, d2, d3);
        val = gather1(s, f);
    }
    epi.post(idx, val, pre, acc);
}

// One output tile (block coordinates bx, by, bz) of the generic staged
// kernel: stage the box, then gather every point of the tile.  The calling
// block is 32 x blockDim.y threads; acc accumulates the epilogue's sums.
template <class Epi>
__device__ __forceinline__ void tile_task(const Dims& g, int K, int H, int E1, int E2, int E3,
                                          int P3, const float* __restrict__ f,
                                          const float* __restrict__ d, const Epi& epi,
                                          float* box, int bx, int by, int bz, double& acc) {
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int i3 = bx * 32 + lane;
    const int i2 = by * blockDim.y + ty;
    const int i1b = bz * K;
    const int o1 = i1b - 1 - H, o2 = by * blockDim.y - 1 - H;
    const int o3 = bx * 32 - 1 - H;
    const bool active = i3 < g.n3 && i2 < g.n2;
    const int kend = min(K, g.n1 - i1b);
    Ahead<Epi> ah[2];
    if (active) {
        if (0 < kend) fetch(ah[0], d, g, epi, i1b, i2, i3);
        if (1 < kend) fetch(ah[1], d, g, epi, i1b + 1, i2, i3);
    }
    // stage the box: one warp per row, lanes along x3 (columns lane, lane+32, ...)
    {
        const int nwarps = blockDim.y;
        int col[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) col[c] = wrap_near(o3 + lane + 32 * c, g.n3);
        const int rows = E1 * E2;
        for (int r = ty; r < rows; r += nwarps) {
            const int a = r / E2, b = r - a * E2;
            const float* src = f + (long long)wrap_near(o1 + a, g.n1) * g.n23 +
                               wrap_near(o2 + b, g.n2) * g.n3;
            float* dst = box + r * P3;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (lane + 32 * c < E3) cp_async4(dst + lane + 32 * c, src + col[c]);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (active) {
        for (int k = 0; k < kend; k += 2) {
            {   // slot 0 (static index: the prefetch ring stays in registers)
                const Ahead<Epi> cur = ah[0];
                if (k + 2 < kend) fetch(ah[0], d, g, epi, i1b + k + 2, i2, i3);
                tile_point(box, E1, E2, E3, P3, o1, o2, o3, epi, f, g, i1b + k, i2, i3, cur.d1,
                           cur.d2, cur.d3, cur.pre, acc);
            }
            if (k + 1 < kend) {
                const Ahead<Epi> cur = ah[1];
                if (k + 3 < kend) fetch(ah[1], d, g, epi, i1b + k + 3, i2, i3);
                tile_point(box, E1, E2, E3, P3, o1, o2, o3, epi, f, g, i1b + k + 1, i2, i3, cur.d1,
                           cur.d2, cur.d3, cur.pre, acc);
            }
        }
    }
}

// ----------------------------------------------- persistent small-grid kernel
// On a small grid (the two-level preconditioner's coarse grid) every launch
// of a matvec's transport is latency bound (a few microseconds of work behind
// a launch, a box load and a tail).  k_matvec_persistent runs the whole
// sequence of one Gauss-Newton matvec's transports in ONE launch: the
// incremental-state set-up, the nt incremental-state steps, the nt
// incremental-adjoint steps with the time integral, and the partial sums of
// <p, b~>, separated by grid-wide barriers.  Every block takes the same tiles
// in every step (so b~ and the levels written at a point are read back by
// the block that wrote them), and boxes are staged with L2-coherent loads,
// because the fields they gather were written earlier in the same launch by
// other blocks.  The barrier waits are bounded (about half a second); a block
// that gives up raises *err, and the host turns the launch's result into NaN.

constexpr long long kBarrierCycles = 1000000000LL;

__device__ __forceinline__ void grid_barrier(unsigned int* count, unsigned int target,
                                             int* err) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        const long long t0 = clock64();
        while (*reinterpret_cast<volatile unsigned int*>(count) < target) {
            if (clock64() - t0 > kBarrierCycles) {
                atomicExch(err, 1);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// tile_task with the box staged by coherent (L2) loads.
template <class Epi>
__device__ __forceinline__ void tile_task_coherent(const Dims& g, int K, int H, int E1, int E2,
                                                   int E3, int P3, const float* f,
                                                   const float* __restrict__ d, const Epi& epi,
                                                   float* box, int bx, int by, int bz,
                                                   double& acc) {
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int i3 = bx * 32 + lane;
    const int i2 = by * blockDim.y + ty;
    const int i1b = bz * K;
    const int o1 = i1b - 1 - H, o2 = by * blockDim.y - 1 - H;
    const int o3 = bx * 32 - 1 - H;
    const bool active = i3 < g.n3 && i2 < g.n2;
    const int kend = min(K, g.n1 - i1b);
    Ahead<Epi> ah[2];
    if (active) {
        if (0 < kend) fetch(ah[0], d, g, epi, i1b, i2, i3);
        if (1 < kend) fetch(ah[1], d, g, epi, i1b + 1, i2, i3);
    }
    {
        const int nwarps = blockDim.y;
        int col[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) col[c] = wrap_near(o3 + lane + 32 * c, g.n3);
        const int rows = E1 * E2;
        for (int r = ty; r < rows; r += nwarps) {
            const int a = r / E2, b = r - a * E2;
            const float* src = f + (long long)wrap_near(o1 + a, g.n1) * g.n23 +
                               wrap_near(o2 + b, g.n2) * g.n3;
            float* dst = box + r * P3;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (lane + 32 * c < E3) dst[lane + 32 * c] = __ldcg(src + col[c]);
        }
    }
    __syncthreads();
    if (active) {
        for (int k = 0; k < kend; k += 2) {
            {
                const Ahead<Epi> cur = ah[0];
                if (k + 2 < kend) fetch(ah[0], d, g, epi, i1b + k + 2, i2, i3);
                tile_point(box, E1, E2, E3, P3, o1, o2, o3, epi, f, g, i1b + k, i2, i3, cur.d1,
                           cur.d2, cur.d3, cur.pre, acc);
            }
            if (k + 1 < kend) {
                const Ahead<Epi> cur = ah[1];
                if (k + 3 < kend) fetch(ah[1], d, g, epi, i1b + k + 3, i2, i3);
                tile_point(box, E1, E2, E3, P3, o1, o2, o3, epi, f, g, i1b + k + 1, i2, i3, cur.d1,
                           cur.d2, cur.d3, cur.pre, acc);
            }
        }
    }
    __syncthreads();   // the box is refilled by the block's next tile
}

struct PersistArgs {
    Dims g;
    int K;                       // points per thread along x1 (block 32 x blockDim.y)
    int Hf, Hb;                  // halos of the forward and adjoint points
    int E1f, E2f, E3f, E1b, E2b, E3b, P3;
    int gx, gy, gz;              // tiles per axis
    int nt;
    float dt;
    const float* vt;             // [3n]
    const float* grad;           // grad rho levels [(nt+1)][3n]
    const float* d_fwd;
    const float* d_adj;
    const float* coef;           // c(x), null when divergence free
    float* u[2];                 // carried incremental state, ping-pong
    float* lam;                  // incremental-adjoint levels [(nt+1) n]
    float* b;                    // b~ [3n]
    const float* dotp;           // [3n]: partial sums of <dotp, b~>
    double* partials;            // [gridDim.x]
    unsigned int* bar;           // barrier counter (zero at launch)
    int* err;                    // raised by a barrier wait that gave up
};

__global__ void __launch_bounds__(256)
k_matvec_persistent(PersistArgs a) {
    extern __shared__ float box[];
    const Dims& g = a.g;
    const long long n = g.n;
    const int ntiles = a.gx * a.gy * a.gz;
    const unsigned int G = gridDim.x;
    unsigned int target = 0;
    auto tile_of = [&](int t, int& bx, int& by, int& bz) {
        bx = t % a.gx;
        by = (t / a.gx) % a.gy;
        bz = t / (a.gx * a.gy);
    };
    // u_0 = dt/2 f_0, f_0 = -v~ . grad rho(t_0), at the points of the block's tiles
    for (int t = blockIdx.x; t < ntiles; t += G) {
        int bx, by, bz;
        tile_of(t, bx, by, bz);
        const int i3 = bx * 32 + threadIdx.x, i2 = by * blockDim.y + threadIdx.y;
        if (i3 >= g.n3 || i2 >= g.n2) continue;
        for (int k = 0; k < a.K && bz * a.K + k < g.n1; ++k) {
            const int idx = ((bz * a.K + k) * g.n2 + i2) * g.n3 + i3;
            const float f0 = -(a.vt[idx] * ld(a.grad, idx) + a.vt[n + idx] * ld(a.grad, n + idx) +
                               a.vt[2 * n + idx] * ld(a.grad, 2 * n + idx));
            a.u[0][idx] = 0.5f * a.dt * f0;
        }
    }
    target += G;
    grid_barrier(a.bar, target, a.err);
    double acc = 0.0;
    for (int j = 0; j < a.nt; ++j) {
        const bool fin = (j == a.nt - 1);
        const EpiIncState epi{fin ? a.lam + a.nt * n : a.u[(j + 1) & 1], a.vt,
                              a.grad + (long long)(j + 1) * 3 * n, n, a.dt, fin ? 1 : 0};
        for (int t = blockIdx.x; t < ntiles; t += G) {
            int bx, by, bz;
            tile_of(t, bx, by, bz);
            tile_task_coherent(g, a.K, a.Hf, a.E1f, a.E2f, a.E3f, a.P3, a.u[j & 1], a.d_fwd, epi,
                               box, bx, by, bz, acc);
        }
        target += G;
        grid_barrier(a.bar, target, a.err);
    }
    acc = 0.0;
    for (int j = a.nt - 1; j >= 0; --j) {
        const bool first = (j == a.nt - 1), last = (j == 0);
        const float w = last ? 0.5f * a.dt : a.dt;
        const EpiAdjAcc epi{last ? nullptr : a.lam + j * n, a.coef,
                            a.grad + (long long)j * 3 * n, a.b, n, w,
                            first ? a.lam + a.nt * n : nullptr,
                            first ? a.grad + (long long)a.nt * 3 * n : nullptr, 0.5f * a.dt,
                            last ? a.dotp : nullptr, a.partials, nullptr};
        for (int t = blockIdx.x; t < ntiles; t += G) {
            int bx, by, bz;
            tile_of(t, bx, by, bz);
            tile_task_coherent(g, a.K, a.Hb, a.E1b, a.E2b, a.E3b, a.P3, a.lam + (j + 1) * n,
                               a.d_adj, epi, box, bx, by, bz, acc);
        }
        if (!last) {
            target += G;
            grid_barrier(a.bar, target, a.err);
        } else {
            // a block whose barrier wait gave up poisons the inner product
            if (*reinterpret_cast<volatile int*>(a.err)) acc = __longlong_as_double(0x7ff8000000000000LL);
            epi.done(acc);
        }
    }
}

template <class Epi>
__global__ void __launch_bounds__(256)
k_tile(Dims g, int K, int H, int E1, int E2, int E3, int P3, const float* __restrict__ f,
       const float* __restrict__ d, Epi epi) {
    extern __shared__ float box[];   // [E1][E2][P3], E3 columns used
    double acc = 0.0;
    tile_task(g, K, H, E1, E2, E3, P3, f, d, epi, box, blockIdx.x, blockIdx.y, blockIdx.z, acc);
    epi.done(acc);
}

// The elements of a box that lie outside the grid, as six disjoint regions
// (planes outside; rows outside of inside planes; columns outside of inside
// rows) of the box's column range [C0, C1), given the in-grid index ranges
// [a_lo, a_hi) x [b_lo, b_hi) x [c_lo, c_hi).  One ordinal e in [0, count())
// enumerates them, so that a thread can load its share before the box's copy
// has landed and store it afterwards.
template <int E2, int C0, int C1>
struct Faces {
    int E1, a_lo, a_hi, b_lo, b_hi, c_lo, c_hi;
    __device__ int count() const {
        constexpr int NC = C1 - C0;
        const int A = a_hi - a_lo, B = b_hi - b_lo;
        return (a_lo + E1 - a_hi) * E2 * NC + A * (b_lo + E2 - b_hi) * NC +
               A * B * (c_lo - C0 + C1 - c_hi);
    }
    // box element (a, b, c) of ordinal e < count()
    __device__ void element(int e, int& a, int& b, int& c) const {
        constexpr int NC = C1 - C0;
        const int A = a_hi - a_lo, B = b_hi - b_lo;
        auto decode = [&](int l, int a0, int b0, int nb, int c0, int nc) {
            c = c0 + l % nc;
            const int r = l / nc;
            b = b0 + r % nb;
            a = a0 + r / nb;
        };
        int n = a_lo * E2 * NC;
        if (e < n) return decode(e, 0, 0, E2, C0, NC);
        e -= n;
        n = (E1 - a_hi) * E2 * NC;
        if (e < n) return decode(e, a_hi, 0, E2, C0, NC);
        e -= n;
        n = A * b_lo * NC;
        if (e < n) return decode(e, a_lo, 0, b_lo, C0, NC);
        e -= n;
        n = A * (E2 - b_hi) * NC;
        if (e < n) return decode(e, a_lo, b_hi, E2 - b_hi, C0, NC);
        e -= n;
        n = A * B * (c_lo - C0);
        if (e < n) return decode(e, a_lo, b_lo, B, C0, c_lo - C0);
        e -= n;
        decode(e, a_lo, b_lo, B, c_hi, C1 - c_hi);
    }
};

// The same kernel with the halo H and the block height WY fixed at compile
// time: every one of the 64 shared-memory offsets of a point is then an
// immediate, and only the base address is computed per point.  The box row
// starts at the 16-byte aligned column o3 = 32 bx - 4, its pitch is 64 words,
// and columns [3 - H, 38 + H) hold every stencil of the tile.  With a tensor
// map (use_tma) one thread stages the whole box with a single TMA copy that
// the block waits for on an mbarrier; the copy reads zeros outside the grid,
// so a block at a face of the periodic domain then reloads those elements
// from their periodic images.  Without one, every thread issues 4-byte
// cp.async copies with the wrap resolved per row.  A block whose wait for the
// copy gives up (bounded, about a second) writes NaN for its points.
constexpr int kWrapAhead = 4;   // periodic-image loads per thread issued before the copy lands

template <class Epi, int H, int WY>
__global__ void __launch_bounds__(32 * WY, 1024 / (32 * WY))
k_tile_fixed(Dims g, int K, const float* __restrict__ f, const float* __restrict__ d, Epi epi,
             const __grid_constant__ CUtensorMap box_map, int use_tma, int inject_timeout) {
    constexpr int E2 = WY + 3 + 2 * H;
    constexpr int P3 = 64;
    constexpr int C0 = 3 - H, C1 = 38 + H;   // columns read by the tile's stencils
    static_assert(C0 >= 0 && C1 <= P3, "box row");
    constexpr int E23 = E2 * P3;
    extern __shared__ __align__(128) float box[];   // [E1][E2][P3], then the mbarrier
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * 32 + lane;
    const int E1 = K + 3 + 2 * H;
    const int i3 = blockIdx.x * 32 + lane;
    const int i2 = blockIdx.y * WY + ty;
    const int i1b = blockIdx.z * K;
    const int o1 = i1b - 1 - H, o2 = blockIdx.y * WY - 1 - H;
    const int o3 = blockIdx.x * 32 - 4;
    const bool active = i3 < g.n3 && i2 < g.n2;
    const int kend = min(K, g.n1 - i1b);
    uint64_t* bar = reinterpret_cast<uint64_t*>(box + E1 * E23);
    const bool tma = use_tma && (smem_u32(box) & 127u) == 0;
    // the first two points' inputs: before the wait for the previous step
    // where none of them is that step's output (the displacements never
    // are; Epi::kPreFixed says whether the epilogue's are)
    Ahead<Epi> ah[2];
    auto prefetch = [&]() {
        if (active) {
            if (0 < kend) fetch(ah[0], d, g, epi, i1b, i2, i3);
            if (1 < kend) fetch(ah[1], d, g, epi, i1b + 1, i2, i3);
        }
    };
    if constexpr (Epi::kPreFixed) prefetch();
    pdl_wait();      // the previous step's level is this step's input
    pdl_trigger();
    if (tma) {
        if (tid == 0) mbar_init(bar, 1);
        __syncthreads();
        if (tid == 0) {
            mbar_expect_tx(bar, (unsigned)(sizeof(float) * E1 * E23));
            if (!inject_timeout) tma_load_box(box, &box_map, bar, o3, o2, o1);
        }
    }
    if constexpr (!Epi::kPreFixed) prefetch();
    bool staged = true;
    if (tma) {
        // the copy reads zeros outside the grid: those elements come from
        // their periodic images, in disjoint parts (planes outside; rows
        // outside of inside planes; columns outside of inside rows).  A
        // thread's first kWrapAhead of them are loaded while the copy is in
        // flight and stored once it has landed, the rest after it.
        const int nthr = 32 * WY;
        const int a_lo = min(max(-o1, 0), E1), a_hi = max(min(g.n1 - o1, E1), a_lo);
        const int b_lo = min(max(-o2, 0), E2), b_hi = max(min(g.n2 - o2, E2), b_lo);
        const int c_lo = min(max(-o3, C0), C1), c_hi = max(min(g.n3 - o3, C1), c_lo);
        const Faces<E2, C0, C1> fc{E1, a_lo, a_hi, b_lo, b_hi, c_lo, c_hi};
        const int total = fc.count();
        auto image = [&](int a, int b, int c) {
            return __ldg(f + (long long)wrap_near(o1 + a, g.n1) * g.n23 +
                         wrap_near(o2 + b, g.n2) * g.n3 + wrap_near(o3 + c, g.n3));
        };
        float wv[kWrapAhead];
        int wi[kWrapAhead];
#pragma unroll
        for (int q = 0; q < kWrapAhead; ++q) {
            const int e = tid + q * nthr;
            wi[q] = -1;
            if (e < total) {
                int a, b, c;
                fc.element(e, a, b, c);
                wi[q] = (a * E2 + b) * P3 + c;
                wv[q] = image(a, b, c);
            }
        }
        const long long limit = inject_timeout ? kInjectWaitCycles : kStageWaitCycles;
        staged = mbar_wait_bounded(bar, 0, limit);
        if (!staged) mbar_wait_bounded(bar, 0, limit);   // let a late copy land before exit
#pragma unroll
        for (int q = 0; q < kWrapAhead; ++q)
            if (wi[q] >= 0) box[wi[q]] = wv[q];
        for (int e = tid + kWrapAhead * nthr; e < total; e += nthr) {
            int a, b, c;
            fc.element(e, a, b, c);
            box[(a * E2 + b) * P3 + c] = image(a, b, c);
        }
    } else {
        int col[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) col[c] = wrap_near(o3 + C0 + lane + 32 * c, g.n3);
        for (int a = 0; a < E1; ++a) {
            const float* plane = f + (long long)wrap_near(o1 + a, g.n1) * g.n23;
            for (int b = ty; b < E2; b += WY) {
                const float* src = plane + wrap_near(o2 + b, g.n2) * g.n3;
                float* dst = box + (a * E2 + b) * P3 + C0;
#pragma unroll
                for (int c = 0; c < 2; ++c)
                    if (lane + 32 * c < C1 - C0) cp_async4(dst + lane + 32 * c, src + col[c]);
            }
        }
        cp_async_wait_all();
    }
    __syncthreads();
    double acc = 0.0;
    if (active) {
        // |floor(d)| <= H for every point by construction of H, so every
        // stencil lies in the box; the clamps only keep non-finite input
        // (which yields a NaN value) inside shared memory.
        const int idx0 = (i1b * g.n2 + i2) * g.n3 + i3;
        const int r2 = i2 - 1 - o2, r3 = i3 - 1 - o3;
        auto point = [&](const Ahead<Epi>& cur, int k) {
            const float fl1 = floorf(cur.d1), fl2 = floorf(cur.d2), fl3 = floorf(cur.d3);
            float w1[4], w2[4], w3[4];
            lagrange4(cur.d1 - fl1, w1);
            lagrange4(cur.d2 - fl2, w2);
            lagrange4(cur.d3 - fl3, w3);
            const int l1 = min(max(k + H + (int)fl1, 0), E1 - 4);   // i1 + fl1 - 1 - o1
            const int l2 = min(max(r2 + (int)fl2, 0), E2 - 4);
            const int l3 = min(max(r3 + (int)fl3, 0), P3 - 4);
            const float* base = box + (l1 * E2 + l2) * P3 + l3;
            const f32x2 w2a = pk(w2[0], w2[1]), w2b = pk(w2[2], w2[3]);
            f32x2 ww3[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) ww3[c] = pk(w3[c], w3[c]);
            float r[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float* pl = base + a * E23;
                // rows (0, 1) and (2, 3) of the plane in packed pairs
                f32x2 s01 = mul2(ww3[0], pk(pl[0], pl[P3]));
                f32x2 s23 = mul2(ww3[0], pk(pl[2 * P3], pl[3 * P3]));
#pragma unroll
                for (int c = 1; c < 4; ++c) {
                    s01 = fma2(ww3[c], pk(pl[c], pl[P3 + c]), s01);
                    s23 = fma2(ww3[c], pk(pl[2 * P3 + c], pl[3 * P3 + c]), s23);
                }
                const float2 t2 = upk(fma2(w2b, s23, mul2(w2a, s01)));
                r[a] = t2.x + t2.y;
            }
            float val = w1[0] * r[0];
            val = fmaf(w1[1], r[1], val);
            val = fmaf(w1[2], r[2], val);
            val = fmaf(w1[3], r[3], val);
            if (!staged) val = __int_as_float(0x7fffffff);
            epi.post(idx0 + k * g.n23, val, cur.pre, acc);
        };
        for (int k = 0; k < kend; k += 2) {
            {
                const Ahead<Epi> cur = ah[0];
                if (k + 2 < kend) fetch(ah[0], d, g, epi, i1b + k + 2, i2, i3);
                point(cur, k);
            }
            if (k + 1 < kend) {
                const Ahead<Epi> cur = ah[1];
                if (k + 3 < kend) fetch(ah[1], d, g, epi, i1b + k + 3, i2, i3);
                point(cur, k + 1);
            }
        }
    }
    epi.done(acc);
}

// The runtime's handle on the driver's tensor-map encoder (null when the
// driver does not offer it; the staged kernel then copies with cp.async).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of the field f (n1 x n2 x n3, x3 fastest) with a box of 64 x E2
// x E1 elements; false (map unused) unless the grid rows are whole 16-byte
// units, f is 16-byte aligned and the grid is at least one box large.
bool box_tensor_map(CUtensorMap* map, const Dims& g, const float* f, int E1, int E2) {
    std::memset(map, 0, sizeof(*map));
    if (g.n3 % 4 || g.n3 < 64 || g.n2 < E2 || g.n1 < E1 || E1 > 256 || E2 > 256 ||
        (reinterpret_cast<uintptr_t>(f) & 15))
        return false;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dim[3] = {(cuuint64_t)g.n3, (cuuint64_t)g.n2, (cuuint64_t)g.n1};
    const cuuint64_t stride[2] = {sizeof(float) * (cuuint64_t)g.n3,
                                  sizeof(float) * (cuuint64_t)g.n23};
    const cuuint32_t boxd[3] = {64, (cuuint32_t)E2, (cuuint32_t)E1};
    const cuuint32_t estride[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(f), dim, stride, boxd,
               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <class Epi, int H, int WY>
cudaError_t run_tile_fixed(const Dims& g, Tile t, const float* f, const float* d,
                           const Epi& epi, cudaStream_t st) {
    constexpr int E2 = WY + 3 + 2 * H;
    constexpr int P3 = 64;
    const int E1 = t.k + 3 + 2 * H;
    // the box, then the 8-byte mbarrier
    const size_t smem = sizeof(float) * (size_t)E1 * E2 * P3 + 16;
    if (smem > 48 * 1024) {
        const int cap = WY >= 16 ? kMaxBoxFloats16 : kMaxBoxFloats;
        const cudaError_t e = cudaFuncSetAttribute(k_tile_fixed<Epi, H, WY>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(sizeof(float) * cap + 16));
        if (e != cudaSuccess) return e;
    }
    CUtensorMap map;
    const int use_tma = t.tma && box_tensor_map(&map, g, f, E1, E2) ? 1 : 0;
    const int inject = use_tma && g_inject_stage.exchange(0) ? 1 : 0;
    return launch_dependent(k_tile_fixed<Epi, H, WY>, march_grid(g, t), dim3(32, WY), smem, st,
                            g, t.k, f, d, epi, map, use_tma, inject);
}

// Tricubic value at displacement (e1, e2, e3) (grid units) of the point of
// local x1 plane kloc, from a staged box laid out as in k_departure_tile
// (H, WY fixed; clamped indices keep every read inside the box).
template <int H, int WY>
__device__ __forceinline__ float box_interp(const float* box, int E1, int kloc, int r2, int r3,
                                            float e1, float e2, float e3) {
    constexpr int E2 = WY + 3 + 2 * H;
    constexpr int E3 = 35 + 2 * H;
    constexpr int P3 = (E3 + 31) & ~31;
    constexpr int E23 = E2 * P3;
    const float fl1 = floorf(e1), fl2 = floorf(e2), fl3 = floorf(e3);
    float w1[4], w2[4], w3[4];
    lagrange4(e1 - fl1, w1);
    lagrange4(e2 - fl2, w2);
    lagrange4(e3 - fl3, w3);
    const int l1 = min(max(kloc + H + (int)fl1, 0), E1 - 4);
    const int l2 = min(max(r2 + (int)fl2, 0), E2 - 4);
    const int l3 = min(max(r3 + (int)fl3, 0), E3 - 4);
    const float* base = box + (l1 * E2 + l2) * P3 + l3;
    const f32x2 w2a = pk(w2[0], w2[1]), w2b = pk(w2[2], w2[3]);
    f32x2 ww3[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ww3[c] = pk(w3[c], w3[c]);
    float r[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float* pl = base + a * E23;
        f32x2 s01 = mul2(ww3[0], pk(pl[0], pl[P3]));
        f32x2 s23 = mul2(ww3[0], pk(pl[2 * P3], pl[3 * P3]));
#pragma unroll
        for (int c = 1; c < 4; ++c) {
            s01 = fma2(ww3[c], pk(pl[c], pl[P3 + c]), s01);
            s23 = fma2(ww3[c], pk(pl[2 * P3 + c], pl[3 * P3 + c]), s23);
        }
        const float2 t2 = upk(fma2(w2b, s23, mul2(w2a, s01)));
        r[a] = t2.x + t2.y;
    }
    float val = w1[0] * r[0];
    val = fmaf(w1[1], r[1], val);
    val = fmaf(w1[2], r[2], val);
    return fmaf(w1[3], r[3], val);
}

// RK2 points of v and -v (Eq. sml-trajectory) from shared memory: the boxes
// of the three velocity components are staged one after the other, and each
// serves both feet of every point of the tile (x - u and x + u, u = dt v(x)
// in grid units, |u| <= H).
template <int H>
__global__ void __launch_bounds__(256)
k_departure_tile(Dims g, int K, const float* __restrict__ v, float dth1, float dth2,
                 float dth3, float* __restrict__ d_fwd, float* __restrict__ d_adj) {
    constexpr int WY = 8;
    constexpr int E2 = WY + 3 + 2 * H;
    constexpr int E3 = 35 + 2 * H;
    constexpr int P3 = (E3 + 31) & ~31;
    extern __shared__ float box[];   // [E1][E2][P3], E3 columns used
    const int lane = threadIdx.x, ty = threadIdx.y;
    const int E1 = K + 3 + 2 * H;
    const int i3 = blockIdx.x * 32 + lane;
    const int i2 = blockIdx.y * WY + ty;
    const int i1b = blockIdx.z * K;
    const int o1 = i1b - 1 - H, o2 = blockIdx.y * WY - 1 - H;
    const int o3 = blockIdx.x * 32 - 1 - H;
    const bool active = i3 < g.n3 && i2 < g.n2;
    const int kend = min(K, g.n1 - i1b);
    const long long n = g.n;
    const int r2 = i2 - 1 - o2, r3 = i3 - 1 - o3;
    int col[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) col[c] = wrap_near(o3 + lane + 32 * c, g.n3);
    for (int comp = 0; comp < 3; ++comp) {
        const float* f = v + comp * n;
        const float dthc = comp == 0 ? dth1 : (comp == 1 ? dth2 : dth3);
        if (comp > 0) __syncthreads();   // every thread is done with the last box
        for (int a = 0; a < E1; ++a) {
            const float* plane = f + (long long)wrap_near(o1 + a, g.n1) * g.n23;
            for (int b = ty; b < E2; b += WY) {
                const float* src = plane + wrap_near(o2 + b, g.n2) * g.n3;
                float* dst = box + (a * E2 + b) * P3;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (lane + 32 * c < E3) cp_async4(dst + lane + 32 * c, src + col[c]);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (!active) continue;
        for (int k = 0; k < kend; ++k) {
            const int idx = ((i1b + k) * g.n2 + i2) * g.n3 + i3;
            const float u1 = __ldg(v + idx) * dth1;
            const float u2 = __ldg(v + n + idx) * dth2;
            const float u3 = __ldg(v + 2 * n + idx) * dth3;
            const float uc = comp == 0 ? u1 : (comp == 1 ? u2 : u3);
            // forward: X* = x - u, X = x - (u + dt v(X*)) / 2
            const float af = box_interp<H, WY>(box, E1, k, r2, r3, -u1, -u2, -u3);
            d_fwd[comp * n + idx] = -0.5f * fmaf(af, dthc, uc);
            if (d_adj) {
                // adjoint (velocity -v): X* = x + u, X = x + (u + dt v(X*)) / 2
                const float aa = box_interp<H, WY>(box, E1, k, r2, r3, u1, u2, u3);
                d_adj[comp * n + idx] = 0.5f * fmaf(aa, dthc, uc);
            }
        }
    }
}

// Tricubic values of the three velocity components at displacement (e1, e2,
// e3) of local point (kloc, r2, r3) from their staged boxes (component c at
// box + c * BOX, pitch 64): one set of weights for the three gathers, each in
// the operation order of box_interp.
template <int H, int WY, int E1>
__device__ __forceinline__ void box_interp3(const float* box, int kloc, int r2, int r3, float e1,
                                            float e2, float e3, float (&out)[3]) {
    constexpr int E2 = WY + 3 + 2 * H;
    constexpr int P3 = 64;
    constexpr int E23 = E2 * P3;
    constexpr int BOX = E1 * E23;
    const float fl1 = floorf(e1), fl2 = floorf(e2), fl3 = floorf(e3);
    float w1[4], w2[4], w3[4];
    lagrange4(e1 - fl1, w1);
    lagrange4(e2 - fl2, w2);
    lagrange4(e3 - fl3, w3);
    const int l1 = min(max(kloc + H + (int)fl1, 0), E1 - 4);
    const int l2 = min(max(r2 + (int)fl2, 0), E2 - 4);
    const int l3 = min(max(r3 + (int)fl3, 0), P3 - 4);
    const f32x2 w2a = pk(w2[0], w2[1]), w2b = pk(w2[2], w2[3]);
    f32x2 ww3[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) ww3[c] = pk(w3[c], w3[c]);
#pragma unroll
    for (int comp = 0; comp < 3; ++comp) {
        const float* base = box + comp * BOX + (l1 * E2 + l2) * P3 + l3;
        float r[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float* pl = base + a * E23;
            f32x2 s01 = mul2(ww3[0], pk(pl[0], pl[P3]));
            f32x2 s23 = mul2(ww3[0], pk(pl[2 * P3], pl[3 * P3]));
#pragma unroll
            for (int c = 1; c < 4; ++c) {
                s01 = fma2(ww3[c], pk(pl[c], pl[P3 + c]), s01);
                s23 = fma2(ww3[c], pk(pl[2 * P3 + c], pl[3 * P3 + c]), s23);
            }
            const float2 t2 = upk(fma2(w2b, s23, mul2(w2a, s01)));
            r[a] = t2.x + t2.y;
        }
        float val = w1[0] * r[0];
        val = fmaf(w1[1], r[1], val);
        val = fmaf(w1[2], r[2], val);
        out[comp] = fmaf(w1[3], r[3], val);
    }
}

// RK2 points of v and -v (Eq. sml-trajectory) from ONE tensor copy of the
// three velocity components' boxes ([3][E1][E2][64] floats, a 4-D tensor map
// over the component-major field; the copy reads zeros outside the grid and
// the block reloads those elements from their periodic images, the loads
// issued while the copy is in flight).  Each foot's weights serve the three
// components, and the point's own velocity comes from the box.  Tile: 4
// points along x1, 8 rows, 32 columns; |u| <= H.  A block whose wait for the
// copy gives up (bounded) writes NaN.  Same values as k_departure_tile.
constexpr int kDepK = 4;

template <int H>
__global__ void __launch_bounds__(256)
k_departure_fixed(Dims g, const float* __restrict__ v, float dth1, float dth2, float dth3,
                  float* __restrict__ d_fwd, float* __restrict__ d_adj,
                  const __grid_constant__ CUtensorMap map, int inject_timeout,
                  unsigned int* __restrict__ dmax) {
    constexpr int K = kDepK, WY = 8;
    constexpr int E1 = K + 3 + 2 * H, E2 = WY + 3 + 2 * H, P3 = 64;
    constexpr int C0 = 3 - H, C1 = 38 + H;
    constexpr int E23 = E2 * P3, BOX = E1 * E23;
    extern __shared__ __align__(128) float box[];   // [3][E1][E2][P3], then the mbarrier
    const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
    const int i3 = blockIdx.x * 32 + lane, i2 = blockIdx.y * WY + ty, i1b = blockIdx.z * K;
    const int o1 = i1b - 1 - H, o2 = blockIdx.y * WY - 1 - H, o3 = blockIdx.x * 32 - 4;
    const bool active = i3 < g.n3 && i2 < g.n2;
    const int kend = min(K, g.n1 - i1b);
    const long long n = g.n;
    uint64_t* bar = reinterpret_cast<uint64_t*>(box + 3 * BOX);
    // the tensor copy wants a 128-byte aligned destination; otherwise every
    // element is loaded as a periodic image (the whole box counts as outside)
    const bool tma = (smem_u32(box) & 127u) == 0;
    if (tma) {
        if (tid == 0) mbar_init(bar, 1);
        __syncthreads();
        if (tid == 0) {
            mbar_expect_tx(bar, (unsigned)(sizeof(float) * 3 * BOX));
            if (!inject_timeout) tma_load_box4(box, &map, bar, o3, o2, o1, 0);
        }
    }
    const int a_lo = tma ? min(max(-o1, 0), E1) : 0;
    const int a_hi = tma ? max(min(g.n1 - o1, E1), a_lo) : 0;
    const int b_lo = min(max(-o2, 0), E2), b_hi = max(min(g.n2 - o2, E2), b_lo);
    const int c_lo = min(max(-o3, C0), C1), c_hi = max(min(g.n3 - o3, C1), c_lo);
    const Faces<E2, C0, C1> fc{E1, a_lo, a_hi, b_lo, b_hi, c_lo, c_hi};
    const int per = fc.count(), total = 3 * per;   // every component's images
    auto image = [&](int e, int& at) {
        const int comp = e / per;
        int a, b, c;
        fc.element(e - comp * per, a, b, c);
        at = comp * BOX + (a * E2 + b) * P3 + c;
        return __ldg(v + comp * n + (long long)wrap_near(o1 + a, g.n1) * g.n23 +
                     wrap_near(o2 + b, g.n2) * g.n3 + wrap_near(o3 + c, g.n3));
    };
    float wv[kWrapAhead];
    int wi[kWrapAhead];
#pragma unroll
    for (int q = 0; q < kWrapAhead; ++q) {
        const int e = tid + q * 256;
        wi[q] = -1;
        if (e < total) wv[q] = image(e, wi[q]);
    }
    bool staged = true;
    if (tma) {
        const long long limit = inject_timeout ? kInjectWaitCycles : kStageWaitCycles;
        staged = mbar_wait_bounded(bar, 0, limit);
        if (!staged) mbar_wait_bounded(bar, 0, limit);   // let a late copy land before exit
    }
#pragma unroll
    for (int q = 0; q < kWrapAhead; ++q)
        if (wi[q] >= 0) box[wi[q]] = wv[q];
    for (int e = tid + kWrapAhead * 256; e < total; e += 256) {
        int at;
        const float x = image(e, at);
        box[at] = x;
    }
    __syncthreads();
    const int r2 = ty + H, r3 = lane + 3;   // i2 - 1 - o2, i3 - 1 - o3
    const float dth[3] = {dth1, dth2, dth3};
    float mf = 0.f, ma = 0.f;   // max |d_fwd|, max |d_adj| of the thread's points
    for (int k = 0; active && k < kend; ++k) {
        const int idx = ((i1b + k) * g.n2 + i2) * g.n3 + i3;
        const int ctr = ((k + 1 + H) * E2 + ty + 1 + H) * P3 + lane + 4;
        const float u[3] = {box[ctr] * dth1, box[BOX + ctr] * dth2, box[2 * BOX + ctr] * dth3};
        float a[3];
        // forward: X* = x - u, X = x - (u + dt v(X*)) / 2
        box_interp3<H, WY, E1>(box, k, r2, r3, -u[0], -u[1], -u[2], a);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float x = staged ? -0.5f * fmaf(a[c], dth[c], u[c]) : __int_as_float(0x7fffffff);
            d_fwd[c * n + idx] = x;
            mf = fmaxf(mf, fabsf(x));
        }
        if (d_adj) {
            // adjoint (velocity -v): X* = x + u, X = x + (u + dt v(X*)) / 2
            box_interp3<H, WY, E1>(box, k, r2, r3, u[0], u[1], u[2], a);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float x = staged ? 0.5f * fmaf(a[c], dth[c], u[c]) : __int_as_float(0x7fffffff);
                d_adj[c * n + idx] = x;
                ma = fmaxf(ma, fabsf(x));
            }
        }
    }
    if (dmax) {
        // the largest |d| of each field, as k_absmax finds it (fmaxf of the
        // absolute values; the bits of non-negative floats order as unsigned
        // integers): a warp, then the block, then one atomic per block
        __shared__ float red[2][8];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mf = fmaxf(mf, __shfl_xor_sync(0xffffffffu, mf, o));
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        }
        if (lane == 0) {
            red[0][ty] = mf;
            red[1][ty] = ma;
        }
        __syncthreads();
        if (tid < 2) {
            float m = 0.f;
            for (int w = 0; w < 8; ++w) m = fmaxf(m, red[tid][w]);
            atomicMax(dmax + tid, __float_as_uint(m));
        }
    }
}

// Tensor map of the velocity (3 x n1 x n2 x n3, x3 fastest) with a box of
// 64 x E2 x E1 x 3 elements; false unless rows are whole 16-byte units, v is
// 16-byte aligned and the grid is at least one box large.
bool velocity_tensor_map(CUtensorMap* map, const Dims& g, const float* v, int E1, int E2) {
    std::memset(map, 0, sizeof(*map));
    if (g.n3 % 4 || g.n3 < 64 || g.n2 < E2 || g.n1 < E1 || E1 > 256 || E2 > 256 ||
        (reinterpret_cast<uintptr_t>(v) & 15))
        return false;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dim[4] = {(cuuint64_t)g.n3, (cuuint64_t)g.n2, (cuuint64_t)g.n1, 3};
    const cuuint64_t stride[3] = {sizeof(float) * (cuuint64_t)g.n3,
                                  sizeof(float) * (cuuint64_t)g.n23,
                                  sizeof(float) * (cuuint64_t)g.n};
    const cuuint32_t boxd[4] = {64, (cuuint32_t)E2, (cuuint32_t)E1, 3};
    const cuuint32_t estride[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(v), dim, stride, boxd,
               estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// The TMA-staged departure kernel when its tensor map can be made; false
// (nothing launched) otherwise.
template <int H>
bool run_departure_fixed(const Dims& g, const float* v, float dth1, float dth2, float dth3,
                         float* d_fwd, float* d_adj, cudaStream_t st, cudaError_t* err,
                         unsigned int* dmax) {
    constexpr int E1 = kDepK + 3 + 2 * H, E2 = 8 + 3 + 2 * H;
    const size_t smem = sizeof(float) * 3 * (size_t)E1 * E2 * 64 + 16;
    CUtensorMap map;
    if (!velocity_tensor_map(&map, g, v, E1, E2)) return false;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(k_departure_fixed<H>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (attr != cudaSuccess) {
        *err = attr;
        return true;
    }
    const int inject = g_inject_stage.exchange(0) ? 1 : 0;
    const dim3 grid((g.n3 + 31) / 32, (g.n2 + 7) / 8, (g.n1 + kDepK - 1) / kDepK);
    if (dmax) {
        *err = cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned int), st);
        if (*err != cudaSuccess) return true;
    }
    k_departure_fixed<H><<<grid, dim3(32, 8), smem, st>>>(g, v, dth1, dth2, dth3, d_fwd, d_adj,
                                                          map, inject, dmax);
    *err = cudaGetLastError();
    return true;
}

template <int H>
cudaError_t run_departure_tile(const Dims& g, Tile t, const float* v, float dth1, float dth2,
                               float dth3, float* d_fwd, float* d_adj, cudaStream_t st) {
    constexpr int E2 = 8 + 3 + 2 * H;
    constexpr int P3 = ((35 + 2 * H) + 31) & ~31;
    const size_t smem = sizeof(float) * (size_t)(t.k + 3 + 2 * H) * E2 * P3;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_departure_tile<H>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(sizeof(float) * kMaxBoxFloats));
        if (e != cudaSuccess) return e;
    }
    k_departure_tile<H><<<march_grid(g, t), dim3(32, 8), smem, st>>>(g, t.k, v, dth1, dth2, dth3,
                                                                    d_fwd, d_adj);
    return cudaGetLastError();
}

dim3 march_grid(const Dims& g, Tile t) {
    return dim3((g.n3 + 31) / 32, (g.n2 + t.wy - 1) / t.wy, (g.n1 + t.k - 1) / t.k);
}

template <class Epi>
cudaError_t run_march(const Dims& g, Tile t, const float* f, const float* d, const Epi& epi,
                      cudaStream_t st) {
    if (t.k < 1 || t.wy < 1) return cudaErrorInvalidValue;
    // the register-window kernel marches in groups of 4 points; 1 or 2
    // points per thread only for the staged kernels (small grids)
    if ((t.k < 4 || (t.k & 3)) && !tile_staged(t)) return cudaErrorInvalidValue;
    if (t.wy == 16) {
        // 16-row blocks exist only as the fixed-halo staged kernel
        if (!tile_staged(t) || t.halo > 3) return cudaErrorInvalidValue;
        if (t.halo <= 1) return run_tile_fixed<Epi, 1, 16>(g, t, f, d, epi, st);
        if (t.halo == 2) return run_tile_fixed<Epi, 2, 16>(g, t, f, d, epi, st);
        return run_tile_fixed<Epi, 3, 16>(g, t, f, d, epi, st);
    }
    if (32 * t.wy > 256) return cudaErrorInvalidValue;
    if (tile_staged(t) && t.wy == 8 && t.halo <= 3) {
        if (t.halo <= 1) return run_tile_fixed<Epi, 1, 8>(g, t, f, d, epi, st);
        if (t.halo == 2) return run_tile_fixed<Epi, 2, 8>(g, t, f, d, epi, st);
        return run_tile_fixed<Epi, 3, 8>(g, t, f, d, epi, st);
    }
    if (tile_staged(t)) {
        const int H = t.halo < 1 ? 1 : t.halo;
        const int E1 = t.k + 3 + 2 * H, E2 = t.wy + 3 + 2 * H, E3 = 35 + 2 * H;
        const int P3 = (E3 + 31) & ~31;
        {
            const size_t smem = sizeof(float) * (size_t)E1 * E2 * P3;
            if (smem > 48 * 1024) {
                const cudaError_t e = cudaFuncSetAttribute(
                    k_tile<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                    (int)(sizeof(float) * kMaxBoxFloats));
                if (e != cudaSuccess) return e;
            }
            k_tile<Epi><<<march_grid(g, t), dim3(32, t.wy), smem, st>>>(g, t.k, H, E1, E2, E3, P3,
                                                                         f, d, epi);
            return cudaGetLastError();
        }
    }
    k_march<Epi><<<march_grid(g, t), dim3(32, t.wy), 0, st>>>(g, t.k, f, d, epi);
    return cudaGetLastError();
}

__global__ void k_absmax(const float* __restrict__ d, long long count, unsigned int* out) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < count;
         i += (long long)gridDim.x * kThreads)
        m = fmaxf(m, fabsf(d[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// ------------------------------------------------------- streaming kernels

__global__ void __launch_bounds__(kThreads)
k_incstate_init(Dims g, const float* __restrict__ vt, const float* __restrict__ g0, float dt,
                float* __restrict__ u0) {
    pdl_wait();
    pdl_trigger();
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    const long long n = g.n;
    const float f0 = -fmaf(vt[2 * n + idx], ld(g0, 2 * n + idx),
                           fmaf(vt[n + idx], ld(g0, n + idx), vt[idx] * ld(g0, idx)));
    u0[idx] = 0.5f * dt * f0;
}


// rho~_j = u_j - dt/2 f_j = u_j + dt/2 v~ . grad rho_j (the incremental state
// from the carried u_j = rho~_j + dt/2 f_j).
__global__ void __launch_bounds__(kThreads)
k_inc_state_level(Dims g, const float* __restrict__ u, const float* __restrict__ vt,
                  const float* __restrict__ gj, float dt, float* __restrict__ out) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    const long long n = g.n;
    const float vg = fmaf(vt[2 * n + idx], ld(gj, 2 * n + idx),
                          fmaf(vt[n + idx], ld(gj, n + idx), vt[idx] * ld(gj, idx)));
    out[idx] = fmaf(0.5f * dt, vg, u[idx]);
}

// b += w lam grad_f (3 components): one term of int lam grad rho~ dt.
__global__ void __launch_bounds__(kThreads)
k_acc_scaled_grad(Dims g, const float* __restrict__ lam, const float* __restrict__ gf, float w,
                  float* __restrict__ b) {
    const int idx = blockIdx.x * kThreads + threadIdx.x;
    if (idx >= g.n) return;
    const long long n = g.n;
    const float l = w * lam[idx];
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c * n + idx] = fmaf(l, gf[c * n + idx], b[c * n + idx]);
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

void arm_stage_timeout(int on) { g_inject_stage.store(on ? 1 : 0); }

namespace {
std::atomic<bool> g_dependent_launch{true};
}
bool dependent_launch_enabled() { return g_dependent_launch.load(std::memory_order_relaxed); }
void set_dependent_launch(bool on) { g_dependent_launch.store(on); }

cudaError_t launch_absmax(const float* d, long long count, unsigned int* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    int nb = (int)((count + kThreads - 1) / kThreads);
    if (nb > 152 * 8) nb = 152 * 8;
    k_absmax<<<nb, kThreads, 0, st>>>(d, count, out);
    return cudaGetLastError();
}

// The staged kernel's box: (k + 3 + 2H) x (wy + 3 + 2H) rows of 35 + 2H
// columns, stored with a row pitch that is a multiple of 32 words so that
// lanes whose stencil bases differ by a row or a plane still hit distinct
// shared-memory banks.
bool tile_staged(const Tile& t) {
    if (t.halo < 0) return false;
    const int H = t.halo < 1 ? 1 : t.halo;   // halo 0 runs the H = 1 kernel
    const long long E3 = 35 + 2 * H, P3 = (E3 + 31) & ~31LL;
    const long long cap = t.wy >= 16 ? kMaxBoxFloats16 : kMaxBoxFloats;
    return E3 <= 96 && (t.k + 3 + 2LL * H) * (t.wy + 3 + 2LL * H) * P3 <= cap;
}

int march_blocks(const Dims& g, Tile t) {
    const dim3 gr = march_grid(g, t);
    return (int)(gr.x * gr.y * gr.z);
}

cudaError_t launch_departure(const Dims& g, Tile t, const float* v, float dt, float* d_fwd,
                             float* d_adj, cudaStream_t st, unsigned int* dmax, bool* maxed) {
    if (maxed) *maxed = false;
    const float two_pi = 6.283185307179586f;
    const float dth1 = dt * g.n1 / two_pi, dth2 = dt * g.n2 / two_pi, dth3 = dt * g.n3 / two_pi;
    if (t.halo >= 0 && t.halo <= 3 && t.tma) {
        // one tensor copy of the three components' boxes per block
        cudaError_t e = cudaSuccess;
        bool done;
        unsigned int* m = d_adj ? dmax : nullptr;
        if (t.halo <= 1) done = run_departure_fixed<1>(g, v, dth1, dth2, dth3, d_fwd, d_adj, st, &e, m);
        else if (t.halo == 2) done = run_departure_fixed<2>(g, v, dth1, dth2, dth3, d_fwd, d_adj, st, &e, m);
        else done = run_departure_fixed<3>(g, v, dth1, dth2, dth3, d_fwd, d_adj, st, &e, m);
        if (done) {
            if (maxed && m && e == cudaSuccess) *maxed = true;
            return e;
        }
    }
    // the per-thread staged kernel tiles rows by 8 whatever the transports'
    // tile (the same arithmetic as the tensor-copy kernel: equal points)
    Tile td = t;
    td.wy = 8;
    if (td.halo >= 0 && td.halo <= 3 && tile_staged(td)) {
        if (td.halo <= 1) return run_departure_tile<1>(g, td, v, dth1, dth2, dth3, d_fwd, d_adj, st);
        if (td.halo == 2) return run_departure_tile<2>(g, td, v, dth1, dth2, dth3, d_fwd, d_adj, st);
        return run_departure_tile<3>(g, td, v, dth1, dth2, dth3, d_fwd, d_adj, st);
    }
    k_departure<<<nblocks(g.n), kThreads, 0, st>>>(g, v, dth1, dth2, dth3, d_fwd, d_adj);
    return cudaGetLastError();
}

cudaError_t launch_interp(const Dims& g, Tile t, const float* f, const float* d, float* out,
                          cudaStream_t st) {
    return run_march(g, t, f, d, EpiStore{out}, st);
}

cudaError_t launch_state_step(const Dims& g, Tile t, const float* rho_in, const float* d,
                              float* rho_out, const float* rho_R, float* lam_out,
                              double* partials, int max_partials, int* nblk_out,
                              cudaStream_t st) {
    if (!rho_R) return run_march(g, t, rho_in, d, EpiStore{rho_out}, st);
    const int nb = march_blocks(g, t);
    if (nb > max_partials) return cudaErrorInvalidValue;
    if (nblk_out) *nblk_out = nb;
    return run_march(g, t, rho_in, d, EpiStateFinal{rho_out, rho_R, lam_out, partials}, st);
}

// Eq. (sml-advection) for the adjoint source f = lam div v with
// f_0 = nu_0 (div v)(X): lam_new = nu_0 + dt/2 (nu_0 dX + (nu_0 + dt nu_0 dX) dv)
// = c(x) nu_0 with c = 1 + dt/2 (dX + dv + dt dX dv), fixed for a given v.
cudaError_t launch_adjoint_acc(const Dims& g, Tile t, const float* lam_in, const float* d,
                               const float* c, float* lam_out, const float* grad, float w,
                               float* b, const float* lam_first, const float* grad_first,
                               float w_first, const float* dotp, double* partials,
                               int max_partials, int* nblk_out, cudaStream_t st,
                               const float* add, const Fin* fin) {
    const int nb = march_blocks(g, t);
    if (dotp && nb > max_partials) return cudaErrorInvalidValue;
    if (nblk_out) *nblk_out = nb;
    const Fin f = (fin && dotp) ? *fin : Fin{};
    if (add)
        return run_march(g, t, lam_in, d,
                         EpiAdjAccT<true>{lam_out, c, grad, b, g.n, w, lam_first, grad_first,
                                          w_first, dotp, partials, add, f},
                         st);
    return run_march(g, t, lam_in, d,
                     EpiAdjAcc{lam_out, c, grad, b, g.n, w, lam_first, grad_first, w_first, dotp,
                               partials, nullptr, f},
                     st);
}

// The persistent small-grid matvec transport (k_matvec_persistent): one
// cooperative launch with one block per (co-resident) slot, tiles of one point
// per thread along x1 and 8 rows; nb_out = blocks (= partial sums).
// cudaErrorNotSupported when the boxes do not fit (halo > 3) or the grid is
// not small; the caller then launches the steps one by one.
cudaError_t launch_matvec_persistent(const Dims& g, int halo_fwd, int halo_adj, int nt, float dt,
                                     const float* vt, const float* grad, const float* d_fwd,
                                     const float* d_adj, const float* coef, float* u0, float* u1,
                                     float* lam, float* b, const float* dotp, double* partials,
                                     int max_partials, unsigned int* bar, int* err, int* nb_out,
                                     cudaStream_t st) {
    if (halo_fwd < 0 || halo_adj < 0 || halo_fwd > 3 || halo_adj > 3) return cudaErrorNotSupported;
    PersistArgs a;
    a.g = g;
    a.K = 1;
    const int WY = 8;
    a.Hf = halo_fwd < 1 ? 1 : halo_fwd;
    a.Hb = halo_adj < 1 ? 1 : halo_adj;
    a.E1f = a.K + 3 + 2 * a.Hf; a.E2f = WY + 3 + 2 * a.Hf; a.E3f = 35 + 2 * a.Hf;
    a.E1b = a.K + 3 + 2 * a.Hb; a.E2b = WY + 3 + 2 * a.Hb; a.E3b = 35 + 2 * a.Hb;
    a.P3 = 64;
    a.gx = (g.n3 + 31) / 32;
    a.gy = (g.n2 + WY - 1) / WY;
    a.gz = (g.n1 + a.K - 1) / a.K;
    a.nt = nt;
    a.dt = dt;
    a.vt = vt; a.grad = grad; a.d_fwd = d_fwd; a.d_adj = d_adj; a.coef = coef;
    a.u[0] = u0; a.u[1] = u1; a.lam = lam; a.b = b; a.dotp = dotp; a.partials = partials;
    a.bar = bar; a.err = err;
    const int E1 = a.E1f > a.E1b ? a.E1f : a.E1b, E2 = a.E2f > a.E2b ? a.E2f : a.E2b;
    const size_t smem = sizeof(float) * (size_t)E1 * E2 * a.P3;
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    static int per_sm = 0, sms = 0;
    std::call_once(once, [&] {
        attr = cudaFuncSetAttribute(k_matvec_persistent,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(float) * kMaxBoxFloats));
        int dev = 0;
        if (attr == cudaSuccess) attr = cudaGetDevice(&dev);
        if (attr == cudaSuccess)
            attr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // occupancy at the largest box (halo 3): a grid that fits any launch
        const size_t smax = sizeof(float) * (1 + 3 + 6) * (WY + 3 + 6) * 64;
        if (attr == cudaSuccess)
            attr = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_matvec_persistent,
                                                                 32 * WY, smax);
    });
    if (attr != cudaSuccess) return attr;
    const int ntiles = a.gx * a.gy * a.gz;
    int G = per_sm * sms;
    if (G > ntiles) G = ntiles;
    if (G > max_partials) G = max_partials;
    if (G < 1) return cudaErrorNotSupported;
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(32, WY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr_coop[1];
    attr_coop[0].id = cudaLaunchAttributeCooperative;
    attr_coop[0].val.cooperative = 1;
    cfg.attrs = attr_coop;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_matvec_persistent, a);
    if (e != cudaSuccess) return e;
    if (nb_out) *nb_out = G;
    return cudaSuccess;
}

cudaError_t launch_source_step(const Dims& g, Tile t, const float* s_old, const float* d,
                               const float* divv, const float* s_new, float dt, float* out,
                               cudaStream_t st) {
    return run_march(g, t, s_old, d, EpiSrcAdd{out, divv, s_new, dt}, st);
}

cudaError_t launch_inc_state_level(const Dims& g, const float* u, const float* vt,
                                   const float* grad_j, float dt, float* out, cudaStream_t st) {
    k_inc_state_level<<<nblocks(g.n), kThreads, 0, st>>>(g, u, vt, grad_j, dt, out);
    return cudaGetLastError();
}

cudaError_t launch_acc_scaled_grad(const Dims& g, const float* lam, const float* grad_f, float w,
                                   float* b, cudaStream_t st) {
    k_acc_scaled_grad<<<nblocks(g.n), kThreads, 0, st>>>(g, lam, grad_f, w, b);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_coef(const Dims& g, Tile t, const float* divv, const float* d_adj,
                                float dt, float* c, cudaStream_t st) {
    return run_march(g, t, divv, d_adj, EpiCoef{c, divv, dt}, st);
}

// Algorithm 2 step rho~_{j+1} = I[rho~_j](X) + dt/2 (I[f_j](X) + f_{j+1}(x)).
// The interpolant is linear in the field, so with u_j = rho~_j + dt/2 f_j:
// rho~_{j+1} = I[u_j](X) + dt/2 f_{j+1}(x) and u_{j+1} = I[u_j](X) + dt f_{j+1}(x).
cudaError_t launch_incstate_step(const Dims& g, Tile t, const float* u_in, const float* d,
                                 const float* vt, const float* grad_j1, float dt, int final_step,
                                 float* out, cudaStream_t st) {
    return run_march(g, t, u_in, d, EpiIncState{out, vt, grad_j1, g.n, dt, final_step}, st);
}

cudaError_t launch_incstate_init(const Dims& g, const float* vt, const float* grad0, float dt,
                                 float* u0, cudaStream_t st) {
    return launch_dependent(k_incstate_init, dim3(nblocks(g.n)), dim3(kThreads), 0, st, g, vt,
                            grad0, dt, u0);
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
