// Shared device helpers and the internal launcher interface of libreg.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cufft.h>
#include <stdint.h>

namespace reg {

// Grid geometry.  n <= 2^30 so a point index fits in int; component offsets
// (c * n) use long long.
struct Dims {
    int n1, n2, n3;
    int n23;          // n2 * n3
    int n;            // n1 * n2 * n3
    int m3;           // n3 / 2 + 1 (half spectrum along x3)
    int nc;           // n1 * n2 * m3 complex coefficients per field
};

inline Dims make_dims(int n1, int n2, int n3) {
    Dims d;
    d.n1 = n1; d.n2 = n2; d.n3 = n3;
    d.n23 = n2 * n3;
    d.n = n1 * n2 * n3;
    d.m3 = n3 / 2 + 1;
    d.nc = n1 * n2 * d.m3;
    return d;
}

// ------------------------------------------------------------ device side

// i mod n for any int i (n > 0).
__device__ __forceinline__ int wrap(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// Cubic Lagrange basis on the nodes -1, 0, 1, 2 at t in [0, 1]:
//   l_-1 = -t(t-1)(t-2)/6, l_0 = (t+1)(t-1)(t-2)/2,
//   l_1 = -(t+1)t(t-2)/2,   l_2 = (t+1)t(t-1)/6,
// with p = t(t-1) and q = (t+1)(t-2) = p - 2 shared (10 operations).
__device__ __forceinline__ void lagrange4(float t, float w[4]) {
    const float p = fmaf(t, t, -t);
    const float q = p - 2.f;
    w[0] = p * fmaf(t, -1.f / 6.f, 1.f / 3.f);
    w[1] = q * fmaf(t, 0.5f, -0.5f);
    w[2] = q * (-0.5f * t);
    w[3] = p * fmaf(t, 1.f / 6.f, 1.f / 6.f);
}

// Programmatic dependent launch: a kernel launched with launch_dependent()
// may start while its predecessor on the stream is still running.  It must
// pass pdl_wait() -- which returns once the predecessor has completed and its
// memory operations are visible -- before it reads or writes global memory
// that the predecessor (or anything before it) touches, and it lets its own
// dependents start (pdl_trigger) only after that wait, so a kernel that
// starts early can rely on everything before its predecessor being complete.
// Both are no-ops in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Process-wide switch of launch_dependent (reg_set_dependent_launch).
bool dependent_launch_enabled();
void set_dependent_launch(bool on);

// Launch kern<<<grid, block, smem, st>>>(args...) with programmatic stream
// serialisation (when enabled): the kernel must call pdl_wait() first.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = dependent_launch_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Finish of a reduction kernel's per-block FP64 partial sums inside the same
// launch (no separate launch_finalize): every block, once its partials are
// visible, draws a ticket from an atomic counter; the block that draws the
// last one (no block waits for another) sums each slot t's partials in the
// order launch_finalize uses (thread-strided, warp shuffles, then the warps in
// order), writes sc[out[t]] = sum * scale, then sc[copy_to] = sc[copy_from]
// when copy_to >= 0, and resets the counter for the next launch.  The
// counter belongs to one context, whose launches on its stream do not
// overlap.
struct Fin {
    unsigned int* count;   // null: no finish (the partials are left for launch_finalize)
    double* sc;
    double scale;
    int out[3];
    int copy_from, copy_to;
};

template <int NS>
__device__ __forceinline__ void finish_partials(const double* partials, int nblk, const Fin& f) {
    __shared__ unsigned int ticket;
    __shared__ double red[32];
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    __threadfence();   // this block's partials before its ticket
    __syncthreads();
    if (tid == 0) ticket = atomicAdd(f.count, 1u);
    __syncthreads();
    if (ticket != (unsigned int)nblk - 1u) return;
    __threadfence();
    for (int t = 0; t < NS; ++t) {
        double acc = 0.0;
        for (int i = tid; i < nblk; i += nthr) acc += __ldcg(partials + (long long)t * nblk + i);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int i = 0; i < nthr / 32; ++i) s += red[i];
            f.sc[f.out[t]] = s * f.scale;
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (f.copy_to >= 0) f.sc[f.copy_to] = f.sc[f.copy_from];
        *f.count = 0u;
    }
}

// Packed FP32 pairs (Blackwell f32x2 ALU): two independent IEEE FP32
// multiply-adds per instruction.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float2 upk(f32x2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// The 4 x 4 x 4 stencil of the point i + d (grid units): wrapped element
// offsets per axis and the Lagrange weights.
struct Stencil {
    int o1[4], o2[4], o3[4];
    float w1[4], w2[4], w3[4];
};

__device__ __forceinline__ void axis_stencil(int i, float d, int n, int stride,
                                             int o[4], float w[4]) {
    const float fl = floorf(d);
    lagrange4(d - fl, w);
    int b = wrap(i + (int)fl - 1, n);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        o[a] = b * stride;
        b = (b + 1 == n) ? 0 : b + 1;
    }
}

__device__ __forceinline__ void make_stencil(Stencil& s, const Dims& g, int i1, int i2,
                                             int i3, float d1, float d2, float d3) {
    axis_stencil(i1, d1, g.n1, g.n23, s.o1, s.w1);
    axis_stencil(i2, d2, g.n2, g.n3, s.o2, s.w2);
    axis_stencil(i3, d3, g.n3, 1, s.o3, s.w3);
}

// sum_{abc} w1 w2 w3 f[...] for one scalar field.
__device__ __forceinline__ float gather1(const Stencil& s, const float* __restrict__ f) {
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float acc2 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const float* row = f + s.o1[a] + s.o2[b];
            float r = s.w3[0] * __ldg(row + s.o3[0]);
            r = fmaf(s.w3[1], __ldg(row + s.o3[1]), r);
            r = fmaf(s.w3[2], __ldg(row + s.o3[2]), r);
            r = fmaf(s.w3[3], __ldg(row + s.o3[3]), r);
            acc2 = fmaf(s.w2[b], r, acc2);
        }
        acc = fmaf(s.w1[a], acc2, acc);
    }
    return acc;
}

// Decompose a point index into (i1, i2, i3).
__device__ __forceinline__ void unflatten(const Dims& g, int idx, int& i1, int& i2, int& i3) {
    i1 = idx / g.n23;
    const int r = idx - i1 * g.n23;
    i2 = r / g.n3;
    i3 = r - i2 * g.n3;
}

// ------------------------------------------------------------ launchers

// Tile of the x1-marching interpolation kernels: a block is 32 (x3) x wy (x2)
// threads and each thread walks k consecutive points along x1.
struct Tile {
    int k;          // points per thread along x1 (multiple of 4)
    int wy;         // threads per block along x2 (1, 2, 4 or 8)
    int halo = -1;  // bound on |floor(displacement)| (cells) of the launch's
                    // points; >= 0 selects the shared-memory staged kernel,
                    // -1 (unknown) the register-window kernel
    int tma = 1;    // staged box by one TMA copy where the grid allows (1) or
                    // by per-thread cp.async copies (0)
};

// Largest shared-memory box (floats) of the staged interpolation kernel.
constexpr int kMaxBoxFloats = 18432;
// Blocks of 16 rows (512 threads) stage up to this many floats (110 KB: two
// resident blocks, 32 warps, per SM).
constexpr int kMaxBoxFloats16 = 28224;

// out[0] = max over i < count of |d[i]| as float bits (d: 3 components).
cudaError_t launch_absmax(const float* d, long long count, unsigned int* out, cudaStream_t st);

// transport.cu
// t.halo (>= ceil of the predictor's largest displacement, grid units) and
// the tile select the shared-memory staged kernel when it applies.  dmax
// (may be null; 2 words): where the tensor-copy kernel runs with d_adj, it
// also leaves max |d_fwd| and max |d_adj| there as launch_absmax would, and
// sets *maxed (else *maxed = false and dmax is untouched).
cudaError_t launch_departure(const Dims& g, Tile t, const float* v, float dt, float* d_fwd,
                             float* d_adj, cudaStream_t st, unsigned int* dmax = nullptr,
                             bool* maxed = nullptr);
// out = I[f](x + d) for one scalar field.
cudaError_t launch_interp(const Dims& g, Tile t, const float* f, const float* d, float* out,
                          cudaStream_t st);
// State step rho_out = I[rho_in](x + d).  With rho_R != nullptr (last step)
// also lam_out = rho_R - rho_out (if lam_out != nullptr) and per-block FP64
// partial sums of (rho_out - rho_R)^2 into partials[0 .. nblocks).
cudaError_t launch_state_step(const Dims& g, Tile t, const float* rho_in, const float* d,
                              float* rho_out, const float* rho_R, float* lam_out,
                              double* partials, int max_partials, int* nblk_out,
                              cudaStream_t st);
// Adjoint / incremental-adjoint tau-step lam_out = c(x) I[lam_in](x + d)
// (c == nullptr: divergence-free velocity, c = 1), fused with the trapezoid
// time integral b = sum_j w_j lam_j grad rho_j: lam_out may be null (last
// step), and at every point b += w lam_out grad.  lam_first != nullptr (first
// step): b starts from w_first lam_first grad_first instead of its stored
// value.  dotp != nullptr (last step): per-block FP64 partials of <dotp, b>
// into partials[0 .. *nblk_out).
// add != nullptr: lam_out = c(x) I[lam_in](x + d) + add(x) (the known-source
// part of a full-Newton incremental adjoint step, from launch_source_step).
cudaError_t launch_adjoint_acc(const Dims& g, Tile t, const float* lam_in, const float* d,
                               const float* c, float* lam_out, const float* grad, float w,
                               float* b, const float* lam_first, const float* grad_first,
                               float w_first, const float* dotp, double* partials,
                               int max_partials, int* nblk_out, cudaStream_t st,
                               const float* add = nullptr, const Fin* fin = nullptr);
// One Gauss-Newton matvec's transports (incremental state from v~, the
// incremental adjoint with the time integral b~, partial sums of <dotp, b~>)
// in one persistent cooperative launch for small grids (grid-wide barriers
// between the steps, bounded waits raising *err); *nb_out = partial sums.
// cudaErrorNotSupported when it does not apply (halo > 3).
cudaError_t launch_matvec_persistent(const Dims& g, int halo_fwd, int halo_adj, int nt, float dt,
                                     const float* vt, const float* grad, const float* d_fwd,
                                     const float* d_adj, const float* coef, float* u0, float* u1,
                                     float* lam, float* b, const float* dotp, double* partials,
                                     int max_partials, unsigned int* bar, int* err, int* nb_out,
                                     cudaStream_t st);
// Known-source part of an adjoint tau-step: out = dt/2 (1 + dt dv(x))
// I[s_old](x + d) + dt/2 s_new(x), dv = divv (null: divergence free, dv = 0).
cudaError_t launch_source_step(const Dims& g, Tile t, const float* s_old, const float* d,
                               const float* divv, const float* s_new, float dt, float* out,
                               cudaStream_t st);
// rho~_j = u_j + dt/2 v~ . grad rho_j from the carried incremental state u_j.
cudaError_t launch_inc_state_level(const Dims& g, const float* u, const float* vt,
                                   const float* grad_j, float dt, float* out, cudaStream_t st);
// b[3][n] += w lam[n] grad_f[3][n].
cudaError_t launch_acc_scaled_grad(const Dims& g, const float* lam, const float* grad_f, float w,
                                   float* b, cudaStream_t st);
// c(x) = 1 + dt/2 (dX + dv + dt dX dv), dv = div v(x), dX = I[div v](x + d_adj).
cudaError_t launch_adjoint_coef(const Dims& g, Tile t, const float* divv, const float* d_adj,
                                float dt, float* c, cudaStream_t st);
// Incremental state, carried as u_j = rho~_j + dt/2 f_j, f = -v~ . grad rho(t_j):
//   u_{j+1} = I[u_j](x + d) + dt f_{j+1}(x);  final step writes
//   lam~(1) = -(I[u_{nt-1}](x + d) + dt/2 f_nt(x)) instead.
// grad_j1 is grad rho(t_{j+1}).
cudaError_t launch_incstate_step(const Dims& g, Tile t, const float* u_in, const float* d,
                                 const float* vt, const float* grad_j1, float dt, int final_step,
                                 float* out, cudaStream_t st);
// u_0 = -dt/2 v~ . grad rho(t_0)
cudaError_t launch_incstate_init(const Dims& g, const float* vt, const float* grad0, float dt,
                                 float* u0, cudaStream_t st);
// det(I + grad u) pointwise from the nine derivative fields
// gu[(3 c + j) n ..] = d_j u_c.
cudaError_t launch_jacobian_det(const float* gu, float* det, long long n, cudaStream_t st);
// Deformation displacement step: u_{j+1} = I[u_j](X) + dt/2 (I[-v](X) - v(x)).
cudaError_t launch_deformation_step(const Dims& g, const float* u_in, const float* v,
                                    const float* d, float dt, float* u_out,
                                    cudaStream_t st);
// float <-> bfloat16 copies (count elements).
cudaError_t launch_to_bf16(const float* in, __nv_bfloat16* out, long long count,
                           cudaStream_t st);
cudaError_t launch_from_bf16(const __nv_bfloat16* in, float* out, long long count,
                             cudaStream_t st);
int march_blocks(const Dims& g, Tile t);   // blocks of one marching launch
// Arm (1) or disarm (0) the bounded-wait test of the next TMA-staged launch.
void arm_stage_timeout(int on);
bool tile_staged(const Tile& t);           // t runs the shared-memory staged kernel

// spectral.cu -- multipliers on the half spectrum (cufftComplex = float2).
// All scale by 1/n (the unnormalised inverse FFT).
enum SpecOp {
    SPEC_GRAD = 0,      // out[3] = i k' in[1]
    SPEC_DIV = 1,       // out[1] = i k' . in[3]
    SPEC_ASSEMBLE = 2,  // out[3] = beta A in_a[3] + (P) in_b[3]   (in_a or in_b may be null)
    SPEC_PRECOND = 3,   // out[3] = M (P) in[3]
    SPEC_GAUSS = 4,     // out[1] = G in[1]
    SPEC_LERAY = 5,     // out[3] = P in[3]
    SPEC_REG = 6        // out[3] = beta A in[3]
};
struct SpecArgs {
    const float2* in_a;
    const float2* in_b;
    float2* out;
    double beta;
    int kind;           // REG_H1 / REG_H2 / REG_H1DIV
    int project;        // apply P
    float s1, s2, s3;   // Gaussian widths
    int normalised;     // in_a holds normalised coefficients (F f / n): no 1/n
};
cudaError_t launch_spectral(const Dims& g, SpecOp op, const SpecArgs& a, cudaStream_t st);
// Per-block FP64 partials of sum_k weight(k) A(k) |V(k)|^2 over 3 fields
// (Hermitian weights on the half spectrum).
cudaError_t launch_spec_energy(const Dims& g, const float2* v, int kind, double* partials,
                               int nblk, cudaStream_t st);
// Spectral Krylov kernels (normalised half-spectrum coefficients, 3 fields).
// Partials: slot t of block b at partials[t * nblk + b].  The preconditioner
// is M = 1 / (beta A + shift) (shift 0: the inverse regularisation operator).
cudaError_t launch_sp_init(const Dims& g, const float2* gh, float2* r, float2* s, float2* p,
                           float2* pc, double beta, double shift, int kind, int project,
                           double* partials, int nblk, cudaStream_t st);
// fin (may be null): finish the partials in the same launch (Fin).
cudaError_t launch_sp_update(const Dims& g, float2* s, float2* r, const float2* p,
                             const float2* B, double* sc, int irz, int ipap, int ipb, int ipq,
                             double beta, double shift, int kind, int project,
                             double* partials, int nblk, cudaStream_t st,
                             const Fin* fin = nullptr);
cudaError_t launch_sp_direction(const Dims& g, const float2* r, float2* p, float2* pc,
                                const double* sc, int irznew, int irz, int zero_beta,
                                double beta, double shift, int kind, int project,
                                double* partials, int nblk, cudaStream_t st,
                                const Fin* fin = nullptr);
cudaError_t launch_sp_gradient(const Dims& g, const float2* v, const float2* B, float2* gout,
                               double beta, int kind, int project, double* partials, int nblk,
                               cudaStream_t st);
cudaError_t launch_sp_axpy(const Dims& g, float2* out, float2* copy, const float2* x,
                           const float2* y, float a, int kind, int project, double* partials,
                           int nblk, cudaStream_t st);
// s += a p, r -= a q and the partial sums of herm |r|^2 in one pass.
cudaError_t launch_sp_fcg_update(const Dims& g, float2* s, float2* r, const float2* p,
                                 const float2* q, float a, double* partials, int nblk,
                                 cudaStream_t st);
cudaError_t launch_sp_dot(const Dims& g, const float2* a, const float2* b, double* partials,
                          int nblk, cudaStream_t st);
cudaError_t launch_sp_normalise(const Dims& g, const float2* in, float2* out, int project,
                                cudaStream_t st);

// Two-level preconditioner between a fine grid gf and a coarse grid gc (both
// with normalised half-spectrum coefficients, 3 fields): restriction to the
// modes L = {|k_j| < nc_j / 2} scaled by `scale` (coarse Nyquist planes 0);
// z = y on L, M P r elsewhere, with partials <r, z>.
cudaError_t launch_sp_restrict(const Dims& gf, const Dims& gc, const float2* in, float2* out,
                               float scale, cudaStream_t st);
cudaError_t launch_sp_twolevel(const Dims& gf, const Dims& gc, const float2* r, const float2* y,
                               float2* z, double beta, double shift, int kind, int project,
                               double* partials, int nblk, cudaStream_t st);

// deriv.cu -- spectral first derivative along one axis by one-dimensional
// FFTs in shared memory: out (+)= d_axis f (i k' with the Nyquist entry 0).
// Grids whose axes are powers of two (n1, n2 in 16..512, n3 in 32..512)
// and f, out 16-byte aligned (the kernels move 16-byte vectors);
// cudaErrorNotSupported elsewhere.  deriv_supported(g, f, out): the same test
// (a null pointer is not checked).
bool deriv_supported(const Dims& g, const void* f = nullptr, const void* out = nullptr);
cudaError_t launch_deriv(const Dims& g, int axis, const float* f, float* out, int accumulate,
                         cudaStream_t st);
// out3[a] = d_a f for a = 0, 1, 2 in one launch (components n apart), on cubic
// grids of 32..256 points a side (deriv_supported's conditions besides);
// cudaErrorNotSupported elsewhere, with nothing launched.
cudaError_t launch_grad(const Dims& g, const float* f, float* out3, cudaStream_t st);

// blas.cu
int blas_blocks();   // number of partial-sum blocks used by reductions
cudaError_t launch_dot_partials(const float* a, const float* b, long long count,
                                double* partials, int nblk, cudaStream_t st);
// result[0] = scale * sum(partials[0..nblk)).
cudaError_t launch_finalize(const double* partials, int nblk, double scale, double* result,
                            cudaStream_t st);
cudaError_t launch_axpy(float* y, const float* x, float alpha, long long count,
                        cudaStream_t st);           // y += alpha x
cudaError_t launch_axpby_out(float* out, const float* x, const float* y, float a, float b,
                             long long count, cudaStream_t st);   // out = a x + b y
// result[k] = scale * sum(partials[k * stride .. k * stride + nblk)) for k < count
cudaError_t launch_finalize_multi(const double* partials, int nblk, int stride, int count,
                                  double scale, double* result, cudaStream_t st);
cudaError_t launch_scale(float* y, float alpha, long long count, cudaStream_t st);
// out[3][n] = s[n] * v[3][n] (pointwise, per component)
cudaError_t launch_mul_fields(const float* s, const float* v, float* out, long long n,
                              cudaStream_t st);

}  // namespace reg
