// The registration context behind the opaque reg_ctx handle, and the
// internal operations shared by the C-ABI entry points and the solver.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"
#include "reg.h"

struct reg_ctx {
    reg::Dims g;
    int nt;
    double beta;
    int kind;
    int incompressible;
    int precision;
    cudaStream_t stream;
    cudaStream_t capture_stream;  // owned; used to capture CUDA graphs
    std::string err;
    bool dead;            // a CUDA error happened: refuse further work

    // cuFFT plans: one field and three fields (batched)
    cufftHandle r2c1, c2r1, r2c3, c2r3;
    bool plans[4];

    // images (FP32 copies; bf16 copies in mixed precision)
    float* rho_T;
    float* rho_R;
    __nv_bfloat16* img_bf;        // [2n] rho_T, rho_R in bf16 (mixed precision)
    bool have_images;

    // linearisation point
    bool have_lin;
    float* d_fwd;        // [3n]
    float* d_adj;        // [3n]
    float* divv;         // [n] (compressible)
    float* rho_hist;     // [(nt+1) n]
    float* grad_hist;    // [(nt+1) 3n] grad rho(t_j), FP32 (gradient and FP32 matvec)
    bool grad0_valid;    // grad_hist level 0 = grad rho(t_0) of the current images
                         // (rho(t_0) = rho_T for every v: computed once per image set)

    // scratch
    float* lam_hist;     // [(nt+1) n] adjoint / incremental-adjoint levels
    float* coef;         // [n] adjoint step factor c(x) (compressible)
    float2* buf[2];      // [n] float2 each (2n floats): ping-pong scratch
    float* bacc;         // [3n] b / b~
    float* tmp3;         // [3n] real scratch
    float2* spec[2];     // [3 nc] complex scratch each
    double* partials;    // FP64 partial sums
    int npartials;
    double* dsc;         // device scalars [32]
    double* hsc;         // pinned host mirror [32]
    double pshift;       // shift of the solver's spectral preconditioner (reg_solve)
    // the device-controlled PCG graph, reused while the kernels it captured
    // stay the same: key = (halo_fwd, halo_adj, tile k, tile wy, hessian),
    // the preconditioner shift and beta
    cudaGraphExec_t pcg_exec;
    int pcg_key[5];
    double pcg_key_shift, pcg_key_beta;
    reg::Tile tile;      // tile of the interpolation kernels (k, wy)
    int halo_fwd, halo_adj;   // ceil(max |X - x|) of d_fwd / d_adj (-1: unknown)
    unsigned int* dabs;  // [2] device scratch for max |d| (float bits)
    unsigned int* gsync; // [4] persistent kernel: barrier counter, error flag; [2] the
                         // ticket counter of reductions finished in their own launch
    bool persistent;     // small grids: one persistent launch per matvec transport

    // Hessian: REG_HESS_GAUSS_NEWTON (default) or REG_HESS_FULL_NEWTON; the
    // full Newton matvec keeps the adjoint levels of the linearisation point
    // and every level of the incremental state (allocated when selected)
    int hessian;
    float* lam_lin;      // [(nt+1) n] lam(t_j) at the linearisation point
    float* rt_hist;      // [nt n] carried incremental state u_j, j < nt

    // solver vectors: real [3n] each, spectral [3 nc] each (ss[8], the
    // flexible PCG's H p, only with the two-level preconditioner)
    float* sv[4];
    float2* ss[9];
    bool have_solver;

    // two-level preconditioner: a context on the coarse grid (n_j / factor)
    // holding the restricted images, linearised at the restricted velocity
    reg_ctx* coarse;
    int coarse_factor;
    int coarse_tile_k, coarse_tile_wy;   // the coarse grid's tile; 0: autotuned
    long long img_version, coarse_img_version;   // restrict the images again when they change

    // timing
    bool timing;
    bool capturing;       // recording a CUDA graph: event pairs go to graph_pairs
    struct Pending { int phase; cudaEvent_t a, b; double bytes; };
    std::vector<Pending> pending;
    std::vector<Pending> graph_pairs;   // re-recorded on every replay of the graph
    std::vector<cudaEvent_t> free_events;
    reg_timing acc;
};

namespace reg {

// Largest number of partial-sum slots one reduction kernel writes (each slot
// holds blas_blocks() doubles); the partials buffer is sized for it.
constexpr int kMaxSlots = 4;

int fail(reg_ctx* c, int status, const std::string& msg);
int fail_cuda(reg_ctx* c, cudaError_t e, const char* what, int line);

#define REG_CK(ctx, call)                                                     \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::reg::fail_cuda(ctx, e_, #call, __LINE__); \
    } while (0)

#define REG_TRY(call)                     \
    do {                                  \
        int s_ = (call);                  \
        if (s_ != REG_OK) return s_;      \
    } while (0)

// Phase timing: begin() before a launch, end() after it (no-ops when off).
void phase_begin(reg_ctx* c, cudaEvent_t* ev);
void phase_end(reg_ctx* c, int phase, cudaEvent_t ev, double bytes);
// RAII helper around one launch.
struct Phase {
    reg_ctx* c; int ph; double bytes; cudaEvent_t ev;
    Phase(reg_ctx* c_, int ph_, double bytes_) : c(c_), ph(ph_), bytes(bytes_) {
        phase_begin(c, &ev);
    }
    ~Phase() { phase_end(c, ph, ev, bytes); }
};
// After a replay of a captured graph has completed: add its event pairs.
int harvest_graph_timing(reg_ctx* c);
// When the graph is destroyed: return its events to the pool.
void release_graph_timing(reg_ctx* c);

// Internal operations (device pointers; all on c->stream).
// maxed (may be null): when the kernel also left max |d_fwd|, max |d_adj| in
// c->dabs[0..1] (float bits), *maxed = true.
int op_departure(reg_ctx* c, const float* v, float* d_fwd, float* d_adj, bool* maxed = nullptr);
int op_fft_r2c(reg_ctx* c, const float* in, float2* out, int ncomp);
int op_fft_c2r(reg_ctx* c, float2* in, float* out, int ncomp);
int op_spectral(reg_ctx* c, SpecOp op, const SpecArgs& a, int ncomp_bytes_fields);
int op_grad(reg_ctx* c, const float* f, float* out3);
int op_div(reg_ctx* c, const float* v3, float* out);
int op_inner(reg_ctx* c, const float* a, const float* b, long long count, int slot);
// Linearisation at v: points, div v and c(x), state history, grad rho
// levels, adjoint, and b = int lam grad rho dt into bacc.
// state_ready: op_trial_state(c, v) ran last for this v (its points, state
// history and mismatch are reused).
// v_hat (may be null): the normalised coefficients of v, when the caller has
// them (div v then needs one inverse transform).
int op_linearize(reg_ctx* c, const float* v, bool state_ready = false,
                 const float2* v_hat = nullptr);
// J's mismatch at v with the points and state history kept in the
// linearisation buffers (the solver's line search: an accepted trial point
// is linearised next without redoing them).  Invalidates the linearisation.
int op_trial_state(reg_ctx* c, const float* v);
int op_gradient(reg_ctx* c, const float* v, float* g, int slot_J);
int op_objective(reg_ctx* c, const float* v, int slot_J);
// dsc[SC_JMIS] = 1/2 ||rho(1) - rho_R||^2_h for v (scratch buffers only).
int op_mismatch(reg_ctx* c, const float* v);
int op_matvec(reg_ctx* c, const float* vt, float* out);
// The transports of one GN matvec with the time integral fused into the
// incremental adjoint steps: bacc = b~ = sum_j w_j lam~_j grad rho_j; with
// dotp, dsc[slot] = <dotp, b~>_h.
int op_matvec_transport(reg_ctx* c, const float* vt, const float* dotp, int slot);
int op_precond(reg_ctx* c, const float* r, float* z);
// The in-launch finish of a reduction (Fin) on c's ticket counter and device
// scalars: slot t's sum times scale into dsc[slot_t], then dsc[copy_to] =
// dsc[copy_from] when copy_to >= 0.
Fin finish_into(reg_ctx* c, double scale, int slot0, int slot1 = 0, int copy_from = 0,
                int copy_to = -1);
int op_leray(reg_ctx* c, const float* v, float* out);
int read_scalars(reg_ctx* c, int first, int count);   // dsc -> hsc, synchronises
int bind_stream(reg_ctx* c, cudaStream_t s);         // launch stream + cuFFT plans
// ceil(scale max |d|) over a field [3n] (synchronises the stream).
int op_halo(reg_ctx* c, const float* d, int* halo, float scale = 1.f);
reg::Tile tile_with(const reg_ctx* c, int halo);
int ensure_solver(reg_ctx* c);

// Batches (solver.cu): the executable graph of one Newton step's PCG loops of
// all active pairs, kept while the pairs' captured kernels stay the same.
struct BatchGraphCache {
    cudaGraphExec_t exec = nullptr;
    std::vector<double> key;
};
// Lockstep Gauss-Newton over the pairs (see solver.cu); the per-pair outputs
// as reg_batch_solve; *graphs_launched = PCG graphs launched (one per step).
int batch_solve_graph(const std::vector<reg_ctx*>& ctx, float* const* v_io,
                      const float* const* rho_T, const float* const* rho_R, int presmooth,
                      int autotune, const reg_solve_opts* opts, reg_solve_stats* stats,
                      double* latency_ms, int* status_out, int workers, cudaStream_t launch,
                      BatchGraphCache* cache, int* graphs_launched);

// Device scalar slots.
enum {
    SC_JMIS = 0, SC_JREG = 1, SC_J = 2, SC_TMP = 3,
    SC_RZ = 4, SC_PQ = 5, SC_RR = 6, SC_RZNEW = 7, SC_GG = 8, SC_GS = 9,
    SC_INNER = 10, SC_ZERO = 11, SC_PAP = 12, SC_PB = 13,
    // device-controlled PCG loop: iteration count, exit flag, tol^2, cap
    SC_IT = 20, SC_FLAG = 21, SC_TOL2 = 22, SC_MAXIT = 23
};

}  // namespace reg
