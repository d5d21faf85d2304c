// Batched registration of independent image pairs of uneven sizes, and the
// interpolation-tile autotuner.
//
// Every pair owns a context and a non-blocking CUDA stream.  Default mode
// (REG_BATCH_ONE_GRAPH): the pairs advance in lockstep Newton steps; the
// gradients and line searches run on host worker threads, each pair on its
// stream, and the PCG solves of a Newton step of every active pair are one
// CUDA graph holding one device-controlled while-loop per pair, each ending
// at its own stopping test (solver.cu, batch_solve_graph).  REG_BATCH_THREADS:
// worker threads take whole solves from a queue ordered by cost (grid points
// x time steps, largest first), each solve with its own device-controlled PCG
// graph per Newton step.  The autotuner times the interpolation kernels of a
// linearised context for a few tile shapes and keeps the fastest; results are
// cached per (grid, halo) for the process.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "ctx.h"

struct reg_batch {
    std::vector<reg_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    int workers;
    int mode;                      // REG_BATCH_ONE_GRAPH or REG_BATCH_THREADS
    cudaStream_t launch;           // the one-graph mode's launch stream
    reg::BatchGraphCache cache;
    int graphs_launched;
    std::string err;
};

namespace reg {

namespace {

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune_cache;

// `reps` matvec transports captured as one executable graph, or nullptr
// (context error state untouched) when the capture is refused.
cudaGraphExec_t capture_transports(reg_ctx* c, const float* vt, int reps) {
    cudaStream_t user = c->stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = bind_stream(c, c->capture_stream) == REG_OK &&
              cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        int s = REG_OK;
        for (int r = 0; r < reps && s == REG_OK; ++r) s = op_matvec_transport(c, vt, nullptr, 0);
        ok = cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && s == REG_OK;
    }
    if (ok && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        exec = nullptr;
        ok = false;
    }
    if (graph) cudaGraphDestroy(graph);
    if (bind_stream(c, user) != REG_OK) ok = false;
    if (!ok) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        c->dead = false;   // a refused capture is not a device fault
        c->err.clear();
    }
    return exec;
}

// Simple timing: the mean of `reps` launches of the matvec transports (nt
// incremental-state and nt incremental-adjoint steps, the latter with the
// time integral), replayed as one CUDA graph like the PCG loop that runs
// them: timed from the host's launches instead, a small grid measures the
// host's enqueue cost, which exceeds the kernels' own time there.
int time_transports(reg_ctx* c, const float* vt, int reps, float* ms) {
    cudaEvent_t a, b;
    REG_CK(c, cudaEventCreate(&a));
    REG_CK(c, cudaEventCreate(&b));
    cudaGraphExec_t exec = capture_transports(c, vt, reps);
    if (exec) {
        REG_CK(c, cudaGraphLaunch(exec, c->stream));   // warm
        REG_CK(c, cudaEventRecord(a, c->stream));
        REG_CK(c, cudaGraphLaunch(exec, c->stream));
        REG_CK(c, cudaEventRecord(b, c->stream));
    } else {
        REG_TRY(op_matvec_transport(c, vt, nullptr, 0));   // warm
        REG_CK(c, cudaEventRecord(a, c->stream));
        for (int r = 0; r < reps; ++r) REG_TRY(op_matvec_transport(c, vt, nullptr, 0));
        REG_CK(c, cudaEventRecord(b, c->stream));
    }
    REG_CK(c, cudaEventSynchronize(b));
    REG_CK(c, cudaEventElapsedTime(ms, a, b));
    *ms /= reps;
    if (exec) cudaGraphExecDestroy(exec);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return REG_OK;
}

}  // namespace

}  // namespace reg

using namespace reg;

extern "C" {

int reg_autotune(reg_ctx* c, int* k_out, int* wy_out) {
    if (!c) return REG_EINVAL;
    if (c->dead) return fail(c, REG_ECUDA, "context unusable after a CUDA error");
    if (!c->have_lin) return fail(c, REG_ENOTREADY, "reg_gradient must come first");
    const auto key = std::make_tuple(c->g.n1, c->g.n2, c->g.n3, c->halo_fwd, c->halo_adj);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c->tile.k = it->second.first;
            c->tile.wy = it->second.second;
            if (k_out) *k_out = c->tile.k;
            if (wy_out) *wy_out = c->tile.wy;
            return REG_OK;
        }
    }
    // a smooth direction for the timing: the cached gradient of rho(t_0)
    const float* vt = c->grad_hist;
    const Tile keep = c->tile;
    const bool timing = c->timing;
    c->timing = false;
    // k = 1 or 2 points per thread give small grids (the two-level
    // preconditioner's coarse grid) more warps; they are tried only where
    // the default tile fills less than two waves of the 152 SMs
    static const int cand[][2] = {{4, 8}, {8, 8}, {16, 8}, {8, 4}, {16, 4}, {8, 16}, {16, 16},
                                  {1, 8}, {2, 8}, {1, 16}, {2, 4}};
    const int ncand = march_blocks(c->g, Tile{8, 8}) < 2 * 152 ? 11 : 7;
    float best = 1e30f;
    int bk = keep.k, bw = keep.wy;
    for (int ci = 0; ci < ncand; ++ci) {
        const auto& kw = cand[ci];
        c->tile.k = kw[0];
        c->tile.wy = kw[1];
        float ms = 0.f;
        const int s = time_transports(c, vt, 4, &ms);
        if (s != REG_OK) {
            c->tile = keep;
            c->timing = timing;
            return s;
        }
        if (ms < best) { best = ms; bk = kw[0]; bw = kw[1]; }
    }
    c->timing = timing;
    c->tile = keep;
    c->tile.k = bk;
    c->tile.wy = bw;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = std::make_pair(bk, bw);
    }
    if (k_out) *k_out = bk;
    if (wy_out) *wy_out = bw;
    return REG_OK;
}

int reg_batch_create(int npairs, const int* dims, int nt, double beta, int reg_kind,
                     int incompressible, int precision, reg_batch** out) {
    if (!out) return REG_EINVAL;
    *out = nullptr;
    if (npairs < 1 || !dims) return REG_EINVAL;
    reg_batch* b = new (std::nothrow) reg_batch();
    if (!b) return REG_ENOMEM;
    b->workers = std::min(npairs, 8);
    b->mode = REG_BATCH_ONE_GRAPH;
    b->launch = nullptr;
    b->graphs_launched = 0;
    int status = REG_OK;
    if (cudaStreamCreateWithFlags(&b->launch, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return REG_ECUDA;
    }
    for (int i = 0; i < npairs && status == REG_OK; ++i) {
        reg_ctx* c = nullptr;
        status = reg_create(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], nt, beta, reg_kind,
                            incompressible, &c);
        if (status != REG_OK) break;
        b->ctx.push_back(c);
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            status = REG_ECUDA;
            break;
        }
        b->streams.push_back(s);
        status = reg_set_stream(c, s);
        // the pairs' PCG loops run side by side: no cooperative launches
        if (status == REG_OK) status = reg_set_persistent(c, 0);
        if (status == REG_OK && precision) status = reg_set_precision(c, precision);
    }
    if (status != REG_OK) {
        for (auto c : b->ctx) reg_destroy(c);
        for (auto s : b->streams) cudaStreamDestroy(s);
        cudaStreamDestroy(b->launch);
        delete b;
        return status;
    }
    *out = b;
    return REG_OK;
}

int reg_batch_destroy(reg_batch* b) {
    if (!b) return REG_OK;
    if (b->launch) cudaStreamSynchronize(b->launch);
    if (b->cache.exec) cudaGraphExecDestroy(b->cache.exec);
    for (auto c : b->ctx) reg_destroy(c);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->launch) cudaStreamDestroy(b->launch);
    delete b;
    return REG_OK;
}

int reg_batch_set_mode(reg_batch* b, int mode) {
    if (!b || (mode != REG_BATCH_ONE_GRAPH && mode != REG_BATCH_THREADS)) return REG_EINVAL;
    b->mode = mode;
    return REG_OK;
}

int reg_batch_graphs_launched(const reg_batch* b, int* count) {
    if (!b || !count) return REG_EINVAL;
    *count = b->graphs_launched;
    return REG_OK;
}

int reg_batch_solve(reg_batch* b, float* const* v_inout, const float* const* rho_T,
                    const float* const* rho_R, int presmooth, int autotune,
                    const reg_solve_opts* opts, reg_solve_stats* stats, double* latency_ms,
                    int* status_out) {
    if (!b || !v_inout || !rho_T || !rho_R) return REG_EINVAL;
    const int np = (int)b->ctx.size();
    if (b->mode == REG_BATCH_ONE_GRAPH) {
        b->graphs_launched = 0;
        return batch_solve_graph(b->ctx, v_inout, rho_T, rho_R, presmooth, autotune, opts, stats,
                                 latency_ms, status_out, b->workers, b->launch, &b->cache,
                                 &b->graphs_launched);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return REG_ECUDA;
    // cost order, largest first
    std::vector<int> order(np);
    for (int i = 0; i < np; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        const long long cx = (long long)b->ctx[x]->g.n * b->ctx[x]->nt;
        const long long cy = (long long)b->ctx[y]->g.n * b->ctx[y]->nt;
        return cx > cy;
    });
    std::atomic<int> next(0);
    std::vector<int> st(np, REG_OK);
    std::vector<reg_solve_stats> local(np);
    std::vector<double> lat(np, 0.0);
    auto work = [&]() {
        cudaSetDevice(dev);
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= np) break;
            const int i = order[q];
            const auto t_start = std::chrono::steady_clock::now();
            reg_ctx* c = b->ctx[i];
            int s = reg_set_images(c, rho_T[i], rho_R[i], presmooth);
            if (s == REG_OK && autotune) {
                // linearise at the initial guess, tune, then solve
                float* g = nullptr;
                s = ensure_solver(c);
                if (s == REG_OK) {
                    g = c->sv[3];
                    s = reg_gradient(c, v_inout[i], g, nullptr);
                }
                if (s == REG_OK) s = reg_autotune(c, nullptr, nullptr);
            }
            if (s == REG_OK || s == REG_EMAXITER) {
                memset(&local[i], 0, sizeof(reg_solve_stats));
                s = reg_solve(c, v_inout[i], opts, &local[i]);
            }
            cudaStreamSynchronize(c->stream);
            st[i] = s;
            lat[i] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() -
                                                               t_start)
                         .count();
        }
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < b->workers; ++w) pool.emplace_back(work);
    for (auto& t : pool) t.join();
    int status = REG_OK;
    for (int i = 0; i < np; ++i) {
        if (stats) stats[i] = local[i];
        if (latency_ms) latency_ms[i] = lat[i];
        if (status_out) status_out[i] = st[i];
        if (st[i] != REG_OK && st[i] != REG_EMAXITER && status == REG_OK) status = st[i];
    }
    return status;
}

}  // extern "C"
