// Forward state transport for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc: code inside another
// library's callback that must not touch the allocator, programs whose device
// memory is owned by a fixed pool or arena that must not grow, and
// latency-critical loops where an allocation (which may synchronise the
// device) is not acceptable.  This file gives them
// reg_state_transport_noalloc: the same state transport as
// reg_state_transport, with no context and no allocation.  Its one
// intermediate time level lives in the file-scope array g_level below, a fixed
// 16 MiB that every GPU loading the library keeps until the process exits.
#include <mutex>

#include "common.cuh"
#include "reg.h"

namespace {

// Largest grid the static intermediate level can hold: 2^22 points (16 MiB).
constexpr long long kMaxPoints = 1LL << 22;
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_level[kMaxPoints];

// Device address of g_level per device.  In host code the name g_level is a
// host-side stand-in, not a device address: the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  Only a
// successful lookup is kept, so a failed one (for instance while the device
// was not yet usable) is retried by the next call.
float* g_level_addr[kMaxDevices];
std::mutex g_level_mutex;

float* level_address(int dev) {
    std::lock_guard<std::mutex> lk(g_level_mutex);
    if (!g_level_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_level) == cudaSuccess) {
            g_level_addr[dev] = static_cast<float*>(p);
        } else {
            cudaGetLastError();   // leave no error behind for the caller
        }
    }
    return g_level_addr[dev];
}

}  // namespace

extern "C" int reg_state_transport_noalloc(int n1, int n2, int n3, int nt, const float* rho0,
                                           const float* d_fwd, float* rho1, void* stream) {
    if (n1 < 4 || n2 < 4 || n3 < 4 || nt < 1 || nt > 64) return REG_EINVAL;
    if ((long long)n1 * n2 * n3 > kMaxPoints) return REG_EINVAL;   // larger than g_level
    if (!rho0 || !d_fwd || !rho1 || rho0 == rho1) return REG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return REG_ECUDA;
    }
    float* level = level_address(dev);
    if (!level) return REG_ECUDA;
    const reg::Dims g = reg::make_dims(n1, n2, n3);
    const reg::Tile t{8, 4};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Level j (1 <= j < nt) lives in rho1 when nt - j is even, else in g_level,
    // so consecutive steps never read and write the same buffer and the last
    // step writes rho1.  Every level is written before it is read: nothing in
    // g_level has to start at zero.
    const float* in = rho0;
    for (int j = 1; j <= nt; ++j) {
        float* out = ((nt - j) % 2 == 0) ? rho1 : level;
        const cudaError_t err = reg::launch_state_step(g, t, in, d_fwd, out, nullptr, nullptr,
                                                       nullptr, 0, nullptr, st);
        if (err != cudaSuccess) return REG_ECUDA;
        in = out;
    }
    return REG_OK;
}
