// Fourier resampling between grids of different sizes (Sec. III-B1: a field is
// its Fourier series on the periodic grid).  R2C on the input grid, a copy of
// the retained half-spectrum coefficients (scaled by 1 / n_in) into the zeroed
// output half-spectrum, C2R on the output grid.
#include <cufft.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "reg.h"

namespace {

struct Plans {
    cufftHandle r2c = 0, c2r = 0;
    cufftComplex* spec_in = nullptr;
    cufftComplex* spec_out = nullptr;
    int ncomp = 0;
};

typedef std::tuple<int, int, int, int, int, int, int> Key;
std::mutex g_mu;
std::map<Key, Plans>* g_plans = nullptr;

// Keep mode k of a length-n_in axis in a length-n_out axis: index of the
// same wavenumber there, or -1 when |k| >= min(n_in, n_out) / 2.
__device__ __forceinline__ int remap(int i, int nin, int nout) {
    const int k = i <= nin / 2 ? i : i - nin;
    const int lim = (nin < nout ? nin : nout);
    if (2 * (k < 0 ? -k : k) >= lim) return -1;
    return k >= 0 ? k : k + nout;
}

__global__ void k_resample_copy(const cufftComplex* __restrict__ in, cufftComplex* __restrict__ out,
                                int a1, int a2, int a3, int b1, int b2, int b3, int ncomp,
                                float scale) {
    const int h_in = a3 / 2 + 1, h_out = b3 / 2 + 1;
    const long long m_in = (long long)a1 * a2 * h_in;
    const long long m_out = (long long)b1 * b2 * h_out;
    const long long total = m_in * ncomp;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / m_in);
        long long r = t - c * m_in;
        const int i3 = (int)(r % h_in);
        r /= h_in;
        const int i2 = (int)(r % a2);
        const int i1 = (int)(r / a2);
        const int j1 = remap(i1, a1, b1), j2 = remap(i2, a2, b2);
        const int lim3 = a3 < b3 ? a3 : b3;
        if (j1 < 0 || j2 < 0 || 2 * i3 >= lim3) continue;
        cufftComplex v = in[t];
        v.x *= scale;
        v.y *= scale;
        out[c * m_out + ((long long)j1 * b2 + j2) * h_out + i3] = v;
    }
}

int get_plans(const int* a, const int* b, int ncomp, Plans** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_plans) g_plans = new std::map<Key, Plans>();
    Key key(a[0], a[1], a[2], b[0], b[1], b[2], ncomp);
    auto it = g_plans->find(key);
    if (it != g_plans->end()) {
        *out = &it->second;
        return REG_OK;
    }
    Plans p;
    p.ncomp = ncomp;
    int na[3] = {a[0], a[1], a[2]}, nb[3] = {b[0], b[1], b[2]};
    const long long ha = (long long)a[0] * a[1] * (a[2] / 2 + 1);
    const long long hb = (long long)b[0] * b[1] * (b[2] / 2 + 1);
    const long long ra = (long long)a[0] * a[1] * a[2], rb = (long long)b[0] * b[1] * b[2];
    if (cufftPlanMany(&p.r2c, 3, na, nullptr, 1, (int)ra, nullptr, 1, (int)ha, CUFFT_R2C, ncomp) !=
        CUFFT_SUCCESS)
        return REG_ECUFFT;
    if (cufftPlanMany(&p.c2r, 3, nb, nullptr, 1, (int)hb, nullptr, 1, (int)rb, CUFFT_C2R, ncomp) !=
        CUFFT_SUCCESS) {
        cufftDestroy(p.r2c);
        return REG_ECUFFT;
    }
    if (cudaMalloc(&p.spec_in, sizeof(cufftComplex) * ha * ncomp) != cudaSuccess ||
        cudaMalloc(&p.spec_out, sizeof(cufftComplex) * hb * ncomp) != cudaSuccess) {
        cudaGetLastError();
        cufftDestroy(p.r2c);
        cufftDestroy(p.c2r);
        cudaFree(p.spec_in);
        return REG_ENOMEM;
    }
    auto res = g_plans->emplace(key, p);
    *out = &res.first->second;
    return REG_OK;
}

}  // namespace

extern "C" int reg_spectral_resample(const int* nin, const int* nout, int ncomp, const float* in,
                                     float* out, void* stream) {
    if (!nin || !nout || !in || !out || ncomp < 1 || ncomp > 16) return REG_EINVAL;
    for (int d = 0; d < 3; ++d)
        if (nin[d] < 2 || nout[d] < 2 || nin[d] > 4096 || nout[d] > 4096) return REG_EINVAL;
    if ((long long)nin[0] * nin[1] * nin[2] * ncomp > (1LL << 31) ||
        (long long)nout[0] * nout[1] * nout[2] * ncomp > (1LL << 31))
        return REG_EINVAL;
    Plans* p = nullptr;
    int s = get_plans(nin, nout, ncomp, &p);
    if (s != REG_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the plan handles are shared: bind them to this stream and enqueue under
    // the lock (the device work of two calls with the same sizes is ordered
    // only if their streams are)
    std::lock_guard<std::mutex> lk(g_mu);
    const long long hb = (long long)nout[0] * nout[1] * (nout[2] / 2 + 1);
    const long long ra = (long long)nin[0] * nin[1] * nin[2];
    if (cufftSetStream(p->r2c, st) != CUFFT_SUCCESS || cufftSetStream(p->c2r, st) != CUFFT_SUCCESS)
        return REG_ECUFFT;
    if (cufftExecR2C(p->r2c, const_cast<float*>(in), p->spec_in) != CUFFT_SUCCESS)
        return REG_ECUFFT;
    if (cudaMemsetAsync(p->spec_out, 0, sizeof(cufftComplex) * hb * ncomp, st) != cudaSuccess)
        return REG_ECUDA;
    const long long ha = (long long)nin[0] * nin[1] * (nin[2] / 2 + 1);
    long long blocks = (ha * ncomp + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_resample_copy<<<(int)blocks, 256, 0, st>>>(p->spec_in, p->spec_out, nin[0], nin[1], nin[2],
                                                 nout[0], nout[1], nout[2], ncomp,
                                                 (float)(1.0 / (double)ra));
    if (cudaGetLastError() != cudaSuccess) return REG_ECUDA;
    if (cufftExecC2R(p->c2r, p->spec_out, out) != CUFFT_SUCCESS) return REG_ECUFFT;
    return REG_OK;
}
