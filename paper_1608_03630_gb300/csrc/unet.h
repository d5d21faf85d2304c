// Internal interface of the U-Net kernels (unet_kernels.cu, unet.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace reg {
namespace unet {

enum { MODE_FWD = 0, MODE_BWD_DATA = 1, MODE_BWD_WEIGHT = 2 };

struct ConvGeom {
    int D, H, W, V;   // volume and voxel count
    int Ci, Co;       // channels in / out
    int ks;           // kernel size (3 or 1), zero padding ks / 2
};

struct IgemmArgs {
    ConvGeom g;
    const __nv_bfloat16* A_src;   // FWD, BWD_WEIGHT: X [V][Ci]; BWD_DATA: dY [V][Co]
    const __nv_bfloat16* B_src;   // FWD: w [ks^3 Ci][Co]; BWD_DATA: wt [ks^3 Co][Ci]; BWD_WEIGHT: dY [V][Co]
    __nv_bfloat16* out_bf;        // FWD output (bf16) ...
    float* out_f;                 // ... or FP32 (one of the two)
    int out_stride, out_off;      // FWD / BWD_DATA output row stride and channel offset
    const float* bias;            // FWD
    int relu;                     // FWD: apply max(0, .)
    float* dX;                    // BWD_DATA output [V][out_stride]
    float* dW;                    // BWD_WEIGHT output [ks^3 Ci][Co] (accumulated)
    int kchunk;                   // BWD_WEIGHT: voxels per block
    const __nv_bfloat16* Bt_src;  // FWD on tcgen05: wt [ks^3][Co][Ci] (K-major B)
};

cudaError_t launch_igemm(int mode, const IgemmArgs& a, cudaStream_t st);

// Forward 3x3x3 convolution on the tcgen05 tensor cores (unet_tc.cu): usable
// when Co is 16, 32, 64 or 128, Ci a multiple of 8, one output -- BF16 with
// bias / ReLU, or FP32 plain sums (no bias, no ReLU) -- with row stride and
// channel offset multiples of 8, and every pointer 16-byte aligned.
bool conv_fwd_tc_ok(const IgemmArgs& a);
cudaError_t launch_conv_fwd_tc(const IgemmArgs& a, cudaStream_t st);

}  // namespace unet
}  // namespace reg
