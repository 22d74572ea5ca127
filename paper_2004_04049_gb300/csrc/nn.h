// nn.h - building blocks of the learned GS warm-start network (conv kernels in nn_conv.cu,
// elementwise and reduction kernels in nn_ops.cu, the network in warmstart.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace holo {
namespace nn {

enum ConvMode : int { kConvFwd = 0, kConvDgrad = 1, kConvWgrad = 2 };

struct ConvArgs {
    int B, H, W;                      // batch and spatial size (input = output, 3x3, pad 1)
    int Cin, Cout;                    // GEMM channels: forward Cin -> Cout; dgrad: layer Cout -> Cin
    const __nv_bfloat16* in;          // forward/wgrad: x [B][H][W][Cin]; dgrad: dy [B][H][W][Cin]
    const __nv_bfloat16* wmat;        // forward: W [Cout][9*Cin]; dgrad: Wt [Cout][9*Cin]
    const __nv_bfloat16* dy;          // wgrad: [B][H][W][Cout]
    const float* bias;                // forward: [Cout] or null
    const __nv_bfloat16* residual;    // forward: [B][H][W][Cout] added before the ReLU, or null
    int relu;                         // forward: apply max(., 0)
    int flip;                         // dgrad: offsets (1-ky, 1-kx)
    __nv_bfloat16* out;               // forward/dgrad output [B][H][W][Cout] or null
    float* out_f32;                   // optional float32 copy of the output
    float* dw;                        // wgrad: [Cout][9*Cin], accumulated
    int kchunk;                       // wgrad: pixels per split (set by conv3x3)
};

// mode: kConvFwd, kConvDgrad (forward kernel with flip = 1) or kConvWgrad. Forward and
// input gradient run on tcgen05 (nn_conv_tc05.cu) when the output width is 32, 64 or 128,
// the input has at least 32 channels and the tensors are 16-byte aligned; `legacy` forces
// the mma.sync kernel (comparisons).
int conv3x3(const ConvArgs& a, int mode, cudaStream_t st, bool legacy = false);
bool conv3x3_tc05_supported(const ConvArgs& a);
int conv3x3_tc05(const ConvArgs& a, int mode, cudaStream_t st);
// reads (and optionally clears) the flag a tcgen05 conv kernel sets when a bounded wait expires
int conv3x3_tc05_fault(int* out, bool clear);

// ---- elementwise / reductions (nn_ops.cu); tensors are [B][H][W][C] bf16, C % 8 == 0
int prep_input(const float* target, int B, int Hs, int Ws, int H, int W, __nv_bfloat16* x, int C,
               cudaStream_t st);
int avgpool2(const __nv_bfloat16* x, int B, int H, int W, int C, __nv_bfloat16* y, cudaStream_t st);
// dx (+)= avgpool2 backward of dy (accumulate != 0 adds to dx)
int avgpool2_bwd(const __nv_bfloat16* dy, int B, int H, int W, int C, __nv_bfloat16* dx, int accumulate,
                 cudaStream_t st);
int upsample2(const __nv_bfloat16* x, int B, int H, int W, int C, __nv_bfloat16* y, cudaStream_t st);
int upsample2_bwd(const __nv_bfloat16* dy, int B, int H, int W, int C, __nv_bfloat16* dx, cudaStream_t st);
// g = d * (y > 0), in place on d
int relu_bwd(__nv_bfloat16* d, const __nv_bfloat16* y, size_t n, cudaStream_t st);
// a += b
int add_inplace(__nv_bfloat16* a, const __nv_bfloat16* b, size_t n, cudaStream_t st);
// db[c] += sum over pixels of g[p][c]
int bias_grad(const __nv_bfloat16* g, size_t pixels, int C, float* db, cudaStream_t st);
// Offset-invariant phase loss of out[p][0..1] (float32, channel stride C) against the label
// phases (radians) with weights target^2; writes loss (mean over the batch) and the
// gradient into gout[p][0..1] (bf16, channel stride C, other channels zeroed).
int phase_loss(const float* out, int C, const float* label, const float* target, int B, int HW,
               float* scratch, float* loss, __nv_bfloat16* gout, cudaStream_t st);
// Adam step on float32 master weights, then the bf16 copies used by the kernels
int adam(float* w, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2, float eps,
         int step, cudaStream_t st);
// W [Cout][9][Cin] float32 -> wmat [Cout][9*Cin] bf16 and wt [Cin][9*Cout] bf16
int pack_weights(const float* w, int Cout, int Cin, __nv_bfloat16* wmat, __nv_bfloat16* wt, cudaStream_t st);
// phase = atan2(v, u) of out[.][0..1] at H x W, bilinearly resampled on (u, v) to Ho x Wo
int phase_out(const float* out, int C, int H, int W, int Ho, int Wo, float* phase, cudaStream_t st);

}  // namespace nn
}  // namespace holo
