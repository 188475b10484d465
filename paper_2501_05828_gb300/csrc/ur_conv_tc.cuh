// 3x3 convolution (zero padding, stride 1) on the 5th-generation tensor cores:
// internal interface between the denoiser (ur_nn.cu) and ur_conv_tc.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

namespace urnn {

struct ConvTC {
    const __nv_bfloat16 *x;      // input, NHWC [N][H][W][C], C a multiple of 32
    int C, N, H, W;
    const __nv_bfloat16 *w;      // weights [taps][Cout][C], tap = 3 ky + kx
    int Cout;                    // a multiple of 32
    int taps;                    // 9, or 1: the input already holds the neighbourhood (weights [1][Cout][C])
    const float *bias;           // [Cout] or null
    const __nv_bfloat16 *mask;   // [N][H][W][Cout] or null: outputs where mask <= 0 become 0
    __nv_bfloat16 *y;            // output NHWC [N][H][W][Cout]
    int relu;                    // max(0, .) after the bias
    float *dbias = nullptr;      // [Cout] or null: += sum over pixels of the (masked) output, FP32
};

// Enqueues the convolution on `stream`.  `d_err` (device int) receives a
// non-zero code if a pipeline wait inside the kernel gave up (bounded waits);
// the caller reads it at its next synchronisation.  Returns a CUDA error for
// launch failures and fills `why` for rejected shapes.
cudaError_t conv3x3_tc(const ConvTC &p, int *d_err, int n_sm, cudaStream_t stream, std::string *why);

// dw[tap][co][ci] += sum over pixels of dy[p][co] x[p + offset(tap)][ci]
// (zero outside the image), FP32 accumulation on the tensor cores, atomically
// added into dw (the caller zeroes it).  taps = 1 uses the centre tap only and
// writes dw[0][co][ci].
struct WgradTC {
    const __nv_bfloat16 *x;      // forward input NHWC [N][H][W][Cin]
    int Cin, N, H, W;
    const __nv_bfloat16 *dy;     // gradient at the convolution's output NHWC [N][H][W][Cout], Cout in {32, 64, 128, 256}
    int Cout, taps;
    float *dw;                   // [taps][Cout][Cin]
};

cudaError_t wgrad3x3_tc(const WgradTC &p, int *d_err, int n_sm, cudaStream_t stream, std::string *why);

}  // namespace urnn
