// 3x3 convolution (zero padding, stride 1) on the 5th-generation tensor cores:
// internal interface between the denoiser (ur_nn.cu) and ur_conv_tc.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

namespace urnn {

// Residual 1x1 head (32 -> 2 channels) evaluated in the epilogue of a 32-channel convolution
// with ReLU: y = xn + Wh a + bh on the BF16-rounded activations a.  Inference writes y (times
// scale) and stores no activations; training (t_rf set) adds the mean squared error against
// the targets to loss, the head's parameter gradients to dwh / dbh, and stores the gradient at
// the ReLU output (masked by a > 0) in place of the activations, with its column sums added to
// the convolution's dbias.
struct HeadTC {
    const float *xn;                 // [P][2] normalised input (the residual)
    const float *wh, *bh;            // [2][32], [2]
    float scale;                     // output scale
    float *out_rf, *out_quad;        // [P] or null
    const float *t_rf, *t_quad;      // [P] targets (training) or null
    float inv_scale, inv_n;          // target normalisation; 1 / (2 P)
    double *loss;                    // += sum of squared differences x inv_n
    float *dwh, *dbh;                // += head gradients
};

struct ConvTC {
    const __nv_bfloat16 *x;      // input, NHWC [N][H][W][C], C a multiple of 32 (see x_low)
    int C, N, H, W;
    const __nv_bfloat16 *w;      // weights [taps][Cout][C], tap = 3 ky + kx
    int Cout;                    // a multiple of 32
    int taps;                    // 9, or 1: the input already holds the neighbourhood (weights [1][Cout][C])
    const float *bias;           // [Cout] or null
    const __nv_bfloat16 *mask;   // [N][H][W][Cout] or null: outputs where mask <= 0 become 0
    __nv_bfloat16 *y;            // output NHWC [N][H][W][Cout]
    int relu;                    // max(0, .) after the bias
    float *dbias = nullptr;      // [Cout] or null: += sum over pixels of the (masked) output, FP32
    __nv_bfloat16 *y2 = nullptr; // or null; else the output is split: channels [0, c_split) go to y
    int c_split = 0;             // ([N][H][W][c_split]) and [c_split, Cout) to y2 ([N][H][W][Cout - c_split]);
                                 // c_split a multiple of 32
    const HeadTC *head = nullptr; // or null; C_out = 32, 9 taps, ReLU only
    // Decoder input read from two tensors (9 taps, C_out in {32, 64, 96}, H and W even): channels
    // [0, c1) are x_low [N][H/2][W/2][c1] upsampled 2x (nearest), channels [c1, C) are
    // x [N][H][W][C - c1]; c1 a multiple of the channel chunk (64 if C % 64 == 0, else 32).
    const __nv_bfloat16 *x_low = nullptr;
    int c1 = 0;
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
    const __nv_bfloat16 *x;      // forward input NHWC [N][H][W][Cin] (see x_low)
    int Cin, N, H, W;
    const __nv_bfloat16 *dy;     // gradient at the convolution's output NHWC [N][H][W][Cout], Cout in {32, 64, 128, 256}
    int Cout, taps;
    float *dw;                   // [taps][Cout][Cin]
    // two-source input as in ConvTC (9 taps): channels [0, c1) from x_low upsampled, c1 % 32 == 0
    const __nv_bfloat16 *x_low = nullptr;
    int c1 = 0;
};

cudaError_t wgrad3x3_tc(const WgradTC &p, int *d_err, int n_sm, cudaStream_t stream, std::string *why);

}  // namespace urnn
