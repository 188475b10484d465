// Channel-data denoiser: a 4-level 2D U-Net over the analytic channel data of
// one transmit (an n_el x n_s image with 2 channels, rf and quad), trained to
// map low-ray-count channel data to high-ray-count channel data.  BF16 weights
// and activations (NHWC), FP32 accumulation, FP32 master weights with Adam.
// Forward, data-gradient and weight-gradient convolutions run on the
// 5th-generation tensor cores (TMA-fed tcgen05.mma with TMEM accumulators,
// ur_conv_tc.cu).  Decoder inputs (nearest-neighbour upsampling of the lower
// level concatenated with the skip tensor) are read by the convolutions from
// the two tensors, the upsampling done by the tensor map; only the quarter-
// resolution one is gathered into one NHWC buffer first.
#include "ultraray.h"
#include "ur_conv_tc.cuh"
#include "ur_device.cuh"
#include "ur_fastdiv.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

typedef __nv_bfloat16 bf16;

using ur::Div32;
using ur::divmod32;
using ur::make_div32;

namespace {

// Convolution input: channels [0, c1) from x1 (at half resolution when low1),
// channels [c1, c1 + c2) from x2 (full resolution).
struct ConvIn {
    const bf16 *x1;
    int c1, low1;
    const bf16 *x2;
    int c2;
};

// ------------------------------------------------------------------ small kernels

__device__ __forceinline__ void unpack8(const uint4 &u, float (&f)[8]) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

__device__ __forceinline__ uint4 pack8(const float (&f)[8]) {
    uint4 u;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
    return u;
}

#define GRID_STRIDE(i, n) \
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// The same over 32-bit indices: the activations' element counts stay below 2^32 (checked when
// a network is created), and pixel and channel indices come from division by invariant
// integers (ur_fastdiv.h) rather than 64-bit division.
#define GRID_STRIDE32(i, n) \
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += gridDim.x * blockDim.x)

// rf, quad [B][H][W] (fp32, the tracer's layout) -> the normalised BF16-rounded
// input xn [B][H][W][2] (fp32) and its 3x3 neighbourhood as 32 BF16 channels per
// pixel (channel 2 t + c = input channel c at tap t = 3 ky + kx, zero outside the
// image and from channel 18 on), so the first convolution is one K = 32 GEMM.
__global__ void k_prep(const float *rf, const float *quad, int B, int H, int W, Div32 dW, Div32 dH, float inv_scale,
                       bf16 *xcol, float *xn) {
    GRID_STRIDE32(p, (uint32_t)B * H * W) {
        uint32_t xu, yu;
        const uint32_t r = divmod32(p, dW, xu);
        const int b = (int)divmod32(r, dH, yu);
        const int x = (int)xu, y = (int)yu;
        float v[32];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
            float a = 0.f, q = 0.f;
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                const size_t o = ((size_t)b * H + yy) * W + xx;
                a = __bfloat162float(__float2bfloat16_rn(rf[o] * inv_scale));
                q = __bfloat162float(__float2bfloat16_rn(quad[o] * inv_scale));
            }
            v[2 * t] = a;
            v[2 * t + 1] = q;
        }
#pragma unroll
        for (int k = 18; k < 32; ++k) v[k] = 0.f;
        uint4 *dst = reinterpret_cast<uint4 *>(xcol + (size_t)p * 32);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) f[j] = v[8 * g + j];
            dst[g] = pack8(f);
        }
        xn[2 * p] = v[8];
        xn[2 * p + 1] = v[9];
    }
}

// Single-tap weights of the first convolution: wp[co][2 t + c] = w[t][co][c].
__global__ void k_pack_first(const bf16 *w, int C, bf16 *wp) {
    GRID_STRIDE(i, (long long)C * 32) {
        const int co = (int)(i / 32), k = (int)(i % 32);
        wp[i] = k < 18 ? w[((size_t)(k / 2) * C + co) * 32 + (k % 2)] : __float2bfloat16_rn(0.f);
    }
}

// dw[t][co][c] += dwp[co][2 t + c]: gradient of the single-tap form back to [9][C][32].
__global__ void k_unpack_first_grad(const float *dwp, int C, float *dw) {
    GRID_STRIDE(i, (long long)C * 18) {
        const int co = (int)(i / 18), k = (int)(i % 18);
        dw[((size_t)(k / 2) * C + co) * 32 + (k % 2)] += dwp[(size_t)co * 32 + k];
    }
}

// Decoder input: cat[b, y, x, 0:c1] = low[b, y/2, x/2, :] (nearest-neighbour
// upsampling), cat[b, y, x, c1:c1+c2] = skip[b, y, x, :]; 16-byte granules.
__global__ void k_upcat(const bf16 *low, int c1, const bf16 *skip, int c2, int B, int H, int W, Div32 dG, Div32 dW,
                        Div32 dH, bf16 *cat) {
    const int g1 = c1 / 8, G = (c1 + c2) / 8;
    GRID_STRIDE32(i, (uint32_t)B * H * W * G) {
        uint32_t gu, xu, yu;
        const uint32_t p = divmod32(i, dG, gu);
        const uint32_t r = divmod32(p, dW, xu);
        const int b = (int)divmod32(r, dH, yu);
        const int g = (int)gu, x = (int)xu, y = (int)yu;
        const bf16 *src = g < g1 ? low + (((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * c1 + g * 8
                                 : skip + (size_t)p * c2 + (g - g1) * 8;
        reinterpret_cast<uint4 *>(cat)[i] = *reinterpret_cast<const uint4 *>(src);
    }
}

// 2x2 average pooling, NHWC bf16, 8 channels per thread.
__global__ void k_pool2(const bf16 *x, bf16 *y, int B, int H, int W, int C, Div32 dG, Div32 dWo, Div32 dHo) {
    const int Ho = H / 2, Wo = W / 2, G = C / 8;
    const uint4 *xg = reinterpret_cast<const uint4 *>(x);
    GRID_STRIDE32(i, (uint32_t)B * Ho * Wo * G) {
        uint32_t gu, xu, yu;
        const uint32_t r = divmod32(divmod32(i, dG, gu), dWo, xu);
        const int b = (int)divmod32(r, dHo, yu);
        const int g = (int)gu, xo = (int)xu, yo = (int)yu;
        const size_t base = (((size_t)b * H + 2 * yo) * W + 2 * xo) * G + g;
        float s[8], t[8];
        unpack8(xg[base], s);
        unpack8(xg[base + G], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] += t[j];
        unpack8(xg[base + (size_t)W * G], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] += t[j];
        unpack8(xg[base + (size_t)W * G + G], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] = 0.25f * (s[j] + t[j]);
        reinterpret_cast<uint4 *>(y)[i] = pack8(s);
    }
}

// Per-channel sums of a thread block: thread t owns channels 8 (t % G) .. +8 of its
// pixels (G = C / 8 divides the 256-thread block); db[c] += the block's total.
__device__ __forceinline__ void flush_channel_sums(float (&acc)[8], int G, float *db) {
    __shared__ float s[256][9];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) s[threadIdx.x][j] = acc[j];
    __syncthreads();
    if ((int)threadIdx.x < G) {
        float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = threadIdx.x; q < (int)blockDim.x; q += G)
#pragma unroll
            for (int j = 0; j < 8; ++j) t[j] += s[q][j];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (t[j] != 0.f) atomicAdd(&db[8 * threadIdx.x + j], t[j]);
    }
}

// Gradient of a concatenated decoder input, first part ([B][H][W][C1]; the data-gradient
// convolution writes the skip channels straight to their own gradient): the C1 channels
// came from the nearest-upsampled half-resolution tensor, so dlow (half resolution) is the
// sum over each 2x2 block; it is the gradient at the lower level's last ReLU output, so it
// is masked by that activation `act` here and its column sums (that layer's bias gradient)
// go to db.
__global__ void __launch_bounds__(256) k_unconcat_low(const bf16 *dcat, int B, int H, int W, int C1, Div32 dWo,
                                                      Div32 dHo, const bf16 *act, bf16 *dlow, float *db) {
    const int Ho = H / 2, Wo = W / 2, G1 = C1 / 8, G = G1;
    const int gi = threadIdx.x % G1, lanes = blockDim.x / G1, pl = threadIdx.x / G1;
    const uint4 *dg = reinterpret_cast<const uint4 *>(dcat);
    const uint4 *ag = reinterpret_cast<const uint4 *>(act);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint32_t P = (uint32_t)B * Ho * Wo;
    for (uint32_t p = blockIdx.x * (uint32_t)lanes + pl; p < P; p += gridDim.x * (uint32_t)lanes) {
        uint32_t xu, yu;
        const int b = (int)divmod32(divmod32(p, dWo, xu), dHo, yu);
        const int xo = (int)xu, yo = (int)yu;
        const size_t base = (((size_t)b * H + 2 * yo) * W + 2 * xo) * G + gi;
        float v[8], t[8], m[8];
        unpack8(dg[base], v);
        unpack8(dg[base + G], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] += t[j];
        unpack8(dg[base + (size_t)W * G], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] += t[j];
        unpack8(dg[base + (size_t)W * G + G], t);
        unpack8(ag[(size_t)p * G1 + gi], m);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = m[j] > 0.f ? v[j] + t[j] : 0.f;
            acc[j] += v[j];
        }
        reinterpret_cast<uint4 *>(dlow)[(size_t)p * G1 + gi] = pack8(v);
    }
    flush_channel_sums(acc, G1, db);
}

// d[b, y, x, c] += dp[b, y/2, x/2, c] / 4 (gradient of 2x2 average pooling); the sum is
// the gradient at the encoder block's last ReLU output, so it is masked by that
// activation `act` and its column sums (the layer's bias gradient) go to db.
__global__ void __launch_bounds__(256) k_pool2_bwd_mask(bf16 *d, const bf16 *dp, const bf16 *act, int B, int H,
                                                        int W, int C, Div32 dW, Div32 dH, float *db) {
    const int G = C / 8, gi = threadIdx.x % G, lanes = blockDim.x / G, pl = threadIdx.x / G;
    uint4 *dg = reinterpret_cast<uint4 *>(d);
    const uint4 *pg = reinterpret_cast<const uint4 *>(dp);
    const uint4 *ag = reinterpret_cast<const uint4 *>(act);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint32_t P = (uint32_t)B * H * W;
    for (uint32_t p = blockIdx.x * (uint32_t)lanes + pl; p < P; p += gridDim.x * (uint32_t)lanes) {
        uint32_t xu, yu;
        const int b = (int)divmod32(divmod32(p, dW, xu), dH, yu);
        const int x = (int)xu, y = (int)yu;
        const size_t i = (size_t)p * G + gi;
        float v[8], a[8], m[8];
        unpack8(dg[i], v);
        unpack8(pg[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * G + gi], a);
        unpack8(ag[i], m);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            v[j] = m[j] > 0.f ? v[j] + 0.25f * a[j] : 0.f;
            acc[j] += v[j];
        }
        dg[i] = pack8(v);
    }
    flush_channel_sums(acc, G, db);
}

// Weights of the data gradients, every layer in one launch: for layer l (table entry j),
// W'[tap][ci][co] = W[8 - tap][co][ci], both at the layer's offset of the packed vector.
struct WtransTable {
    int n;
    long long start[15];   // prefix sums of 9 C_in C_out over the entries
    long long off[14];
    int cin[14], cout[14];
};
__global__ void k_wtrans_all(const bf16 *w, bf16 *wt, const WtransTable T) {
    GRID_STRIDE(i, T.start[T.n]) {
        int j = 0;
        while (j + 1 < T.n && i >= T.start[j + 1]) ++j;
        const long long li = i - T.start[j];
        const int Cout = T.cout[j], Cin = T.cin[j];
        const int co = (int)(li % Cout);
        const long long r = li / Cout;
        const int ci = (int)(r % Cin);
        const int tap = (int)(r / Cin);
        wt[T.off[j] + li] = w[T.off[j] + ((long long)(8 - tap) * Cout + co) * Cin + ci];
    }
}

// Adam (bias-corrected moments) on the fp32 master parameters; refreshes the bf16 copies.
__global__ void k_adam(float *p, const float *g, float *m, float *v, bf16 *pb, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void k_to_bf16(const float *p, bf16 *pb, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

int grid_for(long long n, int block = 256) { return (int)std::min<long long>(4096, (n + block - 1) / block + 1); }

// ------------------------------------------------------------------ network

constexpr int kNumConv = 14;

struct Fail {
    ur_status code;
    std::string msg;
};
[[noreturn]] void fail(ur_status c, const std::string &m) { throw Fail{c, m}; }
void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? UR_ERR_OOM : UR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

struct Tensor {
    bf16 *p = nullptr;
    int H = 0, W = 0, C = 0;
};

}  // namespace

struct ur_nn {
    int device = 0, sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int max_batch = 0, H = 0, W = 0, width = 32;
    float scale = 1.f;
    long long step = 0;
    unsigned long long launches = 0;   // kernels enqueued since creation
    // parameters: per conv [9][Cout][Cin] then [Cout]; head [2][C] then [2]
    int cin[kNumConv], cout[kNumConv];
    size_t woff[kNumConv], boff[kNumConv], hw_off = 0, hb_off = 0, n_params = 0;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *pbf = nullptr, *wt = nullptr;   // bf16 copies; the data gradients' (transposed) weights
    // activations and gradients
    bf16 *x = nullptr;
    float *xn = nullptr;
    Tensor act[kNumConv];    // post-ReLU outputs of every conv
    Tensor pool[3];          // pooled e1, e2, e3
    // training buffers (allocated by the first training step), in units of B*H*W*C BF16 values:
    // gA gradient at d1b's output (1), gB block scratch (1), gcat input gradient of a block (3),
    // gLow gradient of the half-resolution decoder input (1/2), gSkip skip-tensor gradients (1, 1/2, 1/4)
    bf16 *gcat = nullptr, *gA = nullptr, *gB = nullptr, *gSkip[3] = {nullptr, nullptr, nullptr}, *gLow = nullptr;
    bf16 *cat[1] = {nullptr};   // decoder input (upsampled lower level ++ skip) of d3a
    bf16 *wfirst = nullptr;  // first convolution as one tap over the 32 neighbourhood channels [C][32]
    float *dwfirst = nullptr;
    double *loss = nullptr;
    int *d_err = nullptr, *h_err = nullptr;   // bounded-wait failures inside the convolution kernels
    float *stage[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // host-buffer staging
    std::vector<void *> allocs;

    void *alloc(size_t bytes) {
        void *p = nullptr;
        ck(cudaMalloc(&p, std::max<size_t>(bytes, 256)), "cudaMalloc");
        allocs.push_back(p);
        return p;
    }
};

namespace {

template <class F>
ur_status nn_guard(ur_nn *nn, F &&f) {
    if (!nn) return UR_ERR_INVALID_ARG;
    try {
        nn->err.clear();
        f();
        return UR_OK;
    } catch (const Fail &e) {
        nn->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        nn->err = "host allocation failed";
        return UR_ERR_OOM;
    } catch (...) {
        nn->err = "unexpected host exception";
        return UR_ERR_CUDA;
    }
}

// Input of a convolution: x, or for a decoder input read from two tensors the skip tensor x and
// the half-resolution x_low whose upsampling gives channels [0, c1).
struct In {
    const bf16 *x, *x_low;
    int c1;
};

void conv_fwd(ur_nn *nn, In in, int B, int H, int W, int Cin, int Cout, const bf16 *w, const float *bias,
              const bf16 *mask, bf16 *y, bool relu, int taps = 9, float *dbias = nullptr, bf16 *y2 = nullptr,
              int c_split = 0, const urnn::HeadTC *head = nullptr) {
    urnn::ConvTC P{in.x, Cin, B, H, W, w, Cout, taps, bias, mask, y, relu ? 1 : 0, dbias, y2, c_split, head,
                   in.x_low, in.c1};
    std::string why;
    ++nn->launches;
    const cudaError_t e = urnn::conv3x3_tc(P, nn->d_err, nn->sms, nn->stream, &why);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorInvalidValue ? UR_ERR_INVALID_ARG : UR_ERR_CUDA,
             why.empty() ? std::string("conv kernel: ") + cudaGetErrorString(e) : why);
    }
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device view of a [batch][n_el][n_s] FP32 argument: the pointer itself, or a
// staging buffer (slot) filled from host memory on the network's stream.
float *staged(ur_nn *nn, int slot, const float *p, int batch, bool copy_in) {
    if (dev_ptr(p)) return const_cast<float *>(p);
    const size_t n = (size_t)nn->max_batch * nn->H * nn->W;
    if (!nn->stage[slot]) nn->stage[slot] = (float *)nn->alloc(sizeof(float) * n);
    if (copy_in)
        ck(cudaMemcpyAsync(nn->stage[slot], p, sizeof(float) * (size_t)batch * nn->H * nn->W, cudaMemcpyHostToDevice,
                           nn->stream),
           "copy input");
    return nn->stage[slot];
}

// Synchronises the network's stream and reports a convolution that gave up waiting.
void sync_check(ur_nn *nn, const char *what) {
    ck(cudaMemcpyAsync(nn->h_err, nn->d_err, sizeof(int), cudaMemcpyDeviceToHost, nn->stream), "read status");
    ck(cudaStreamSynchronize(nn->stream), what);
    if (*nn->h_err) {
        *nn->h_err = 0;
        ck(cudaMemsetAsync(nn->d_err, 0, sizeof(int), nn->stream), "reset status");
        fail(UR_ERR_TIMEOUT, std::string(what) + ": a convolution pipeline wait timed out");
    }
}

void conv_wgrad(ur_nn *nn, const bf16 *x, const bf16 *dy, int B, int H, int W, int Cin, int Cout, float *dw,
                int taps = 9, const bf16 *x_low = nullptr, int c1 = 0) {
    urnn::WgradTC P{x, Cin, B, H, W, dy, Cout, taps, dw, x_low, c1};
    std::string why;
    ++nn->launches;
    const cudaError_t e = urnn::wgrad3x3_tc(P, nn->d_err, nn->sms, nn->stream, &why);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorInvalidValue ? UR_ERR_INVALID_ARG : UR_ERR_CUDA,
             why.empty() ? std::string("wgrad kernel: ") + cudaGetErrorString(e) : why);
    }
}

// Grid of a kernel whose threads own 8 of C channels of every (256 / (C / 8))-th pixel and whose
// blocks end by adding their per-channel sums atomically: four blocks per SM, so each block
// covers many pixels and the C atomics per block (all to the same C addresses) stay few.
int channel_grid(const ur_nn *nn, long long P, int C) {
    const int lanes = 256 / (C / 8);
    return (int)std::min<long long>(4ll * std::max(1, nn->sms), (P + lanes - 1) / lanes);
}

// Inputs of every conv of the network at batch B.
struct Layer {
    ConvIn in;
    int H, W;
};

Layer layer_in(ur_nn *nn, int l) {
    const int H = nn->H, W = nn->W;
    auto full = [](const Tensor &t) { return ConvIn{t.p, t.C, 0, nullptr, 0}; };
    switch (l) {
        case 0: return {ConvIn{nn->x, 32, 0, nullptr, 0}, H, W};
        case 1: return {full(nn->act[0]), H, W};
        case 2: return {full(nn->pool[0]), H / 2, W / 2};
        case 3: return {full(nn->act[2]), H / 2, W / 2};
        case 4: return {full(nn->pool[1]), H / 4, W / 4};
        case 5: return {full(nn->act[4]), H / 4, W / 4};
        case 6: return {full(nn->pool[2]), H / 8, W / 8};
        case 7: return {full(nn->act[6]), H / 8, W / 8};
        case 8: return {ConvIn{nn->act[7].p, nn->act[7].C, 1, nn->act[5].p, nn->act[5].C}, H / 4, W / 4};
        case 9: return {full(nn->act[8]), H / 4, W / 4};
        case 10: return {ConvIn{nn->act[9].p, nn->act[9].C, 1, nn->act[3].p, nn->act[3].C}, H / 2, W / 2};
        case 11: return {full(nn->act[10]), H / 2, W / 2};
        case 12: return {ConvIn{nn->act[11].p, nn->act[11].C, 1, nn->act[1].p, nn->act[1].C}, H, W};
        default: return {full(nn->act[12]), H, W};
    }
}

// Input of conv l.  The decoder inputs of d2a and d1a are read by their convolutions straight
// from the lower level (upsampled by the tensor map) and the skip tensor; that of d3a (quarter
// resolution, 384 channels: the per-tap kernel) lives in nn->cat[0], built by the forward pass
// (build = true) and reused by the backward pass.
In conv_input(ur_nn *nn, int B, int l, bool build) {
    const Layer L = layer_in(nn, l);
    if (!L.in.x2) return In{L.in.x1, nullptr, 0};
    if (l != 8) return In{L.in.x2, L.in.x1, L.in.c1};
    bf16 *cat = nn->cat[0];
    if (build) {
        ++nn->launches;
        k_upcat<<<grid_for((long long)B * L.H * L.W * nn->cin[l] / 8), 256, 0, nn->stream>>>(
            L.in.x1, L.in.c1, L.in.x2, L.in.c2, B, L.H, L.W, make_div32((uint32_t)(nn->cin[l] / 8)),
            make_div32((uint32_t)L.W), make_div32((uint32_t)L.H), cat);
        ck(cudaGetLastError(), "upcat kernel");
    }
    return In{cat, nullptr, 0};
}

// Forward pass; the residual head runs in the last convolution's epilogue.  Inference writes
// out_rf / out_quad; training (t_rf, t_quad) adds the loss and the head's gradients and leaves
// the gradient at d1b's ReLU output (masked, bias sums added) in gA instead of d1b's output.
void forward(ur_nn *nn, int B, const float *rf, const float *quad, float *out_rf, float *out_quad,
             const float *t_rf = nullptr, const float *t_quad = nullptr) {
    const long long P = (long long)B * nn->H * nn->W;
    ++nn->launches;
    k_prep<<<grid_for(P), 256, 0, nn->stream>>>(rf, quad, B, nn->H, nn->W, make_div32((uint32_t)nn->W),
                                                make_div32((uint32_t)nn->H), 1.f / nn->scale, nn->x, nn->xn);
    ck(cudaGetLastError(), "prep kernel");
    ++nn->launches;
    k_pack_first<<<grid_for(32ll * nn->width), 256, 0, nn->stream>>>(nn->pbf + nn->woff[0], nn->width, nn->wfirst);
    ck(cudaGetLastError(), "pack kernel");
    for (int l = 0; l < kNumConv; ++l) {
        const Layer L = layer_in(nn, l);
        const In in = conv_input(nn, B, l, true);
        if (l == 0) {   // neighbourhood already in the 32 input channels: one tap
            conv_fwd(nn, in, B, L.H, L.W, 32, nn->cout[0], nn->wfirst, nn->params + nn->boff[0], nullptr, nn->act[0].p,
                     true, 1);
        } else if (l == kNumConv - 1) {   // d1b with the residual head (and the loss) in its epilogue
            const urnn::HeadTC h{nn->xn, nn->params + nn->hw_off, nn->params + nn->hb_off, nn->scale, out_rf, out_quad,
                                 t_rf, t_quad, 1.f / nn->scale, 1.f / (2.f * (float)P), nn->loss,
                                 nn->grads + nn->hw_off, nn->grads + nn->hb_off};
            conv_fwd(nn, in, B, L.H, L.W, nn->cin[l], nn->cout[l], nn->pbf + nn->woff[l], nn->params + nn->boff[l],
                     nullptr, t_rf ? nn->gA : nn->act[l].p, true, 9, t_rf ? nn->grads + nn->boff[l] : nullptr, nullptr,
                     0, &h);
        } else {
            conv_fwd(nn, in, B, L.H, L.W, nn->cin[l], nn->cout[l], nn->pbf + nn->woff[l], nn->params + nn->boff[l],
                     nullptr, nn->act[l].p, true);
        }
        if (l == 1 || l == 3 || l == 5) {   // pool after each encoder block
            const int q = l / 2;
            ++nn->launches;
            k_pool2<<<grid_for((long long)B * L.H * L.W * nn->cout[l] / 4), 256, 0, nn->stream>>>(
                nn->act[l].p, nn->pool[q].p, B, L.H, L.W, nn->cout[l], make_div32((uint32_t)(nn->cout[l] / 8)),
                make_div32((uint32_t)(L.W / 2)), make_div32((uint32_t)(L.H / 2)));
            ck(cudaGetLastError(), "pool kernel");
        }
    }
}

// Backward of one block (convs la, lb) given the gradient at lb's output, already
// masked by lb's ReLU with lb's bias gradient summed by the kernel that produced it;
// leaves the gradient of la's input in `din` if din; for a decoder block (dskip) the
// input's first c1 channels (upsampled lower level) go to din and the rest to dskip.
void block_bwd(ur_nn *nn, int B, int la, int lb, bf16 *d_out, bf16 *scratch, bf16 *din, bf16 *dskip = nullptr,
               int c1 = 0) {
    const Layer La = layer_in(nn, la), Lb = layer_in(nn, lb);
    conv_wgrad(nn, nn->act[la].p, d_out, B, Lb.H, Lb.W, nn->cin[lb], nn->cout[lb], nn->grads + nn->woff[lb]);
    // gradient at la's output, masked by la's ReLU in the epilogue, which also sums la's bias gradient
    conv_fwd(nn, In{d_out, nullptr, 0}, B, Lb.H, Lb.W, nn->cout[lb], nn->cin[lb], nn->wt + nn->woff[lb], nullptr,
             nn->act[la].p, scratch, false, 9, nn->grads + nn->boff[la]);
    if (la == 0) {   // first layer: single-tap gradient over the neighbourhood channels, then back to [9][C][32]
        ck(cudaMemsetAsync(nn->dwfirst, 0, sizeof(float) * 32 * nn->width, nn->stream), "memset");
        conv_wgrad(nn, nn->x, scratch, B, La.H, La.W, 32, nn->cout[0], nn->dwfirst, 1);
        ++nn->launches;
        k_unpack_first_grad<<<grid_for(18ll * nn->width), 256, 0, nn->stream>>>(nn->dwfirst, nn->width,
                                                                               nn->grads + nn->woff[0]);
    } else {
        const In in = conv_input(nn, B, la, false);
        conv_wgrad(nn, in.x, scratch, B, La.H, La.W, nn->cin[la], nn->cout[la], nn->grads + nn->woff[la], 9, in.x_low,
                   in.c1);
    }
    if (din) {
        conv_fwd(nn, In{scratch, nullptr, 0}, B, La.H, La.W, nn->cout[la], nn->cin[la], nn->wt + nn->woff[la], nullptr,
                 nullptr, din, false, 9, nullptr, dskip, c1);
    }
    ck(cudaGetLastError(), "block backward");
}

// gcat (gradient of the upsampled part of a decoder input, [B][H][W][C1]) -> gLow (masked
// by act[l_low], bias sums of layer l_low).
void unconcat(ur_nn *nn, int B, int H, int W, int C1, int l_low) {
    ++nn->launches;
    k_unconcat_low<<<channel_grid(nn, (long long)B * (H / 2) * (W / 2), C1), 256, 0, nn->stream>>>(
        nn->gcat, B, H, W, C1, make_div32((uint32_t)(W / 2)), make_div32((uint32_t)(H / 2)), nn->act[l_low].p,
        nn->gLow, nn->grads + nn->boff[l_low]);
    ck(cudaGetLastError(), "unconcat");
}

// d (gradient at layer l's output, H x W) += pooling gradient of gcat, masked by act[l], bias sums.
void pool_bwd(ur_nn *nn, int B, int H, int W, int C, int l, bf16 *d) {
    ++nn->launches;
    k_pool2_bwd_mask<<<channel_grid(nn, (long long)B * H * W, C), 256, 0, nn->stream>>>(
        d, nn->gcat, nn->act[l].p, B, H, W, C, make_div32((uint32_t)W), make_div32((uint32_t)H), nn->grads + nn->boff[l]);
    ck(cudaGetLastError(), "pooling backward");
}

void ensure_train_buffers(ur_nn *nn) {
    if (nn->gA) return;
    const size_t B = nn->max_batch, H = nn->H, W = nn->W, C = nn->width, unit = B * H * W * C;
    nn->gA = (bf16 *)nn->alloc(sizeof(bf16) * unit);
    nn->gB = (bf16 *)nn->alloc(sizeof(bf16) * unit);
    nn->gcat = (bf16 *)nn->alloc(sizeof(bf16) * 3 * unit);
    nn->gLow = (bf16 *)nn->alloc(sizeof(bf16) * unit / 2);
    for (int q = 0; q < 3; ++q) nn->gSkip[q] = (bf16 *)nn->alloc(sizeof(bf16) * (unit >> q));
}

double train(ur_nn *nn, int B, const float *rf, const float *quad, const float *t_rf, const float *t_quad) {
    ensure_train_buffers(nn);
    ck(cudaMemsetAsync(nn->loss, 0, sizeof(double), nn->stream), "memset loss");
    ck(cudaMemsetAsync(nn->grads, 0, sizeof(float) * nn->n_params, nn->stream), "memset grads");
    // forward with the loss, the head's gradients and the gradient at d1b's output (gA); every
    // block's incoming gradient below arrives masked by its ReLU with its bias gradient summed
    forward(nn, B, rf, quad, nullptr, nullptr, t_rf, t_quad);
    {   // the data gradients' weights of layers 1..13 (layer 0 has no data gradient), one launch
        WtransTable T{};
        T.n = kNumConv - 1;
        for (int j = 0; j < T.n; ++j) {
            const int l = j + 1;
            T.off[j] = (long long)nn->woff[l];
            T.cin[j] = nn->cin[l];
            T.cout[j] = nn->cout[l];
            T.start[j + 1] = T.start[j] + 9ll * nn->cin[l] * nn->cout[l];
        }
        ++nn->launches;
        k_wtrans_all<<<grid_for(T.start[T.n]), 256, 0, nn->stream>>>(nn->pbf, nn->wt, T);
        ck(cudaGetLastError(), "weight transpose");
    }
    const int C = nn->width;
    const int H = nn->H, W = nn->W;
    // decoder level 1: input concat(up(d2), e1)
    block_bwd(nn, B, 12, 13, nn->gA, nn->gB, nn->gcat, nn->gSkip[0], 2 * C);
    unconcat(nn, B, H, W, 2 * C, 11);
    // decoder level 2: the gradient of d2 (half resolution) is gLow
    block_bwd(nn, B, 10, 11, nn->gLow, nn->gB, nn->gcat, nn->gSkip[1], 4 * C);
    unconcat(nn, B, H / 2, W / 2, 4 * C, 9);
    block_bwd(nn, B, 8, 9, nn->gLow, nn->gB, nn->gcat, nn->gSkip[2], 8 * C);
    unconcat(nn, B, H / 4, W / 4, 8 * C, 7);
    // bottleneck: the gradient of e4 is gLow; encoder blocks leave d(pooled input) in gcat
    block_bwd(nn, B, 6, 7, nn->gLow, nn->gB, nn->gcat);
    pool_bwd(nn, B, H / 4, W / 4, 4 * C, 5, nn->gSkip[2]);
    block_bwd(nn, B, 4, 5, nn->gSkip[2], nn->gB, nn->gcat);
    pool_bwd(nn, B, H / 2, W / 2, 2 * C, 3, nn->gSkip[1]);
    block_bwd(nn, B, 2, 3, nn->gSkip[1], nn->gB, nn->gcat);
    pool_bwd(nn, B, H, W, C, 1, nn->gSkip[0]);
    block_bwd(nn, B, 0, 1, nn->gSkip[0], nn->gB, nullptr);
    ck(cudaGetLastError(), "backward");
    double loss = 0.0;
    ck(cudaMemcpyAsync(&loss, nn->loss, sizeof(double), cudaMemcpyDeviceToHost, nn->stream), "read loss");
    sync_check(nn, "train step");
    return loss;
}

// deterministic standard normals for the initial weights (splitmix64 + Box-Muller)
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uni() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return std::sqrt(-2.0 * std::log(uni())) * std::cos(6.283185307179586 * uni()); }
};

}  // namespace

extern "C" {

ur_status ur_nn_create(ur_nn **out, int device, void *cuda_stream, int max_batch, int n_el, int n_s, int width,
                       uint64_t seed) {
    if (!out) return UR_ERR_INVALID_ARG;
    *out = nullptr;
    ur_nn *nn = new (std::nothrow) ur_nn();
    if (!nn) return UR_ERR_OOM;
    ur_status st = nn_guard(nn, [&] {
        if (max_batch < 1 || max_batch > 64 || n_el < 8 || n_s < 8 || n_el % 8 || n_s % 8 || width != 32)
            fail(UR_ERR_INVALID_ARG, "need 1 <= batch <= 64, n_el and n_s multiples of 8, width 32");
        // the elementwise kernels index 16-byte granules of the largest activation (3 width
        // channels at full resolution) and pixels with 32-bit integers
        if ((uint64_t)max_batch * (uint64_t)n_el * (uint64_t)n_s * 3ull * (uint64_t)width / 8ull >= (1ull << 32))
            fail(UR_ERR_INVALID_ARG, "batch x n_el x n_s too large for the network's 32-bit indexing");
        int n = 0;
        ck(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
        if (device < 0 || device >= n) fail(UR_ERR_INVALID_ARG, "bad device index");
        nn->device = device;
        ck(cudaSetDevice(device), "cudaSetDevice");
        ck(cudaDeviceGetAttribute(&nn->sms, cudaDevAttrMultiProcessorCount, device), "SM count");
        if (cuda_stream) {
            nn->stream = (cudaStream_t)cuda_stream;
        } else {
            ck(cudaStreamCreateWithFlags(&nn->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            nn->own_stream = true;
        }
        nn->max_batch = max_batch;
        nn->H = n_el;
        nn->W = n_s;
        nn->width = width;
        const int C = width;
        const int ci[kNumConv] = {32, C, C, 2 * C, 2 * C, 4 * C, 4 * C, 8 * C, 12 * C, 4 * C, 6 * C, 2 * C, 3 * C, C};
        const int co[kNumConv] = {C, C, 2 * C, 2 * C, 4 * C, 4 * C, 8 * C, 8 * C, 4 * C, 4 * C, 2 * C, 2 * C, C, C};
        size_t off = 0;
        for (int l = 0; l < kNumConv; ++l) {
            nn->cin[l] = ci[l];
            nn->cout[l] = co[l];
            nn->woff[l] = off;
            off += 9ull * ci[l] * co[l];
            nn->boff[l] = off;
            off += co[l];
            off = (off + 7) / 8 * 8;   // keep every weight tensor 16-byte aligned in bf16
        }
        nn->hw_off = off;
        off += 2ull * C;
        nn->hb_off = off;
        off += 2;
        nn->n_params = (off + 7) / 8 * 8;
        // He-normal initialisation on the true fan-in (the first conv sees 2 real channels)
        std::vector<float> h(nn->n_params, 0.f);
        Rng rng{seed * 0x2545F4914F6CDD1Dull + 1};
        for (int l = 0; l < kNumConv; ++l) {
            const int real_ci = l == 0 ? 2 : ci[l];
            const double sd = std::sqrt(2.0 / (9.0 * real_ci));
            for (int t = 0; t < 9; ++t)
                for (int o = 0; o < co[l]; ++o)
                    for (int i = 0; i < real_ci; ++i) h[nn->woff[l] + ((size_t)t * co[l] + o) * ci[l] + i] = (float)(sd * rng.normal());
        }
        for (int i = 0; i < 2 * C; ++i) h[nn->hw_off + i] = (float)(std::sqrt(2.0 / C) * 0.1 * rng.normal());
        nn->params = (float *)nn->alloc(sizeof(float) * nn->n_params);
        nn->grads = (float *)nn->alloc(sizeof(float) * nn->n_params);
        nn->m = (float *)nn->alloc(sizeof(float) * nn->n_params);
        nn->v = (float *)nn->alloc(sizeof(float) * nn->n_params);
        nn->pbf = (bf16 *)nn->alloc(sizeof(bf16) * nn->n_params);
        nn->wt = (bf16 *)nn->alloc(sizeof(bf16) * nn->n_params);   // data-gradient weights at the same offsets
        ck(cudaMemcpy(nn->params, h.data(), sizeof(float) * nn->n_params, cudaMemcpyHostToDevice), "copy params");
        ck(cudaMemset(nn->m, 0, sizeof(float) * nn->n_params), "memset");
        ck(cudaMemset(nn->v, 0, sizeof(float) * nn->n_params), "memset");
        ++nn->launches;
        k_to_bf16<<<grid_for((long long)nn->n_params), 256, 0, nn->stream>>>(nn->params, nn->pbf, (long long)nn->n_params);
        ck(cudaGetLastError(), "to bf16");
        // activations
        const size_t B = max_batch, H = n_el, W = n_s;
        const int lh[kNumConv] = {1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1};
        for (int l = 0; l < kNumConv; ++l) {
            nn->act[l] = Tensor{(bf16 *)nn->alloc(sizeof(bf16) * B * (H / lh[l]) * (W / lh[l]) * co[l]), (int)(H / lh[l]),
                                (int)(W / lh[l]), co[l]};
        }
        for (int q = 0; q < 3; ++q) {
            const int f = 2 << q, c = C << q;
            nn->pool[q] = Tensor{(bf16 *)nn->alloc(sizeof(bf16) * B * (H / f) * (W / f) * c), (int)(H / f), (int)(W / f), c};
        }
        nn->x = (bf16 *)nn->alloc(sizeof(bf16) * B * H * W * 32);
        nn->xn = (float *)nn->alloc(sizeof(float) * B * H * W * 2);
        nn->cat[0] = (bf16 *)nn->alloc(sizeof(bf16) * B * (H >> 2) * (W >> 2) * 12 * C);   // d3a: [H/4][W/4][12C]
        nn->wfirst = (bf16 *)nn->alloc(sizeof(bf16) * 32 * C);
        nn->dwfirst = (float *)nn->alloc(sizeof(float) * 32 * C);
        nn->loss = (double *)nn->alloc(sizeof(double));
        nn->d_err = (int *)nn->alloc(sizeof(int));
        ck(cudaMemset(nn->d_err, 0, sizeof(int)), "memset status");
        ck(cudaMallocHost(&nn->h_err, sizeof(int)), "cudaMallocHost");
        *nn->h_err = 0;
        ck(cudaStreamSynchronize(nn->stream), "init");
    });
    if (st != UR_OK) {
        for (void *p : nn->allocs) cudaFree(p);
        if (nn->h_err) cudaFreeHost(nn->h_err);
        if (nn->own_stream) cudaStreamDestroy(nn->stream);
        delete nn;
        return st;
    }
    *out = nn;
    return UR_OK;
}

ur_status ur_nn_destroy(ur_nn *nn) {
    if (!nn) return UR_ERR_INVALID_ARG;
    cudaSetDevice(nn->device);
    cudaStreamSynchronize(nn->stream);
    for (void *p : nn->allocs) cudaFree(p);
    if (nn->h_err) cudaFreeHost(nn->h_err);
    if (nn->own_stream) cudaStreamDestroy(nn->stream);
    delete nn;
    return UR_OK;
}

const char *ur_nn_last_error(const ur_nn *nn) { return nn ? nn->err.c_str() : "null network"; }

ur_status ur_nn_param_count(const ur_nn *nn, uint64_t *n) {
    if (!nn || !n) return UR_ERR_INVALID_ARG;
    *n = nn->n_params;
    return UR_OK;
}

ur_status ur_nn_launch_count(const ur_nn *nn, uint64_t *n) {
    if (!nn || !n) return UR_ERR_INVALID_ARG;
    *n = nn->launches;
    return UR_OK;
}

ur_status ur_nn_params(ur_nn *nn, float *get, const float *set) {
    return nn_guard(nn, [&] {
        ck(cudaSetDevice(nn->device), "cudaSetDevice");
        ck(cudaStreamSynchronize(nn->stream), "pending work");
        if (get) ck(cudaMemcpy(get, nn->params, sizeof(float) * nn->n_params, cudaMemcpyDefault), "get params");
        if (set) {
            ck(cudaMemcpy(nn->params, set, sizeof(float) * nn->n_params, cudaMemcpyDefault), "set params");
            ++nn->launches;
            k_to_bf16<<<grid_for((long long)nn->n_params), 256, 0, nn->stream>>>(nn->params, nn->pbf, (long long)nn->n_params);
            ck(cudaGetLastError(), "to bf16");
            ck(cudaMemsetAsync(nn->m, 0, sizeof(float) * nn->n_params, nn->stream), "reset m");
            ck(cudaMemsetAsync(nn->v, 0, sizeof(float) * nn->n_params, nn->stream), "reset v");
            nn->step = 0;
            ck(cudaStreamSynchronize(nn->stream), "set params");
        }
    });
}

ur_status ur_nn_set_scale(ur_nn *nn, float scale) {
    return nn_guard(nn, [&] {
        if (!(scale > 0.f) || !std::isfinite(scale)) fail(UR_ERR_INVALID_ARG, "scale must be positive");
        nn->scale = scale;
    });
}

ur_status ur_nn_forward(ur_nn *nn, const float *rf, const float *quad, int batch, float *out_rf, float *out_quad) {
    return nn_guard(nn, [&] {
        ck(cudaSetDevice(nn->device), "cudaSetDevice");
        if (batch < 1 || batch > nn->max_batch) fail(UR_ERR_INVALID_ARG, "batch out of range");
        if (!rf || !quad || !out_rf || !out_quad) fail(UR_ERR_INVALID_ARG, "inputs and outputs are required");
        const size_t n = (size_t)batch * nn->H * nn->W;
        float *o_rf = staged(nn, 4, out_rf, batch, false), *o_q = staged(nn, 5, out_quad, batch, false);
        forward(nn, batch, staged(nn, 0, rf, batch, true), staged(nn, 1, quad, batch, true), o_rf, o_q);
        if (o_rf != out_rf) ck(cudaMemcpyAsync(out_rf, o_rf, sizeof(float) * n, cudaMemcpyDeviceToHost, nn->stream), "copy out");
        if (o_q != out_quad) ck(cudaMemcpyAsync(out_quad, o_q, sizeof(float) * n, cudaMemcpyDeviceToHost, nn->stream), "copy out");
        sync_check(nn, "forward");
    });
}

ur_status ur_nn_train_step(ur_nn *nn, const float *rf, const float *quad, const float *t_rf, const float *t_quad,
                           int batch, float lr, float *loss, float *grad_out) {
    return nn_guard(nn, [&] {
        ck(cudaSetDevice(nn->device), "cudaSetDevice");
        if (batch < 1 || batch > nn->max_batch) fail(UR_ERR_INVALID_ARG, "batch out of range");
        if (!rf || !quad || !t_rf || !t_quad) fail(UR_ERR_INVALID_ARG, "inputs and targets are required");
        if (!(lr >= 0.f)) fail(UR_ERR_INVALID_ARG, "lr must be >= 0");
        const double l = train(nn, batch, staged(nn, 0, rf, batch, true), staged(nn, 1, quad, batch, true),
                               staged(nn, 2, t_rf, batch, true), staged(nn, 3, t_quad, batch, true));
        if (loss) *loss = (float)l;
        if (grad_out) ck(cudaMemcpy(grad_out, nn->grads, sizeof(float) * nn->n_params, cudaMemcpyDefault), "grad out");
        if (lr > 0.f) {
            nn->step += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - std::pow(b1, (float)nn->step), c2 = 1.f - std::pow(b2, (float)nn->step);
            ++nn->launches;
            k_adam<<<grid_for((long long)nn->n_params), 256, 0, nn->stream>>>(nn->params, nn->grads, nn->m, nn->v, nn->pbf,
                                                                            (long long)nn->n_params, lr, b1, b2, 1e-8f, c1, c2);
            ck(cudaGetLastError(), "adam kernel");
        }
    });
}

}  // extern "C"
