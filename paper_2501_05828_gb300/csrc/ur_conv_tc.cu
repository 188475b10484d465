// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores.
//
// A tile is 128 consecutive pixels of one image row (the M dimension, one TMEM
// lane per pixel) by BN output channels (N); persistent CTAs stride over tiles.  The K loop
// walks the 9 taps and, within each, the input channels in chunks of BK (64:
// 128-byte rows, or 32: 64-byte rows).  For every K step one thread issues two
// TMA loads into a ring of shared-memory stages:
//   A: the 128 x BK box of the NHWC input at (x0 + kx - 1, y + ky - 1), so the
//      zero padding of the convolution is TMA's out-of-bounds fill,
//   B: the BN x BK box of the weights [9][Cout][Cin] at this tap,
// both written in the canonical K-major swizzled layout the tensor core reads.
// A second thread issues tcgen05.mma (M = 128, N = BN, K = 16, BF16 inputs,
// FP32 accumulator in TMEM, two accumulators in turn) and releases each stage
// with tcgen05.commit.  Four epilogue warps read a finished accumulator with
// tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) .. +31) and apply bias, ReLU and
// an optional ReLU mask (for data gradients) before storing BF16, while the
// next tile's MMAs run.
//
// Below it: k_conv_kx, the 3x3 form for C_out <= 96 with the three kx taps read
// from one staged input row (and row-stacked tiles), and k_wgrad_tc, the weight
// gradient.
//
// Every mbarrier wait is bounded by the global timer; a wait that gives up
// records an error code for the host and the block still frees its TMEM.
#include "ur_conv_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

namespace urnn {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kBM = 128;         // pixels per tile = TMEM lanes
constexpr int kThreads = 128;    // 4 warps: TMA producer (warp 0), MMA issuer (warp 1), all four in the epilogue
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s: far above any tile's run time

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of the given parity to complete; false once the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline) {
    while (!mbar_test(bar, parity))
        if (now_ns() > deadline) return false;
    return true;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// Row of a half-resolution tensor that nearest upsampling maps to full-resolution row yy (>= -1).
__device__ __forceinline__ int low_row(int yy) { return yy >= 0 ? yy >> 1 : -1; }

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 with BF16 operands and FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives on the mbarrier once every MMA this thread issued so far has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory descriptor of a K-major operand in the canonical swizzled layout:
// rows of `row_bytes` (128: 128-byte swizzle, 64: 64-byte swizzle), 8-row groups
// 8 * row_bytes apart (stride byte offset); the leading byte offset is unused for
// swizzled K-major operands; descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t row_bytes) {
    const uint64_t layout = row_bytes == 128 ? 2ull : 4ull;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)((8u * row_bytes) >> 4) << 32) | (1ull << 46) |
           (layout << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

constexpr int kConvThreads = 192;   // warp 0 TMA producer, warp 1 MMA issuer, warps 2-5 epilogue

template <int BN, int BK>
struct Cfg {
    static constexpr int ROW = BK * 2;                    // bytes per operand row
    static constexpr int A_BYTES = kBM * ROW;
    static constexpr int B_BYTES = BN * ROW;
    static constexpr int A_PAD = (A_BYTES + 1023) / 1024 * 1024;
    static constexpr int B_PAD = (B_BYTES + 1023) / 1024 * 1024;
    static constexpr int BUDGET = BN >= 192 ? 200 * 1024 : 100 * 1024;   // one CTA per SM from 192 columns on
    static constexpr int S_RAW = BUDGET / (A_PAD + B_PAD);
    static constexpr int S = S_RAW < 2 ? 2 : (S_RAW > 6 ? 6 : S_RAW);
    static constexpr int ACC_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;   // one accumulator
    static constexpr int TMEM_COLS = 2 * ACC_COLS;                                            // double-buffered
    static constexpr int N_BARS = 2 * S + 4;   // full[S], empty[S], acc_full[2], acc_empty[2]
    static constexpr int SMEM = S * (A_PAD + B_PAD) + 1024 + 8 * N_BARS + 16;
};

struct Args {
    int N, H, W, C, Cout, nxb, relu, taps, n_tiles, n_ntiles;
    int stages, wres;   // kx-fused kernel: input stages per CTA, weights resident in shared memory
    int rows, nyb;      // kx-fused kernel: output rows per tile (several only with resident weights), row blocks
    const float *bias;
    const bf16 *mask;
    bf16 *y;
    float *dbias;   // nullable: += column sums of the output over all pixels
    bf16 *y2;       // nullable: output columns [c_split, Cout) go to y2 (and [0, c_split) to y)
    int c_split;
    int *err;
    int has_head;   // kx-fused kernel with BN = 32: the residual head in the epilogue
    HeadTC head;
    int c1;         // kx-fused kernel: input channels [0, c1) from the upsampled half-resolution map
};

// Sum over the 32 lanes of each of the 32 values v[j]; lane l ends with the total of
// v[l] (recursive halving: 31 shuffles).
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int j = 0; j < w; ++j) {
            // keep the half of the values whose index bit w matches this lane's bit w
            const float send = upper ? v[j] : v[j + w];
            const float keep = upper ? v[j + w] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, w);
        }
    }
    return v[0];
}

// Destination of output columns co .. co + 31 of pixel pix: y, or, when the output is split,
// y [pix][c_split] for the first c_split columns and y2 [pix][Cout - c_split] for the rest.
__device__ __forceinline__ bf16 *out_cols(const Args &a, size_t pix, int co) {
    if (!a.y2) return a.y + pix * a.Cout + co;
    return co < a.c_split ? a.y + pix * a.c_split + co : a.y2 + pix * (a.Cout - a.c_split) + (co - a.c_split);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ...; tile t = (M tile, N tile) with the N
// tile fastest, M tile = (image n, row y, 128-pixel block).  The producer runs ahead across
// tiles; the accumulator is double-buffered in TMEM so the epilogue of one tile overlaps the
// MMAs of the next.
template <int BN, int BK>
__global__ void __launch_bounds__(kConvThreads, 1)
    k_conv_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw, const Args a) {
    using K = Cfg<BN, BK>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = s_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;          // swizzled operands want 1024-byte alignment
    uint8_t *sm = smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + K::S * K::A_PAD;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + K::S * (K::A_PAD + K::B_PAD));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + K::N_BARS);
    const uint32_t full0 = s_addr(bars), empty0 = s_addr(bars + K::S);
    const uint32_t accf0 = s_addr(bars + 2 * K::S), acce0 = s_addr(bars + 2 * K::S + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kc = a.C / BK, nk = a.taps * kc;
    const uint64_t deadline = now_ns() + kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K::S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);   // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(s_addr(tslot), K::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    bool ok = true;

    auto decode = [&](int t, int &n, int &y, int &x0, int &co0) {
        const int nt = t % a.n_ntiles;
        int m = t / a.n_ntiles;
        const int xb = m % a.nxb;
        m /= a.nxb;
        y = m % a.H;
        n = m / a.H;
        x0 = xb * kBM;
        co0 = nt * BN;
    };

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            int it = 0;
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x) {
                int n, y, x0, co0;
                decode(t, n, y, x0, co0);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % K::S;
                    if (!mbar_wait(empty0 + 8 * s, ((uint32_t)(it / K::S) & 1u) ^ 1u, deadline)) {
                        ok = false;
                        break;
                    }
                    const int tap = kt / kc, c0 = (kt - tap * kc) * BK;
                    const int ky = a.taps == 1 ? 1 : tap / 3, kx = a.taps == 1 ? 1 : tap - 3 * (tap / 3);
                    mbar_expect_tx(full0 + 8 * s, (uint32_t)(K::A_BYTES + K::B_BYTES));
                    tma_load_4d(sA + s * K::A_PAD, &tmx, c0, x0 + kx - 1, y + ky - 1, n, full0 + 8 * s);
                    tma_load_3d(sB + s * K::B_PAD, &tmw, c0, co0, tap, full0 + 8 * s);
                }
            }
            if (!ok)   // let the copies already in flight land before the block can exit
                for (int j = it > K::S ? it - K::S : 0; j < it; ++j)
                    mbar_wait(full0 + 8 * (j % K::S), (uint32_t)(j / K::S) & 1u, deadline + kWaitNs / 20);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = idesc_bf16<BN>();
            int it = 0, i = 0;
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x, ++i) {
                const int b = i & 1;
                if (!mbar_wait(acce0 + 8 * b, ((uint32_t)(i >> 1) & 1u) ^ 1u, deadline)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * K::ACC_COLS);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % K::S;
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)(it / K::S) & 1u, deadline)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = sA + s * K::A_PAD, b0 = sB + s * K::B_PAD;
#pragma unroll
                    for (int k = 0; k < BK / 16; ++k)
                        mma_bf16(d, sdesc(a0 + 32 * k, K::ROW), sdesc(b0 + 32 * k, K::ROW), idesc, (kt | k) != 0);
                    mma_commit(empty0 + 8 * s);
                }
                mma_commit(accf0 + 8 * b);   // accumulator b complete (or abandoned: the status word says so)
            }
        }
        __syncwarp();
    } else {   // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
        const int q = warp & 3;
        float dsum[BN / 32];   // lane l: running column sum of channel c + l of this CTA's N tile
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) dsum[c] = 0.f;
        int dsum_co0 = -1;
        int i = 0;
        for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ready = mbar_wait(accf0 + 8 * b, (uint32_t)(i >> 1) & 1u, deadline);
            if (__all_sync(0xffffffffu, ready) == 0) {
                ok = false;
                break;
            }
            tc_fence_after();
            int n, y, x0, co0;
            decode(t, n, y, x0, co0);
            if (a.dbias && co0 != dsum_co0) {   // N tile changed: flush the running column sums
                if (dsum_co0 >= 0)
#pragma unroll
                    for (int c = 0; c < BN / 32; ++c) atomicAdd(a.dbias + dsum_co0 + 32 * c + lane, dsum[c]);
#pragma unroll
                for (int c = 0; c < BN / 32; ++c) dsum[c] = 0.f;
                dsum_co0 = co0;
            }
            const int x = x0 + q * 32 + lane;
            const size_t pix = ((size_t)n * a.H + y) * a.W + x;
#pragma unroll
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(b * K::ACC_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)c, r);
                const bool in = x < a.W;
                const int co = co0 + c;
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = in ? __uint_as_float(r[j]) : 0.f;
                if (in) {
                    if (a.bias) {
                        const float4 *b4 = reinterpret_cast<const float4 *>(a.bias + co);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 bb = b4[j];
                            v[4 * j] += bb.x;
                            v[4 * j + 1] += bb.y;
                            v[4 * j + 2] += bb.z;
                            v[4 * j + 3] += bb.w;
                        }
                    }
                    if (a.relu) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                    }
                    if (a.mask) {
                        const uint4 *m4 = reinterpret_cast<const uint4 *>(a.mask + pix * a.Cout + co);
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const uint4 mv = m4[g];
                            const __nv_bfloat162 *mb = reinterpret_cast<const __nv_bfloat162 *>(&mv);
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const float2 f = __bfloat1622float2(mb[h]);
                                if (!(f.x > 0.f)) v[8 * g + 2 * h] = 0.f;
                                if (!(f.y > 0.f)) v[8 * g + 2 * h + 1] = 0.f;
                            }
                        }
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(out_cols(a, pix, co));
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        uint4 o;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * g], v[8 * g + 1]);
                        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * g + 2], v[8 * g + 3]);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * g + 4], v[8 * g + 5]);
                        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * g + 6], v[8 * g + 7]);
                        o.x = *reinterpret_cast<uint32_t *>(&h0);
                        o.y = *reinterpret_cast<uint32_t *>(&h1);
                        o.z = *reinterpret_cast<uint32_t *>(&h2);
                        o.w = *reinterpret_cast<uint32_t *>(&h3);
                        dst[g] = o;
                    }
                }
                if (a.dbias) dsum[c / 32] += warp_transpose_sum(v, lane);   // column sums over the warp's pixels
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);   // accumulator b may be overwritten
        }
        if (a.dbias && dsum_co0 >= 0)
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) atomicAdd(a.dbias + dsum_co0 + 32 * c + lane, dsum[c]);
    }
    if (!ok) atomicExch(a.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, K::TMEM_COLS);
    }
}

// ------------------------------------------------------------------ kx-fused convolution
//
// For C_out = BN in {32, 64, 96}: a stage holds the input pixels x0 - 1 .. x0 + 128 of row
// y + ky - 1 (130 rows of BK channels) and the weights of the three kx taps of kernel row ky
// (consecutive rows 3 ky C_out .. of the weight view [9 C_out][C_in]).  Tap kx reads the
// A operand from row kx of the staged tile: the tensor core applies the swizzle from the
// shared-memory address bits, so a descriptor that starts one or two 128- (or 64-) byte rows
// into a tile written by TMA still reads the rows TMA wrote there.  The three taps accumulate
// into one accumulator of 128 output pixels, and the input is read once per kernel row instead
// of once per tap; the epilogue is the plain one (bias, ReLU, mask, BF16 store).
//
// Row-stacked tiles (BN in {32, 64} when the weights fit): a tile is R = 128 / BN output rows
// y .. y + R - 1, their accumulators side by side in TMEM.  Input row y - 1 + r (r = 0 .. R + 1)
// contributes to the output rows y + o, o = max(0, r - 2) .. min(R - 1, r), with kernel rows
// ky = r - o, so one MMA adds it to all of them if its B operand is the run W(ky = r - o_lo),
// W(ky - 1), ... of BN-row weight blocks (N = BN x the rows it touches, D at column o_lo BN).  The
// resident weights of a channel chunk hold, per kx, the blocks W(2), W(1), W(0) in that order, so
// every such run is contiguous.  The first K slice of an input row that starts a new output row
// (o = r) is issued as two MMAs: the rows already under way accumulate, the new one is
// initialised.  An input row is staged (R + 2) / R times per output row instead of 3, and each
// staged row costs 3 BK / 16 MMAs of up to 3 BN columns instead of up to 3 x 3 BK / 16 of BN
// columns (the tensor core re-reads the A operand for every MMA).
constexpr int kKxRows = kBM + 2;   // staged input pixels per kernel row

// Weights: when all 3 kc blocks of one C_out tile fit beside a few input stages they are
// loaded once per CTA and stay in shared memory (every CTA reads the same few KB, which
// otherwise come from a handful of L2 slices at every stage); otherwise each stage carries its
// kernel row's block.  The stage count and this choice are set per launch.
constexpr int kKxMaxStages = 8;

template <int BN, int BK>
struct KxCfg {
    static constexpr int ROW = BK * 2;
    static constexpr int NB = 3 * BN;                      // weight rows per block: the three kx taps
    static constexpr int A_BYTES = kKxRows * ROW;
    static constexpr int B_BYTES = NB * ROW;
    static constexpr int A_PAD = (A_BYTES + 2 * ROW + 1023) / 1024 * 1024;   // room for 132 upsampled rows
    static constexpr int B_PAD = (B_BYTES + 1023) / 1024 * 1024;
    static constexpr int MAX_ROWS = 128 / BN;              // output rows per tile: R BN <= 128 columns
    static constexpr int TMEM_COLS = 256;                  // two accumulator sets of 128 columns
    static constexpr int ACC_COLS = 128;
    static constexpr int N_BARS = 2 * kKxMaxStages + 5;    // full, empty, acc_full[2], acc_empty[2], weights
    static constexpr int TAIL = 8 * N_BARS + 16;           // barriers and the TMEM address slot
    static constexpr int BLK = BN * ROW;                    // one BN-row weight block
    // row-stacked weights of one channel chunk: per kx the blocks W(2), W(1), W(0)
    static constexpr int STK_BYTES = (9 * BLK + 1023) / 1024 * 1024;
    // shared memory of a launch: alignment slack, resident weights, stages, tail
    static int smem(int kc, bool wres, int stages) {
        return 1024 + (wres ? 3 * kc * B_PAD : 0) + stages * (A_PAD + (wres ? 0 : B_PAD)) + TAIL;
    }
};

template <int BN, int BK>
__global__ void __launch_bounds__(kConvThreads, 2)
    k_conv_kx(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
              const __grid_constant__ CUtensorMap tml, const Args a) {
    using K = KxCfg<BN, BK>;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = s_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (base - raw);
    const int kc = a.C / BK, nk = 3 * kc;   // weight blocks of the layer: kernel rows x channel chunks
    const bool wres = a.wres != 0;
    const int S = a.stages;
    const int R = a.rows;   // R > 1: row-stacked tile (resident stacked weights)
    const uint32_t wb_stk = R > 1 ? (uint32_t)K::STK_BYTES : 0u;   // stacked weights per channel chunk
    const uint32_t w_bytes = R > 1 ? (uint32_t)kc * wb_stk : wres ? (uint32_t)(3 * kc * K::B_PAD) : 0u;
    const uint32_t stage = (uint32_t)(K::A_PAD + (wres ? 0 : K::B_PAD));
    const uint32_t sW = base, sS = base + w_bytes;   // resident weights; stage s: A at sS + s stage, then B
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + w_bytes + (uint32_t)S * stage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + K::N_BARS);
    const uint32_t full0 = s_addr(bars), empty0 = s_addr(bars + kKxMaxStages);
    const uint32_t accf0 = s_addr(bars + 2 * kKxMaxStages), acce0 = s_addr(bars + 2 * kKxMaxStages + 2);
    const uint32_t wfull = s_addr(bars + 2 * kKxMaxStages + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t deadline = now_ns() + kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, 4);
        }
        mbar_init(wfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(s_addr(tslot), K::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    bool ok = true;

    auto decode = [&](int t, int &n, int &y, int &x0) {   // y: the tile's first output row
        const int xb = t % a.nxb;
        const int m = t / a.nxb;
        y = (m % a.nyb) * R;
        n = m / a.nyb;
        x0 = xb * kBM;
    };

    if (warp == 0) {
        if (lane == 0) {   // TMA producer
            if (R > 1) {   // stacked: W(ky) of (chunk, kx) at block 3 kx + 2 - ky of the chunk
                mbar_expect_tx(wfull, (uint32_t)(kc * 9 * K::BLK));
                for (int cc = 0; cc < kc; ++cc)
                    for (int kx = 0; kx < 3; ++kx)
                        for (int ky = 0; ky < 3; ++ky)
                            tma_load_2d(sW + (uint32_t)cc * wb_stk + (uint32_t)((3 * kx + 2 - ky) * K::BLK),
                                        &tmw, cc * BK, (3 * ky + kx) * BN, wfull);
            } else if (wres) {   // every weight block once: block kt = (ky, channel chunk) at sW + kt B_PAD
                mbar_expect_tx(wfull, (uint32_t)(nk * K::B_BYTES));
                for (int kt = 0; kt < nk; ++kt) {
                    const int ky = kt / kc, c0 = (kt - ky * kc) * BK;
                    for (int kx = 0; kx < 3; ++kx)   // boxes of BN rows (a box is at most 256 rows)
                        tma_load_2d(sW + (uint32_t)(kt * K::B_PAD + kx * BN * K::ROW), &tmw, c0, (3 * ky + kx) * BN, wfull);
                }
            }
            int it = 0, s = 0;
            uint32_t ph = 0;
            const int nr = (R + 2) * kc;   // stages per tile: input rows x channel chunks
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x) {
                int n, y, x0;
                decode(t, n, y, x0);
                for (int kt = 0; kt < nr; ++kt, ++it) {
                    if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, deadline)) {
                        ok = false;
                        break;
                    }
                    const int ky = kt / kc, c0 = (kt - ky * kc) * BK;   // ky: input row y - 1 + ky (= kernel row if R = 1)
                    const uint32_t sa = sS + (uint32_t)s * stage;
                    const bool low = c0 < a.c1;   // upsampled chunk: 132 pixels from x0 - 2, each low pixel twice
                    mbar_expect_tx(full0 + 8 * s, (uint32_t)((low ? K::A_BYTES + 2 * K::ROW : K::A_BYTES) +
                                                             (wres ? 0 : K::B_BYTES)));
                    if (low)
                        tma_load_5d(sa, &tml, c0, 0, x0 / 2 - 1, low_row(y + ky - 1), n, full0 + 8 * s);
                    else
                        tma_load_4d(sa, &tmx, c0 - a.c1, x0 - 1, y + ky - 1, n, full0 + 8 * s);
                    if (!wres)
                        for (int kx = 0; kx < 3; ++kx)
                            tma_load_2d(sa + K::A_PAD + (uint32_t)(kx * BN * K::ROW), &tmw, c0, (3 * ky + kx) * BN,
                                        full0 + 8 * s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
            }
            // let the copies already in flight land before the block can exit
            if (wres) mbar_wait(wfull, 0u, deadline + kWaitNs / 20);
            if (!ok)
                for (int j = it > S ? it - S : 0; j < it; ++j)
                    mbar_wait(full0 + 8 * (j % S), (uint32_t)(j / S) & 1u, deadline + kWaitNs / 20);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = idesc_bf16<BN>();
            // row-stacked: N = BN x rows columns (kind::f16, FP32 accumulator, BF16 operands, M = 128)
            auto idesc_rows = [](int rows) {
                return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((rows * BN) >> 3) << 17) |
                       ((uint32_t)(kBM >> 4) << 24);
            };
            if (wres && !mbar_wait(wfull, 0u, deadline)) ok = false;
            int i = 0, s = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < a.n_tiles && ok; t += gridDim.x, ++i) {
                const int b = i & 1;
                if (!mbar_wait(acce0 + 8 * b, ((uint32_t)(i >> 1) & 1u) ^ 1u, deadline)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * K::ACC_COLS);
                const int nr = (R + 2) * kc;
                for (int kt = 0; kt < nr; ++kt) {
                    if (!mbar_wait(full0 + 8 * s, ph, deadline)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int r = kt / kc, kcc = kt - r * kc;   // staged input row y - 1 + r, channel chunk kcc
                    // stage row i is pixel x0 - 1 + i, or x0 - 2 + i for an upsampled chunk
                    const uint32_t st0 = sS + (uint32_t)s * stage;
                    const uint32_t a0 = st0 + (kcc * BK < a.c1 ? (uint32_t)K::ROW : 0u);
                    if (R > 1) {   // one MMA per tap column and K slice: every output row this input row touches
                        const uint32_t wc = sW + (uint32_t)kcc * wb_stk;
                        const int o_lo = r > 2 ? r - 2 : 0, o_hi = r < R - 1 ? r : R - 1, nr_o = o_hi - o_lo + 1;
                        const uint32_t dst = d + (uint32_t)(o_lo * BN);
                        const bool opens = kcc == 0 && o_hi == r;   // output row y + r starts here
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx) {
                            const uint32_t b0 = wc + (uint32_t)((3 * kx + 2 - (r - o_lo)) * K::BLK);   // W(ky = r - o_lo)
#pragma unroll
                            for (int k = 0; k < BK / 16; ++k) {
                                const uint64_t ad = sdesc(a0 + (uint32_t)(kx * K::ROW) + 32 * k, K::ROW);
                                if (opens && kx == 0 && k == 0) {   // older rows accumulate, row r is initialised
                                    if (nr_o > 1)
                                        mma_bf16(dst, ad, sdesc(b0, K::ROW), idesc_rows(nr_o - 1), 1u);
                                    mma_bf16(d + (uint32_t)(r * BN), ad, sdesc(wc + (uint32_t)(2 * K::BLK), K::ROW),
                                             idesc_rows(1), 0u);
                                } else {
                                    mma_bf16(dst, ad, sdesc(b0 + 32 * k, K::ROW), idesc_rows(nr_o), 1u);
                                }
                            }
                        }
                    } else {
                        const uint32_t b0 = wres ? sW + (uint32_t)((r * kc + kcc) * K::B_PAD) : st0 + K::A_PAD;
#pragma unroll
                        for (int kx = 0; kx < 3; ++kx)   // output pixel x0 + i reads input row i + kx of the stage
#pragma unroll
                            for (int k = 0; k < BK / 16; ++k)
                                mma_bf16(d, sdesc(a0 + (uint32_t)(kx * K::ROW) + 32 * k, K::ROW),
                                         sdesc(b0 + (uint32_t)(kx * BN * K::ROW) + 32 * k, K::ROW), idesc,
                                         (kt | kx | k) != 0);
                    }
                    mma_commit(empty0 + 8 * s);
                    if (++s == S) {
                        s = 0;
                        ph ^= 1u;
                    }
                }
                mma_commit(accf0 + 8 * b);
            }
        }
        __syncwarp();
    } else {   // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31
        const int q = warp & 3;
        float dsum[BN / 32];
#pragma unroll
        for (int c = 0; c < BN / 32; ++c) dsum[c] = 0.f;
        float hloss = 0.f, hb0 = 0.f, hb1 = 0.f, hw0 = 0.f, hw1 = 0.f;   // residual head (training)
        int i = 0;
        constexpr int HR = BN == 32 ? K::MAX_ROWS : 1;   // rows of head inputs fetched per tile
        for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            int n, y0, x0;
            decode(t, n, y0, x0);
            const int x = x0 + q * 32 + lane;
            const bool in = x < a.W;
            // the head's per-pixel inputs of every row of the tile, requested before the accumulator wait
            float2 hx[HR], ht[HR];
            if (BN == 32 && a.has_head) {
#pragma unroll
                for (int o = 0; o < HR; ++o) {
                    hx[o] = ht[o] = make_float2(0.f, 0.f);
                    if (o < R && y0 + o < a.H && in) {
                        const size_t p = ((size_t)n * a.H + y0 + o) * a.W + x;
                        hx[o] = reinterpret_cast<const float2 *>(a.head.xn)[p];
                        if (a.head.t_rf) ht[o] = make_float2(a.head.t_rf[p], a.head.t_quad[p]);
                    }
                }
            }
            const bool ready = mbar_wait(accf0 + 8 * b, (uint32_t)(i >> 1) & 1u, deadline);
            if (__all_sync(0xffffffffu, ready) == 0) {
                ok = false;
                break;
            }
            tc_fence_after();
#pragma unroll 1
            for (int o = 0; o < R && y0 + o < a.H; ++o) {   // output row y0 + o: accumulator columns o BN ..
            const size_t pix = ((size_t)n * a.H + y0 + o) * a.W + x;
#pragma unroll
            for (int c = 0; c < BN; c += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + (uint32_t)(b * K::ACC_COLS) + ((uint32_t)(q * 32) << 16) + (uint32_t)(o * BN + c), r);
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = in ? __uint_as_float(r[j]) : 0.f;
                if (in) {
                    if (a.bias) {
                        const float4 *b4 = reinterpret_cast<const float4 *>(a.bias + c);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 bb = b4[j];
                            v[4 * j] += bb.x;
                            v[4 * j + 1] += bb.y;
                            v[4 * j + 2] += bb.z;
                            v[4 * j + 3] += bb.w;
                        }
                    }
                    if (a.relu) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.f);
                    }
                    if (a.mask) {
                        const uint4 *m4 = reinterpret_cast<const uint4 *>(a.mask + pix * a.Cout + c);
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            const uint4 mv = m4[g];
                            const __nv_bfloat162 *mb = reinterpret_cast<const __nv_bfloat162 *>(&mv);
#pragma unroll
                            for (int h = 0; h < 4; ++h) {
                                const float2 f = __bfloat1622float2(mb[h]);
                                if (!(f.x > 0.f)) v[8 * g + 2 * h] = 0.f;
                                if (!(f.y > 0.f)) v[8 * g + 2 * h + 1] = 0.f;
                            }
                        }
                    }
                }
                if (BN == 32 && a.has_head) {   // residual head on the BF16-rounded activations
                    const HeadTC &hd = a.head;
                    float g0 = 0.f, g1 = 0.f;
                    if (in) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = __bfloat162float(__float2bfloat16_rn(v[j]));
                        float2 xo = hx[0], to = ht[0];   // row o's inputs (selected, not indexed: registers)
#pragma unroll
                        for (int u = 1; u < HR; ++u)
                            if (o == u) {
                                xo = hx[u];
                                to = ht[u];
                            }
                        float s0 = hd.bh[0] + xo.x, s1 = hd.bh[1] + xo.y;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            s0 += hd.wh[j] * v[j];
                            s1 += hd.wh[32 + j] * v[j];
                        }
                        if (hd.out_rf) {
                            hd.out_rf[pix] = s0 * hd.scale;
                            hd.out_quad[pix] = s1 * hd.scale;
                        }
                        if (hd.t_rf) {   // squared error and its gradient at the head's output
                            const float d0 = s0 - to.x * hd.inv_scale, d1 = s1 - to.y * hd.inv_scale;
                            hloss += d0 * d0 + d1 * d1;
                            g0 = 2.f * d0 * hd.inv_n;
                            g1 = 2.f * d1 * hd.inv_n;
                            hb0 += g0;
                            hb1 += g1;
                        }
                    }
                    if (hd.t_rf) {   // head weight gradients (column sums over the warp's pixels), then the
                                     // gradient at the ReLU output replaces the activations
                        float t[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) t[j] = g0 * v[j];
                        hw0 += warp_transpose_sum(t, lane);
#pragma unroll
                        for (int j = 0; j < 32; ++j) t[j] = g1 * v[j];
                        hw1 += warp_transpose_sum(t, lane);
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = v[j] > 0.f ? g0 * hd.wh[j] + g1 * hd.wh[32 + j] : 0.f;
                    }
                }
                if (in && !(BN == 32 && a.has_head && !a.head.t_rf)) {   // inference with the head stores nothing
                    uint4 *dst = reinterpret_cast<uint4 *>(out_cols(a, pix, c));
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        uint4 o4;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * g], v[8 * g + 1]);
                        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * g + 2], v[8 * g + 3]);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * g + 4], v[8 * g + 5]);
                        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * g + 6], v[8 * g + 7]);
                        o4.x = *reinterpret_cast<uint32_t *>(&h0);
                        o4.y = *reinterpret_cast<uint32_t *>(&h1);
                        o4.z = *reinterpret_cast<uint32_t *>(&h2);
                        o4.w = *reinterpret_cast<uint32_t *>(&h3);
                        dst[g] = o4;
                    }
                }
                if (a.dbias) dsum[c / 32] += warp_transpose_sum(v, lane);
            }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce0 + 8 * b);
        }
        if (a.dbias)
#pragma unroll
            for (int c = 0; c < BN / 32; ++c) atomicAdd(a.dbias + 32 * c + lane, dsum[c]);
        if (BN == 32 && a.has_head && a.head.t_rf) {
            atomicAdd(a.head.dwh + lane, hw0);
            atomicAdd(a.head.dwh + 32 + lane, hw1);
            for (int off = 16; off > 0; off >>= 1) {
                hloss += __shfl_down_sync(0xffffffffu, hloss, off);
                hb0 += __shfl_down_sync(0xffffffffu, hb0, off);
                hb1 += __shfl_down_sync(0xffffffffu, hb1, off);
            }
            if (lane == 0) {
                atomicAdd(a.head.loss, (double)(hloss * a.head.inv_n));
                atomicAdd(a.head.dbh, hb0);
                atomicAdd(a.head.dbh + 1, hb1);
            }
        }
    }
    if (!ok) atomicExch(a.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_free(tmem, K::TMEM_COLS);
    }
}

// ------------------------------------------------------------------ weight gradient
//
// dW[tap][co][ci] = sum_p dy[p][co] x[p + offset(tap)][ci] as D = A B^T with
// M = (tap, ci) rows, N = co, K = pixels.  Both operands are read MN-major from
// the NHWC tensors: a K step is 64 consecutive pixels of one image row; A is
// made of three or four 32-row groups (the MMA's other rows are not read back),
// each the TMA box of the tap-shifted input for 32 input channels (zero padding
// from the out-of-bounds fill), B of BN/32 boxes
// of dy.  Boxes are 64 pixels x 32 channels with 64-byte swizzle: 32-element
// MN chunks 4 KB apart (leading byte offset), 8-pixel K groups 512 B apart
// (stride byte offset).  K is split across CTAs; partial tiles are added into
// dW (FP32) with atomics, 32 consecutive ci per warp instruction.
//
// KX (9 taps; C_out tiles of BN in {32, 64}): with q = p + (0, kx - 1),
// dW[3 ky + kx] = sum_q x[q + (ky - 1, 0)] dy[q - (0, kx - 1)], so the rows are
// (ky, ci) from input boxes shifted by rows only and the N = 3 BN columns are
// (kx, co) from dy shifted by -(kx - 1) pixels: each input row is read once per
// kernel row instead of once per tap.  The three shifts come from one box of
// kWK + 2 pixels x BN channels (dy at x0 - 1 .. x0 + kWK): in the MN-major
// layout a pixel is one BN-channel row of the box, so column block j = 2 - kx
// starts j rows into it and the B descriptor's leading byte offset (the stride
// between its BN-column blocks) is one pixel row.  The tensor core swizzles from
// the shared-memory address bits, so the shifted blocks read the rows TMA wrote.
constexpr int kWK = 64;                 // pixels per K step (128 for the fused-kx form on wide images)
constexpr int kChunk = 32 * kWK * 2;    // one 32-channel x 64-pixel box: 4 KB

// A operand: 32-channel MN chunks `chunk` bytes apart (one box of 32 channels x the step's pixels)
__device__ __forceinline__ uint64_t sdesc_mn64(uint32_t addr, uint32_t chunk = kChunk) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(chunk >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           (1ull << 46) | (4ull << 61);
}

// B operand of the KX weight gradient: pixel rows of ROW = 2 BN bytes (64-byte swizzle for
// BN = 32, 128-byte for BN = 64), 8-pixel K groups 8 ROW apart, BN-column blocks one row apart.
template <int BN>
__device__ __forceinline__ uint64_t sdesc_mn_shift(uint32_t addr) {
    constexpr uint32_t ROW = 2 * BN;
    constexpr uint64_t layout = BN == 64 ? 2ull : 4ull;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(ROW >> 4) << 16) | ((uint64_t)((8 * ROW) >> 4) << 32) |
           (1ull << 46) | (layout << 61);
}

template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16_mn() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

// BN: C_out tile; KX: the fused-kx form (MMA N = 3 BN, one shifted dy box per stage); WK: pixels
// per K step.
template <int BN, bool KX, int WK = kWK>
struct WCfg {
    static constexpr int NB = KX ? 3 * BN : BN;   // MMA N
    static constexpr int CHUNK = 32 * WK * 2;      // one 32-channel box
    static constexpr int A_BYTES = 4 * CHUNK;
    static constexpr int B_TX = KX ? (WK + 2) * BN * 2 : (BN / 32) * CHUNK;   // bytes the B boxes deliver
    static constexpr int B_BYTES = (B_TX + 1023) / 1024 * 1024;                  // their stage slot
    // KX with 64-pixel steps: two CTAs per SM (stages within half the SM's shared memory), so one
    // CTA's epilogue overlaps the other's main loop; 128-pixel steps: one CTA per SM, four stages
    static constexpr int S_RAW =
        (KX ? (WK > 64 ? 200 * 1024 : 110 * 1024) : BN >= 128 ? 200 * 1024 : 100 * 1024) / (A_BYTES + B_BYTES);
    static constexpr int S = S_RAW < 2 ? 2 : (S_RAW > 6 ? 6 : S_RAW);
    static constexpr int TMEM_COLS = NB <= 32 ? 32 : NB <= 64 ? 64 : NB <= 128 ? 128 : 256;
    static constexpr int SMEM = S * (A_BYTES + B_BYTES) + 1024 + 8 * (2 * S + 1) + 16;
};

struct WArgs {
    int N, H, W, Cin, Cout, taps, nxb, steps, per_split;
    int gpt;   // 32-row groups per M tile (3 or 4)
    float *dw;
    int *err;
    int c1;   // input channels [0, c1) from the upsampled half-resolution map
};

template <int BN, bool KX, int WK>
__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmd,
               const __grid_constant__ CUtensorMap tml, const WArgs a) {
    using K = WCfg<BN, KX, WK>;
    constexpr int NB = K::NB;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = s_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *sm = smem_raw + (base - raw);
    const uint32_t sA = base, sB = base + K::S * K::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + K::S * (K::A_BYTES + K::B_BYTES));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * K::S + 1);
    const uint32_t full0 = s_addr(bars), empty0 = s_addr(bars + K::S), accb = s_addr(bars + 2 * K::S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int rows = (KX ? 3 : a.taps) * a.Cin;
    const int r0 = blockIdx.x * 32 * a.gpt;
    const int n_groups = min(a.gpt, (rows - r0) / 32);
    const int co0 = blockIdx.y * BN;
    const int s_begin = blockIdx.z * a.per_split;
    const int s_end = min(a.steps, s_begin + a.per_split);
    const int nk = s_end - s_begin;
    const uint64_t deadline = now_ns() + kWaitNs;

    if (threadIdx.x == 0) {
        for (int s = 0; s < K::S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(s_addr(tslot), K::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tslot);
    bool ok = true;

    if (warp == 0) {
        if (lane == 0 && nk > 0) {   // TMA producer
            int issued = 0;
            const uint32_t bytes = (uint32_t)(n_groups * K::CHUNK + K::B_TX);
            for (int kt = 0; kt < nk; ++kt) {
                const int st = kt % K::S;
                if (!mbar_wait(empty0 + 8 * st, ((uint32_t)(kt / K::S) & 1u) ^ 1u, deadline)) {
                    ok = false;
                    break;
                }
                // K steps run down the image rows fastest: the rows a step loads for ky = 0, 1, 2 are
                // loaded again by the next two steps (ky shifted by one), while still in L2
                int q = s_begin + kt;
                const int y = q % a.H;
                q /= a.H;
                const int xb = q % a.nxb, n = q / a.nxb, x0 = xb * WK;
                mbar_expect_tx(full0 + 8 * st, bytes);
                for (int g = 0; g < n_groups; ++g) {
                    const int r = r0 + 32 * g, tap = r / a.Cin, ci0 = r - tap * a.Cin;
                    int ky, kx;
                    if (KX) {   // row group (ky, ci0): input shifted by rows only
                        ky = tap;
                        kx = 1;
                    } else {
                        ky = a.taps == 1 ? 1 : tap / 3;
                        kx = a.taps == 1 ? 1 : tap - 3 * (tap / 3);
                    }
                    if (ci0 < a.c1)   // upsampled: 32 low pixels, each twice (kx = 1 here: no pixel shift)
                        tma_load_5d(sA + st * K::A_BYTES + g * K::CHUNK, &tml, ci0, 0, x0 / 2, low_row(y + ky - 1), n,
                                    full0 + 8 * st);
                    else
                        tma_load_4d(sA + st * K::A_BYTES + g * K::CHUNK, &tmx, ci0 - a.c1, x0 + kx - 1, y + ky - 1, n,
                                    full0 + 8 * st);
                }
                if (KX) {   // dy at pixels x0 - 1 .. x0 + WK: the three kx shifts are rows 2 - kx on
                    tma_load_4d(sB + st * K::B_BYTES, &tmd, co0, x0 - 1, y, n, full0 + 8 * st);
                } else {
                    for (int c = 0; c < BN / 32; ++c)
                        tma_load_4d(sB + st * K::B_BYTES + c * K::CHUNK, &tmd, co0 + 32 * c, x0, y, n, full0 + 8 * st);
                }
                issued = kt + 1;
            }
            if (!ok)
                for (int kt = issued > K::S ? issued - K::S : 0; kt < issued; ++kt)
                    mbar_wait(full0 + 8 * (kt % K::S), (uint32_t)(kt / K::S) & 1u, deadline + kWaitNs / 20);
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && nk > 0) {   // MMA issuer
            constexpr uint32_t idesc = idesc_bf16_mn<NB>();
            for (int kt = 0; kt < nk; ++kt) {
                const int st = kt % K::S;
                if (!mbar_wait(full0 + 8 * st, (uint32_t)(kt / K::S) & 1u, deadline)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = sA + st * K::A_BYTES, b0 = sB + st * K::B_BYTES;
#pragma unroll
                for (int k = 0; k < WK / 16; ++k) {   // 16 pixels: two 8-row K groups
                    const uint64_t bd =
                        KX ? sdesc_mn_shift<BN>(b0 + (uint32_t)(16 * 2 * BN * k)) : sdesc_mn64(b0 + 1024 * k, K::CHUNK);
                    mma_bf16(tmem, sdesc_mn64(a0 + 1024 * k, K::CHUNK), bd, idesc, (kt | k) != 0);
                }
                mma_commit(empty0 + 8 * st);
            }
            mma_commit(accb);
        }
        __syncwarp();
    }

    const bool acc_ready = nk > 0 && mbar_wait(accb, 0, deadline + kWaitNs / 10);
    const bool warp_ready = __all_sync(0xffffffffu, acc_ready) != 0;
    if (nk > 0 && !acc_ready) ok = false;
    tc_fence_after();
    if (warp_ready && warp < n_groups) {
        const int r = r0 + 32 * warp, tr = r / a.Cin, ci = r - tr * a.Cin + lane;
#pragma unroll 1
        for (int c = 0; c < NB; c += 32) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            const int tap = KX ? 3 * tr + 2 - c / BN : tr;   // KX: row = ky, column block j = 2 - kx
            const int co = co0 + (KX ? c % BN : c);
            float *dst = a.dw + ((size_t)tap * a.Cout + co) * a.Cin + ci;
#pragma unroll
            for (int j = 0; j < 32; ++j) atomicAdd(dst + (size_t)j * a.Cin, __uint_as_float(v[j]));
        }
    }
    if (!ok) atomicExch(a.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(tmem, K::TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

template <typename KernelT>
cudaError_t ctas_per_sm(KernelT kernel, int smem, int tmem_cols, int *occ);

// Persistent grid: as many CTAs as fit on the SMs at once (shared memory and TMEM), at most one per tile.
template <int BN, int BK>
cudaError_t launch(const CUtensorMap &mx, const CUtensorMap &mw, const Args &a, int n_sm, cudaStream_t stream) {
    using K = Cfg<BN, BK>;
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    if (e == cudaSuccess)   // all of the unified L1/shared array as shared memory, so several CTAs fit per SM
        e = cudaFuncSetAttribute(k_conv_tc<BN, BK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int occ = 1;
    if ((e = ctas_per_sm(k_conv_tc<BN, BK>, K::SMEM, K::TMEM_COLS, &occ)) != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(a.n_tiles, (long long)occ * std::max(1, n_sm));
    k_conv_tc<BN, BK><<<grid, kConvThreads, K::SMEM, stream>>>(mx, mw, a);
    return cudaGetLastError();
}

// co-resident CTAs per SM from shared memory (with the per-block reserve), registers, warps and TMEM
template <typename KernelT>
cudaError_t ctas_per_sm(KernelT kernel, int smem, int tmem_cols, int *occ) {
    int dev = 0, smem_sm = 0, reserve = 0;
    cudaFuncAttributes fa{};
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess)
        return e;
    const int regs = ((std::max(fa.numRegs, 1) + 7) / 8) * 8 * kConvThreads;
    *occ = std::max(1, std::min({smem_sm / (smem + reserve), 65536 / regs, 64 / (kConvThreads / 32), 512 / tmem_cols}));
    return cudaSuccess;
}

// Stages and weight residency of a kx-fused launch: two CTAs per SM (the epilogues of two tiles
// overlap), with resident weights when two input stages fit beside them, else with the weights
// streamed with the input; one CTA per SM only when neither fits.
template <int BN, int BK>
cudaError_t launch_kx(const CUtensorMap &mx, const CUtensorMap &mw, const CUtensorMap &ml, Args a, int n_sm,
                      cudaStream_t stream) {
    using K = KxCfg<BN, BK>;
    int dev = 0, smem_sm = 0, reserve = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return e;
    const int kc = a.C / BK, two = smem_sm / 2 - reserve;
    // Row-stacked tiles (R = 128 / BN output rows) when the stacked weights and two input stages fit
    // twice per SM (at one CTA per SM stacked tiles were slower than single-row tiles at two,
    // measured on the denoiser's layers).  Otherwise one output row per tile with the weights
    // resident (two CTAs per SM, else one) or streamed with each stage.
    int R = 1, stages = 0, smem = 0;
    bool wres = true;
    if (K::MAX_ROWS > 1) {
        const int fixed = 1024 + kc * K::STK_BYTES + K::TAIL;
        const int n = std::min((two - fixed) / K::A_PAD, kKxMaxStages);
        if (n >= 2) {
            R = K::MAX_ROWS;
            stages = n;
            smem = fixed + n * K::A_PAD;
        }
    }
    if (R == 1) {
        auto fit = [&](int budget, bool w) {
            const int n = (budget - K::smem(kc, w, 0)) / (K::A_PAD + (w ? 0 : K::B_PAD));
            return std::min(n, kKxMaxStages);
        };
        stages = fit(two, true);
        if (stages < 2) {
            wres = false;
            stages = fit(two, false);
        }
        if (stages < 2) {
            wres = true;
            stages = fit(optin, true);
        }
        if (stages < 2) {
            wres = false;
            stages = fit(optin, false);
        }
        if (stages < 2) return cudaErrorInvalidValue;
        smem = K::smem(kc, wres, stages);
    }
    a.stages = stages;
    a.wres = wres ? 1 : 0;
    a.rows = R;
    a.nyb = (a.H + R - 1) / R;
    const long long row_tiles = (long long)a.N * a.nxb;
    if (row_tiles * a.nyb > 0x7fffffffll) return cudaErrorInvalidValue;
    a.n_tiles = (int)(row_tiles * a.nyb);
    e = cudaFuncSetAttribute(k_conv_kx<BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_conv_kx<BN, BK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    int occ = 1;
    if (e == cudaSuccess) e = ctas_per_sm(k_conv_kx<BN, BK>, smem, K::TMEM_COLS, &occ);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>(a.n_tiles, (long long)occ * std::max(1, n_sm));
    k_conv_kx<BN, BK><<<grid, kConvThreads, smem, stream>>>(mx, mw, ml, a);
    return cudaGetLastError();
}

template <int BK>
cudaError_t launch_bn(int BN, const CUtensorMap &mx, const CUtensorMap &mw, const Args &a, int n_sm,
                      cudaStream_t stream) {
    switch (BN) {
        case 32: return launch<32, BK>(mx, mw, a, n_sm, stream);
        case 64: return launch<64, BK>(mx, mw, a, n_sm, stream);
        case 96: return launch<96, BK>(mx, mw, a, n_sm, stream);
        case 128: return launch<128, BK>(mx, mw, a, n_sm, stream);
        case 192: return launch<192, BK>(mx, mw, a, n_sm, stream);
        default: return launch<256, BK>(mx, mw, a, n_sm, stream);
    }
}

int pick_bn(int cout) {
    if (cout <= 256) return (cout == 32 || cout == 64 || cout == 96 || cout == 128 || cout == 192 || cout == 256) ? cout : 0;
    for (int bn : {256, 192, 128, 64, 32})
        if (cout % bn == 0) return bn;
    return 0;
}

}  // namespace

cudaError_t conv3x3_tc(const ConvTC &p, int *d_err, int n_sm, cudaStream_t stream, std::string *why) {
    const int BK = p.C % 64 == 0 ? 64 : 32;
    const int BN = pick_bn(p.Cout);
    if (p.C < 32 || p.C % 32 || BN == 0 || (p.taps != 9 && p.taps != 1) || p.N < 1 || p.H < 1 || p.W < 1 || !p.x || !p.w || !p.y || !d_err ||
        (reinterpret_cast<uintptr_t>(p.x) & 15) || (reinterpret_cast<uintptr_t>(p.w) & 15) ||
        (reinterpret_cast<uintptr_t>(p.y) & 15) || (p.bias && (reinterpret_cast<uintptr_t>(p.bias) & 15)) ||
        (p.mask && (reinterpret_cast<uintptr_t>(p.mask) & 15)) ||
        (p.y2 && ((reinterpret_cast<uintptr_t>(p.y2) & 15) || p.c_split <= 0 || p.c_split >= p.Cout || p.c_split % 32)) ||
        (p.head && (p.Cout != 32 || p.taps != 9 || !p.relu || p.mask || p.y2 || !p.head->xn || !p.head->wh ||
                    !p.head->bh || (!p.head->out_rf != !p.head->out_quad) || (!p.head->t_rf != !p.head->t_quad) ||
                    (p.head->t_rf && (!p.head->loss || !p.head->dwh || !p.head->dbh)))) ||
        (p.x_low && (p.taps != 9 || !(p.Cout == 32 || p.Cout == 64 || p.Cout == 96) || (p.H | p.W) & 1 ||
                     p.c1 <= 0 || p.c1 >= p.C || p.c1 % BK || (p.C - p.c1) % BK ||
                     (reinterpret_cast<uintptr_t>(p.x_low) & 15)))) {
        if (why) *why = "conv3x3_tc: unsupported shape or alignment";
        return cudaErrorInvalidValue;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) {
        if (why) *why = "cuTensorMapEncodeTiled is not available from the driver";
        return cudaErrorNotSupported;
    }
    const CUtensorMapSwizzle sw = BK == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    alignas(64) CUtensorMap mx, mw, mlow;
    {
        const int cx = p.x_low ? p.C - p.c1 : p.C;   // channels of x itself
        const cuuint64_t dims[4] = {(cuuint64_t)cx, (cuuint64_t)p.W, (cuuint64_t)p.H, (cuuint64_t)p.N};
        const cuuint64_t strides[3] = {(cuuint64_t)cx * 2, (cuuint64_t)p.W * cx * 2, (cuuint64_t)p.H * p.W * cx * 2};
        const bool kx = p.taps == 9 && (p.Cout == 32 || p.Cout == 64 || p.Cout == 96);   // kx-fused: 130 staged pixels
        const cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)(kx ? kKxRows : kBM), 1, 1};
        const cuuint32_t es[4] = {1, 1, 1, 1};
        const CUresult r = enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(p.x), dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            if (why) *why = "tensor map of the convolution input rejected (" + std::to_string((int)r) + ")";
            return cudaErrorInvalidValue;
        }
    }
    if (p.x_low) {   // (c, repeat 2 with stride 0, x / 2, y / 2, n): a box of 66 low pixels gives 132 upsampled rows
        const int c1 = p.c1, wl = p.W / 2, hl = p.H / 2;
        const cuuint64_t dims[5] = {(cuuint64_t)c1, 2, (cuuint64_t)wl, (cuuint64_t)hl, (cuuint64_t)p.N};
        const cuuint64_t strides[4] = {0, (cuuint64_t)c1 * 2, (cuuint64_t)wl * c1 * 2, (cuuint64_t)hl * wl * c1 * 2};
        const cuuint32_t box[5] = {(cuuint32_t)BK, 2, (cuuint32_t)(kKxRows / 2 + 1), 1, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        const CUresult r = enc(&mlow, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(p.x_low), dims, strides, box,
                               es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            if (why) *why = "tensor map of the upsampled input rejected (" + std::to_string((int)r) + ")";
            return cudaErrorInvalidValue;
        }
    }
    {
        const cuuint64_t dims[3] = {(cuuint64_t)p.C, (cuuint64_t)p.Cout, (cuuint64_t)p.taps};
        const cuuint64_t strides[2] = {(cuuint64_t)p.C * 2, (cuuint64_t)p.Cout * p.C * 2};
        const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BN, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        const CUresult r = enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16 *>(p.w), dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            if (why) *why = "tensor map of the weights rejected (" + std::to_string((int)r) + ")";
            return cudaErrorInvalidValue;
        }
    }
    if (p.taps == 9 && (p.Cout == 32 || p.Cout == 64 || p.Cout == 96)) {   // kx taps from row-shifted stages
        alignas(64) CUtensorMap mw2;
        const cuuint64_t dims[2] = {(cuuint64_t)p.C, 9ull * p.Cout};
        const cuuint64_t strides[1] = {(cuuint64_t)p.C * 2};
        const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)p.Cout};
        const cuuint32_t es[2] = {1, 1};
        if (enc(&mw2, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16 *>(p.w), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            if (why) *why = "tensor map of the stacked weights rejected";
            return cudaErrorInvalidValue;
        }
        const int nxk = (p.W + kBM - 1) / kBM;
        const long long nt = (long long)p.N * p.H * nxk;
        if (nt > 0x7fffffffll) {
            if (why) *why = "conv3x3_tc: too many tiles";
            return cudaErrorInvalidValue;
        }
        Args a{p.N, p.H, p.W, p.C, p.Cout, nxk, p.relu, p.taps, (int)nt, 1, 0, 0, 1, p.H, p.bias, p.mask, p.y, p.dbias,
               p.y2, p.c_split, d_err};
        if (p.head) {
            a.has_head = 1;
            a.head = *p.head;
        }
        a.c1 = p.x_low ? p.c1 : 0;
        const CUtensorMap &ml = p.x_low ? mlow : mx;
        if (p.Cout == 32)
            return BK == 64 ? launch_kx<32, 64>(mx, mw2, ml, a, n_sm, stream) : launch_kx<32, 32>(mx, mw2, ml, a, n_sm, stream);
        if (p.Cout == 96)
            return BK == 64 ? launch_kx<96, 64>(mx, mw2, ml, a, n_sm, stream) : launch_kx<96, 32>(mx, mw2, ml, a, n_sm, stream);
        return BK == 64 ? launch_kx<64, 64>(mx, mw2, ml, a, n_sm, stream) : launch_kx<64, 32>(mx, mw2, ml, a, n_sm, stream);
    }
    const int nxb = (p.W + kBM - 1) / kBM;
    const long long n_tiles = (long long)p.N * p.H * nxb * (p.Cout / BN);
    if (n_tiles > 0x7fffffffll) {
        if (why) *why = "conv3x3_tc: too many tiles";
        return cudaErrorInvalidValue;
    }
    Args a{p.N, p.H, p.W, p.C, p.Cout, nxb, p.relu, p.taps, (int)n_tiles, p.Cout / BN, 0, 0, 1, p.H, p.bias, p.mask, p.y,
           p.dbias, p.y2, p.c_split, d_err};
    return BK == 64 ? launch_bn<64>(BN, mx, mw, a, n_sm, stream) : launch_bn<32>(BN, mx, mw, a, n_sm, stream);
}

namespace {

template <int BN, bool KX, int WK = kWK>
cudaError_t launch_w(const CUtensorMap &mx, const CUtensorMap &md, const CUtensorMap &ml, const WArgs &a, dim3 grid,
                     cudaStream_t stream) {
    using K = WCfg<BN, KX, WK>;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<BN, KX, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, K::SMEM);
    if (e == cudaSuccess)   // all of the unified L1/shared array as shared memory: two CTAs per SM
        e = cudaFuncSetAttribute(k_wgrad_tc<BN, KX, WK>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    k_wgrad_tc<BN, KX, WK><<<grid, kThreads, K::SMEM, stream>>>(mx, md, ml, a);
    return cudaGetLastError();
}

bool encode_nhwc(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap *m, const bf16 *p, int C, int N, int H, int W,
                 int box_c, int box_px, CUtensorMapSwizzle sw) {
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)N};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {(cuuint32_t)box_c, (cuuint32_t)box_px, 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t wgrad3x3_tc(const WgradTC &p, int *d_err, int n_sm, cudaStream_t stream, std::string *why) {
    const int BN = p.Cout <= 256 ? p.Cout : 0;
    if (p.Cin < 32 || p.Cin % 32 || (BN != 32 && BN != 64 && BN != 128 && BN != 256) || (p.taps != 9 && p.taps != 1) ||
        p.N < 1 || p.H < 1 || p.W < 1 || !p.x || !p.dy || !p.dw || !d_err || (reinterpret_cast<uintptr_t>(p.x) & 15) ||
        (reinterpret_cast<uintptr_t>(p.dy) & 15) ||
        (p.x_low && (p.taps != 9 || (p.H | p.W) & 1 || p.c1 <= 0 || p.c1 >= p.Cin || p.c1 % 32 ||
                     (reinterpret_cast<uintptr_t>(p.x_low) & 15)))) {
        if (why) *why = "wgrad3x3_tc: unsupported shape or alignment";
        return cudaErrorInvalidValue;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) {
        if (why) *why = "cuTensorMapEncodeTiled is not available from the driver";
        return cudaErrorNotSupported;
    }
    const bool kx = p.taps == 9;   // C_out tiles of 32 (C_out = 32) or 64 columns x 3 taps
    const int kx_bn = p.Cout == 32 ? 32 : 64;
    // pixels per K step: 128 for the fused-kx form where the image width fills 128-pixel blocks or
    // is wide enough that a ragged last block costs little (half as many K steps, each twice the
    // MMAs per pipeline round trip), else 64
    const int wk = kx && (p.W % 128 == 0 || p.W >= 1024) ? 128 : kWK;
    alignas(64) CUtensorMap mx, md, mlow;
    if (p.x_low) {   // (c, repeat 2 with stride 0, x / 2, y / 2, n): 32 low pixels give a 64-pixel box
        const int c1 = p.c1, wl = p.W / 2, hl = p.H / 2;
        const cuuint64_t dims[5] = {(cuuint64_t)c1, 2, (cuuint64_t)wl, (cuuint64_t)hl, (cuuint64_t)p.N};
        const cuuint64_t strides[4] = {0, (cuuint64_t)c1 * 2, (cuuint64_t)wl * c1 * 2, (cuuint64_t)hl * wl * c1 * 2};
        const cuuint32_t box[5] = {32, 2, (cuuint32_t)(wk / 2), 1, 1};
        const cuuint32_t es[5] = {1, 1, 1, 1, 1};
        if (enc(&mlow, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16 *>(p.x_low), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
            if (why) *why = "wgrad3x3_tc: tensor map of the upsampled input rejected";
            return cudaErrorInvalidValue;
        }
    }
    const int cx = p.x_low ? p.Cin - p.c1 : p.Cin;   // channels of x itself
    const bool md_ok = kx ? encode_nhwc(enc, &md, p.dy, p.Cout, p.N, p.H, p.W, kx_bn, wk + 2,
                                        kx_bn == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B)
                          : encode_nhwc(enc, &md, p.dy, p.Cout, p.N, p.H, p.W, 32, kWK, CU_TENSOR_MAP_SWIZZLE_64B);
    if (!encode_nhwc(enc, &mx, p.x, cx, p.N, p.H, p.W, 32, wk, CU_TENSOR_MAP_SWIZZLE_64B) || !md_ok) {
        if (why) *why = "wgrad3x3_tc: tensor map rejected";
        return cudaErrorInvalidValue;
    }
    const int nxb = (p.W + wk - 1) / wk;
    const long long steps = (long long)p.N * p.H * nxb;
    // M tiles of 4 groups of 32 (tap, ci) rows, or of 3 where that gives as many tiles with equal
    // work (96 input channels: three tiles of 96 rows instead of 128, 128 and 32)
    const int groups = (kx ? 3 : p.taps) * p.Cin / 32;
    const int gpt = (groups % 4 != 0 && groups % 3 == 0 && groups / 3 == (groups + 3) / 4) ? 3 : 4;
    const int m_tiles = (groups + gpt - 1) / gpt;
    if (steps > 0x7fffffffll) {
        if (why) *why = "wgrad3x3_tc: too many pixels";
        return cudaErrorInvalidValue;
    }
    int smem = 0;
    switch (kx ? kx_bn : 1000 + BN) {
        case 32: smem = wk == 128 ? WCfg<32, true, 128>::SMEM : WCfg<32, true>::SMEM; break;
        case 64: smem = wk == 128 ? WCfg<64, true, 128>::SMEM : WCfg<64, true>::SMEM; break;
        case 1032: smem = WCfg<32, false>::SMEM; break;
        case 1064: smem = WCfg<64, false>::SMEM; break;
        case 1128: smem = WCfg<128, false>::SMEM; break;
        default: smem = WCfg<256, false>::SMEM; break;
    }
    int dev = 0, smem_sm = 0, reserve = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
        return e;
    // one wave of CTAs (as many as fit on the SMs at once), each a run of at least 8 K steps down
    // the image rows: partial tiles are added once per CTA
    const int occ = std::max(1, std::min(2, smem_sm / (smem + reserve)));
    const long long target = (long long)occ * (n_sm > 0 ? n_sm : 148);
    const int n_tiles = kx ? p.Cout / kx_bn : 1;
    long long splits = std::max<long long>(1, target / ((long long)m_tiles * n_tiles));
    splits = std::min<long long>(splits, std::max<long long>(1, steps / 8));
    const int per = (int)((steps + splits - 1) / splits);
    splits = (steps + per - 1) / per;
    WArgs a{p.N, p.H, p.W, p.Cin, p.Cout, p.taps, nxb, (int)steps, per, gpt, p.dw, d_err, p.x_low ? p.c1 : 0};
    const CUtensorMap &ml = p.x_low ? mlow : mx;
    const dim3 grid((unsigned)m_tiles, (unsigned)n_tiles, (unsigned)splits);
    if (kx && wk == 128)
        return kx_bn == 32 ? launch_w<32, true, 128>(mx, md, ml, a, grid, stream)
                           : launch_w<64, true, 128>(mx, md, ml, a, grid, stream);
    if (kx) return kx_bn == 32 ? launch_w<32, true>(mx, md, ml, a, grid, stream) : launch_w<64, true>(mx, md, ml, a, grid, stream);
    switch (BN) {
        case 32: return launch_w<32, false>(mx, md, ml, a, grid, stream);
        case 64: return launch_w<64, false>(mx, md, ml, a, grid, stream);
        case 128: return launch_w<128, false>(mx, md, ml, a, grid, stream);
        default: return launch_w<256, false>(mx, md, ml, a, grid, stream);
    }
}

}  // namespace urnn
