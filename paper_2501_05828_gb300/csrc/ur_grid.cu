// Scatterer grid: columns in x and y, each indexed by z cells, cells numbered
// with z fastest.  A scatterer is referenced by every column its capture square
// [p - r_m, p + r_m] (r_m slightly above r_s) overlaps in x and y, but only in
// the z cell that holds it, so the references of one column are grouped by z
// and a range of z cells is one contiguous range of references.  A ray segment
// visits the columns it passes and, in each, the references whose z lies within
// r_m of the z it spans there.  Built on the device: bounding box, per-cell
// counts, exclusive scan, fill.
#include "ur_device.cuh"

namespace ur {
namespace {

__device__ __forceinline__ unsigned int ordered(float f) {
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_bbox(const float4 *scat, int n, unsigned int *lohi) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float4 p = scat[j];
        mn[0] = fminf(mn[0], p.x); mx[0] = fmaxf(mx[0], p.x);
        mn[1] = fminf(mn[1], p.y); mx[1] = fmaxf(mx[1], p.y);
        mn[2] = fminf(mn[2], p.z); mx[2] = fmaxf(mx[2], p.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const unsigned int lo = __reduce_min_sync(0xffffffffu, ordered(mn[a]));
        const unsigned int hi = __reduce_max_sync(0xffffffffu, ordered(mx[a]));
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&lohi[a], lo);
            atomicMax(&lohi[3 + a], hi);
        }
    }
}

// Columns (x, y) whose cells a scatterer at p is referenced from, and its z cell.
__device__ __forceinline__ void cell_range(const GridBuildP &G, float4 p, int3 &c0, int3 &c1) {
    c0.x = min(max((int)floorf((p.x - G.r_m - G.lo.x) * G.inv_h.x), 0), G.dim.x - 1);
    c0.y = min(max((int)floorf((p.y - G.r_m - G.lo.y) * G.inv_h.y), 0), G.dim.y - 1);
    c1.x = min(max((int)floorf((p.x + G.r_m - G.lo.x) * G.inv_h.x), 0), G.dim.x - 1);
    c1.y = min(max((int)floorf((p.y + G.r_m - G.lo.y) * G.inv_h.y), 0), G.dim.y - 1);
    c0.z = c1.z = min(max((int)floorf((p.z - G.lo.z) * G.inv_h.z), 0), G.dim.z - 1);
}

__global__ void k_grid_count(const GridBuildP G) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G.n_scat; j += gridDim.x * blockDim.x) {
        int3 c0, c1;
        cell_range(G, G.scat[j], c0, c1);
        for (int y = c0.y; y <= c1.y; ++y)
            for (int x = c0.x; x <= c1.x; ++x)
                atomicAdd(&G.cell_count[((uint32_t)x * G.dim.y + y) * G.dim.z + c0.z], 1u);
    }
}

__global__ void k_grid_fill(const GridBuildP G) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G.n_scat; j += gridDim.x * blockDim.x) {
        const float4 p = G.scat[j];
        G.amp[j] = p.w;
        int3 c0, c1;
        cell_range(G, p, c0, c1);
        for (int y = c0.y; y <= c1.y; ++y)
            for (int x = c0.x; x <= c1.x; ++x) {
                const uint32_t c = ((uint32_t)x * G.dim.y + y) * G.dim.z + c0.z;
                const uint32_t slot = atomicAdd(&G.cell_fill[c], 1u);
                G.refs[G.cell_start[c] + slot] = make_float4(p.x, p.y, p.z, __uint_as_float((uint32_t)j));
            }
    }
}

// ---- exclusive scan of n u32 values: out[0..n], out[n] = total ----
constexpr int kScanBlock = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanBlock * kScanPer;

__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[31];
    const uint32_t r = (wid ? s_warp[wid - 1] : 0u) + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const uint32_t *in, uint32_t n, uint32_t *block_sums) {
    __shared__ uint32_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q)
        if (base + q < n) s += in[base + q];
    uint32_t total;
    block_exclusive(s, s_warp, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(uint32_t *block_sums, uint32_t nb) {
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < nb ? block_sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive(v, s_warp, total);
        if (i < nb) block_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) block_sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const uint32_t *in, uint32_t n, const uint32_t *block_sums,
                                                             uint32_t nb, uint32_t *out) {
    __shared__ uint32_t s_warp[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        v[q] = base + q < n ? in[base + q] : 0u;
        s += v[q];
    }
    uint32_t total;
    uint32_t ex = block_exclusive(s, s_warp, total) + block_sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanPer; ++q) {
        if (base + q < n) out[base + q] = ex;
        ex += v[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = block_sums[nb];
}

}  // namespace

void launch_bbox(const float4 *scat, int n, float *lohi, cudaStream_t s) {
    k_bbox<<<min(1024, (n + 255) / 256 + 1), 256, 0, s>>>(scat, n, reinterpret_cast<unsigned int *>(lohi));
}

void launch_grid_count(const GridBuildP &G, cudaStream_t s) {
    k_grid_count<<<min(4096, (G.n_scat + 255) / 256 + 1), 256, 0, s>>>(G);
}

void launch_grid_fill(const GridBuildP &G, cudaStream_t s) {
    k_grid_fill<<<min(4096, (G.n_scat + 255) / 256 + 1), 256, 0, s>>>(G);
}

// block_sums needs (n / 4096 + 2) entries.
void launch_scan_u32(const uint32_t *in, uint32_t *out, uint32_t *block_sums, uint32_t n, cudaStream_t s) {
    const uint32_t nb = (n + kScanTile - 1) / kScanTile + (n == 0);
    k_scan_reduce<<<nb, kScanBlock, 0, s>>>(in, n, block_sums);
    k_scan_blocks<<<1, kScanBlock, 0, s>>>(block_sums, nb);
    k_scan_apply<<<nb, kScanBlock, 0, s>>>(in, n, block_sums, nb, out);
}

}  // namespace ur
