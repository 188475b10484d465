// Ray order of a mixed transmit sequence.  With per-ray transmit mixing
// (Sec. 2.3) ray i of the sequence draws its transmit k(i) from its own Philox
// counter, so neighbouring rays belong to different transmits and a warp that
// traces consecutive rays diverges at once.  A ray's path is a function of
// (i, k(i)) alone, so the order in which the tracer visits the rays is free:
// these kernels counting-sort the ray indices by (drawn transmit, emitting
// element), and the tracer takes its slots from that list, giving each warp
// neighbouring rays of one element and one transmit as in an unmixed trace.
#include "ur_device.cuh"

#include <algorithm>

namespace ur {
namespace {

// Bin of ray i: its drawn transmit k (the tracer's draw, counter (i, 0, 0, 1))
// times n_el plus its emitting element, or k alone when the (transmit, element)
// bins do not fit in shared memory.
__device__ __forceinline__ uint32_t mix_bin(const MixP &M, uint32_t i) {
    const uint4 y = philox(make_uint4(i, 0u, 0u, 1u), M.key);
    const uint32_t k = (uint32_t)(((uint64_t)(y.x >> 8) * (uint64_t)M.n_tx) >> 24);
    return M.per_element ? k * M.n_el + i % M.n_el : k;
}

// Contiguous ray range of this CTA (64-bit: n may come close to 2^32).
__device__ __forceinline__ void mix_range(uint64_t n, uint64_t &b, uint64_t &e) {
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    b = min(n, (uint64_t)blockIdx.x * per);
    e = min(n, b + per);
}

__global__ void k_mix_count(const MixP M) {
    extern __shared__ uint32_t hist[];   // [n_bins]
    for (uint32_t q = threadIdx.x; q < M.n_bins; q += blockDim.x) hist[q] = 0u;
    __syncthreads();
    uint64_t b, e;
    mix_range(M.n_rays, b, e);
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&hist[mix_bin(M, (uint32_t)i)], 1u);
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < M.n_bins; q += blockDim.x)
        if (hist[q]) atomicAdd(&M.count[q], hist[q]);
}

// Exclusive scan of the bin counts (one CTA of 1024 threads; n_bins <= kMixMaxBins).
__global__ void k_mix_scan(const MixP M) {
    __shared__ uint32_t part[1024];
    const uint32_t per = (M.n_bins + blockDim.x - 1) / blockDim.x;
    const uint32_t q0 = min(M.n_bins, threadIdx.x * per), q1 = min(M.n_bins, q0 + per);
    uint32_t s = 0;
    for (uint32_t q = q0; q < q1; ++q) s += M.count[q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (uint32_t off = 1; off < blockDim.x; off <<= 1) {   // inclusive Hillis-Steele scan
        const uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (uint32_t q = q0; q < q1; ++q) {
        M.offset[q] = run;
        run += M.count[q];
    }
}

// Each CTA reserves room for its rays in every bin, then writes them there.
__global__ void k_mix_scatter(const MixP M) {
    extern __shared__ uint32_t pos[];   // [n_bins]: the CTA's count, then its next write position
    for (uint32_t q = threadIdx.x; q < M.n_bins; q += blockDim.x) pos[q] = 0u;
    __syncthreads();
    uint64_t b, e;
    mix_range(M.n_rays, b, e);
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) atomicAdd(&pos[mix_bin(M, (uint32_t)i)], 1u);
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < M.n_bins; q += blockDim.x)
        if (pos[q]) pos[q] = M.offset[q] + atomicAdd(&M.fill[q], pos[q]);
    __syncthreads();
    for (uint64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
        const uint32_t p = atomicAdd(&pos[mix_bin(M, (uint32_t)i)], 1u);
        if (p < M.n_rays) M.list[p] = (uint32_t)i;
    }
}

}  // namespace

int mix_bins(int n_tx, int n_el, bool *per_element) {
    const long long both = (long long)n_tx * (long long)n_el;
    *per_element = both <= kMixMaxBins;
    if (*per_element) return (int)both;
    return n_tx <= kMixMaxBins ? n_tx : 0;
}

cudaError_t launch_mix_plan(const MixP &M, int sms, cudaStream_t s) {
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * 4, ((uint64_t)M.n_rays + 4095) / 4096));
    const size_t smem = sizeof(uint32_t) * M.n_bins;
    cudaError_t err = cudaMemsetAsync(M.count, 0, sizeof(uint32_t) * M.n_bins, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(M.fill, 0, sizeof(uint32_t) * M.n_bins, s);
    if (err != cudaSuccess) return err;
    k_mix_count<<<grid, 256, smem, s>>>(M);
    k_mix_scan<<<1, 1024, 0, s>>>(M);
    k_mix_scatter<<<grid, 256, smem, s>>>(M);
    return cudaGetLastError();
}

}  // namespace ur
