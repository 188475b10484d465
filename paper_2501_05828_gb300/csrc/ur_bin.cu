// Binning of arrivals into the analytic channel data (Eq. 14, deposited at the
// exact arrival time).  Arrivals are counting-sorted by row (transmit x element)
// and cut into work items of at most `chunk` arrivals; one CTA accumulates an
// item's pulse taps for its whole row in shared memory (n_s complex samples)
// with shared-memory atomics and flushes the row with coalesced global
// reductions.
#include "ur_device.cuh"

#include <algorithm>

namespace ur {
namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

// Arrivals are split into one contiguous range per CTA.  With few rows (one
// transmit has n_el rows) every arrival of a frame lands on one of a handful of
// counters, so the row histogram is kept per CTA in shared memory and added to
// the global counts once per (CTA, row); with more rows than fit, the counts go
// straight to global memory (warp-aggregated).
__device__ __forceinline__ void cta_range(uint64_t n, uint64_t &b, uint64_t &e) {
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    b = min(n, (uint64_t)blockIdx.x * per);
    e = min(n, b + per);
}

__global__ void k_bin_count(const BinP B) {
    extern __shared__ uint32_t hist[];   // [n_rows] when B.priv_rows
    const uint64_t n = min((uint64_t)*B.arr_count, B.arr_cap);
    const bool priv = B.priv_rows;
    if (priv) {
        for (int r = threadIdx.x; r < B.n_rows; r += blockDim.x) hist[r] = 0u;
        __syncthreads();
    }
    uint64_t b, e;
    cta_range(n, b, e);
    for (uint64_t idx = b + threadIdx.x; idx < e; idx += blockDim.x) {
        const uint32_t row = B.arr[idx].x;
        const unsigned peers = __match_any_sync(__activemask(), row);
        if ((threadIdx.x & 31) == __ffs(peers) - 1)
            atomicAdd(priv ? &hist[row] : &B.row_count[row], (uint32_t)__popc(peers));
    }
    if (priv) {
        __syncthreads();
        for (int r = threadIdx.x; r < B.n_rows; r += blockDim.x)
            if (hist[r]) atomicAdd(&B.row_count[r], hist[r]);
    }
}

// Single-CTA scan: row offsets (exclusive scan of counts) and the work-item list.
__global__ void __launch_bounds__(1024) k_bin_plan(const BinP B) {
    __shared__ uint32_t s_warp[2][32];
    __shared__ uint32_t s_carry[2];
    if (threadIdx.x == 0) {
        s_carry[0] = 0;
        s_carry[1] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // Work-item size: enough items for several waves of the deposit grid, within [chunk_min, chunk].
    const uint64_t total = min((uint64_t)*B.arr_count, B.arr_cap);
    const uint32_t chunk = (uint32_t)min((uint64_t)B.chunk,
                                         max((uint64_t)B.chunk_min, (total + B.target_items - 1) / B.target_items));
    for (int base = 0; base < B.n_rows; base += 1024) {
        const int row = base + (int)threadIdx.x;
        const uint32_t cnt = row < B.n_rows ? B.row_count[row] : 0u;
        const uint32_t nit = row < B.n_rows ? max(1u, (cnt + chunk - 1) / chunk) : 0u;
        // inclusive warp scans of (cnt, nit)
        uint32_t a = cnt, c = nit;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ya = __shfl_up_sync(0xffffffffu, a, off);
            const uint32_t yc = __shfl_up_sync(0xffffffffu, c, off);
            if (lane >= off) {
                a += ya;
                c += yc;
            }
        }
        if (lane == 31) {
            s_warp[0][wid] = a;
            s_warp[1][wid] = c;
        }
        __syncthreads();
        if (wid == 0) {
            uint32_t wa = s_warp[0][lane], wc = s_warp[1][lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t ya = __shfl_up_sync(0xffffffffu, wa, off);
                const uint32_t yc = __shfl_up_sync(0xffffffffu, wc, off);
                if (lane >= off) {
                    wa += ya;
                    wc += yc;
                }
            }
            s_warp[0][lane] = wa;
            s_warp[1][lane] = wc;
        }
        __syncthreads();
        const uint32_t pre_a = (wid ? s_warp[0][wid - 1] : 0u) + a - cnt + s_carry[0];
        const uint32_t pre_c = (wid ? s_warp[1][wid - 1] : 0u) + c - nit + s_carry[1];
        if (row < B.n_rows) {
            B.row_off[row] = pre_a;
            for (uint32_t q = 0; q < nit; ++q) {
                const uint32_t it = pre_c + q;
                if (it < B.max_items) {
                    const uint32_t b0 = pre_a + q * chunk;
                    const uint32_t b1 = min(pre_a + cnt, b0 + chunk);
                    B.items[it] = make_uint4((uint32_t)row, b0, b1, 0u);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry[0] += s_warp[0][31];
            s_carry[1] += s_warp[1][31];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.row_off[B.n_rows] = s_carry[0];
        *B.n_items = min(s_carry[1], B.max_items);
    }
}

// Counting-sort scatter.  With the shared histogram each CTA counts its range
// again, reserves one block of positions per row with a single global atomic,
// then hands out positions inside the block with shared-memory atomics.
__global__ void k_bin_scatter(const BinP B) {
    extern __shared__ uint32_t hist[];   // [n_rows]: local counts, then next free position
    const uint64_t n = min((uint64_t)*B.arr_count, B.arr_cap);
    const unsigned lt = lanemask_lt();
    uint64_t b, e;
    cta_range(n, b, e);
    if (!B.priv_rows) {
        for (uint64_t idx = b + threadIdx.x; idx < e; idx += blockDim.x) {
            const uint4 a = B.arr[idx];
            const uint32_t row = a.x;
            const unsigned peers = __match_any_sync(__activemask(), row);
            const int leader = __ffs(peers) - 1;
            uint32_t base = 0;
            if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&B.row_fill[row], (uint32_t)__popc(peers));
            base = __shfl_sync(peers, base, leader);
            const uint32_t pos = B.row_off[row] + base + (uint32_t)__popc(peers & lt);
            B.sorted[pos] = make_float4(__uint_as_float(a.y), __uint_as_float(a.z), __uint_as_float(a.w), 0.f);
        }
        return;
    }
    for (int r = threadIdx.x; r < B.n_rows; r += blockDim.x) hist[r] = 0u;
    __syncthreads();
    for (uint64_t idx = b + threadIdx.x; idx < e; idx += blockDim.x) {
        const uint32_t row = B.arr[idx].x;
        const unsigned peers = __match_any_sync(__activemask(), row);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&hist[row], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int r = threadIdx.x; r < B.n_rows; r += blockDim.x) {
        const uint32_t c = hist[r];
        if (c) hist[r] = B.row_off[r] + atomicAdd(&B.row_fill[r], c);
    }
    __syncthreads();
    for (uint64_t idx = b + threadIdx.x; idx < e; idx += blockDim.x) {
        const uint4 a = B.arr[idx];
        const uint32_t row = a.x;
        const unsigned peers = __match_any_sync(__activemask(), row);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&hist[row], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        B.sorted[base + (uint32_t)__popc(peers & lt)] =
            make_float4(__uint_as_float(a.y), __uint_as_float(a.z), __uint_as_float(a.w), 0.f);
    }
}

// ceil / floor of a float-float value hi + lo
__device__ __forceinline__ int ff_ceil(float hi, float lo) {
    const float c = ceilf(hi);
    return (int)c + ((c == hi && lo > 0.f) ? 1 : 0);
}
__device__ __forceinline__ int ff_floor(float hi, float lo) {
    const float f = floorf(hi);
    return (int)f - ((f == hi && lo < 0.f) ? 1 : 0);
}

// One CTA per work item (a chunk of one row's arrivals): the row's complex
// samples accumulate in shared memory and are flushed with one global reduction
// each.  A warp loads 32 arrivals at once (one per lane, coalesced); each lane
// evaluates the carrier phase of its own arrival at that arrival's first tap,
// and the warp then deposits the 32 arrivals one after the other, lanes taking
// consecutive taps.  A lane's phase is the broadcast first-tap phase rotated by
// its lane offset, advanced by the exact rotation of 32 samples per step; the
// Gaussian envelope is evaluated per tap.
__global__ void __launch_bounds__(512) k_bin_deposit(const BinP B) {
    extern __shared__ float acc[];  // [2][n_s]: real, quadrature
    const uint32_t n_items = *B.n_items;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float rl_s, rl_c;   // carrier rotation over `lane` samples
    sincospif((float)lane * B.phase_per_sample, &rl_s, &rl_c);
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint4 item = B.items[it];
        for (int n = threadIdx.x; n < 2 * B.n_s; n += blockDim.x) acc[n] = 0.f;
        __syncthreads();
        for (uint32_t q0 = item.y + 32u * (uint32_t)wid; q0 < item.z; q0 += 32u * (uint32_t)nw) {
            const uint32_t q = q0 + (uint32_t)lane;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            int n0 = 0, n1 = -1;
            float bs = 0.f, bc = 1.f;
            if (q < item.z) {
                a = B.sorted[q];
                n0 = max(ff_ceil(a.x - B.K, a.y), 0);
                n1 = min(ff_floor(a.x + B.K, a.y), B.n_s - 1);
                sincospif((((float)n0 - a.x) - a.y) * B.phase_per_sample, &bs, &bc);
            }
            const int cnt = (int)min(32u, item.z - q0);
            for (int j = 0; j < cnt; ++j) {
                const int jn0 = __shfl_sync(0xffffffffu, n0, j);
                const int jn1 = __shfl_sync(0xffffffffu, n1, j);
                const float t_hi = __shfl_sync(0xffffffffu, a.x, j);
                const float t_lo = __shfl_sync(0xffffffffu, a.y, j);
                const float amp = __shfl_sync(0xffffffffu, a.z, j);
                const float js = __shfl_sync(0xffffffffu, bs, j);
                const float jc = __shfl_sync(0xffffffffu, bc, j);
                int n = jn0 + lane;
                if (n > jn1) continue;
                float sn = fmaf(js, rl_c, jc * rl_s);
                float cs = fmaf(jc, rl_c, -js * rl_s);
                float tau = ((float)n - t_hi) - t_lo;   // (n - t_hi) is exact
                for (;;) {
                    const float g = amp * exp2f(-tau * tau * B.inv_2s2_log2e);
                    atomicAdd(&acc[n], g * sn);
                    atomicAdd(&acc[B.n_s + n], -g * cs);
                    n += 32;
                    if (n > jn1) break;
                    tau += 32.f;
                    const float s2 = fmaf(sn, B.rot32_c, cs * B.rot32_s);
                    cs = fmaf(cs, B.rot32_c, -sn * B.rot32_s);
                    sn = s2;
                }
            }
        }
        __syncthreads();
        float *rf = B.rf + (size_t)item.x * B.n_s;
        float *qd = B.quad + (size_t)item.x * B.n_s;
        for (int n = threadIdx.x; n < B.n_s; n += blockDim.x) {
            const float vr = acc[n], vq = acc[B.n_s + n];
            if (vr != 0.f) atomicAdd(&rf[n], vr);
            if (vq != 0.f) atomicAdd(&qd[n], vq);
        }
        __syncthreads();
    }
}

__global__ void k_unpack_debug(const uint4 *arr, const uint2 *dbg, const unsigned long long *count, uint64_t cap_in,
                               const DebugOut D) {
    const uint64_t n = min(min((uint64_t)*count, cap_in), D.cap);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a = arr[i];
        const uint2 b = dbg[i];
        D.row[i] = a.x;
        D.t_hi[i] = __uint_as_float(a.y);
        D.t_lo[i] = __uint_as_float(a.z);
        D.amp[i] = __uint_as_float(a.w);
        D.ray[i] = b.x;
        D.event[i] = b.y;
    }
}

}  // namespace

void launch_unpack_debug(const uint4 *arr, const uint2 *dbg, const unsigned long long *count, uint64_t cap_in,
                         const DebugOut &D, cudaStream_t s) {
    k_unpack_debug<<<1024, 256, 0, s>>>(arr, dbg, count, cap_in, D);
}

int bin_sort_smem(int n_rows) {
    return n_rows <= kBinPrivRows ? n_rows * (int)sizeof(uint32_t) : 0;
}

void launch_bin_sort(const BinP &B, int sms, cudaStream_t s) {
    const int smem = B.priv_rows ? bin_sort_smem(B.n_rows) : 0;
    // CTAs per SM: up to 4 x 512 threads, fewer when the histogram is large
    const int per_sm = smem ? std::max(1, std::min(4, (200 << 10) / (smem + 1024))) : 4;
    const int grid = sms * per_sm;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k_bin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_bin_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
    k_bin_count<<<grid, 512, smem, s>>>(B);
    k_bin_plan<<<1, 1024, 0, s>>>(B);
    k_bin_scatter<<<grid, 512, smem, s>>>(B);
}

void launch_bin_deposit(const BinP &B, int sms, cudaStream_t s) {
    const int smem = 2 * B.n_s * (int)sizeof(float);
    cudaFuncSetAttribute(k_bin_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kMaxNs * (int)sizeof(float));
    k_bin_deposit<<<sms * 4, 512, smem, s>>>(B);
}

}  // namespace ur
