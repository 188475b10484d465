// Binning of arrivals into the analytic channel data (Eq. 14, deposited at the
// exact arrival time).  Arrivals are counting-sorted by row (transmit x element)
// and cut into work items of at most `chunk` arrivals; one CTA accumulates an
// item's pulse taps for its whole row in shared memory (n_s complex samples)
// with shared-memory atomics and flushes the row with coalesced global
// reductions.
#include "ur_device.cuh"

namespace ur {
namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    return (1u << (threadIdx.x & 31)) - 1u;
}

__global__ void k_bin_count(const BinP B) {
    const uint64_t n = min((uint64_t)*B.arr_count, B.arr_cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const uint32_t row = B.arr[idx].x;
        const unsigned peers = __match_any_sync(__activemask(), row);
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&B.row_count[row], (uint32_t)__popc(peers));
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
    for (int base = 0; base < B.n_rows; base += 1024) {
        const int row = base + (int)threadIdx.x;
        const uint32_t cnt = row < B.n_rows ? B.row_count[row] : 0u;
        const uint32_t nit = row < B.n_rows ? max(1u, (cnt + B.chunk - 1) / B.chunk) : 0u;
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
                    const uint32_t b0 = pre_a + q * B.chunk;
                    const uint32_t b1 = min(pre_a + cnt, b0 + B.chunk);
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

__global__ void k_bin_scatter(const BinP B) {
    const uint64_t n = min((uint64_t)*B.arr_count, B.arr_cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
        const uint4 a = B.arr[idx];
        const uint32_t row = a.x;
        const unsigned peers = __match_any_sync(__activemask(), row);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&B.row_fill[row], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        const uint32_t pos = B.row_off[row] + base + (uint32_t)__popc(peers & lanemask_lt());
        B.sorted[pos] = make_float4(__uint_as_float(a.y), __uint_as_float(a.z), __uint_as_float(a.w), 0.f);
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

__global__ void __launch_bounds__(512) k_bin_deposit(const BinP B) {
    extern __shared__ float acc[];  // [2][n_s]: real, quadrature
    const uint32_t n_items = *B.n_items;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint4 item = B.items[it];
        for (int n = threadIdx.x; n < 2 * B.n_s; n += blockDim.x) acc[n] = 0.f;
        __syncthreads();
        for (uint32_t q = item.y + (uint32_t)wid; q < item.z; q += (uint32_t)nw) {
            const float4 a = B.sorted[q];
            const int n0 = max(ff_ceil(a.x - B.K, a.y), 0);
            const int n1 = min(ff_floor(a.x + B.K, a.y), B.n_s - 1);
            for (int n = n0 + lane; n <= n1; n += 32) {
                const float tau = ((float)n - a.x) - a.y;   // (n - t_hi) is exact
                const float g = a.z * expf(-tau * tau * B.inv_2s2);
                float sn, cs;
                sincospif(tau * B.phase_per_sample, &sn, &cs);
                atomicAdd(&acc[n], g * sn);
                atomicAdd(&acc[B.n_s + n], -g * cs);
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

void launch_bin_sort(const BinP &B, int sms, cudaStream_t s) {
    const int blk = 256;
    const int grid = sms * 8;
    k_bin_count<<<grid, blk, 0, s>>>(B);
    k_bin_plan<<<1, 1024, 0, s>>>(B);
    k_bin_scatter<<<grid, blk, 0, s>>>(B);
}

void launch_bin_deposit(const BinP &B, int sms, cudaStream_t s) {
    const int smem = 2 * B.n_s * (int)sizeof(float);
    cudaFuncSetAttribute(k_bin_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kMaxNs * (int)sizeof(float));
    k_bin_deposit<<<sms * 2, 512, smem, s>>>(B);
}

}  // namespace ur
