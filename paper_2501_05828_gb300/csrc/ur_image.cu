// Image formation: plane-wave delay-and-sum of the analytic channel data with
// coherent compounding over transmits, envelope, global maximum and log
// compression.  Delays are evaluated in float-float so that the interpolation
// position is exact to well below 1e-6 samples at any depth.
#include "ur_device.cuh"

namespace ur {
namespace {

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ int ff_floor_i(ff a) {
    const float f = floorf(a.hi);
    return (int)f - ((f == a.hi && a.lo < 0.f) ? 1 : 0);
}

// One thread per pixel; threadIdx.x runs along depth so neighbouring threads
// read neighbouring samples of the same channel.  CONVEX: element centres (x, z)
// from the table of a convex array, else on z = 0 at x_first + e pitch.
template <bool CONVEX>
__global__ void __launch_bounds__(256) k_das(const ImageP I) {
    extern __shared__ ff s_xe[];  // element centres, float-float: x [n_el] (then z [n_el] if CONVEX)
    for (int e = threadIdx.x; e < I.n_el; e += blockDim.x) {
        if (CONVEX) {
            s_xe[e] = I.elem_xz[2 * e];
            s_xe[I.n_el + e] = I.elem_xz[2 * e + 1];
        } else {
            const float pe = (float)e * I.pitch;
            const ff ep = {pe, __fmaf_rn((float)e, I.pitch, -pe)};
            s_xe[e] = ff_add(I.x_first, ep);
        }
    }
    __syncthreads();
    const int iz = blockIdx.x * blockDim.x + threadIdx.x;
    const int ix = blockIdx.y;
    const int img = blockIdx.z;
    const int q0 = I.img_items ? I.img_begin[img] : 0;
    const int q1 = I.img_items ? I.img_begin[img + 1] : I.n_tx;
    float env = 0.f;
    if (iz < I.nz) {
        const float x = I.x_px[ix], z = I.z_px[iz];
        const ff zz = ff_sqr_f(z);
        const float top = (float)(I.n_s - 1);
        float sr = 0.f, si = 0.f;
        for (int qi = q0; qi < q1; ++qi) {
            const int item = I.img_items ? I.img_items[qi] : qi;
            const int k = I.img_items ? I.item_angle[item] : item;
            // transmit delay to (x, z): plane wave; distance from a virtual source; through a focus
            const int kind = I.tx_kind ? I.tx_kind[k] : UR_TX_PLANE;
            ff T;
            if (kind == UR_TX_PLANE) {
                T = ff_add(ff_mul_f(x, I.tx_sin[k]), ff_mul_f(z, I.tx_cos[k]));
                T = ff_mul(ff_add(T, ff_neg(I.tx_m[k])), I.q);
            } else {
                const ff ddx = ff_add_f(ff_neg(I.tx_sin[k]), x), ddz = ff_add_f(ff_neg(I.tx_cos[k]), z);
                const ff r = ff_sqrt(ff_add(ff_mul(ddx, ddx), ff_mul(ddz, ddz)));
                if (kind == UR_TX_DIVERGING)
                    T = ff_mul(ff_add(r, ff_neg(I.tx_m[k])), I.q);
                else
                    T = ff_mul(ff_add(I.tx_m[k], (z >= I.tx_cos[k].hi) ? r : ff_neg(r)), I.q);
            }
            const float *rf = I.rf + (size_t)item * I.n_el * I.n_s;
            const float *qd = I.quad + (size_t)item * I.n_el * I.n_s;
            for (int e = 0; e < I.n_el; ++e) {
                const ff dx = ff_add_f(ff_neg(s_xe[e]), x);
                ff r2;
                if (CONVEX) {
                    const ff dz = ff_add_f(ff_neg(s_xe[I.n_el + e]), z);
                    r2 = ff_add(ff_mul(dz, dz), ff_mul(dx, dx));
                } else {
                    r2 = ff_add(zz, ff_mul(dx, dx));
                }
                const ff tau = ff_add(T, ff_mul(ff_sqrt(r2), I.q));
                if (tau.hi < 0.f || (tau.hi == 0.f && tau.lo < 0.f) || ff_gt(tau, top)) continue;
                const int i0 = ff_floor_i(tau);
                const float f = ((tau.hi - (float)i0) + tau.lo);
                const int i1 = min(i0 + 1, I.n_s - 1);
                const size_t row = (size_t)e * I.n_s;
                const float a0 = __ldg(rf + row + i0), a1 = __ldg(rf + row + i1);
                const float b0 = __ldg(qd + row + i0), b1 = __ldg(qd + row + i1);
                sr += a0 * (1.f - f) + a1 * f;
                si += b0 * (1.f - f) + b1 * f;
            }
        }
        const size_t px = ((size_t)img * I.nz + iz) * I.nx + ix;
        if (I.iq) I.iq[px] = make_float2(sr, si);
        env = sqrtf(sr * sr + si * si);
        if (I.env) I.env[px] = env;
    }
    const unsigned int m = __reduce_max_sync(0xffffffffu, __float_as_uint(env));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&I.env_max[img], m);
}

__global__ void k_log(const ImageP I) {
    const int n = I.nx * I.nz;
    const int img = blockIdx.y;
    const float mx = __uint_as_float(I.env_max[img]);
    const float *env = I.env + (size_t)img * n;
    float *db = I.db + (size_t)img * n;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float e = env[p];
        float v = (mx > 0.f && e > 0.f) ? 20.f * log10f(e / mx) : -I.dyn_range_db;
        db[p] = fmaxf(v, -I.dyn_range_db);
    }
}

}  // namespace

void launch_das(const ImageP &I, cudaStream_t s) {
    dim3 grid((I.nz + 255) / 256, I.nx, I.img_items ? I.n_images : 1);
    if (I.elem_xz)
        k_das<true><<<grid, 256, 2 * I.n_el * sizeof(ff), s>>>(I);
    else
        k_das<false><<<grid, 256, I.n_el * sizeof(ff), s>>>(I);
}

void launch_log(const ImageP &I, cudaStream_t s) {
    const int n = I.nx * I.nz;
    dim3 grid(min(4096, (n + 255) / 256), I.img_items ? I.n_images : 1);
    k_log<<<grid, 256, 0, s>>>(I);
}

}  // namespace ur
