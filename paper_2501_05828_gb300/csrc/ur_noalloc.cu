// ur_beamform_noalloc: delay-and-sum, envelope and log compression for callers
// that may not allocate device memory.  All per-call scratch (transmit tables,
// pixel coordinates, the envelope maximum and, if the caller passes no envelope
// buffer, the envelope itself) lives in one file-scope device array that every
// GPU loading the library holds until the process exits.  The transmit angles
// travel to the table kernel as a by-value kernel parameter, so no copy reads
// the context's host memory.
#include "ultraray.h"
#include "ur_device.cuh"

#include <cmath>
#include <mutex>

namespace {

constexpr int kMaxDevices = 64;

struct Scratch {
    unsigned int env_max;
    unsigned int pad[63];
    ur::ff tx_sin[UR_NOALLOC_MAX_TX], tx_cos[UR_NOALLOC_MAX_TX], tx_m[UR_NOALLOC_MAX_TX];
    float px[2 * UR_NOALLOC_MAX_AXIS];
    float env[UR_NOALLOC_MAX_PIXELS];
};
static_assert(sizeof(Scratch) <= UR_NOALLOC_SCRATCH_BYTES, "scratch exceeds its documented size");

// The scratch itself.  Host code must not use this name as an address: in host
// code it is only a stand-in, the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[UR_NOALLOC_SCRATCH_BYTES];

Scratch *g_dev_ptr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Device address of the scratch on `device` (which must be current); looked up
// once per device.
cudaError_t scratch_on(int device, Scratch **out) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_dev_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[device] = static_cast<Scratch *>(p);
    }
    *out = g_dev_ptr[device];
    return cudaSuccess;
}

__device__ __forceinline__ ur::ff split_dev(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

// The transmit angles, passed by value (4 KiB of kernel parameters).
struct Angles {
    float a[UR_NOALLOC_MAX_TX];
};

// Per-transmit tables of the delay-and-sum (sin, cos, min_e x_e sin) in double,
// split into float-float, like the context's own tables.
__global__ void k_tables(Scratch *S, const __grid_constant__ Angles ang, int n_tx, int n_el, float pitch) {
    for (int k = threadIdx.x; k < n_tx; k += blockDim.x) {
        const double th = (double)ang.a[k];
        const double sn = sin(th), cs = cos(th);
        const double x0 = -0.5 * (double)(n_el - 1) * (double)pitch;
        double mn = INFINITY;
        for (int e = 0; e < n_el; ++e) mn = fmin(mn, (x0 + e * (double)pitch) * sn);
        S->tx_sin[k] = split_dev(sn);
        S->tx_cos[k] = split_dev(cs);
        S->tx_m[k] = split_dev(mn);
    }
}

// Device (or managed) memory of `device`: memory of another GPU would be a peer
// access the kernels are not set up for.
bool on_device(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" ur_status ur_beamform_noalloc(ur_ctx *ctx, const float *rf, const float *quad, const float *x_px, int nx,
                                         const float *z_px, int nz, float dyn_range_db, float *iq, float *env,
                                         float *db) {
    ur::CtxView v;
    if (!ctx) return UR_ERR_INVALID_ARG;
    if (!ur::ctx_view(ctx, &v)) return UR_ERR_STATE;
    if (!v.plane_waves || !v.linear) return UR_ERR_INVALID_ARG;   // its tables hold plane waves of a linear array
    if (!rf || !quad || !x_px || !z_px || (!iq && !env && !db)) return UR_ERR_INVALID_ARG;
    if (v.n_tx > UR_NOALLOC_MAX_TX || nx < 1 || nz < 1 || nx > UR_NOALLOC_MAX_AXIS || nz > UR_NOALLOC_MAX_AXIS)
        return UR_ERR_INVALID_ARG;
    if (!env && (long long)nx * nz > UR_NOALLOC_MAX_PIXELS) return UR_ERR_INVALID_ARG;
    if (db && !(dyn_range_db > 0.f)) return UR_ERR_INVALID_ARG;
    const int dev = v.device;
    if (!on_device(rf, dev) || !on_device(quad, dev) || (iq && !on_device(iq, dev)) ||
        (env && !on_device(env, dev)) || (db && !on_device(db, dev)))
        return UR_ERR_INVALID_ARG;
    if (cudaSetDevice(dev) != cudaSuccess) return UR_ERR_CUDA;
    // An error left by earlier, unrelated work stays where it is: it is reported, not cleared.
    if (cudaPeekAtLastError() != cudaSuccess) return UR_ERR_CUDA;
    Scratch *S = nullptr;
    if (scratch_on(v.device, &S) != cudaSuccess) {
        cudaGetLastError();
        return UR_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)v.stream;
    Angles ang;
    for (int k = 0; k < v.n_tx; ++k) ang.a[k] = v.angles[k];
    if (cudaMemcpyAsync(S->px, x_px, sizeof(float) * nx, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(S->px + nx, z_px, sizeof(float) * nz, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemsetAsync(&S->env_max, 0, sizeof(unsigned int), s) != cudaSuccess) {
        cudaGetLastError();
        return UR_ERR_CUDA;
    }
    k_tables<<<1, 256, 0, s>>>(S, ang, v.n_tx, v.arr.n_el, v.arr.pitch);
    if (cudaGetLastError() != cudaSuccess) return UR_ERR_CUDA;
    ur::ImageP I{};
    I.rf = rf;
    I.quad = quad;
    I.n_tx = v.n_tx;
    I.n_el = v.arr.n_el;
    I.n_s = v.arr.n_s;
    I.x_px = S->px;
    I.z_px = S->px + nx;
    I.nx = nx;
    I.nz = nz;
    const double q = (double)v.arr.fs / (double)v.arr.c_bf;
    const double xf = -0.5 * (double)(v.arr.n_el - 1) * (double)v.arr.pitch;
    I.q = {(float)q, (float)(q - (double)(float)q)};
    I.x_first = {(float)xf, (float)(xf - (double)(float)xf)};
    I.pitch = v.arr.pitch;
    I.tx_sin = S->tx_sin;
    I.tx_cos = S->tx_cos;
    I.tx_m = S->tx_m;
    I.iq = (float2 *)iq;
    I.env = env ? env : S->env;
    I.db = db;
    I.env_max = &S->env_max;
    I.dyn_range_db = dyn_range_db;
    ur::launch_das(I, s);
    if (cudaGetLastError() != cudaSuccess) return UR_ERR_CUDA;
    if (db) {
        ur::launch_log(I, s);
        if (cudaGetLastError() != cudaSuccess) return UR_ERR_CUDA;
    }
    return UR_OK;
}
