// Primary-ray tracer: emission (Eq. 6), traversal with reflection/refraction
// at analytic boundaries (Eqs. 7-11), transducer sampling of point scatterers
// through straight connection rays with the receive directivity (Eq. 13), and
// recording of returns to the aperture.  FP32 geometry, float-float time of
// flight; arrivals are appended to a global queue for the binning stage.
#include "ur_device.cuh"

namespace ur {
namespace {

// Nearest boundary hit along o + t d, t in (kTmin, inf).  `skip` is the
// primitive the ray is leaving: a plane cannot be met again, a sphere or
// cylinder only at its far root.  With `terminals`, the array plane z = 0
// (id n_bnd, upward rays) and the absorbing plane z = z_max (id n_bnd + 1,
// downward rays) take part.
__device__ __forceinline__ int nearest(const SceneP &S, float3 o, float3 d, int skip, bool terminals,
                                       float &t_out) {
    float best = INFINITY;
    int hit = -1;
    for (int p = 0; p < S.n_bnd; ++p) {
        const Bnd &B = S.bnd[p];
        float t;
        if (B.kind == kPlaneZ) {
            if (p == skip || d.z == 0.f) continue;
            t = (B.p[0] - o.z) / d.z;
        } else if (B.kind == kSphere) {
            const float3 oc = make_float3(o.x - B.p[0], o.y - B.p[1], o.z - B.p[2]);
            const float b = dot3(oc, d);
            if (p == skip) {
                t = -2.f * b;
            } else {
                const float3 f = oc - b * d;
                const float disc = B.p[3] * B.p[3] - dot3(f, f);
                if (disc < 0.f) continue;
                const float s = sqrtf(disc);
                t = -b - s;
                if (!(t > kTmin)) t = -b + s;
            }
        } else {
            const float ocx = o.x - B.p[0], ocz = o.z - B.p[1];
            const float a = d.x * d.x + d.z * d.z;
            if (a == 0.f) continue;
            const float b = (ocx * d.x + ocz * d.z) / a;
            if (p == skip) {
                t = -2.f * b;
            } else {
                const float fx = ocx - b * d.x, fz = ocz - b * d.z;
                const float disc = (B.p[2] * B.p[2] - (fx * fx + fz * fz)) / a;
                if (disc < 0.f) continue;
                const float s = sqrtf(disc);
                t = -b - s;
                if (!(t > kTmin)) t = -b + s;
            }
        }
        if (t > kTmin && t < best) {
            best = t;
            hit = p;
        }
    }
    if (terminals) {
        if (d.z < 0.f) {
            const float t = -o.z / d.z;
            if (t > kTmin && t < best) {
                best = t;
                hit = S.n_bnd;
            }
        } else if (d.z > 0.f) {
            const float t = (S.z_max - o.z) / d.z;
            if (t > kTmin && t < best) {
                best = t;
                hit = S.n_bnd + 1;
            }
        }
    }
    t_out = best;
    return hit;
}

__device__ __forceinline__ float3 outward(const Bnd &B, float3 h) {
    if (B.kind == kPlaneZ) return make_float3(0.f, 0.f, 1.f);
    if (B.kind == kSphere) return unit3(make_float3(h.x - B.p[0], h.y - B.p[1], h.z - B.p[2]));
    return unit3(make_float3(h.x - B.p[0], 0.f, h.z - B.p[1]));
}

// Snell (speed ratio) and the fluid-fluid pressure reflection coefficient.
// Returns false on total internal reflection.
__device__ __forceinline__ bool fresnel(float cos_i, float c1, float Z1, float c2, float Z2, float &r,
                                        float &cos_t) {
    const float eta = c2 / c1;
    const float k = 1.f - eta * eta * (1.f - cos_i * cos_i);
    if (k < 0.f) return false;
    cos_t = sqrtf(k);
    r = (Z2 * cos_i - Z1 * cos_t) / (Z2 * cos_i + Z1 * cos_t);
    return true;
}

// Eq. 13 through cosines: 1 inside the main beam, 0 beyond the cutoff, linear in angle between.
__device__ __forceinline__ float directivity(const TraceP &P, float cos_a) {
    if (cos_a >= P.cos_am) return 1.f;
    if (cos_a < P.cos_ac) return 0.f;
    const float al = acosf(fminf(cos_a, 1.f));
    return (P.ac - al) / (P.ac - P.am);
}

// Straight connection ray from p to the element centre (x_e, 0, 0): product of
// sqrt(1 - R) over the boundaries it crosses (0 if one reflects totally),
// travel time (samples) and attenuation exponent.
__device__ float connection(const SceneP &S, float3 p, int med, float xe, ff &t_conn, float &att) {
    float3 o = p;
    float3 w = make_float3(xe - p.x, -p.y, -p.z);
    float rem = sqrtf(dot3(w, w));
    w = make_float3(w.x / rem, w.y / rem, w.z / rem);
    float fac = 1.f, a = 0.f;
    ff t = {0.f, 0.f};
    int m = med, skip = -1;
    for (int it = 0; it < kMaxCross; ++it) {
        float th;
        const int hit = nearest(S, o, w, skip, false, th);
        const Medium &M = S.med[m];
        if (hit < 0 || th >= rem) {
            t = ff_add(t, ff_mul_f(rem, M.slow));
            a += M.a * rem;
            break;
        }
        t = ff_add(t, ff_mul_f(th, M.slow));
        a += M.a * th;
        float3 h = o + th * w;
        const Bnd &B = S.bnd[hit];
        if (B.kind == kPlaneZ) h.z = B.p[0];
        const float3 n = outward(B, h);
        const float dn = dot3(w, n);
        const int m2 = dn > 0.f ? B.med_pos : B.med_neg;
        float r, ct;
        if (!fresnel(fabsf(dn), M.c, M.Z, S.med[m2].c, S.med[m2].Z, r, ct)) return 0.f;
        fac *= sqrtf(1.f - r * r);
        m = m2;
        o = h;
        rem -= th;
        skip = hit;
    }
    t_conn = t;
    att = a;
    return fac;
}

// Warp-aggregated append to the arrival queue (one atomic per converged group).
template <bool DBG>
__device__ __forceinline__ void emit(const TraceP &P, uint32_t row, ff t, float amp, uint32_t ray, uint32_t ev) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(P.arr_count, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    const unsigned long long idx = base + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
    if (idx < P.arr_cap) {
        P.arr[idx] = make_uint4(row, __float_as_uint(t.hi), __float_as_uint(t.lo), __float_as_uint(amp));
        if (DBG) P.arr_dbg[idx] = make_uint2(ray, ev);
    }
}

struct Counters {
    uint32_t rays, segments, interactions, candidates, connections, arrivals;
};

// A scatterer within r_s of the segment: choose an element uniformly (Philox
// keyed by ray, transmit, segment and scatterer), weigh by Eq. 13 and cast the
// connection ray.
template <bool DBG>
__device__ __forceinline__ void scatter_event(const TraceP &P, uint32_t i, uint32_t k, float4 q, float tca, ff t,
                                              float w, int med, int b, Counters &cn) {
    const uint32_t j = __float_as_uint(q.w);
    const uint4 x = philox(make_uint4(i, k, 2u | ((uint32_t)b << 8), j), P.key);
    const uint32_t e = (uint32_t)(((uint64_t)(x.x >> 8) * (uint64_t)P.n_el) >> 24);
    const float xe = P.x_first + (float)e * P.pitch;
    const float vx = xe - q.x;
    const float D = sqrtf(vx * vx + q.y * q.y + q.z * q.z);
    const float fd = directivity(P, q.z / D);
    cn.candidates++;
    if (!(fd > 0.f)) return;
    cn.connections++;
    ff tc;
    float att;
    const float fac = connection(P.S, make_float3(q.x, q.y, q.z), med, xe, tc, att);
    if (fac == 0.f) return;
    const Medium &M = P.S.med[med];
    const ff ta = ff_add(ff_add(t, ff_mul_f(tca, M.slow)), tc);
    if (ff_gt(ta, P.t_last)) return;
    const float amp = w * expf(-M.a * tca) * P.S.amp[j] * (float)P.n_el * fd * fac * expf(-att);
    emit<DBG>(P, k * (uint32_t)P.n_el + e, ta, amp, i, ((uint32_t)b << 24) | j);
    cn.arrivals++;
}

// Every scatterer whose closest approach to the open segment o + t d,
// 0 < t < seg, is closer than r_s.  Uniform grid walked with a 3D DDA; each
// cell tests only closest-approach parameters inside its own [t_enter, t_exit)
// range, so a scatterer referenced by several cells is found exactly once.
template <bool DBG>
__device__ void segment_scatterers(const TraceP &P, uint32_t i, uint32_t k, float3 o, float3 d, float seg, ff t,
                                   float w, int med, int b, Counters &cn) {
    const SceneP &S = P.S;
    const float hi_x = S.g_lo.x + (float)S.g_dim.x * S.g_h.x;
    const float hi_y = S.g_lo.y + (float)S.g_dim.y * S.g_h.y;
    const float hi_z = S.g_lo.z + (float)S.g_dim.z * S.g_h.z;
    float t0 = 0.f, t1 = seg;
    const float ix = 1.f / d.x, iy = 1.f / d.y, iz = 1.f / d.z;
    if (d.x != 0.f) {
        const float ta = (S.g_lo.x - o.x) * ix, tb = (hi_x - o.x) * ix;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    } else if (o.x < S.g_lo.x || o.x > hi_x) {
        return;
    }
    if (d.y != 0.f) {
        const float ta = (S.g_lo.y - o.y) * iy, tb = (hi_y - o.y) * iy;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    } else if (o.y < S.g_lo.y || o.y > hi_y) {
        return;
    }
    if (d.z != 0.f) {
        const float ta = (S.g_lo.z - o.z) * iz, tb = (hi_z - o.z) * iz;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    } else if (o.z < S.g_lo.z || o.z > hi_z) {
        return;
    }
    if (!(t0 < t1)) return;

    int cx = (int)floorf((o.x + t0 * d.x - S.g_lo.x) * S.g_inv_h.x);
    int cy = (int)floorf((o.y + t0 * d.y - S.g_lo.y) * S.g_inv_h.y);
    int cz = (int)floorf((o.z + t0 * d.z - S.g_lo.z) * S.g_inv_h.z);
    cx = min(max(cx, 0), S.g_dim.x - 1);
    cy = min(max(cy, 0), S.g_dim.y - 1);
    cz = min(max(cz, 0), S.g_dim.z - 1);
    const int sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0);
    const int sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
    const int sz = d.z > 0.f ? 1 : (d.z < 0.f ? -1 : 0);
    const float tdx = sx ? S.g_h.x * fabsf(ix) : INFINITY;
    const float tdy = sy ? S.g_h.y * fabsf(iy) : INFINITY;
    const float tdz = sz ? S.g_h.z * fabsf(iz) : INFINITY;
    float tmx = sx ? (S.g_lo.x + (float)(cx + (sx > 0)) * S.g_h.x - o.x) * ix : INFINITY;
    float tmy = sy ? (S.g_lo.y + (float)(cy + (sy > 0)) * S.g_h.y - o.y) * iy : INFINITY;
    float tmz = sz ? (S.g_lo.z + (float)(cz + (sz > 0)) * S.g_h.z - o.z) * iz : INFINITY;

    float t_enter = -INFINITY;
    const int guard_max = S.g_dim.x + S.g_dim.y + S.g_dim.z + 3;
    for (int guard = 0; guard < guard_max; ++guard) {
        const int axis = (tmx <= tmy && tmx <= tmz) ? 0 : (tmy <= tmz ? 1 : 2);
        const float t_exit = axis == 0 ? tmx : (axis == 1 ? tmy : tmz);
        bool last = !(t_exit < t1);
        if (!last) {
            const int nc = axis == 0 ? cx + sx : (axis == 1 ? cy + sy : cz + sz);
            const int dm = axis == 0 ? S.g_dim.x : (axis == 1 ? S.g_dim.y : S.g_dim.z);
            last = nc < 0 || nc >= dm;
        }
        const float t_acc = last ? INFINITY : t_exit;
        const uint32_t cell = ((uint32_t)cz * (uint32_t)S.g_dim.y + (uint32_t)cy) * (uint32_t)S.g_dim.x + (uint32_t)cx;
        const uint32_t r0 = S.cell_start[cell], r1 = S.cell_start[cell + 1];
        for (uint32_t r = r0; r < r1; ++r) {
            const float4 q = S.refs[r];
            const float3 v = make_float3(q.x - o.x, q.y - o.y, q.z - o.z);
            const float tca = dot3(v, d);
            if (!(tca > 0.f && tca < seg)) continue;
            if (tca < t_enter || !(tca < t_acc)) continue;
            const float3 pe = v - tca * d;
            if (!(dot3(pe, pe) < S.r2)) continue;
            scatter_event<DBG>(P, i, k, q, tca, t, w, med, b, cn);
        }
        if (last) break;
        t_enter = t_exit;
        if (axis == 0) {
            cx += sx;
            tmx += tdx;
        } else if (axis == 1) {
            cy += sy;
            tmy += tdy;
        } else {
            cz += sz;
            tmz += tdz;
        }
    }
}

// One primary ray: emission (Eq. 6) and traversal until termination.
template <bool DBG>
__device__ void trace_ray(const TraceP &P, uint32_t i, uint32_t k, uint32_t e, Counters &cn) {
    const SceneP &S = P.S;
    const uint4 x = philox(make_uint4(i, k, 0u, 0u), P.key);
    const float2 sc = P.txdir[k];
    const float xe = P.x_first + (float)e * P.pitch;
    float3 o = make_float3(xe + (u24(x.x) - 0.5f) * P.pitch, (u24(x.y) - 0.5f) * P.H, 0.f);
    float3 d = make_float3(sc.x, 0.f, sc.y);
    ff t = P.delay[k * (uint32_t)P.n_el + e];
    float w = sc.y * P.inv_n;
    int med = S.med_array, b = 0, prev = -1, reason = kEndPath;
    float L = 0.f;
    uint64_t h = kFnvOffset;
    for (int guard = 0; guard < kMaxSeg; ++guard) {
        float th;
        const int hit = nearest(S, o, d, prev, true, th);
        float seg = th;
        bool clipped = false;
        if (L + seg > P.max_path) {
            seg = P.max_path - L;
            clipped = true;
        }
        cn.segments++;
        if (S.n_scat > 0) segment_scatterers<DBG>(P, i, k, o, d, seg, t, w, med, b, cn);
        const Medium &M = S.med[med];
        t = ff_add(t, ff_mul_f(seg, M.slow));
        w *= expf(-M.a * seg);
        L += seg;
        o = o + seg * d;
        if (clipped) {
            reason = kEndPath;
            break;
        }
        if (hit == S.n_bnd) {  // array plane: only paths returning to the aperture are kept
            o.z = 0.f;
            const float xl = P.x_first - 0.5f * P.pitch;
            if (fabsf(o.y) <= 0.5f * P.H && o.x >= xl && o.x < xl + (float)P.n_el * P.pitch) {
                int el = (int)floorf((o.x - xl) / P.pitch);
                if (el > P.n_el - 1) el = P.n_el - 1;
                const float fd = directivity(P, -d.z);
                if (fd > 0.f && !ff_gt(t, P.t_last)) {
                    emit<DBG>(P, k * (uint32_t)P.n_el + (uint32_t)el, t, w * fd, i, 0x80000000u | ((uint32_t)b << 24));
                    cn.arrivals++;
                }
                reason = kEndAperture;
            } else {
                reason = kEndArrayMiss;
            }
            break;
        }
        if (hit == S.n_bnd + 1) {
            reason = kEndBottom;
            break;
        }
        const Bnd &B = S.bnd[hit];
        if (B.kind == kPlaneZ) o.z = B.p[0];
        if (ff_gt(t, P.t_last)) {
            reason = kEndTime;
            break;
        }
        if (b >= P.max_b) {
            reason = kEndMaxB;
            break;
        }
        // boundary interaction (Eqs. 7-11), Monte Carlo choice reflect if y < r^2
        const float3 n_out = outward(B, o);
        const float dn = dot3(d, n_out);
        const int m2 = dn > 0.f ? B.med_pos : B.med_neg;
        const float3 n = dn > 0.f ? make_float3(-n_out.x, -n_out.y, -n_out.z) : n_out;
        const float cos_i = -dot3(n, d);
        const float3 dr = unit3(d + (2.f * cos_i) * n);
        const Medium &M2 = S.med[m2];
        float r, cos_t;
        uint32_t branch;
        if (!fresnel(cos_i, M.c, M.Z, M2.c, M2.Z, r, cos_t)) {
            branch = 2;
            d = dr;
        } else {
            const float R = r * r;
            const uint4 y = philox(make_uint4(i, k, 1u | ((uint32_t)b << 8), 0u), P.key);
            if (u24(y.x) < R) {
                branch = 0;
                w *= r / R;
                d = dr;
            } else {
                branch = 1;
                const float eta = M2.c / M.c;
                w *= 1.f / sqrtf(1.f - R);
                d = unit3(eta * d + (eta * cos_i - cos_t) * n);
                med = m2;
            }
        }
        cn.interactions++;
        if (DBG) h = fnv_step(h, 0x10000u | ((uint32_t)hit << 4) | branch);
        b += 1;
        prev = hit;
    }
    if (DBG) P.path_hash[(uint64_t)k * P.n_rays + i] = fnv_step(h, 0x20000u | (uint32_t)reason);
    cn.rays++;
}

// Slots are element-major so that a warp traces neighbouring rays of one
// element (coherent scatterer-grid cells); slot -> ray i = m * n_el + e.
template <bool DBG>
__global__ void __launch_bounds__(256) k_trace(const __grid_constant__ TraceP P, uint64_t n_slots) {
    Counters cn = {0, 0, 0, 0, 0, 0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_slots; g += stride) {
        const uint32_t m = (uint32_t)(g % P.rays_per_el);
        const uint64_t q = g / P.rays_per_el;
        const uint32_t e = (uint32_t)(q % (uint64_t)P.n_el);
        const uint32_t k = (uint32_t)(q / (uint64_t)P.n_el);
        const uint32_t i = m * (uint32_t)P.n_el + e;
        if (i < P.n_rays) trace_ray<DBG>(P, i, k, e, cn);
    }
    if (P.stats) {
        const uint32_t v[6] = {cn.rays, cn.segments, cn.interactions, cn.candidates, cn.connections, cn.arrivals};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const uint32_t s = __reduce_add_sync(0xffffffffu, v[c]);
            if ((threadIdx.x & 31) == 0 && s) atomicAdd(&P.stats[c], (unsigned long long)s);
        }
    }
}

}  // namespace

int trace_occupancy(int block, bool debug) {
    int n = 0;
    if (debug)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false>, block, 0);
    return n > 0 ? n : 1;
}

void launch_trace(const TraceP &P, bool debug, int block, int grid, cudaStream_t s) {
    const uint64_t n_slots = (uint64_t)P.n_tx * (uint64_t)P.n_el * (uint64_t)P.rays_per_el;
    if (debug)
        k_trace<true><<<grid, block, 0, s>>>(P, n_slots);
    else
        k_trace<false><<<grid, block, 0, s>>>(P, n_slots);
}

}  // namespace ur
