// Primary-ray tracer: emission (Eq. 6), traversal with reflection/refraction
// at analytic boundaries (Eqs. 7-11), transducer sampling of point scatterers
// through straight connection rays with the receive directivity (Eq. 13), and
// recording of returns to the aperture.  FP32 geometry, float-float time of
// flight; arrivals are appended to a global queue for the binning stage.
#include "ur_device.cuh"

namespace ur {
namespace {

// Philox blocks of the plane-wave tracer come from one out-of-line copy: the kernel's hot loop
// stays smaller, and instruction fetch is its first stall (layered frame 8.59 -> 8.17 ms); the
// extended tracers keep them inline (there the call cost more than the code it saved).
__device__ __noinline__ uint4 philox_outline(uint4 c, uint2 k) { return philox(c, k); }

template <bool INLINE>
__device__ __forceinline__ uint4 draw(uint4 c, uint2 k) { return INLINE ? philox(c, k) : philox_outline(c, k); }

// Straight connection ray from p to the element centre (x_e, 0, 0): product of
// sqrt(1 - R) over the boundaries it crosses (0 if one reflects totally),
// travel time (samples) and attenuation exponent.  skip0: the boundary p lies
// on (-1 inside a medium).
template <bool MESH>
__device__ float connection(const SceneP &S, float3 p, int med, int skip0, float xe, ff &t_conn, float &att) {
    float3 o = p;
    float3 w = make_float3(xe - p.x, -p.y, -p.z);
    const float w2 = dot3(w, w), iw = rsqrtf(w2);
    float rem = sqrtf(w2);   // the length sets the travel time: correctly rounded
    w = make_float3(w.x * iw, w.y * iw, w.z * iw);
    float fac = 1.f, a = 0.f;
    ff t = {0.f, 0.f};
    int m = med, skip = skip0;
    for (int it = 0; it < kMaxCross; ++it) {
        float th;
        const int hit = nearest<MESH>(S, o, w, skip, false, th);
        const Medium &M = S.med[m];
        if (hit < 0 || th >= rem) {
            t = ff_add(t, ff_mul_f(rem, M.slow));
            a += M.a * rem;
            break;
        }
        t = ff_add(t, ff_mul_f(th, M.slow));
        a += M.a * th;
        float3 h = o + th * w, n;
        int m_neg, m_pos;
        float alpha;
        surface<MESH>(S, hit, h, n, m_neg, m_pos, alpha);
        const float dn = dot3(w, n);
        const int m2 = dn > 0.f ? m_pos : m_neg;
        float r, ct;
        if (!fresnel(fabsf(dn), M.c, M.Z, S.med[m2].c, S.med[m2].Z, r, ct)) return 0.f;
        fac *= sqrtf(transmitted(fabsf(dn), ct, M.Z, S.med[m2].Z));
        m = m2;
        o = h;
        rem -= th;
        skip = hit;
    }
    t_conn = t;
    att = a;
    return fac;
}

// ---------------------------------------------------------------- rough boundaries (Eq. 12)
constexpr float kPiF = 3.14159265358979f;

// GGX density of microfacet normals at c = n.h, a2 = alpha^2; the denominator
// written as (1 - c^2) + a2 c^2 stays positive when c rounds to 1.
__device__ __forceinline__ float ggx_d(float c, float a2) {
    if (!(c > 0.f)) return 0.f;
    const float c2 = c * c;
    const float k = fmaf(a2, c2, 1.f - c2);
    return a2 / (kPiF * k * k);
}

// Smith masking of one direction at cosine c to the macro normal.
__device__ __forceinline__ float ggx_g1(float c, float a2) {
    const float t2 = (1.f - c * c) / (c * c);
    return 2.f / (1.f + sqrtf(1.f + a2 * t2));
}

// Microfacet normal with density D(m)(m.n) about unit n: tan^2 theta = alpha^2 xi1 / (1 - xi1),
// phi = 2 pi xi2, in the tangent frame of Duff et al. (JCGT 2017).
__device__ __forceinline__ float3 ggx_sample(float3 n, float a2, float xi1, float xi2, float &ct) {
    const float tan2 = a2 * xi1 / (1.f - xi1);
    ct = 1.f / sqrtf(1.f + tan2);
    const float st = sqrtf(tan2) * ct;
    float sp, cp;
    sincospif(2.f * xi2, &sp, &cp);
    const float sg = n.z >= 0.f ? 1.f : -1.f;
    const float a = -1.f / (sg + n.z);
    const float b = n.x * n.y * a;
    const float3 t1 = make_float3(1.f + sg * n.x * n.x * a, sg * b, -sg * n.x);
    const float3 t2 = make_float3(b, sg + n.y * n.y * a, -n.y);
    return (st * cp) * t1 + (st * sp) * t2 + ct * n;
}

// Scattering of a rough boundary from incident direction d (n: unit macro normal
// on the incident side) into o: returns f |o.n| in the amplitude form (r or
// sqrt(1 - R) of the half-vector microfacet) and the solid-angle density of o
// under microfacet sampling and the reflect-if-y < R branch.
__device__ float rough_eval(float3 d, float3 n, float3 o, float a2, const Medium &M1, const Medium &M2,
                           float &pdf) {
    pdf = 0.f;
    const float3 i = make_float3(-d.x, -d.y, -d.z);
    const float cos_i = dot3(i, n), cos_o = dot3(o, n);
    if (!(cos_i > 0.f) || cos_o == 0.f) return 0.f;
    float3 h;
    float coef, pb, jac;
    if (cos_o > 0.f) {
        h = unit3(i + o);
        const float ih = dot3(i, h);
        if (!(dot3(h, n) > 0.f) || !(ih > 0.f)) return 0.f;
        float r, ct;
        const bool ok = fresnel(ih, M1.c, M1.Z, M2.c, M2.Z, r, ct);
        coef = ok ? r : 1.f;
        pb = ok ? r * r : 1.f;
        jac = 0.25f / dot3(o, h);
    } else {
        const float eta = M2.c / M1.c;
        h = unit3(eta * i + o);   // along i/c1 + o/c2
        if (dot3(h, n) < 0.f) h = make_float3(-h.x, -h.y, -h.z);
        const float ih = dot3(i, h), oh = dot3(o, h);
        if (!(dot3(h, n) > 0.f) || !(ih > 0.f) || !(oh < 0.f)) return 0.f;
        float r, ct;
        if (!fresnel(ih, M1.c, M1.Z, M2.c, M2.Z, r, ct)) return 0.f;
        const float den = fmaf(eta, ih, oh);   // c2 (i.h / c1 + o.h / c2)
        if (!(den * den > 1e-30f)) return 0.f;
        pb = transmitted(ih, ct, M1.Z, M2.Z);
        coef = sqrtf(pb);
        jac = -oh / (den * den);
    }
    const float hn = dot3(h, n);
    const float D = ggx_d(hn, a2);
    const float G = ggx_g1(cos_i, a2) * ggx_g1(fabsf(cos_o), a2);
    pdf = D * hn * jac * pb;
    return coef * G * D * dot3(i, h) * jac / cos_i;
}

// The same toward an arbitrary element centre q (convex arrays).
template <bool MESH>
__device__ float connection_to(const SceneP &S, float3 p, int med, int skip0, float3 q, ff &t_conn, float &att) {
    float3 o = p;
    float3 w = make_float3(q.x - p.x, q.y - p.y, q.z - p.z);
    const float w2 = dot3(w, w), iw = rsqrtf(w2);
    float rem = sqrtf(w2);   // the length sets the travel time: correctly rounded
    w = make_float3(w.x * iw, w.y * iw, w.z * iw);
    float fac = 1.f, a = 0.f;
    ff t = {0.f, 0.f};
    int m = med, skip = skip0;
    for (int it = 0; it < kMaxCross; ++it) {
        float th;
        const int hit = nearest<MESH>(S, o, w, skip, false, th);
        const Medium &M = S.med[m];
        if (hit < 0 || th >= rem) {
            t = ff_add(t, ff_mul_f(rem, M.slow));
            a += M.a * rem;
            break;
        }
        t = ff_add(t, ff_mul_f(th, M.slow));
        a += M.a * th;
        float3 h = o + th * w, n;
        int m_neg, m_pos;
        float alpha;
        surface<MESH>(S, hit, h, n, m_neg, m_pos, alpha);
        const float dn = dot3(w, n);
        const int m2 = dn > 0.f ? m_pos : m_neg;
        float r, ct;
        if (!fresnel(fabsf(dn), M.c, M.Z, S.med[m2].c, S.med[m2].Z, r, ct)) return 0.f;
        fac *= sqrtf(transmitted(fabsf(dn), ct, M.Z, S.med[m2].Z));
        m = m2;
        o = h;
        rem -= th;
        skip = hit;
    }
    t_conn = t;
    att = a;
    return fac;
}

// Centre c and unit normal n of element e: on the arc of a convex array (radius > 0;
// z written as -2 R sin^2(phi/2) to avoid cancellation near the apex), else (x_e, 0, 0), +z.
template <bool CVX>
__device__ __forceinline__ void elem_frame(const TraceP &P, uint32_t e, float3 &c, float3 &n) {
    if (CVX) {
        const float ph = P.phi0 + (float)e * P.dphi;
        float sn, cs, sh, ch;
        sincosf(ph, &sn, &cs);
        sincosf(0.5f * ph, &sh, &ch);
        n = make_float3(sn, 0.f, cs);
        c = make_float3(P.radius * sn, 0.f, -2.f * P.radius * sh * sh);
    } else {
        c = make_float3(P.x_first + (float)e * P.pitch, 0.f, 0.f);
        n = make_float3(0.f, 0.f, 1.f);
    }
}

// Warp-aggregated append to the arrival queue (one atomic per converged group);
// with DBG or REC the arrival's (ray, event) words go to arr_dbg as well.
template <bool DBG, bool REC>
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
        if (DBG || REC) P.arr_dbg[idx] = make_uint2(ray, ev);
    }
}

struct Counters {
    uint32_t rays, segments, interactions, candidates, connections, arrivals;
};

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;
constexpr int kQueue = 64;     // scatterer-event ring per warp (power of two, >= 63 entries needed)
constexpr int kPool = kTracePool;

// Lane states: walking a segment's columns, segment walked (to be finished), waiting for a
// new ray, ray placed or redirected (its next segment to be set up), no rays left.
enum { kInSeg = 0, kSegDone = 1, kNeedRay = 2, kFinished = 3, kNeedSeg = 4 };

// Scatterer events waiting for their connection ray, one ring per warp (SoA).
struct WarpQueue {
    uint32_t ray[kQueue], kmb[kQueue], j[kQueue];
    float tca[kQueue], t_hi[kQueue], t_lo[kQueue], w[kQueue];
};

// Step direction marking a segment that walks one of the fine columns (vertical segments).
constexpr int kFineColumn = 2;

// Per-lane state: the primary ray, its current segment and the column walk over it.
struct Lane {
    float3 o, d;
    ff t;
    float w, L;
    int med, b, prev, scene;
    uint32_t i, item, stream;
    uint64_t h;
    float seg;
    int hit;
    bool clipped;
    int cx, cy, sx, sy;
    float tmx, tmy, tdx, tdy, t_enter, t_end;
    int state;
    // rough boundaries: the path left a rough vertex mp with direction density mpdf and has
    // crossed only by transmission since (its aperture hit takes a balance-heuristic weight)
    bool mis;
    float3 mp;
    float mpdf;
};

__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1u; }

// Segment from the current position to the nearest boundary (clipped by the
// path-length budget); set up the column walk over the part inside the grid box.
// The walk steps in x and y only: a column visit covers the segment's stretch
// through the column, and its references are those within g_rm of the z that
// stretch spans.  The first visit accepts closest approaches from g_rm before the
// grid box on (none can lie there; the margin only keeps rounding out of play).
template <int GEO, bool FINE>
__device__ __forceinline__ void start_segment(const TraceP &P, Lane &R, Counters &cn) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0, MESH = (GEO & kGeoMesh) != 0;
    const SceneP &S = P.S[R.scene];
    float th;
    R.hit = nearest<MESH>(S, R.o, R.d, R.prev, true, th, CVX ? P.radius : 0.f);
    R.seg = th;
    R.clipped = false;
    if (R.L + R.seg > P.max_path) {
        R.seg = P.max_path - R.L;
        R.clipped = true;
    }
    cn.segments++;
    R.state = kSegDone;
    if (S.n_scat == 0) return;
    const float3 o = R.o, d = R.d;
    const float hi_x = S.g_lo.x + (float)S.g_dim.x * S.g_h.x;
    const float hi_y = S.g_lo.y + (float)S.g_dim.y * S.g_h.y;
    const float hi_z = S.g_lo.z + (float)S.g_dim.z * S.g_h.z;
    float t0 = 0.f, t1 = R.seg;
    // Reciprocals of the direction for the box clip and the column steps.  They only place
    // column boundaries, which the g_rm margin of the references absorbs, so the approximate
    // form serves (a few ulp, and no slow path for the zero components of in-plane and
    // vertical rays: in a y-invariant scene every ray has d.y = 0).
    const float ix = __fdividef(1.f, d.x), iy = __fdividef(1.f, d.y), iz = __fdividef(1.f, d.z);
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
    if (FINE && d.x == 0.f && d.y == 0.f && S.f_refs) {   // vertical: one visit of a fine column
        R.cx = min(max((int)floorf((o.x - S.f_lo.x) * S.f_inv_h.x), 0), S.f_dim.x - 1);
        R.cy = min(max((int)floorf((o.y - S.f_lo.y) * S.f_inv_h.y), 0), S.f_dim.y - 1);
        R.sx = kFineColumn;
        R.sy = 0;
        R.tdx = R.tdy = R.tmx = R.tmy = INFINITY;
    } else {
        R.cx = min(max((int)floorf((o.x + t0 * d.x - S.g_lo.x) * S.g_inv_h.x), 0), S.g_dim.x - 1);
        R.cy = min(max((int)floorf((o.y + t0 * d.y - S.g_lo.y) * S.g_inv_h.y), 0), S.g_dim.y - 1);
        R.sx = d.x > 0.f ? 1 : (d.x < 0.f ? -1 : 0);
        R.sy = d.y > 0.f ? 1 : (d.y < 0.f ? -1 : 0);
        R.tdx = R.sx ? S.g_h.x * fabsf(ix) : INFINITY;
        R.tdy = R.sy ? S.g_h.y * fabsf(iy) : INFINITY;
        R.tmx = R.sx ? (S.g_lo.x + (float)(R.cx + (R.sx > 0)) * S.g_h.x - o.x) * ix : INFINITY;
        R.tmy = R.sy ? (S.g_lo.y + (float)(R.cy + (R.sy > 0)) * S.g_h.y - o.y) * iy : INFINITY;
    }
    R.t_enter = t0 - S.g_rm;
    R.t_end = t1;
    R.state = kInSeg;
}

template <bool DBG>
__device__ __forceinline__ void end_ray(const TraceP &P, Lane &R, int reason, Counters &cn) {
    if (DBG) P.path_hash[P.items[R.item].hash_begin + R.i] = fnv_step(R.h, 0x20000u | (uint32_t)reason);
    cn.rays++;
    R.state = kNeedRay;
}

// Emission (Eq. 6) of ray i of item `item` (a transmit of one scene) from element e.
// With transmit mixing the ray first draws its transmit (Sec. 2.3); a synthetic-
// aperture transmit emits every ray from its one element.
template <bool DBG, bool EXT, int GEO>
__device__ __forceinline__ void start_ray(const TraceP &P, Lane &R, uint32_t item, const ItemP &slot_item,
                                          uint32_t i, uint32_t e, Counters &cn) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0, EMIT = EXT && (GEO & kGeoEmit) != 0;
    if (EMIT && P.mix_tx > 0) {
        const uint4 y = philox(make_uint4(i, 0u, 0u, 1u), P.key);
        item = (uint32_t)(((uint64_t)(y.x >> 8) * (uint64_t)P.mix_tx) >> 24);
    }
    const ItemP &IT = EMIT && P.mix_tx > 0 ? P.items[item] : slot_item;
    if (EMIT && IT.kind == UR_TX_SYNTHETIC) e = (uint32_t)IT.vx;
    const uint4 x = draw<EXT>(make_uint4(i, IT.stream, 0u, 0u), P.key);
    const float xe = P.x_first + (float)e * P.pitch;
    R.o = make_float3(xe + (u24(x.x) - 0.5f) * P.pitch, (u24(x.y) - 0.5f) * P.H, 0.f);
    float3 nrm = make_float3(0.f, 0.f, 1.f);   // normal at the emission point
    if (CVX) {                                  // a point of the element's arc face
        const float ph = P.phi0 + ((float)e + u24(x.x) - 0.5f) * P.dphi;
        float sn, cs, sh, ch;
        sincosf(ph, &sn, &cs);
        sincosf(0.5f * ph, &sh, &ch);
        nrm = make_float3(sn, 0.f, cs);
        R.o = make_float3(P.radius * sn, R.o.y, -2.f * P.radius * sh * sh);
    }
    if (!EXT || IT.kind == UR_TX_PLANE) {
        R.d = make_float3(IT.sin_t, 0.f, IT.cos_t);
    } else if (EMIT && IT.kind == UR_TX_SYNTHETIC) {   // uniform angle to the face normal in (-pi/2, pi/2)
        const float th = ((float)(int)((x.z >> 8) - (1u << 23)) + 0.5f) * (kPiF * 0x1p-24f);
        float st, ct;
        sincosf(th, &st, &ct);
        R.d = make_float3(nrm.x * ct + nrm.z * st, 0.f, nrm.z * ct - nrm.x * st);
    } else {   // along the line from the virtual source, or toward the focus, in the xz plane
        const float sg = IT.kind == UR_TX_DIVERGING ? 1.f : -1.f;
        const float dx = sg * (R.o.x - IT.vx), dz = sg * (R.o.z - IT.vz);
        const float l = sqrtf(dx * dx + dz * dz);
        R.d = make_float3(dx / l, 0.f, dz / l);
    }
    R.t = P.delay[(uint32_t)IT.angle * (uint32_t)P.n_el + e];
    R.w = (EXT ? dot3(R.d, nrm) : R.d.z) * IT.inv_n;   // Eq. 6: cosine to the face normal over N
    R.scene = IT.scene;
    R.med = P.S[IT.scene].med_array;
    R.b = 0;
    R.prev = -1;
    R.L = 0.f;
    R.i = i;
    R.item = item;
    R.stream = IT.stream;
    R.h = kFnvOffset;
    R.mis = false;
    if (EXT && !(R.w > 0.f)) {   // aimed into a convex probe: no ray
        end_ray<DBG>(P, R, kEndArrayMiss, cn);
        return;
    }
    R.state = kNeedSeg;   // set up by the resolve loop, with the other lanes that need a segment
}

// Secondary ray of a rough vertex to a uniformly drawn element centre, weighted
// against BSDF sampling of the same direction by the balance heuristic.
template <bool DBG, bool REC, int GEO>
__device__ void rough_connection(const TraceP &P, const SceneP &S, const Lane &R, float3 n, int m2, float a2,
                                 Counters &cn) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0, MESH = (GEO & kGeoMesh) != 0;
    const uint4 x = philox(make_uint4(R.i, R.stream, 4u | ((uint32_t)R.b << 8), 0u), P.key);
    const uint32_t e = (uint32_t)(((uint64_t)(x.x >> 8) * (uint64_t)P.n_el) >> 24);
    float3 ce, ne;
    elem_frame<CVX>(P, e, ce, ne);
    const float3 v = ce - R.o;
    const float D = sqrtf(dot3(v, v));
    const float3 o = make_float3(v.x / D, v.y / D, v.z / D);
    const float cos_e = -dot3(o, ne);   // at the element, to its normal
    const float fd = directivity(P, -dot3(v, ne), cross2(v, ne));
    if (!(fd > 0.f)) return;
    const Medium &M = S.med[R.med], &M2 = S.med[m2];
    float pdf;
    const float f = rough_eval(R.d, n, o, a2, M, M2, pdf);
    if (!(f > 0.f)) return;
    cn.connections++;
    ff tc;
    float att;
    const float fac = connection_to<MESH>(S, R.o, dot3(o, n) > 0.f ? R.med : m2, R.hit, ce, tc, att);
    if (fac == 0.f) return;
    const ff ta = ff_add(R.t, tc);
    if (ff_gt(ta, P.t_last)) return;
    const float omega = P.pitch * P.H * cos_e / (D * D);   // element solid angle seen from the vertex
    const float p_nee = 1.f / ((float)P.n_el * omega);
    const float amp = R.w * f * fd * fac * expf(-att) / (p_nee + pdf);
    emit<DBG, REC>(P, R.item * (uint32_t)P.n_el + e, ta, amp, R.i,
                   0x80000000u | ((uint32_t)R.b << 24) | (uint32_t)(R.hit + 1));
    cn.arrivals++;
}

// Microfacet sampling at a rough vertex: normal from D(m)(m.n), the smooth branch
// about it, weight |i.m| G / (|i.n| |m.n|).  Returns false if the sample is not
// admissible (back-facing microfacet or a direction on the wrong side).
__device__ bool rough_scatter(const TraceP &P, const SceneP &S, Lane &R, float3 n, int m2, float a2,
                              uint32_t &branch) {
    const float cos_i = -dot3(n, R.d);
    const uint4 x = philox(make_uint4(R.i, R.stream, 3u | ((uint32_t)R.b << 8), 0u), P.key);
    float mn;   // m.n, the sampled cosine (exact where a dot product would cancel for grazing m)
    const float3 m = ggx_sample(n, a2, u24(x.x), u24(x.y), mn);
    const float c_im = -dot3(R.d, m);
    if (!(c_im > 0.f)) return false;
    const Medium &M = S.med[R.med], &M2 = S.med[m2];
    float r, cos_t;
    const bool tir = !fresnel(c_im, M.c, M.Z, M2.c, M2.Z, r, cos_t);
    float3 o;
    float fac, pb, jac;
    bool far = false;
    if (tir) {
        branch = 2;
        o = unit3(R.d + (2.f * c_im) * m);
        fac = 1.f;
        pb = 1.f;
        jac = 0.25f / c_im;
    } else {
        const uint4 y = philox(make_uint4(R.i, R.stream, 1u | ((uint32_t)R.b << 8), 0u), P.key);
        const float Rs = r * r;
        if (u24(y.x) < Rs) {
            branch = 0;
            o = unit3(R.d + (2.f * c_im) * m);
            fac = r / Rs;
            pb = Rs;
            jac = 0.25f / c_im;
        } else {
            branch = 1;
            const float eta = M2.c / M.c;
            o = unit3(eta * R.d + (eta * c_im - cos_t) * m);
            pb = transmitted(c_im, cos_t, M.Z, M2.Z);
            fac = 1.f / sqrtf(pb);
            const float om = dot3(o, m);
            const float den = fmaf(eta, c_im, om);
            jac = -om / (den * den);
            far = true;
        }
    }
    const float on = dot3(o, n);
    if (far ? !(on < 0.f) : !(on > 0.f)) return false;
    const float G = ggx_g1(cos_i, a2) * ggx_g1(fabsf(on), a2);
    R.w *= fac * c_im * G / (cos_i * mn);
    R.mis = true;
    R.mp = R.o;
    R.mpdf = ggx_d(mn, a2) * mn * jac * pb;
    R.d = o;
    if (far) R.med = m2;
    return true;
}

// End of a segment: time of flight and attenuation along it, then the array
// plane (aperture return), the absorbing bottom, the time window, the bounce
// budget, or a boundary interaction (Eqs. 7-11) and the next segment.
template <bool DBG, bool SPLIT, bool REC, bool ROUGH, int GEO>
__device__ void finish_segment(const TraceP &P, Lane &R, Counters &cn) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0, MESH = (GEO & kGeoMesh) != 0;
    const SceneP &S = P.S[R.scene];
    const Medium &M = S.med[R.med];
    R.t = ff_add(R.t, ff_mul_f(R.seg, M.slow));
    R.w *= expf(-M.a * R.seg);
    R.L += R.seg;
    R.o = R.o + R.seg * R.d;
    if (R.clipped) {
        end_ray<DBG>(P, R, kEndPath, cn);
        return;
    }
    if (CVX && R.hit == S.n_bnd + 2) {   // passed beside a convex probe
        end_ray<DBG>(P, R, kEndArrayMiss, cn);
        return;
    }
    if (R.hit == S.n_bnd) {  // array surface: only paths returning to the aperture are kept
        int el = -1;
        if (CVX) {   // the probe's cylinder: the element whose arc holds the hit
            const float u = (atan2f(R.o.x, R.o.z + P.radius) - P.phi0) / P.dphi + 0.5f;
            if (fabsf(R.o.y) <= 0.5f * P.H && u >= 0.f && u < (float)P.n_el) el = min((int)floorf(u), P.n_el - 1);
        } else {
            R.o.z = 0.f;
            const float xl = P.x_first - 0.5f * P.pitch;
            if (fabsf(R.o.y) <= 0.5f * P.H && R.o.x >= xl && R.o.x < xl + (float)P.n_el * P.pitch) {
                el = (int)floorf((R.o.x - xl) / P.pitch);
                if (el > P.n_el - 1) el = P.n_el - 1;
            }
        }
        int reason = kEndArrayMiss;
        if (el >= 0) {
            float3 ce = make_float3(0.f, 0.f, 0.f), ne = make_float3(0.f, 0.f, 1.f);
            if (ROUGH) elem_frame<CVX>(P, (uint32_t)el, ce, ne);
            const float fd = ROUGH ? directivity(P, -dot3(R.d, ne), cross2(R.d, ne))
                                   : directivity(P, -R.d.z, R.d.x * R.d.x + R.d.y * R.d.y);
            if (fd > 0.f && !ff_gt(R.t, P.t_last)) {
                float wa = R.w * fd;
                if (ROUGH && R.mis) {   // balance heuristic against the rough vertex's secondary ray
                    const float3 v = ce - R.mp;
                    const float D2 = dot3(v, v);
                    const float omega = P.pitch * P.H * (-dot3(v, ne) / sqrtf(D2)) / D2;
                    if (omega > 0.f) wa *= 1.f / (1.f + 1.f / ((float)P.n_el * omega * R.mpdf));
                }
                emit<DBG, REC>(P, R.item * (uint32_t)P.n_el + (uint32_t)el, R.t, wa, R.i,
                          0x80000000u | ((uint32_t)R.b << 24));
                cn.arrivals++;
            }
            reason = kEndAperture;
        }
        end_ray<DBG>(P, R, reason, cn);
        return;
    }
    if (R.hit == S.n_bnd + 1) {
        end_ray<DBG>(P, R, kEndBottom, cn);
        return;
    }
    const bool on_tri = MESH && R.hit >= S.tri_base;
    if (!on_tri && S.bnd[R.hit].kind == kPlaneZ) R.o.z = S.bnd[R.hit].p[0];
    if (ff_gt(R.t, P.t_last)) {
        end_ray<DBG>(P, R, kEndTime, cn);
        return;
    }
    if (R.b >= P.max_b) {
        end_ray<DBG>(P, R, kEndMaxB, cn);
        return;
    }
    float3 n_out;
    int m_neg, m_pos;
    float alpha;
    if (on_tri) {
        surface_tri(S, R.hit, n_out, m_neg, m_pos, alpha);
    } else {
        const Bnd &B = S.bnd[R.hit];
        n_out = outward(B, R.o);
        m_neg = B.med_neg;
        m_pos = B.med_pos;
        alpha = B.alpha;
    }
    const float dn = dot3(R.d, n_out);
    const int m2 = dn > 0.f ? m_pos : m_neg;
    const float3 n = dn > 0.f ? make_float3(-n_out.x, -n_out.y, -n_out.z) : n_out;
    if (ROUGH && alpha > 0.f) {   // rough boundary: secondary ray first, then the BSDF sample
        const float a2 = alpha * alpha;
        rough_connection<DBG, REC, GEO>(P, S, R, n, m2, a2, cn);
        cn.interactions++;
        uint32_t rb = 0;
        if (!rough_scatter(P, S, R, n, m2, a2, rb)) {
            end_ray<DBG>(P, R, kEndRough, cn);
            return;
        }
        if (DBG) R.h = fnv_step(R.h, 0x10000u | ((uint32_t)R.hit << 4) | rb);
        R.b += 1;
        R.prev = R.hit;
        R.state = kNeedSeg;   // set up by the resolve loop, with the other lanes that need a segment
        return;
    }
    const float cos_i = -dot3(n, R.d);
    const float3 dr = unit3(R.d + (2.f * cos_i) * n);
    const Medium &M2 = S.med[m2];
    float r, cos_t, Rs, rs, cts = 0.f;
    bool tir;
    uint32_t branch;
    if (!SPLIT) {   // the media decide their own branches
        tir = !fresnel(cos_i, M.c, M.Z, M2.c, M2.Z, r, cos_t);
        Rs = r * r;
    } else {        // frozen sampling media decide the branch and its probability
        tir = !fresnel(cos_i, S.cs[R.med], S.Zs[R.med], S.cs[m2], S.Zs[m2], rs, cts) ||
              !fresnel(cos_i, M.c, M.Z, M2.c, M2.Z, r, cos_t);
        Rs = rs * rs;
    }
    if (tir) {
        branch = 2;
        R.d = dr;
    } else {
        const uint4 y = draw<ROUGH>(make_uint4(R.i, R.stream, 1u | ((uint32_t)R.b << 8), 0u), P.key);
        if (u24(y.x) < Rs) {
            branch = 0;
            R.w *= r / Rs;
            R.d = dr;
        } else {
            branch = 1;
            const float eta = M2.c / M.c;
            // 1 - R as 4 Z1 Z2 cos_i cos_t / (Z2 cos_i + Z1 cos_t)^2: no cancellation near the critical angle
            const float T = transmitted(cos_i, cos_t, M.Z, M2.Z);
            R.w *= SPLIT ? sqrtf(T) / transmitted(cos_i, cts, S.Zs[R.med], S.Zs[m2]) : rsqrtf(T);
            R.d = unit3(eta * R.d + (eta * cos_i - cos_t) * n);
            R.med = m2;
        }
    }
    cn.interactions++;
    if (ROUGH && branch != 1) R.mis = false;   // a smooth reflection: the secondary ray cannot produce this path
    if (DBG) R.h = fnv_step(R.h, 0x10000u | ((uint32_t)R.hit << 4) | branch);
    R.b += 1;
    R.prev = R.hit;
    R.state = kNeedSeg;   // set up by the resolve loop, with the other lanes that need a segment
}

// A queued scatterer event: element drawn uniformly (Philox keyed by ray,
// transmit, segment and scatterer) and the receive directivity (Eq. 13).  An
// event the element receives goes on to the warp's connection ring with its
// arrival time and amplitude so far (the connection ray's part follows there).
template <bool EXT, int GEO>
__device__ __forceinline__ bool event_element(const TraceP &P, const WarpQueue &Q, int slot, uint32_t &e, ff &t_pre,
                                              float &amp_pre) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0;
    const uint32_t ray = Q.ray[slot], kmb = Q.kmb[slot], j = Q.j[slot];
    const float tca = Q.tca[slot], w = Q.w[slot];
    const ff t = {Q.t_hi[slot], Q.t_lo[slot]};
    const uint32_t item = kmb >> 16;
    const int med = (int)((kmb >> 8) & 0xffu), b = (int)(kmb & 0xffu);
    const ItemP &IT = P.items[item];
    const SceneP &S = P.S[IT.scene];
    const float4 q = S.scat[j];
    const uint4 x = draw<EXT>(make_uint4(ray, IT.stream, 2u | ((uint32_t)b << 8), j), P.key);
    e = (uint32_t)(((uint64_t)(x.x >> 8) * (uint64_t)P.n_el) >> 24);
    float fd;
    if (CVX) {   // convex array: directivity to the element's normal
        float3 ce, ne;
        elem_frame<CVX>(P, e, ce, ne);
        const float3 v = make_float3(q.x - ce.x, q.y - ce.y, q.z - ce.z);
        fd = directivity(P, dot3(v, ne), cross2(v, ne));
    } else {
        const float vx = P.x_first + (float)e * P.pitch - q.x;
        fd = directivity(P, q.z, vx * vx + q.y * q.y);
    }
    if (!(fd > 0.f)) return false;
    const Medium &M = S.med[med];
    t_pre = ff_add(t, ff_mul_f(tca, M.slow));
    amp_pre = w * expf(-M.a * tca) * q.w * (float)P.n_el * fd;
    return true;
}

// Scatterer events waiting for their connection ray to the drawn element, one ring per warp (SoA).
struct ConnQueue {
    uint32_t ray[kQueue], kmb[kQueue], j[kQueue], e[kQueue];
    float t_hi[kQueue], t_lo[kQueue], amp[kQueue];
};

// A queued connection: the straight ray from the scatterer to the element centre,
// its transmission factors, time and attenuation; the arrival goes to the queue.
template <bool DBG, bool REC, bool EXT, int GEO>
__device__ __forceinline__ void process_connection(const TraceP &P, const ConnQueue &C, int slot, Counters &cn) {
    constexpr bool CVX = (GEO & kGeoConvex) != 0, MESH = (GEO & kGeoMesh) != 0;
    const uint32_t ray = C.ray[slot], kmb = C.kmb[slot], j = C.j[slot], e = C.e[slot];
    const uint32_t item = kmb >> 16;
    const int med = (int)((kmb >> 8) & 0xffu), b = (int)(kmb & 0xffu);
    const ItemP &IT = P.items[item];
    const SceneP &S = P.S[IT.scene];
    const float4 q = S.scat[j];
    cn.connections++;
    ff tc;
    float att, fac;
    if (CVX) {
        float3 ce, ne;
        elem_frame<CVX>(P, e, ce, ne);
        fac = connection_to<MESH>(S, make_float3(q.x, q.y, q.z), med, -1, ce, tc, att);
    } else {
        fac = connection<MESH>(S, make_float3(q.x, q.y, q.z), med, -1, P.x_first + (float)e * P.pitch, tc, att);
    }
    if (fac == 0.f) return;
    const ff ta = ff_add({C.t_hi[slot], C.t_lo[slot]}, tc);
    if (ff_gt(ta, P.t_last)) return;
    const float amp = C.amp[slot] * fac * expf(-att);
    emit<DBG, REC>(P, item * (uint32_t)P.n_el + e, ta, amp, ray, ((uint32_t)b << 24) | j);
    cn.arrivals++;
}

// Events [qhead + lane] for the lanes below n: element draw and directivity; the ones the
// element receives join the connection ring, which is traced 32 at a time with all lanes.
template <bool DBG, bool REC, bool EXT, int GEO>
__device__ __forceinline__ void drain_events(const TraceP &P, const WarpQueue &Q, ConnQueue &CQ, int qhead, int n,
                                             int &chead, int &cn_q, Counters &cn) {
    const int lane = threadIdx.x & 31;
    uint32_t e = 0;
    ff t_pre = {0.f, 0.f};
    float amp_pre = 0.f;
    const int slot = (qhead + lane) & (kQueue - 1);
    const bool go = lane < n && event_element<EXT, GEO>(P, Q, slot, e, t_pre, amp_pre);
    const unsigned m = __ballot_sync(0xffffffffu, go);
    if (go) {
        const int c = (chead + cn_q + __popc(m & ((1u << lane) - 1u))) & (kQueue - 1);
        CQ.ray[c] = Q.ray[slot];
        CQ.kmb[c] = Q.kmb[slot];
        CQ.j[c] = Q.j[slot];
        CQ.e[c] = e;
        CQ.t_hi[c] = t_pre.hi;
        CQ.t_lo[c] = t_pre.lo;
        CQ.amp[c] = amp_pre;
    }
    cn_q += __popc(m);
    if (cn_q >= 32) {
        __syncwarp();
        process_connection<DBG, REC, EXT, GEO>(P, CQ, (chead + lane) & (kQueue - 1), cn);
        __syncwarp();
        chead = (chead + 32) & (kQueue - 1);
        cn_q -= 32;
    }
}

// The item whose slot range holds `slot` (item slot ranges are pool-aligned and ascending).
__device__ __forceinline__ uint32_t item_of(const TraceP &P, uint64_t slot) {
    int lo = 0, hi = P.n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.items[mid].slot_begin <= slot) lo = mid; else hi = mid - 1;
    }
    return (uint32_t)lo;
}

// Residency: the usual tracer runs 4 CTAs per SM in 64 registers; the extended ones trade
// warps for registers (3 CTAs, 80 registers: 14.84 instead of 15.18 ms on the paper-settings
// acquisition, 29.6 instead of 32.0 ms on the rough layered frame), the mesh ones more so (2 CTAs, 128 registers: the BVH walk's stack and state
// spilled 1.3 KB per thread at 64 registers; 61.5 instead of 71.5 ms).  The grid is sized for
// 4 CTAs per SM: CTAs that find the ray pools empty exit at once.
template <bool ROUGH, int GEO>
constexpr int trace_ctas_per_sm() { return (GEO & kGeoMesh) ? 2 : ROUGH ? 3 : 4; }

// Persistent tracer.  Each iteration of the warp's loop (1) finishes segments
// and claims new rays for idle lanes, (2) moves every active lane through one
// grid column, the references of all lanes' visits tested 32 at a time across
// the warp, (3) hands scatterer events to a per-warp queue that is drained 32
// events at a time with all lanes busy; the events the drawn element receives
// wait in a second ring for their connection rays, traced 32 at a time as well.
// Ray slots are element-major: a freshly claimed
// batch of lanes traces neighbouring rays of one element; slot -> ray
// i = m * n_el + e.
template <bool DBG, bool SPLIT, bool REC, bool ROUGH, int GEO>
__global__ void __launch_bounds__(kBlock, trace_ctas_per_sm<ROUGH, GEO>()) k_trace(const __grid_constant__ TraceP P) {
    __shared__ WarpQueue s_q[kWarps];
    __shared__ ConnQueue s_c[kWarps];
    WarpQueue &Q = s_q[threadIdx.x >> 5];
    ConnQueue &CQ = s_c[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const uint64_t n_slots = P.n_slots;
    Counters cn = {0, 0, 0, 0, 0, 0};
    Lane R;
    R.state = kNeedRay;
    uint64_t pool_next = 0;
    uint32_t pool_cnt = 0, pool_item = 0;
    bool pool_dry = false;
    int qhead = 0, qn = 0;     // warp-uniform ring bookkeeping: scatterer events
    int chead = 0, cqn = 0;    // and connections

    for (;;) {
        // (1) resolve finished segments and idle lanes, once enough lanes wait
        const unsigned waiting = __ballot_sync(0xffffffffu, R.state == kSegDone || R.state == kNeedRay);
        const bool resolve = __popc(waiting) >= P.resolve_batch || __ballot_sync(0xffffffffu, R.state == kInSeg) == 0u;
        for (int guard = 0; resolve && guard < 256; ++guard) {
            if (R.state == kSegDone) finish_segment<DBG, SPLIT, REC, ROUGH, GEO>(P, R, cn);
            unsigned need = __ballot_sync(0xffffffffu, R.state == kNeedRay);
            uint64_t my_slot = ~0ull;
            while (need) {
                if (pool_cnt == 0) {
                    if (!pool_dry) {
                        unsigned long long base = 0;
                        if (lane == 0) base = atomicAdd(P.next_slot, (unsigned long long)kPool);
                        base = __shfl_sync(0xffffffffu, base, 0);
                        pool_next = base;
                        pool_cnt = base >= n_slots ? 0u : (uint32_t)kPool;
                        pool_dry = pool_cnt == 0;
                        if (!pool_dry) pool_item = item_of(P, base);
                    }
                    if (pool_dry) {
                        if (R.state == kNeedRay) R.state = kFinished;
                        break;
                    }
                }
                const uint32_t take = min((uint32_t)__popc(need), pool_cnt);
                const uint32_t rank = (uint32_t)__popc(need & lanemask_lt());
                if (((need >> lane) & 1u) && rank < take) my_slot = pool_next + rank;
                pool_next += take;
                pool_cnt -= take;
                need = __ballot_sync(0xffffffffu, R.state == kNeedRay && my_slot == ~0ull);
            }
            if (my_slot != ~0ull) {
                // A warp that used up a pool and claimed the next one in the same pass holds slots
                // of both; a slot before the current item's range belongs to an earlier item.
                uint32_t item = pool_item;
                if (my_slot < P.items[item].slot_begin) item = item_of(P, my_slot);
                const ItemP &IT = P.items[item];
                const uint64_t local = my_slot - IT.slot_begin;
                if (ROUGH && (GEO & kGeoEmit) && P.mix_list) {   // a mixed sequence in (drawn transmit, element) order
                    if (local < IT.n_rays) {
                        const uint32_t i = P.mix_list[local];
                        start_ray<DBG, ROUGH, GEO>(P, R, item, IT, i, i % (uint32_t)P.n_el, cn);
                    }
                } else {
                    const uint32_t m = (uint32_t)(local % IT.rays_per_el);
                    const uint64_t e = local / IT.rays_per_el;
                    const uint32_t i = m * (uint32_t)P.n_el + (uint32_t)e;
                    if (e < (uint64_t)P.n_el && i < IT.n_rays) start_ray<DBG, ROUGH, GEO>(P, R, item, IT, i, (uint32_t)e, cn);
                }
            }
            // one call site for every lane that continues its ray or starts a new one
            if (R.state == kNeedSeg) start_segment<GEO, !ROUGH>(P, R, cn);
            if (!__any_sync(0xffffffffu, R.state == kSegDone || R.state == kNeedRay)) break;
        }
        if (__all_sync(0xffffffffu, R.state == kFinished)) break;

        // (2) one column visit per active lane; the references of all visits are numbered
        // across the warp (prefix sum of their counts) and tested 32 at a time, each lane
        // reading the visiting ray of its reference from the owner lane's registers by
        // shuffles (staging the visits in shared memory instead cost L1 capacity: the
        // kernel's register spills and scatterer references live there)
        const bool active = R.state == kInSeg;
        uint32_t cnt = 0;
        float v_hi = 0.f, v_r2 = 0.f;
        unsigned long long v_refs = 0ull;
        int axis = 0;
        float t_exit = 0.f;
        bool last = false;
        if (active) {
            const SceneP &S = P.S[R.scene];
            axis = R.tmx <= R.tmy ? 0 : 1;
            t_exit = axis == 0 ? R.tmx : R.tmy;
            last = !(t_exit < R.t_end);
            if (!last) {
                const int nc = axis == 0 ? R.cx + R.sx : R.cy + R.sy;
                last = nc < 0 || nc >= (axis == 0 ? S.g_dim.x : S.g_dim.y);
            }
            const float t_out = last ? R.t_end : t_exit;
            // the column's grid: fine (a vertical segment of the plane-wave tracer) or the usual; the
            // extended tracers keep to the usual columns (the selection cost the paper-settings
            // trace more than their vertical segments gained)
            const bool fine = !ROUGH && R.sx == kFineColumn;
            const float lo_z = fine ? S.f_lo.z : S.g_lo.z, inv_hz = fine ? S.f_inv_h.z : S.g_inv_h.z;
            const int dim_y = fine ? S.f_dim.y : S.g_dim.y, dim_z = fine ? S.f_dim.z : S.g_dim.z;
            const uint32_t *cs = fine ? S.f_cell_start : S.cell_start;
            const float za = fmaf(R.t_enter, R.d.z, R.o.z), zb = fmaf(t_out, R.d.z, R.o.z);
            const int cza = min(max((int)floorf((fminf(za, zb) - S.g_rm - lo_z) * inv_hz), 0), dim_z - 1);
            const int czb = min(max((int)floorf((fmaxf(za, zb) + S.g_rm - lo_z) * inv_hz), 0), dim_z - 1);
            const uint32_t col = ((uint32_t)R.cx * (uint32_t)dim_y + (uint32_t)R.cy) * (uint32_t)dim_z;
            const uint32_t rb = cs[col + (uint32_t)cza];
            cnt = cs[col + (uint32_t)czb + 1u] - rb;
            v_hi = last ? R.seg : t_exit;
            v_refs = (unsigned long long)(uintptr_t)((fine ? S.f_refs : S.refs) + rb);
            v_r2 = S.r2;
        }
        uint32_t incl = cnt;   // inclusive prefix sum of the visits' reference counts
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        v_refs -= (unsigned long long)(incl - cnt) * sizeof(float4);
        const uint32_t v_kmb = (R.item << 16) | ((uint32_t)R.med << 8) | (uint32_t)R.b;
        for (uint32_t base = 0; base < total; base += 32) {
            const uint32_t k = base + (uint32_t)lane;
            int owner = 0;   // the lane whose visit holds reference k: the first with incl > k
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t v = __shfl_sync(0xffffffffu, incl, owner + step - 1);
                if (v <= k) owner += step;
            }
            bool cand = false;
            float tca = 0.f;
            uint32_t j = 0;
            const float4 A = make_float4(__shfl_sync(0xffffffffu, R.o.x, owner), __shfl_sync(0xffffffffu, R.o.y, owner),
                                         __shfl_sync(0xffffffffu, R.o.z, owner), __shfl_sync(0xffffffffu, R.t_enter, owner));
            const float4 B = make_float4(__shfl_sync(0xffffffffu, R.d.x, owner), __shfl_sync(0xffffffffu, R.d.y, owner),
                                         __shfl_sync(0xffffffffu, R.d.z, owner), __shfl_sync(0xffffffffu, v_hi, owner));
            const unsigned long long rp = __shfl_sync(0xffffffffu, v_refs, owner);
            const float r2 = __shfl_sync(0xffffffffu, v_r2, owner);
            if (k < total) {
                const float4 q = reinterpret_cast<const float4 *>((uintptr_t)rp)[k];
                const float3 v = make_float3(q.x - A.x, q.y - A.y, q.z - A.z);
                tca = v.x * B.x + v.y * B.y + v.z * B.z;
                if (tca > 0.f && tca >= A.w && tca < B.w) {
                    const float3 pe = make_float3(v.x - tca * B.x, v.y - tca * B.y, v.z - tca * B.z);
                    cand = dot3(pe, pe) < r2;
                    j = __float_as_uint(q.w);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, cand);
            if (m) {
                const uint32_t e_ray = __shfl_sync(0xffffffffu, R.i, owner), e_kmb = __shfl_sync(0xffffffffu, v_kmb, owner);
                const float e_thi = __shfl_sync(0xffffffffu, R.t.hi, owner), e_tlo = __shfl_sync(0xffffffffu, R.t.lo, owner);
                const float e_w = __shfl_sync(0xffffffffu, R.w, owner);
                if (cand) {
                    const int slot = (qhead + qn + __popc(m & lanemask_lt())) & (kQueue - 1);
                    Q.ray[slot] = e_ray;
                    Q.kmb[slot] = e_kmb;
                    Q.j[slot] = j;
                    Q.tca[slot] = tca;
                    Q.t_hi[slot] = e_thi;
                    Q.t_lo[slot] = e_tlo;
                    Q.w[slot] = e_w;
                    cn.candidates++;
                }
                qn += __popc(m);
                if (qn >= 32) {
                    __syncwarp();
                    drain_events<DBG, REC, ROUGH, GEO>(P, Q, CQ, qhead, 32, chead, cqn, cn);
                    __syncwarp();
                    qhead = (qhead + 32) & (kQueue - 1);
                    qn -= 32;
                }
            }
        }
        if (active) {
            if (last) {
                R.state = kSegDone;
            } else {
                R.t_enter = t_exit;
                if (axis == 0) {
                    R.cx += R.sx;
                    R.tmx += R.tdx;
                } else {
                    R.cy += R.sy;
                    R.tmy += R.tdy;
                }
            }
        }
    }
    // (3) drain the queues
    __syncwarp();
    drain_events<DBG, REC, ROUGH, GEO>(P, Q, CQ, qhead, qn, chead, cqn, cn);
    __syncwarp();
    if (lane < cqn) process_connection<DBG, REC, ROUGH, GEO>(P, CQ, (chead + lane) & (kQueue - 1), cn);

    if (P.stats) {
        const uint32_t v[6] = {cn.rays, cn.segments, cn.interactions, cn.candidates, cn.connections, cn.arrivals};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const uint32_t s = __reduce_add_sync(0xffffffffu, v[c]);
            if (lane == 0 && s) atomicAdd(&P.stats[c], (unsigned long long)s);
        }
    }
}

}  // namespace

int trace_occupancy(int block, bool debug) {
    int n = 0;
    if (debug)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<true, false, false, false, 0>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_trace<false, false, false, false, 0>, block, 0);
    return n > 0 ? n : 1;
}

// Variants with frozen sampling media, with recorded (ray, event) words and the
// extended variants (rough boundaries, diverging and focused transmits; one per
// geometry: linear or convex array, with or without triangle meshes; with or
// without synthetic-aperture emission and transmit mixing, whose code cost the
// rough layered frame 6 % and the paper-settings acquisition 9 % when every
// extended trace carried it) are compiled separately so the usual kernel carries
// none of their code.  Mesh variants always carry the emission code.  The extended variants never record or freeze sampling media (the
// adjoint and ur_scene_set_media refuse such scenes and transmits).
template <int GEO>
void launch_extended(const TraceP &P, bool debug, int block, int grid, cudaStream_t s) {
    debug ? k_trace<true, false, false, true, GEO><<<grid, block, 0, s>>>(P)
          : k_trace<false, false, false, true, GEO><<<grid, block, 0, s>>>(P);
}

void launch_trace(const TraceP &P, bool debug, int block, int grid, cudaStream_t s, bool point_waves, bool emit) {
    bool split = false, mesh = false, rough = point_waves || P.radius > 0.f;   // convex arrays: extended tracer
    for (int q = 0; q < P.n_scenes && q < kMaxScenes; ++q) {
        split = split || P.S[q].split_sampling != 0;
        mesh = mesh || P.S[q].n_tri > 0;
        for (int b = 0; b < P.S[q].n_bnd; ++b) rough = rough || P.S[q].bnd[b].alpha > 0.f;
    }
    if (rough || mesh || emit) {
        const int cvx = P.radius > 0.f ? kGeoConvex : 0;
        if (mesh) {
            if (cvx) launch_extended<kGeoConvex | kGeoMesh | kGeoEmit>(P, debug, block, grid, s);
            else launch_extended<kGeoMesh | kGeoEmit>(P, debug, block, grid, s);
        } else if (emit) {
            if (cvx) launch_extended<kGeoConvex | kGeoEmit>(P, debug, block, grid, s);
            else launch_extended<kGeoEmit>(P, debug, block, grid, s);
        } else {
            if (cvx) launch_extended<kGeoConvex>(P, debug, block, grid, s);
            else launch_extended<0>(P, debug, block, grid, s);
        }
        return;
    }
    if (debug) {
        split ? k_trace<true, true, false, false, 0><<<grid, block, 0, s>>>(P)
              : k_trace<true, false, false, false, 0><<<grid, block, 0, s>>>(P);
    } else if (P.record) {
        split ? k_trace<false, true, true, false, 0><<<grid, block, 0, s>>>(P)
              : k_trace<false, false, true, false, 0><<<grid, block, 0, s>>>(P);
    } else {
        split ? k_trace<false, true, false, false, 0><<<grid, block, 0, s>>>(P)
              : k_trace<false, false, false, false, 0><<<grid, block, 0, s>>>(P);
    }
}

}  // namespace ur
