// Device-side building blocks of the sm_103a acoustic ray tracer: float-float
// arithmetic for times and delays, Philox4x32-10, parameter blocks shared by
// the kernels, and host-side launcher declarations.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ultraray.h"

namespace ur {

constexpr int kMaxMed = 16;
constexpr int kMaxBnd = 16;
constexpr int kMaxScenes = 16;   // scenes traced together in one launch
constexpr int kAdjMed = 4;       // media the adjoint differentiates (c, Z, alpha each)
constexpr int kTracePool = 32;   // ray slots a tracer warp claims at once (item slot ranges are multiples)
constexpr int kMaxNs = 8192;
constexpr int kMaxSeg = 4096;      // safety bound on primary segments per path
constexpr int kMaxCross = 64;      // boundaries a connection ray may cross
constexpr float kTmin = 1e-7f;     // smallest admissible hit distance (m)
constexpr int kMaxTri = 1 << 22;   // triangles per scene (hit ids stay below 2^24)
constexpr int kBvhStack = 32;      // traversal stack; the host's BVH is never deeper
constexpr int kGeoConvex = 1;      // tracer instantiation bits: convex array,
constexpr int kGeoMesh = 2;        // triangle-mesh boundaries,
constexpr int kGeoEmit = 4;        // synthetic-aperture transmits or transmit mixing
constexpr uint64_t kFnvOffset = 0xcbf29ce484222325ull;
constexpr uint64_t kFnvPrime = 0x100000001b3ull;

enum { kPlaneZ = 0, kSphere = 1, kCylY = 2 };
enum { kEndAperture = 1, kEndArrayMiss = 2, kEndBottom = 3, kEndPath = 4, kEndTime = 5, kEndMaxB = 6, kEndRough = 7 };

// ---------------------------------------------------------------- float-float
// A value hi + lo with |lo| <= ulp(hi)/2 (Dekker / Knuth error-free transforms).
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_quick(float a, float b) {   // requires |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_quick(s.hi, lo);
}

__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = ff_two_sum(a.hi, b);
    return ff_quick(s.hi, __fadd_rn(s.lo, a.lo));
}

// a (float) times b (ff)
__device__ __forceinline__ ff ff_mul_f(float a, ff b) {
    float p = __fmul_rn(a, b.hi);
    float e = __fmaf_rn(a, b.hi, -p);
    e = __fmaf_rn(a, b.lo, e);
    return ff_quick(p, e);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_quick(p, e);
}

__device__ __forceinline__ ff ff_sqr_f(float a) {
    float p = __fmul_rn(a, a);
    return ff_quick(p, __fmaf_rn(a, a, -p));
}

// square root of a non-negative ff (one Newton correction of the float root)
__device__ __forceinline__ ff ff_sqrt(ff a) {
    if (a.hi <= 0.f) return {0.f, 0.f};
    float s = sqrtf(a.hi);
    float r = __fmaf_rn(-s, s, a.hi);
    r = __fadd_rn(r, a.lo);
    return ff_quick(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ bool ff_gt(ff a, float b) { return a.hi > b || (a.hi == b && a.lo > 0.f); }

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds, each two 32x32
// multiplies whose high/low halves are mixed with the other counter words and
// the key; the key advances by the two Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hA = __umulhi(0xD2511F53u, c.x), lA = 0xD2511F53u * c.x;
        const uint32_t hB = __umulhi(0xCD9E8D57u, c.z), lB = 0xCD9E8D57u * c.z;
        c = make_uint4(hB ^ c.y ^ k.x, lB, hA ^ c.w ^ k.y, lA);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Uniform in [0, 1) from the top 24 bits (exact in float).
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }

__device__ __forceinline__ uint64_t fnv_step(uint64_t h, uint32_t w) { return (h ^ (uint64_t)w) * kFnvPrime; }

// ---------------------------------------------------------------- vectors
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// Unit vector by the hardware reciprocal square root (a few ulp; the tracer's directions feed
// geometry whose error budget is set by FP32 positions, and no slow path of an IEEE divide runs).
__device__ __forceinline__ float3 unit3(float3 a) {
    const float il = rsqrtf(dot3(a, a));
    return make_float3(a.x * il, a.y * il, a.z * il);
}

// ---------------------------------------------------------------- parameters
struct Medium {
    float c, Z, a;          // m/s, MRayl, Np/m
    ff slow;                // samples per metre (fs / c)
};

struct Bnd {
    int kind, med_neg, med_pos;
    float alpha;            // GGX roughness (Eq. 12): the larger of the two media's; 0 = smooth
    float p[4];
};

struct SceneP {
    int n_med, n_bnd, med_array;
    float z_max;
    Medium med[kMaxMed];
    Bnd bnd[kMaxBnd];
    // scatterer grid
    int n_scat;
    float r2;               // capture radius squared
    float g_rm;             // grid margin: r_s plus slack above FP32 rounding
    float3 g_lo, g_inv_h, g_h;
    int3 g_dim;
    const float4 *refs;     // (x, y, z, bits(index)) per cell reference; cells (x, y, z) with z fastest;
                            // a scatterer is referenced from the columns within g_rm of it in x and y,
                            // in its own z cell only
    const uint32_t *cell_start;
    // the same structure on narrow columns, walked by exactly vertical segments (null: none)
    float3 f_lo, f_inv_h;
    int3 f_dim;
    const float4 *f_refs;
    const uint32_t *f_cell_start;
    const float *amp;
    const float4 *scat;     // (x, y, z, amplitude) by scatterer index
    // rarely read (after the fields every segment reads, which keep their offsets):
    int split_sampling;               // 1 if some (cs, Zs) differs from the media
    float cs[kMaxMed], Zs[kMaxMed];   // c and Z that decide Monte Carlo branches (normally = med)
    // triangle meshes (tracer instantiations with kGeoMesh): triangle t has hit id tri_base + t
    int n_tri, tri_base;              // tri_base = n_bnd + 3, after the terminal planes
    const float4 *bvh;                // 2 per node: (lo, bits(first child | first triangle)),
                                      // (hi, bits(0 for an inner node | triangle count)); children adjacent
    const float4 *tri;                // 3 per triangle in leaf order: (v0, bits(id)), (v1 - v0), (v2 - v0)
    const float4 *tri_nrm;            // per id: unit normal (v1 - v0) x (v2 - v0), bits(behind | front << 8)
    float rough[kMaxMed];             // GGX roughness per medium (a triangle takes the larger of its two)
};

// One transmit of one scene: a contiguous range of ray slots (element-major,
// padded to a multiple of the tracer's per-warp slot pool).
struct ItemP {
    uint64_t slot_begin;    // first slot of the item
    uint64_t hash_begin;    // first path-hash index (debug output)
    uint32_t n_rays, rays_per_el;
    int scene, angle;
    float sin_t, cos_t, inv_n;
    uint32_t stream;        // Philox counter word identifying the transmit's random stream
    int kind;               // UR_TX_*: plane wave (sin_t, cos_t), diverging, focused or synthetic aperture
    float vx, vz;           // virtual source or focus in the xz plane (m); synthetic aperture: vx = the
                            // firing element's index
};

struct TraceP {
    SceneP S[kMaxScenes];           // scene table (parameter space, indexed per lane)
    int n_scenes;
    // array
    int n_el, n_s;
    float pitch, H, x_first;        // element 0 centre (linear array)
    float radius, dphi, phi0;       // convex array (radius > 0): angle between centres, angle of element 0
    float K, t_last;                // pulse half-width and latest useful arrival (samples)
    float t2am, t2ac, am, ac;   // directivity (Eq. 13): tan^2 of the main-beam and cutoff angles, the angles
    // work: items (transmit x scene) and their slots
    const ItemP *items;
    int n_items;
    uint64_t n_slots;
    const ff *delay;                // [n_angles][n_el] transmit delays (samples)
    uint2 key;
    int max_b;
    float max_path;
    int resolve_batch;              // lanes that must wait before a warp resolves segments
    int mix_tx;                     // > 0: the rays of item 0's slots draw their transmit among items
                                    // 0 .. mix_tx - 1 (extended tracer only)
    const uint32_t *mix_list;       // with mix_tx: the ray index of each of item 0's slots (null: slot order)
    // outputs
    uint4 *arr;                     // (row, t_hi, t_lo, amp), row = item * n_el + element
    uint2 *arr_dbg;                 // (ray, event), debug only
    unsigned long long *arr_count;
    uint64_t arr_cap;
    unsigned long long *next_slot;  // work counter of the persistent tracer (zeroed per launch)
    unsigned long long *path_hash;  // per item and ray, debug only
    unsigned long long *stats;      // 6 counters, nullable
    int record;                     // 1: store (ray, event) of every arrival in arr_dbg (the adjoint's work)
};

// ---------------------------------------------------------------- geometry shared by tracer and adjoint
// Nearest boundary hit along o + t d, t in (kTmin, inf).  `skip` is the
// primitive the ray is leaving: a plane cannot be met again, a sphere or
// cylinder only at its far root.  With `terminals`, the array plane z = 0
// (id n_bnd, upward rays) and the absorbing plane z = z_max (id n_bnd + 1,
// downward rays) take part.
// Moeller-Trumbore: distance along o + t d to the triangle (v0, e1 = v1 - v0, e2 = v2 - v0).
__device__ __forceinline__ bool tri_hit(float4 v0, float4 e1, float4 e2, float3 o, float3 d, float &t) {
    const float px = d.y * e2.z - d.z * e2.y, py = d.z * e2.x - d.x * e2.z, pz = d.x * e2.y - d.y * e2.x;
    const float det = e1.x * px + e1.y * py + e1.z * pz;
    if (det == 0.f) return false;
    const float inv = 1.f / det;
    const float sx = o.x - v0.x, sy = o.y - v0.y, sz = o.z - v0.z;
    const float u = (sx * px + sy * py + sz * pz) * inv;
    if (u < 0.f || u > 1.f) return false;
    const float qx = sy * e1.z - sz * e1.y, qy = sz * e1.x - sx * e1.z, qz = sx * e1.y - sy * e1.x;
    const float v = (d.x * qx + d.y * qy + d.z * qz) * inv;
    if (v < 0.f || u + v > 1.f) return false;
    t = (e2.x * qx + e2.y * qy + e2.z * qz) * inv;
    return true;
}

// Slab test of a BVH box against (0, t_max); axes the ray runs parallel to test the origin.
__device__ __forceinline__ bool box_hit(float4 lo, float4 hi, float3 o, float3 inv, int3 par, float t_max,
                                        float &t_near) {
    float tn = 0.f, tf = t_max;
    if (par.x) {
        if (o.x < lo.x || o.x > hi.x) return false;
    } else {
        const float a = (lo.x - o.x) * inv.x, b = (hi.x - o.x) * inv.x;
        tn = fmaxf(tn, fminf(a, b));
        tf = fminf(tf, fmaxf(a, b));
    }
    if (par.y) {
        if (o.y < lo.y || o.y > hi.y) return false;
    } else {
        const float a = (lo.y - o.y) * inv.y, b = (hi.y - o.y) * inv.y;
        tn = fmaxf(tn, fminf(a, b));
        tf = fminf(tf, fmaxf(a, b));
    }
    if (par.z) {
        if (o.z < lo.z || o.z > hi.z) return false;
    } else {
        const float a = (lo.z - o.z) * inv.z, b = (hi.z - o.z) * inv.z;
        tn = fmaxf(tn, fminf(a, b));
        tf = fminf(tf, fmaxf(a, b));
    }
    t_near = tn;
    return tn <= tf;
}

// Nearest triangle along o + t d with t in (kTmin, best): BVH walk, near child first.
__device__ __forceinline__ void nearest_triangle(const SceneP &S, float3 o, float3 d, int skip, float &best,
                                                 int &hit) {
    const int3 par = make_int3(d.x == 0.f, d.y == 0.f, d.z == 0.f);
    const float3 inv = make_float3(par.x ? 0.f : 1.f / d.x, par.y ? 0.f : 1.f / d.y, par.z ? 0.f : 1.f / d.z);
    int stack[kBvhStack];
    int sp = 0, node = 0;
    float t0;
    if (!box_hit(S.bvh[0], S.bvh[1], o, inv, par, best, t0)) return;
    for (;;) {
        const float4 a = S.bvh[2 * node], b = S.bvh[2 * node + 1];
        const int first = __float_as_int(a.w), cnt = __float_as_int(b.w);
        if (cnt > 0) {
            for (int q = first; q < first + cnt; ++q) {
                const float4 v0 = S.tri[3 * q];
                const int id = S.tri_base + __float_as_int(v0.w);
                float t;
                if (id != skip && tri_hit(v0, S.tri[3 * q + 1], S.tri[3 * q + 2], o, d, t) && t > kTmin &&
                    t < best) {
                    best = t;
                    hit = id;
                }
            }
        } else {
            float tl, tr;
            const bool hl = box_hit(S.bvh[2 * first], S.bvh[2 * first + 1], o, inv, par, best, tl);
            const bool hr = box_hit(S.bvh[2 * first + 2], S.bvh[2 * first + 3], o, inv, par, best, tr);
            if (hl && hr) {
                const bool left_first = tl <= tr;
                if (sp < kBvhStack) stack[sp++] = left_first ? first + 1 : first;
                node = left_first ? first : first + 1;
                continue;
            }
            if (hl || hr) {
                node = hl ? first : first + 1;
                continue;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
}

template <bool MESH = false>
__device__ __forceinline__ int nearest(const SceneP &S, float3 o, float3 d, int skip, bool terminals,
                                       float &t_out, float radius = 0.f) {
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
    if (MESH && S.n_tri > 0) nearest_triangle(S, o, d, skip, best, hit);
    if (terminals && radius > 0.f) {   // convex probe: its cylinder (id n_bnd), the escape plane z = -R (n_bnd + 2)
        const float ox = o.x, oz = o.z + radius;
        const float a = d.x * d.x + d.z * d.z;
        const float b = ox * d.x + oz * d.z;
        if (a > 0.f && b < 0.f) {
            const float disc = b * b - a * ((ox - radius) * (ox + radius) + oz * oz);
            if (disc >= 0.f) {
                const float t = (-b - sqrtf(disc)) / a;
                if (t > kTmin && t < best) {
                    best = t;
                    hit = S.n_bnd;
                }
            }
        }
        if (d.z < 0.f) {
            const float t = (-radius - o.z) / d.z;
            if (t > kTmin && t < best) {
                best = t;
                hit = S.n_bnd + 2;
            }
        } else if (d.z > 0.f) {
            const float t = (S.z_max - o.z) / d.z;
            if (t > kTmin && t < best) {
                best = t;
                hit = S.n_bnd + 1;
            }
        }
    } else if (terminals) {
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

// Triangle hit id -> unit outward normal, media behind and in front, GGX roughness.
__device__ __forceinline__ void surface_tri(const SceneP &S, int hit, float3 &n_out, int &m_neg, int &m_pos,
                                            float &alpha) {
    const float4 q = S.tri_nrm[hit - S.tri_base];
    const int m = __float_as_int(q.w);
    n_out = make_float3(q.x, q.y, q.z);
    m_neg = m & 0xff;
    m_pos = (m >> 8) & 0xff;
    alpha = fmaxf(S.rough[m_neg], S.rough[m_pos]);
}

// The surface a ray met (hit id from nearest): unit outward normal at h (a plane's hit point is
// put on the plane), the media behind and in front, and the GGX roughness.
template <bool MESH>
__device__ __forceinline__ void surface(const SceneP &S, int hit, float3 &h, float3 &n_out, int &m_neg, int &m_pos,
                                        float &alpha) {
    if (MESH && hit >= S.tri_base) {
        surface_tri(S, hit, n_out, m_neg, m_pos, alpha);
        return;
    }
    const Bnd &B = S.bnd[hit];
    if (B.kind == kPlaneZ) h.z = B.p[0];
    n_out = outward(B, h);
    m_neg = B.med_neg;
    m_pos = B.med_pos;
    alpha = B.alpha;
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

// Transmitted intensity fraction 1 - r^2 of the fluid-fluid interface, written as
// 4 Z1 Z2 cos_i cos_t / (Z2 cos_i + Z1 cos_t)^2, without the cancellation of
// 1 - r^2 near the critical angle.
__device__ __forceinline__ float transmitted(float cos_i, float cos_t, float Z1, float Z2) {
    const float s = fmaf(Z2, cos_i, Z1 * cos_t);
    return 4.f * Z1 * Z2 * cos_i * cos_t / (s * s);
}

// Eq. 13 for a direction given by its part ax along the element normal and the squared length
// tr2 of its part across it (any scale): 1 inside the main beam, 0 beyond the cutoff (< 90
// degrees, so ax <= 0 is beyond it), linear in the angle between.  The beam tests compare tan^2,
// with no square root or division; in the taper the angle is atan2(tr, ax), which keeps a few
// ulp of the angle itself where acos of a rounded cosine loses ulp(cos) / sin(angle), an error the
// taper divides by its own small value near the cutoff.
__device__ __forceinline__ float directivity(const TraceP &P, float ax, float tr2) {
    if (!(ax > 0.f)) return 0.f;
    const float ax2 = ax * ax;
    if (tr2 <= P.t2am * ax2) return 1.f;
    if (tr2 > P.t2ac * ax2) return 0.f;
    return (P.ac - atan2f(sqrtf(tr2), ax)) / (P.ac - P.am);
}

// Squared length of v x n for a unit n: the part of v across n, from products that do not cancel.
__device__ __forceinline__ float cross2(float3 v, float3 n) {
    const float a = v.y * n.z - v.z * n.y, b = v.z * n.x - v.x * n.z, c = v.x * n.y - v.y * n.x;
    return a * a + b * b + c * c;
}


// ---------------------------------------------------------------- launchers
void launch_trace(const TraceP &P, bool debug, int block, int grid, cudaStream_t s, bool point_waves,
                  bool emit);
int trace_occupancy(int block, bool debug);   // resident tracer CTAs per SM

// Path-replay adjoint: loss sensitivities in, parameter gradients out.
struct AdjP {
    TraceP T;                   // scene table, array, items, Philox key, limits
    const float *g_rf, *g_q;    // dL/d rf, dL/d quad  [n_items][n_el][n_s]
    double *grad;               // [3 * kAdjMed]: (c, Z, alpha) per medium, accumulated
    float *grad_amp;            // [n_scat] of scene 0, accumulated (nullable)
    float K, inv_2s2, inv_s2, half_cycles, om;   // pulse: half-width, 1/(2 s^2), 1/s^2 (samples), 2 f0/fs, rad/sample
    float fs, k_alpha;          // sampling frequency; d(Np/m)/d(dB/cm/MHz) at f0
    const uint4 *arr;           // arrivals of the forward trace (row, t_hi, t_lo, amp)
    const uint2 *rec;           // their (ray, event) words
    const unsigned long long *n_arr;
    uint64_t arr_cap;
    uint32_t *order;            // [arr_cap]: arrival indices grouped by path shape (filled by launch_adjoint)
    uint32_t *key_count;        // [3 * kAdjKeys] scratch of that counting sort
};
constexpr int kAdjKeys = 256;   // path shapes: aperture return or scatterer event x interactions before it
void launch_adjoint(const AdjP &A, int sms, cudaStream_t s);

struct BinP {
    const uint4 *arr;
    const unsigned long long *arr_count;
    uint64_t arr_cap;
    int n_rows, n_s;
    uint32_t *row_count;    // [n_rows]
    uint32_t *row_fill;     // [n_rows]
    uint32_t *row_off;      // [n_rows + 1]
    uint4 *items;           // (row, begin, end, 0) work items
    uint32_t *n_items;
    uint32_t max_items;
    uint32_t chunk, chunk_min, target_items;   // work items of chunk_min..chunk arrivals, about target_items of them
    int priv_rows;          // row histograms in shared memory (n_rows <= kBinPrivRows)
    float4 *sorted;         // (t_hi, t_lo, amp, 0)
    float *rf, *quad;       // [n_rows][n_s]
    float K, inv_2s2_log2e, phase_per_sample;   // taps |n - t| <= K; log2(e) / (2 s^2); 2 f0 / fs (half-cycles per sample)
    float rot32_s, rot32_c;                     // sin, cos of the carrier phase over 32 samples
};
constexpr int kBinPrivRows = 4096;                  // largest row count with shared-memory histograms
int bin_sort_smem(int n_rows);                      // their bytes per CTA (0: global counters)
void launch_bin_sort(const BinP &B, int sms, cudaStream_t s);      // 3 kernels
void launch_bin_deposit(const BinP &B, int sms, cudaStream_t s);   // 1 kernel

struct GridBuildP {
    const float4 *scat;
    int n_scat;
    float r_m;
    float3 lo, inv_h;
    int3 dim;
    uint32_t *cell_count;   // [n_cells + 1]
    uint32_t *cell_start;   // [n_cells + 1]
    uint32_t *cell_fill;    // [n_cells]
    float4 *refs;
    float *amp;
};
void launch_bbox(const float4 *scat, int n, float *lohi /* 6 floats as ordered ints */, cudaStream_t s);
void launch_grid_count(const GridBuildP &G, cudaStream_t s);
void launch_scan_u32(const uint32_t *in, uint32_t *out, uint32_t *block_sums, uint32_t n, cudaStream_t s);
void launch_grid_fill(const GridBuildP &G, cudaStream_t s);

// Delay-and-sum of items (transmits) into images.  rf/quad hold [n_items][n_el][n_s];
// image z compounds items img_items[img_begin[z] .. img_begin[z+1]); with
// img_items == nullptr there is one image made of items 0..n_tx-1 and item k
// uses angle k.  Outputs are [n_images][nz][nx].
struct ImageP {
    const float *rf, *quad;
    int n_tx, n_el, n_s;
    const int *img_items, *img_begin, *item_angle;
    int n_images;
    const float *x_px, *z_px;
    int nx, nz;
    ff q;                   // fs / c_bf (samples per metre)
    ff x_first;             // element 0 centre
    float pitch;
    const ff *tx_sin, *tx_cos, *tx_m;   // per transmit: plane wave: sin, cos, min_e x_e sin; diverging
                                        // (focused) wave: source (focus) x, z, min (max) element distance
    const int *tx_kind;                 // per transmit UR_TX_* (null: plane waves)
    const ff *elem_xz;                  // convex array: element centres (x, z) per element (null: linear)
    float2 *iq;
    float *env, *db;
    unsigned int *env_max;  // float bits, one per image
    float dyn_range_db;
};
void launch_das(const ImageP &I, cudaStream_t s);

struct DebugOut {
    uint32_t *ray, *event, *row;
    float *t_hi, *t_lo, *amp;
    uint64_t cap;
};
void launch_unpack_debug(const uint4 *arr, const uint2 *dbg, const unsigned long long *count, uint64_t cap_in,
                         const DebugOut &D, cudaStream_t s);
void launch_log(const ImageP &I, cudaStream_t s);

// Read-only view of a context's set-up for entry points living in other files
// (false if the array or the transmits are not set).
struct CtxView {
    int device;
    void *stream;
    ur_array arr;
    int n_tx;
    const float *angles;    // host copy, n_tx entries
    bool plane_waves;       // every transmit is a plane wave
    bool linear;            // the array is linear
};
bool ctx_view(const ur_ctx *c, CtxView *v);

// Counting sort of a mixed transmit sequence's rays by (drawn transmit, emitting element).
constexpr uint32_t kMixMaxBins = 12288;   // bins held in shared memory (48 KB)
struct MixP {
    uint2 key;
    uint32_t n_rays, n_tx, n_el, n_bins;
    bool per_element;                     // bins are (transmit, element); else transmits
    uint32_t *count, *offset, *fill;      // [n_bins]
    uint32_t *list;                       // [n_rays]: ray indices in bin order
};
// Bins for n_tx transmits of n_el elements (0: too many transmits to sort).
int mix_bins(int n_tx, int n_el, bool *per_element);
cudaError_t launch_mix_plan(const MixP &M, int sms, cudaStream_t s);

}  // namespace ur
