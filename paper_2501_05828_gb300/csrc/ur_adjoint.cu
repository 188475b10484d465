// Path-replay adjoint: gradient of a loss on the analytic channel data with
// respect to every medium's sound speed c, impedance Z and attenuation alpha
// and to every scatterer's amplitude.  Each ray is re-emitted from its Philox
// stream and its path replayed (same branch decisions as the forward), carrying
// forward-mode tangents: position, direction, time and path length with
// respect to the sound speeds (the only parameters that move the geometry,
// through refraction), and the logarithmic derivative of the weight with
// respect to all parameters.  Branch probabilities dividing the weights carry
// no derivative.  At every arrival the loss sensitivities dL/d(amplitude) and
// dL/d(time) are formed from dL/d(rf, quad) over the pulse taps (Eq. 14) and
// chained into the parameter gradient.
#include "ur_device.cuh"

#include <algorithm>

namespace ur {
namespace {

constexpr int kAM = kAdjMed;
constexpr int kNP = 3 * kAdjMed;   // parameter 3m + 0: c_m, 3m + 1: Z_m, 3m + 2: alpha_m

struct Tan {
    float3 dO[kAM], dD[kAM];   // d position / d c_m, d direction / d c_m
    float dT[kAM], dL[kAM];    // d time (samples) / d c_m, d path length / d c_m
    float lw[kNP];             // d log|w| / d parameter
};

__device__ __forceinline__ int ceil_ff(float hi, float lo) {
    const float c = ceilf(hi);
    return (int)c + ((c == hi && lo > 0.f) ? 1 : 0);
}
__device__ __forceinline__ int floor_ff(float hi, float lo) {
    const float f = floorf(hi);
    return (int)f - ((f == hi && lo < 0.f) ? 1 : 0);
}

// dL/d(amplitude) and dL/d(time) of one arrival from dL/d(rf, quad) of its row.
__device__ void sensitivities(const AdjP &A, uint32_t row, ff t, float amp, float &g_amp, float &g_t) {
    const int n_s = A.T.n_s;
    const float *gr = A.g_rf + (size_t)row * n_s;
    const float *gq = A.g_q + (size_t)row * n_s;
    const int n0 = max(ceil_ff(t.hi - A.K, t.lo), 0);
    const int n1 = min(floor_ff(t.hi + A.K, t.lo), n_s - 1);
    float sa = 0.f, st = 0.f;
    for (int n = n0; n <= n1; ++n) {
        const float tau = ((float)n - t.hi) - t.lo;
        const float g = expf(-tau * tau * A.inv_2s2);
        float sn, cs;
        sincospif(tau * A.half_cycles, &sn, &cs);
        const float gre = __ldg(gr + n), gim = __ldg(gq + n);
        sa += g * (gre * sn - gim * cs);
        st -= g * (gre * (A.om * cs - tau * A.inv_s2 * sn) + gim * (A.om * sn + tau * A.inv_s2 * cs));
    }
    g_amp = sa;
    g_t = amp * st;
}

__device__ __forceinline__ void accumulate(float *acc, const float *lw, const float *dTa, float g_amp, float g_t,
                                           float amp) {
#pragma unroll
    for (int m = 0; m < kAM; ++m) {
        acc[3 * m + 0] += g_amp * amp * lw[3 * m + 0] + g_t * dTa[m];
        acc[3 * m + 1] += g_amp * amp * lw[3 * m + 1];
        acc[3 * m + 2] += g_amp * amp * lw[3 * m + 2];
    }
}

// Partial derivatives of the pressure reflection coefficient
// r = (Z2 ci - Z1 ct)/(Z2 ci + Z1 ct) with ct = sqrt(1 - eta^2 (1 - ci^2)), eta = c2/c1.
struct RDeriv {
    float r_ci, r_ct, r_Z1, r_Z2, ct_eta, ct_ci;
};
__device__ __forceinline__ RDeriv r_partials(float ci, float ct, float eta, float Z1, float Z2) {
    RDeriv D;
    const float den = Z2 * ci + Z1 * ct;
    const float inv2 = 1.f / (den * den);
    D.r_ci = 2.f * Z1 * Z2 * ct * inv2;
    D.r_ct = -2.f * Z1 * Z2 * ci * inv2;
    D.r_Z1 = -2.f * Z2 * ci * ct * inv2;
    D.r_Z2 = 2.f * Z1 * ci * ct * inv2;
    const float ctg = fmaxf(ct, 1e-12f);
    D.ct_eta = -eta * (1.f - ci * ci) / ctg;
    D.ct_ci = eta * eta * ci / ctg;
    return D;
}

// Connection ray (fixed geometry): factor, time, attenuation and their
// derivatives (log factor and attenuation into lwc, time into dtc).
__device__ float connection_tan(const AdjP &A, const SceneP &S, float3 p, int med, float xe, ff &t_conn,
                                float &att, float *lwc, float *dtc) {
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
        const float leg = (hit < 0 || th >= rem) ? rem : th;
        t = ff_add(t, ff_mul_f(leg, M.slow));
        a += M.a * leg;
        if (m < kAM) {
            dtc[m] -= leg * A.fs / (M.c * M.c);
            lwc[3 * m + 2] -= A.k_alpha * leg;
        }
        if (hit < 0 || th >= rem) break;
        float3 h = o + th * w;
        const Bnd &B = S.bnd[hit];
        if (B.kind == kPlaneZ) h.z = B.p[0];
        const float3 n = outward(B, h);
        const float dn = dot3(w, n);
        const int m2 = dn > 0.f ? B.med_pos : B.med_neg;
        const float ci = fabsf(dn);
        float r, ct;
        const Medium &M2 = S.med[m2];
        if (!fresnel(ci, M.c, M.Z, M2.c, M2.Z, r, ct)) return 0.f;
        const float Tr = transmitted(ci, ct, M.Z, M2.Z);   // 1 - r^2
        fac *= sqrtf(Tr);
        const float eta = M2.c / M.c;
        const RDeriv D = r_partials(ci, ct, eta, M.Z, M2.Z);
        const float coef = -r / Tr;                        // d log sqrt(1 - r^2) / dr
        const float r_eta = D.r_ct * D.ct_eta;
        lwc[3 * m + 0] += coef * r_eta * (-M2.c / (M.c * M.c));
        lwc[3 * m2 + 0] += coef * r_eta * (1.f / M.c);
        lwc[3 * m + 1] += coef * D.r_Z1;
        lwc[3 * m2 + 1] += coef * D.r_Z2;
        m = m2;
        o = h;
        rem -= th;
        skip = hit;
    }
    t_conn = t;
    att = a;
    return fac;
}

// Tangent of the distance to the boundary `hit` along o + t d.
__device__ void hit_tangent(const SceneP &S, int hit, float3 o, float3 d, float th, const Tan &T, float *dseg) {
    if (hit < 0) return;
    if (hit >= S.n_bnd || S.bnd[hit].kind == kPlaneZ) {
#pragma unroll
        for (int m = 0; m < kAM; ++m) dseg[m] = (-T.dO[m].z - th * T.dD[m].z) / d.z;
        return;
    }
    const Bnd &B = S.bnd[hit];
    if (B.kind == kSphere) {
        const float3 h = make_float3(o.x + th * d.x - B.p[0], o.y + th * d.y - B.p[1], o.z + th * d.z - B.p[2]);
        const float den = dot3(h, d);
#pragma unroll
        for (int m = 0; m < kAM; ++m) dseg[m] = -dot3(h, T.dO[m] + th * T.dD[m]) / den;
        return;
    }
    const float hx = o.x + th * d.x - B.p[0], hz = o.z + th * d.z - B.p[1];
    const float den = hx * d.x + hz * d.z;
#pragma unroll
    for (int m = 0; m < kAM; ++m)
        dseg[m] = -(hx * (T.dO[m].x + th * T.dD[m].x) + hz * (T.dO[m].z + th * T.dD[m].z)) / den;
}

struct RayVal {
    float3 o, d;
    ff t;
    float w, L;
    int med, b;
};

// One scatterer event of the current segment with its tangents.
__device__ void event(const AdjP &A, const SceneP &S, uint32_t item, uint32_t stream, uint32_t i, const RayVal &V,
                      const Tan &T, float4 q, float tca, float *acc) {
    const TraceP &P = A.T;
    const uint32_t j = __float_as_uint(q.w);
    const uint4 x = philox(make_uint4(i, stream, 2u | ((uint32_t)V.b << 8), j), P.key);
    const uint32_t e = (uint32_t)(((uint64_t)(x.x >> 8) * (uint64_t)P.n_el) >> 24);
    const float xe = P.x_first + (float)e * P.pitch;
    const float vx = xe - q.x;
    const float fd = directivity(P, q.z, vx * vx + q.y * q.y);
    if (!(fd > 0.f)) return;
    float lw[kNP], dTa[kAM];
#pragma unroll
    for (int k = 0; k < kNP; ++k) lw[k] = T.lw[k];
#pragma unroll
    for (int m = 0; m < kAM; ++m) dTa[m] = 0.f;
    ff tc;
    float att;
    const float3 p = make_float3(q.x, q.y, q.z);
    const float fac = connection_tan(A, S, p, V.med, xe, tc, att, lw, dTa);
    if (fac == 0.f) return;
    const Medium &M = S.med[V.med];
    const ff ta = ff_add(ff_add(V.t, ff_mul_f(tca, M.slow)), tc);
    if (ff_gt(ta, P.t_last)) return;
    const float4 sj = S.scat[j];
    const float amp_wo = V.w * expf(-M.a * tca) * (float)P.n_el * fd * fac * expf(-att);
    const float amp = amp_wo * sj.w;
    const float3 v = p - V.o;
    const float slow = M.slow.hi;
#pragma unroll
    for (int m = 0; m < kAM; ++m) {
        const float dtca = -dot3(T.dO[m], V.d) + dot3(v, T.dD[m]);
        lw[3 * m] -= M.a * dtca;
        dTa[m] += T.dT[m] + dtca * slow;
    }
    if (V.med < kAM) {
        dTa[V.med] -= tca * A.fs / (M.c * M.c);
        lw[3 * V.med + 2] -= A.k_alpha * tca;
    }
    float g_amp, g_t;
    sensitivities(A, item * (uint32_t)P.n_el + e, ta, amp, g_amp, g_t);
    accumulate(acc, lw, dTa, g_amp, g_t, amp);
    if (A.grad_amp) atomicAdd(&A.grad_amp[j], g_amp * amp_wo);
}

// Replay of ray i of `item` with tangents up to the arrival recorded by the
// forward trace: event word ev = b << 24 | j for the connection from scatterer j
// on the segment after b interactions, 0x80000000 | b << 24 for the return to
// the aperture at the end of that segment.
__device__ void replay(const AdjP &A, uint32_t item, const ItemP &IT, uint32_t i, uint32_t e, uint32_t ev,
                       float *acc) {
    const TraceP &P = A.T;
    const SceneP &S = P.S[IT.scene];
    const uint4 x = philox(make_uint4(i, IT.stream, 0u, 0u), P.key);
    const float xe = P.x_first + (float)e * P.pitch;
    RayVal V;
    V.o = make_float3(xe + (u24(x.x) - 0.5f) * P.pitch, (u24(x.y) - 0.5f) * P.H, 0.f);
    V.d = make_float3(IT.sin_t, 0.f, IT.cos_t);
    V.t = P.delay[(uint32_t)IT.angle * (uint32_t)P.n_el + e];
    V.w = IT.cos_t * IT.inv_n;
    V.L = 0.f;
    V.med = S.med_array;
    V.b = 0;
    int prev = -1;
    Tan T;
#pragma unroll
    for (int m = 0; m < kAM; ++m) {
        T.dO[m] = make_float3(0.f, 0.f, 0.f);
        T.dD[m] = make_float3(0.f, 0.f, 0.f);
        T.dT[m] = 0.f;
        T.dL[m] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kNP; ++k) T.lw[k] = 0.f;

    for (int guard = 0; guard < kMaxSeg; ++guard) {
        float th;
        const int hit = nearest(S, V.o, V.d, prev, true, th);
        float seg = th, dseg[kAM] = {0.f, 0.f, 0.f, 0.f};
        hit_tangent(S, hit, V.o, V.d, th, T, dseg);
        bool clipped = false;
        if (V.L + seg > P.max_path) {
            seg = P.max_path - V.L;
            clipped = true;
#pragma unroll
            for (int m = 0; m < kAM; ++m) dseg[m] = -T.dL[m];
        }
        if (!(ev & 0x80000000u) && (uint32_t)V.b == ((ev >> 24) & 0x7fu)) {   // the recorded scatterer event
            const uint32_t j = ev & 0xffffffu;
            const float4 sj = S.scat[j];
            const float3 v = make_float3(sj.x - V.o.x, sj.y - V.o.y, sj.z - V.o.z);
            event(A, S, item, IT.stream, i, V, T, make_float4(sj.x, sj.y, sj.z, __uint_as_float(j)), dot3(v, V.d), acc);
            return;
        }
        // advance along the segment
        const Medium &M = S.med[V.med];
        const float slow = M.slow.hi;
#pragma unroll
        for (int m = 0; m < kAM; ++m) {
            T.dT[m] += dseg[m] * slow;
            T.lw[3 * m] -= M.a * dseg[m];
            T.dO[m] = T.dO[m] + dseg[m] * V.d + seg * T.dD[m];
            T.dL[m] += dseg[m];
        }
        if (V.med < kAM) {
            T.dT[V.med] -= seg * A.fs / (M.c * M.c);
            T.lw[3 * V.med + 2] -= A.k_alpha * seg;
        }
        V.t = ff_add(V.t, ff_mul_f(seg, M.slow));
        V.w *= expf(-M.a * seg);
        V.L += seg;
        V.o = V.o + seg * V.d;
        if (clipped) return;
        if (hit == S.n_bnd) {   // array plane: aperture return
            V.o.z = 0.f;
            const float xl = P.x_first - 0.5f * P.pitch;
            if (fabsf(V.o.y) <= 0.5f * P.H && V.o.x >= xl && V.o.x < xl + (float)P.n_el * P.pitch) {
                int el = (int)floorf((V.o.x - xl) / P.pitch);
                if (el > P.n_el - 1) el = P.n_el - 1;
                const float ax = -V.d.z, tr2 = V.d.x * V.d.x + V.d.y * V.d.y;
                const float fd = directivity(P, ax, tr2);
                if (fd > 0.f && !ff_gt(V.t, P.t_last)) {
                    float lw[kNP];
#pragma unroll
                    for (int k = 0; k < kNP; ++k) lw[k] = T.lw[k];
                    if (tr2 > P.t2am * ax * ax) {      // linear part of Eq. 13: f_d depends on the angle
                        const float s = sqrtf(tr2);    // sin of the angle (unit d)
                        const float al = atan2f(s, ax);
#pragma unroll
                        for (int m = 0; m < kAM; ++m) lw[3 * m] += -(T.dD[m].z / s) / (P.ac - al);
                    }
                    const float amp = V.w * fd;
                    float g_amp, g_t;
                    sensitivities(A, item * (uint32_t)P.n_el + (uint32_t)el, V.t, amp, g_amp, g_t);
                    accumulate(acc, lw, T.dT, g_amp, g_t, amp);
                }
            }
            return;
        }
        if (hit == S.n_bnd + 1 || hit < 0) return;
        const Bnd &B = S.bnd[hit];
        if (B.kind == kPlaneZ) {
            V.o.z = B.p[0];
#pragma unroll
            for (int m = 0; m < kAM; ++m) T.dO[m].z = 0.f;
        }
        if (ff_gt(V.t, P.t_last)) return;
        if (V.b >= P.max_b) return;

        // interaction (Eqs. 7-11) with tangents
        const float3 n_out = outward(B, V.o);
        float3 dn[kAM];
        if (B.kind == kPlaneZ) {
#pragma unroll
            for (int m = 0; m < kAM; ++m) dn[m] = make_float3(0.f, 0.f, 0.f);
        } else {
            float3 vrel;
            if (B.kind == kSphere)
                vrel = make_float3(V.o.x - B.p[0], V.o.y - B.p[1], V.o.z - B.p[2]);
            else
                vrel = make_float3(V.o.x - B.p[0], 0.f, V.o.z - B.p[1]);
            const float inv_len = rsqrtf(dot3(vrel, vrel));
#pragma unroll
            for (int m = 0; m < kAM; ++m) {
                float3 dv = T.dO[m];
                if (B.kind == kCylY) dv.y = 0.f;
                dn[m] = inv_len * (dv - dot3(n_out, dv) * n_out);
            }
        }
        const float dsign = dot3(V.d, n_out) > 0.f ? -1.f : 1.f;
        const int m2 = dsign < 0.f ? B.med_pos : B.med_neg;
        const float3 n = dsign * n_out;
        const float ci = -dot3(n, V.d);
        float dci[kAM];
#pragma unroll
        for (int m = 0; m < kAM; ++m) {
            dn[m] = dsign * dn[m];
            dci[m] = -(dot3(dn[m], V.d) + dot3(n, T.dD[m]));
        }
        const float3 dr = unit3(V.d + (2.f * ci) * n);
        const Medium &M2 = S.med[m2];
        float r, ct, Rs, rs, cts = 0.f;
        bool tir;
        if (!S.split_sampling) {
            tir = !fresnel(ci, M.c, M.Z, M2.c, M2.Z, r, ct);
            Rs = r * r;
        } else {   // frozen sampling media decide the branch and its probability
            tir = !fresnel(ci, S.cs[V.med], S.Zs[V.med], S.cs[m2], S.Zs[m2], rs, cts) ||
                  !fresnel(ci, M.c, M.Z, M2.c, M2.Z, r, ct);
            Rs = rs * rs;
        }
        if (tir) {
#pragma unroll
            for (int m = 0; m < kAM; ++m) T.dD[m] = T.dD[m] + (2.f * dci[m]) * n + (2.f * ci) * dn[m];
            V.d = dr;
        } else {
            const float eta = M2.c / M.c;
            const RDeriv D = r_partials(ci, ct, eta, M.Z, M2.Z);
            float deta[kAM], dct[kAM], drc[kAM];
#pragma unroll
            for (int m = 0; m < kAM; ++m) {
                deta[m] = (m == V.med ? -M2.c / (M.c * M.c) : 0.f) + (m == m2 ? 1.f / M.c : 0.f);
                dct[m] = D.ct_eta * deta[m] + D.ct_ci * dci[m];
                drc[m] = D.r_ct * dct[m] + D.r_ci * dci[m];
            }
            const uint4 y = philox(make_uint4(i, IT.stream, 1u | ((uint32_t)V.b << 8), 0u), P.key);
            // d log(branch factor) / dr: 1/r on reflection, -r/(1 - r^2) on transmission
            const bool refl = u24(y.x) < Rs;
            const float Tr = refl ? 0.f : transmitted(ci, ct, M.Z, M2.Z);   // 1 - r^2
            const float coef = refl ? 1.f / r : -r / Tr;
#pragma unroll
            for (int m = 0; m < kAM; ++m) T.lw[3 * m] += coef * drc[m];
            if (V.med < kAM) T.lw[3 * V.med + 1] += coef * D.r_Z1;
            if (m2 < kAM) T.lw[3 * m2 + 1] += coef * D.r_Z2;
            if (refl) {
                V.w *= r / Rs;
#pragma unroll
                for (int m = 0; m < kAM; ++m) T.dD[m] = T.dD[m] + (2.f * dci[m]) * n + (2.f * ci) * dn[m];
                V.d = dr;
            } else {
                V.w *= S.split_sampling ? sqrtf(Tr) / transmitted(ci, cts, S.Zs[V.med], S.Zs[m2]) : rsqrtf(Tr);   // as the tracer
#pragma unroll
                for (int m = 0; m < kAM; ++m)
                    T.dD[m] = deta[m] * V.d + eta * T.dD[m] + (deta[m] * ci + eta * dci[m] - dct[m]) * n +
                              (eta * ci - ct) * dn[m];
                V.d = unit3(eta * V.d + (eta * ci - ct) * n);
                V.med = m2;
            }
        }
        V.b += 1;
        prev = hit;
    }
}

// Arrivals are replayed grouped by path shape, so that the lanes of a warp replay the same
// number of interactions and end in the same kind of event: key = (aperture return or
// scatterer event, interactions before it), counting-sorted (per-CTA shared-memory
// histograms, one scan, a scatter of the arrival indices).
__device__ __forceinline__ uint32_t shape_key(uint32_t ev) { return ((ev >> 31) << 7) | ((ev >> 24) & 0x7Fu); }

__device__ __forceinline__ void arrival_range(const AdjP &A, uint64_t &b, uint64_t &e) {
    const uint64_t n = min((uint64_t)*A.n_arr, A.arr_cap);
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    b = min(n, (uint64_t)blockIdx.x * per);
    e = min(n, b + per);
}

__global__ void k_adj_count(const AdjP A) {
    __shared__ uint32_t h[kAdjKeys];
    for (int q = threadIdx.x; q < kAdjKeys; q += blockDim.x) h[q] = 0u;
    __syncthreads();
    uint64_t b, e;
    arrival_range(A, b, e);
    for (uint64_t k = b + threadIdx.x; k < e; k += blockDim.x) atomicAdd(&h[shape_key(A.rec[k].y)], 1u);
    __syncthreads();
    for (int q = threadIdx.x; q < kAdjKeys; q += blockDim.x)
        if (h[q]) atomicAdd(&A.key_count[q], h[q]);
}

__global__ void k_adj_scan(const AdjP A) {   // one CTA of kAdjKeys threads: exclusive scan into the offsets
    __shared__ uint32_t part[kAdjKeys];
    const uint32_t v = A.key_count[threadIdx.x];
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kAdjKeys; off <<= 1) {
        const uint32_t y = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    A.key_count[kAdjKeys + threadIdx.x] = part[threadIdx.x] - v;
}

__global__ void k_adj_scatter(const AdjP A) {
    __shared__ uint32_t pos[kAdjKeys];
    for (int q = threadIdx.x; q < kAdjKeys; q += blockDim.x) pos[q] = 0u;
    __syncthreads();
    uint64_t b, e;
    arrival_range(A, b, e);
    for (uint64_t k = b + threadIdx.x; k < e; k += blockDim.x) atomicAdd(&pos[shape_key(A.rec[k].y)], 1u);
    __syncthreads();
    for (int q = threadIdx.x; q < kAdjKeys; q += blockDim.x)
        if (pos[q]) pos[q] = A.key_count[kAdjKeys + q] + atomicAdd(&A.key_count[2 * kAdjKeys + q], pos[q]);
    __syncthreads();
    for (uint64_t k = b + threadIdx.x; k < e; k += blockDim.x) {
        const uint32_t p = atomicAdd(&pos[shape_key(A.rec[k].y)], 1u);
        if (p < A.arr_cap) A.order[p] = (uint32_t)k;
    }
}

// One thread per recorded arrival (only depositing paths have a gradient), in path-shape order.
__global__ void __launch_bounds__(128) k_adjoint(const __grid_constant__ AdjP A) {
    const TraceP &P = A.T;
    float acc[kNP];
#pragma unroll
    for (int k = 0; k < kNP; ++k) acc[k] = 0.f;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n = min((uint64_t)*A.n_arr, A.arr_cap);
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const uint64_t k = A.order[q];
        const uint32_t row = A.arr[k].x;
        const uint2 rec = A.rec[k];
        const uint32_t item = row / (uint32_t)P.n_el;
        if (item >= (uint32_t)P.n_items) continue;
        const ItemP &IT = P.items[item];
        if (rec.x >= IT.n_rays) continue;
        replay(A, item, IT, rec.x, rec.x % (uint32_t)P.n_el, rec.y, acc);
    }
#pragma unroll
    for (int k = 0; k < kNP; ++k) {
        float v = acc[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(&A.grad[k], (double)v);
    }
}

}  // namespace

void launch_adjoint(const AdjP &A, int sms, cudaStream_t s) {
    if (cudaMemsetAsync(A.key_count, 0, sizeof(uint32_t) * 3 * kAdjKeys, s) != cudaSuccess) return;
    k_adj_count<<<sms * 4, 256, 0, s>>>(A);
    k_adj_scan<<<1, kAdjKeys, 0, s>>>(A);
    k_adj_scatter<<<sms * 4, 256, 0, s>>>(A);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint, 128, 0);
    k_adjoint<<<sms * (per_sm > 0 ? per_sm : 1), 128, 0, s>>>(A);
}

}  // namespace ur
