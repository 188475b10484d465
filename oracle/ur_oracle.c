/*
 * FP64 CPU oracle for UltraRay-style full-path acoustic ray tracing.
 * TEST INFRASTRUCTURE ONLY (see ur_oracle.h): slow, brute force, double precision.
 *
 * Readings of the paper used here (where it is silent, garbled or at odds with
 * the physics the tests pin):
 *  - Refraction (Eqs. 8, 10): eta = c2/c1 (acoustic Snell law), not Z1/Z2.
 *  - Fresnel (Eq. 11): pressure reflection coefficient of a fluid-fluid interface,
 *    r = (Z2 cos_i - Z1 cos_t) / (Z2 cos_i + Z1 cos_t); at normal incidence
 *    (Z2 - Z1)/(Z2 + Z1).  Total internal reflection: r = 1.
 *  - Monte Carlo branch (Sec. 2.3, reflect if y < A_r^2): weight r/R on
 *    reflection and sqrt(1-R)/(1-R) on transmission, so that the expected
 *    amplitude is r (reflected) and sqrt(1-R) (transmitted, energy-normalised).
 *  - Emission (Eq. 6): weight cos(theta)/N with N the rays of one transmit.
 *  - Diverging and focused transmits (Sec. 2.3 "Ray Emission" names them beside
 *    plane waves without formulas): element delays make the wavefront of a
 *    virtual source behind the array, or one converging on a focus in front of
 *    it, both in the lateral (xz) plane; each element fires at its delay (first
 *    element at t = 0) and a ray leaves its emission point along the line from
 *    the virtual source, or toward the focus, projected on the xz plane (the
 *    delays act laterally only, so directions keep y = 0 as for plane waves);
 *    the Eq. 6 weight is the cosine to the element normal over N.
 *  - Synthetic aperture (named among the acquisition schemes of Sec. 1 without
 *    formulas): one element fires at t = 0 and every element receives.  All N
 *    rays of the transmit leave uniform points of that element's face, at an
 *    angle to its normal drawn uniformly in (-pi/2, pi/2) in the xz plane (the
 *    angle the plane-wave scheme fixes is drawn here, Sec. 2.3); the Eq. 6 weight
 *    is the cosine of that angle over N.
 *  - Triangle meshes (the paper's bone is a CT-derived mesh, Sec. 4; the method
 *    handles its triangles like any other surface): each triangle separates the
 *    medium behind it (negative side of (v1 - v0) x (v2 - v0)) from the one in
 *    front, with that unit normal, a Fresnel interface like the analytic
 *    boundaries and the GGX roughness of the rougher medium; a ray leaving a
 *    triangle does not meet it again.  Intersections: Moeller-Trumbore (1997)
 *    over every triangle, brute force.
 *  - Transmit mixing (Sec. 2.3: rays of different acquisition events leave
 *    together, each with a randomly selected angle): in this mode n_tx * N rays
 *    are traced and ray i draws its transmit k uniformly from its own counter;
 *    from there it is ray i of transmit k, with the Eq. 6 weight over N, the
 *    expected number of rays per transmit.
 *  - Convex array (Sec. 2.3 describes the transducer by its elements, elevation,
 *    radius and opening angle): element centres lie `pitch` apart on the arc of
 *    radius R about (0, 0, -R), apex at the origin, normals radial; the probe is
 *    the cylinder inside the arc.  A ray leaves a uniform point of its element's
 *    arc face (weight: cosine to the local normal over N; none if that is not
 *    positive); returning rays end on the cylinder, inside the aperture at the
 *    element whose arc holds the hit, and rays passing the probe end on the plane
 *    z = -R.  Connections, directivities and delays use element centres and
 *    normals.
 *  - Transducer sampling: delta (smooth) boundaries contribute only through the
 *    primary ray crossing the array plane; point scatterers contribute only
 *    through a straight connection ray to a uniformly chosen element centre,
 *    with a sqrt(1-R) factor per boundary crossed, 0 on total internal
 *    reflection, and weight n_el (inverse element-choice probability).
 *  - Scatterers: every scatterer within r_s of a ray segment is an event at the
 *    closest-approach distance t_ca along the ray; the connection leaves from
 *    the scatterer position; scatterers do not redirect the ray.
 *  - Attenuation: amplitude factor exp(-a l), a in Np/m from dB/cm/MHz at f0.
 *  - Pulse (Eq. 14): analytic pulse exp(-tau^2/(2 s^2)) (sin(w tau) - j cos(w tau)),
 *    s = n_cycles/(4 f0), deposited at the exact arrival time, truncated at
 *    |tau| <= tcut_sigmas * s.
 *  - Rough boundaries (Sec. 2.3, Eq. 12): a boundary takes the larger GGX
 *    roughness of its two media.  The paper gives only the distribution D; the
 *    rest follows the microfacet model it cites (Walter et al. 2007): the
 *    microfacet normal m is drawn with density D(m)(m.n), the smooth branch of
 *    Eqs. 7-11 is taken about m, and the weight gains |i.m| G / (|i.n| |m.n|)
 *    with the separable Smith G; a sample leaving on the wrong side of the
 *    macro surface ends the ray.  In the amplitude convention above the BSDF
 *    carries the microfacet's r (reflection) or sqrt(1-R) (transmission) where
 *    the intensity form has F or 1-F.
 *  - Transducer sampling at rough boundaries (Sec. 2.3: at each boundary
 *    encounter, before the BSDF is sampled): a connection to a uniformly drawn
 *    element centre with the BSDF toward it and the element's solid angle
 *    A cos / D^2 standing for the integral over the element face.  It and the
 *    direct aperture hits of paths that left a rough vertex (with only smooth
 *    transmissions before the array) are combined by the balance heuristic,
 *    the element's density being 1 / (n_el * solid angle); as the roughness
 *    goes to 0 the direct hits take all the weight and the smooth result returns.
 */
#include "ur_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TMIN 1e-7              /* m: smallest admissible hit distance */
#define OR_MAX_CROSS 64           /* connection rays cross at most this many boundaries */
#define OR_MAX_SEG 4096           /* safety bound on primary segments */
#define OR_FNV_OFFSET 0xcbf29ce484222325ULL
#define OR_FNV_PRIME 0x100000001b3ULL
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications with the
 * Philox multipliers, the key bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0, 1) from the top 24 bits: exact in float and double. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

static void draw(uint64_t seed, uint32_t i, uint32_t k, uint32_t kind_b, uint32_t aux, uint32_t out[4])
{
    uint32_t ctr[4] = {i, k, kind_b, aux};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ---------------------------------------------------------- small helpers */

static double dot3(const double a[3], const double b[3]) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

static void normalize3(double a[3])
{
    double l = sqrt(dot3(a, a));
    a[0] /= l; a[1] /= l; a[2] /= l;
}

static uint64_t fnv(uint64_t h, uint32_t word) { return (h ^ (uint64_t)word) * OR_FNV_PRIME; }

double or_np_per_m(double alpha_db_cm_mhz, double f0)
{
    /* dB/cm/MHz -> dB/m at f0 -> Np/m (amplitude): 1 Np = 20 log10(e) dB */
    double db_per_m = alpha_db_cm_mhz * (f0 * 1e-6) * 100.0;
    return db_per_m / (20.0 * log10(exp(1.0)));
}

/* Eq. 13: piecewise-linear receive directivity in the incidence angle. */
double or_directivity(double alpha, double alpha_m, double alpha_c)
{
    double a = fabs(alpha);
    if (a > alpha_c) return 0.0;
    if (a > alpha_m) return (alpha_c - a) / (alpha_c - alpha_m);
    return 1.0;
}

/* Eq. 14, analytic form: real part sin(2 pi f0 tau) exp(-tau^2/(2 s^2)),
 * quadrature part -cos(2 pi f0 tau) exp(-tau^2/(2 s^2)), s = n_cycles/(4 f0). */
double or_pulse(double tau, double f0, double n_cycles, double *imag)
{
    double s = n_cycles / (4.0 * f0);
    double g = exp(-tau * tau / (2.0 * s * s));
    double ph = 2.0 * OR_PI * f0 * tau;
    if (imag) *imag = -g * cos(ph);
    return g * sin(ph);
}

/* Eqs. 7-11 at one boundary. */
int or_interface(const double d[3], const double n[3], double c1, double Z1,
                 double c2, double Z2, double d_r[3], double d_t[3],
                 double *r, double *R)
{
    double nn[3] = {n[0], n[1], n[2]};
    if (dot3(d, nn) > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
    double cos_i = -dot3(nn, d);                               /* Eq. 7 */
    for (int q = 0; q < 3; ++q) d_r[q] = d[q] + 2.0 * cos_i * nn[q]; /* Eq. 9 */
    normalize3(d_r);
    double eta = c2 / c1;
    double k = 1.0 - eta * eta * (1.0 - cos_i * cos_i);
    if (k < 0.0) {                                             /* total internal reflection */
        d_t[0] = d_t[1] = d_t[2] = 0.0;
        *r = 1.0; *R = 1.0;
        return 1;
    }
    double cos_t = sqrt(k);                                    /* Eq. 8 */
    for (int q = 0; q < 3; ++q) d_t[q] = eta * d[q] + (eta * cos_i - cos_t) * nn[q]; /* Eq. 10 */
    normalize3(d_t);
    *r = (Z2 * cos_i - Z1 * cos_t) / (Z2 * cos_i + Z1 * cos_t); /* Eq. 11 (acoustic) */
    *R = (*r) * (*r);
    return 0;
}

/* ------------------------------------------------------------ scene state */

typedef struct {
    const or_scene *sc;
    const or_array *ar;
    const or_trace_cfg *cfg;
    double *c, *Z, *a, *slow;   /* per medium; slow in samples per metre */
    double *cs, *Zs;            /* per medium: c and Z deciding the Monte Carlo branches */
    double *delay;              /* [n_tx][n_el] transmit delays in samples */
    double *sin_t, *cos_t;      /* per transmit */
    double x0, pitch, H;        /* centre of element 0, pitch, elevation height */
    double K, t_last;           /* pulse half-width; latest useful arrival time (samples) */
    double am, ac;              /* directivity angles (rad) */
    int top, bot;               /* ids of the terminal planes */
    double *alpha_b;            /* per boundary: GGX roughness (0: smooth) */
    double R, dphi, phi0;       /* convex array: radius, angle between centres, angle of element 0 */
    int esc;                    /* id of the escape plane z = -R (convex arrays) */
    int *kind;                  /* per transmit: OR_TX_* */
    double *vx, *vz;            /* per transmit: virtual source or focus (m) */
    int tri0;                   /* hit id of triangle 0 */
} ctx_t;

static double elem_x(const ctx_t *C, int e) { return C->x0 + (double)e * C->pitch; }

/* Centre and unit normal of element e (linear: (x_e, 0, 0), +z). */
static void elem_frame(const ctx_t *C, int e, double c[3], double n[3])
{
    if (C->R > 0.0) {
        double ph = C->phi0 + (double)e * C->dphi;
        n[0] = sin(ph); n[1] = 0.0; n[2] = cos(ph);
        c[0] = C->R * n[0]; c[1] = 0.0; c[2] = C->R * (n[2] - 1.0);
    } else {
        c[0] = elem_x(C, e); c[1] = 0.0; c[2] = 0.0;
        n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    }
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Distance along o + t d to triangle t (Moeller-Trumbore: barycentric u, v of the
 * hit from Cramer's rule on o + t d = v0 + u e1 + v e2), INFINITY if none. */
static double triangle_hit(const or_scene *sc, int t, const double o[3], const double d[3])
{
    const float *v = &sc->tri[9 * t];
    double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
    double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
    double p[3], q[3];
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return INFINITY;             /* ray parallel to the triangle's plane */
    double s[3] = {o[0] - v[0], o[1] - v[1], o[2] - v[2]};
    double u = dot3(s, p) / det;
    if (u < 0.0 || u > 1.0) return INFINITY;
    cross3(s, e1, q);
    double w = dot3(d, q) / det;
    if (w < 0.0 || u + w > 1.0) return INFINITY;
    return dot3(e2, q) / det;
}

/* Nearest boundary along o + t d with t in (OR_TMIN, inf).  `skip` is the
 * primitive the ray is leaving: a plane cannot be hit again, a sphere or
 * cylinder only at its far root.  With terminals, z = 0 (upward rays) and
 * z = z_max (downward rays) are included.  Returns the primitive id or -1. */
static int nearest_boundary(const ctx_t *C, const double o[3], const double d[3], int skip,
                            int terminals, double *t_out)
{
    const or_scene *sc = C->sc;
    double best = INFINITY;
    int hit = -1;
    for (int p = 0; p < sc->n_bnd; ++p) {
        const float *q = &sc->bnd_p[4 * p];
        double t = INFINITY;
        if (sc->bnd_kind[p] == OR_PLANE_Z) {
            if (p == skip || d[2] == 0.0) continue;
            t = ((double)q[0] - o[2]) / d[2];
        } else if (sc->bnd_kind[p] == OR_SPHERE) {
            double oc[3] = {o[0] - q[0], o[1] - q[1], o[2] - q[2]};
            double b = dot3(oc, d);
            if (p == skip) {
                t = -2.0 * b;
            } else {
                double f[3] = {oc[0] - b * d[0], oc[1] - b * d[1], oc[2] - b * d[2]};
                double disc = (double)q[3] * q[3] - dot3(f, f);
                if (disc < 0.0) continue;
                double s = sqrt(disc);
                t = -b - s;
                if (!(t > OR_TMIN)) t = -b + s;
            }
        } else { /* OR_CYL_Y */
            double ocx = o[0] - q[0], ocz = o[2] - q[1];
            double a = d[0] * d[0] + d[2] * d[2];
            if (a == 0.0) continue;
            double b = (ocx * d[0] + ocz * d[2]) / a;
            if (p == skip) {
                t = -2.0 * b;
            } else {
                double fx = ocx - b * d[0], fz = ocz - b * d[2];
                double disc = ((double)q[2] * q[2] - (fx * fx + fz * fz)) / a;
                if (disc < 0.0) continue;
                double s = sqrt(disc);
                t = -b - s;
                if (!(t > OR_TMIN)) t = -b + s;
            }
        }
        if (t > OR_TMIN && t < best) { best = t; hit = p; }
    }
    for (int q = 0; q < sc->n_tri; ++q) {        /* triangles: brute force */
        if (C->tri0 + q == skip) continue;
        double t = triangle_hit(sc, q, o, d);
        if (t > OR_TMIN && t < best) { best = t; hit = C->tri0 + q; }
    }
    if (terminals && C->R > 0.0) {   /* convex probe: its cylinder, the escape plane z = -R, the bottom */
        double ox = o[0], oz = o[2] + C->R;
        double a = d[0] * d[0] + d[2] * d[2];
        if (a > 0.0) {
            double b = ox * d[0] + oz * d[2], cc = ox * ox + oz * oz - C->R * C->R;
            double disc = b * b - a * cc;
            if (disc >= 0.0 && b < 0.0) {
                double t = (-b - sqrt(disc)) / a;
                if (t > OR_TMIN && t < best) { best = t; hit = C->top; }
            }
        }
        if (d[2] < 0.0) {
            double t = (-C->R - o[2]) / d[2];
            if (t > OR_TMIN && t < best) { best = t; hit = C->esc; }
        } else if (d[2] > 0.0) {
            double t = ((double)sc->z_max - o[2]) / d[2];
            if (t > OR_TMIN && t < best) { best = t; hit = C->bot; }
        }
    } else if (terminals) {
        if (d[2] < 0.0) {
            double t = -o[2] / d[2];
            if (t > OR_TMIN && t < best) { best = t; hit = C->top; }
        } else if (d[2] > 0.0) {
            double t = ((double)sc->z_max - o[2]) / d[2];
            if (t > OR_TMIN && t < best) { best = t; hit = C->bot; }
        }
    }
    *t_out = best;
    return hit;
}

/* Outward normal of primitive p at point h (unit). */
static void outward_normal(const ctx_t *C, int p, const double h[3], double n[3])
{
    if (p >= C->tri0) {                          /* triangle: (v1 - v0) x (v2 - v0) */
        const float *v = &C->sc->tri[9 * (p - C->tri0)];
        double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
        double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]};
        cross3(e1, e2, n);
        normalize3(n);
        return;
    }
    const float *q = &C->sc->bnd_p[4 * p];
    if (C->sc->bnd_kind[p] == OR_PLANE_Z) {
        n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    } else if (C->sc->bnd_kind[p] == OR_SPHERE) {
        n[0] = h[0] - q[0]; n[1] = h[1] - q[1]; n[2] = h[2] - q[2];
        normalize3(n);
    } else {
        n[0] = h[0] - q[0]; n[1] = 0.0; n[2] = h[2] - q[1];
        normalize3(n);
    }
}

/* Medium on the far side of primitive p for a ray moving along d at h. */
static int far_medium(const ctx_t *C, int p, const double d[3], const double n_out[3])
{
    const int32_t *m = p >= C->tri0 ? &C->sc->tri_med[2 * (p - C->tri0)] : &C->sc->bnd_med[2 * p];
    return dot3(d, n_out) > 0.0 ? m[1] : m[0];
}

/* Connection (secondary) ray: straight from p to the element centre; `skip0` is
 * the boundary p lies on (-1 for a point inside a medium). */
static double connection_to(const ctx_t *C, const double p[3], int med, int skip0, const double q[3],
                            double *t_samples, double *atten)
{
    double o[3] = {p[0], p[1], p[2]};
    double w[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    double rem = sqrt(dot3(w, w));
    w[0] /= rem; w[1] /= rem; w[2] /= rem;
    double fac = 1.0, t = 0.0, att = 0.0;
    int m = med, skip = skip0;
    for (int it = 0; it < OR_MAX_CROSS; ++it) {
        double th;
        int hit = nearest_boundary(C, o, w, skip, 0, &th);
        if (hit < 0 || th >= rem) {
            t += rem * C->slow[m];
            att += C->a[m] * rem;
            break;
        }
        t += th * C->slow[m];
        att += C->a[m] * th;
        double h[3] = {o[0] + th * w[0], o[1] + th * w[1], o[2] + th * w[2]};
        if (hit < C->sc->n_bnd && C->sc->bnd_kind[hit] == OR_PLANE_Z) h[2] = C->sc->bnd_p[4 * hit];
        double n_out[3];
        outward_normal(C, hit, h, n_out);
        int m2 = far_medium(C, hit, w, n_out);
        double dr[3], dt[3], r, R;
        if (or_interface(w, n_out, C->c[m], C->Z[m], C->c[m2], C->Z[m2], dr, dt, &r, &R))
            return 0.0;
        fac *= sqrt(1.0 - R);
        m = m2;
        o[0] = h[0]; o[1] = h[1]; o[2] = h[2];
        rem -= th;
        skip = hit;
    }
    *t_samples = t;
    *atten = att;
    return fac;
}

static double connection(const ctx_t *C, const double p[3], int med, double x_e,
                         double *t_samples, double *atten)
{
    double q[3] = {x_e, 0.0, 0.0};
    return connection_to(C, p, med, -1, q, t_samples, atten);
}

/* ------------------------------------------------------ rough boundaries */

/* Eq. 12: GGX density of microfacet normals, cos_m = n.h. */
double or_ggx_d(double cos_m, double alpha)
{
    if (!(cos_m > 0.0)) return 0.0;
    double a2 = alpha * alpha;
    double k = cos_m * cos_m * (a2 - 1.0) + 1.0;
    return a2 / (OR_PI * k * k);
}

/* Smith masking of one direction for GGX (Walter et al. 2007, Eq. 34);
 * c = cosine between that direction and the macro normal (c > 0). */
double or_ggx_g1(double c, double alpha)
{
    double tan2 = (1.0 - c * c) / (c * c);
    return 2.0 / (1.0 + sqrt(1.0 + alpha * alpha * tan2));
}

/* Orthonormal basis (t1, t2, n) around a unit n (Duff et al., "Building an
 * orthonormal basis, revisited", JCGT 6(1), 2017). */
static void onb(const double n[3], double t1[3], double t2[3])
{
    double sg = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    t1[0] = 1.0 + sg * n[0] * n[0] * a; t1[1] = sg * b; t1[2] = -sg * n[0];
    t2[0] = b; t2[1] = sg + n[1] * n[1] * a; t2[2] = -n[1];
}

/* Microfacet normal with density D(m)(m.n): tan^2(theta_m) = alpha^2 xi1 / (1 - xi1),
 * phi_m = 2 pi xi2 (the inversion of its CDF, Walter et al. 2007, Eqs. 35-36). */
void or_ggx_sample(const double n[3], double alpha, double xi1, double xi2, double m[3])
{
    double tan2 = alpha * alpha * xi1 / (1.0 - xi1);
    double ct = 1.0 / sqrt(1.0 + tan2);
    double st = sqrt(tan2) * ct;
    double ph = 2.0 * OR_PI * xi2;
    double t1[3], t2[3];
    onb(n, t1, t2);
    for (int q = 0; q < 3; ++q) m[q] = st * cos(ph) * t1[q] + st * sin(ph) * t2[q] + ct * n[q];
}

/* Scattering of a rough boundary from incident direction d (unit, travelling
 * toward the surface; n the unit macro normal facing the incident side) into
 * o: returns f(i, o) |o.n| in the amplitude form and writes the solid-angle
 * density *pdf with which microfacet sampling and the reflect-if-y < R branch
 * produce o.  Reflection (o.n > 0): half vector h = (i + o)/|i + o|,
 * |dw_h/dw_o| = 1/(4 |o.h|), coefficient r(h), branch probability R(h) (1 on
 * total internal reflection).  Transmission (o.n < 0): h along -(i/c1 + o/c2),
 * |dw_h/dw_o| = |o.h| / (c2^2 (i.h/c1 + o.h/c2)^2), coefficient sqrt(1-R(h)),
 * branch probability 1 - R(h).  f |o.n| = coef G D(h) |i.h| |dw_h/dw_o| / |i.n|. */
double or_rough_eval(const double d[3], const double n[3], const double o[3], double alpha,
                     double c1, double Z1, double c2, double Z2, double *pdf)
{
    *pdf = 0.0;
    double i[3] = {-d[0], -d[1], -d[2]};
    double cos_i = dot3(i, n), cos_o = dot3(o, n);
    if (!(cos_i > 0.0) || cos_o == 0.0) return 0.0;
    double h[3], jac, coef, pb;
    if (cos_o > 0.0) {
        for (int q = 0; q < 3; ++q) h[q] = i[q] + o[q];
        normalize3(h);
        double ih = dot3(i, h);
        if (!(dot3(h, n) > 0.0) || !(ih > 0.0)) return 0.0;
        double dr[3], dt[3], r, R;
        int tir = or_interface(d, h, c1, Z1, c2, Z2, dr, dt, &r, &R);
        coef = tir ? 1.0 : r;
        pb = tir ? 1.0 : R;
        jac = 1.0 / (4.0 * dot3(o, h));
    } else {
        for (int q = 0; q < 3; ++q) h[q] = -(i[q] / c1 + o[q] / c2);
        normalize3(h);
        if (dot3(h, n) < 0.0) { h[0] = -h[0]; h[1] = -h[1]; h[2] = -h[2]; }
        double ih = dot3(i, h), oh = dot3(o, h);
        if (!(dot3(h, n) > 0.0) || !(ih > 0.0) || !(oh < 0.0)) return 0.0;
        double dr[3], dt[3], r, R;
        if (or_interface(d, h, c1, Z1, c2, Z2, dr, dt, &r, &R)) return 0.0;
        double den = ih / c1 + oh / c2;
        if (den * den < 1e-300) return 0.0;
        coef = sqrt(1.0 - R);
        pb = 1.0 - R;
        jac = -oh / (c2 * c2 * den * den);
    }
    double hn = dot3(h, n);
    double D = or_ggx_d(hn, alpha);
    double G = or_ggx_g1(cos_i, alpha) * or_ggx_g1(fabs(cos_o), alpha);
    *pdf = D * hn * jac * pb;
    return coef * G * D * dot3(i, h) * jac / cos_i;
}

/* ------------------------------------------------------- arrival buffers */

typedef struct {
    or_arrival a;
    uint64_t order;   /* (tx, ray, sequence) sort key */
    uint32_t seq;
} rec_t;

typedef struct {
    rec_t *v;
    size_t n, cap;
} abuf_t;

static void push(abuf_t *b, int tx, int el, uint32_t ray, uint32_t ev, double t, double amp, uint32_t seq)
{
    if (b->n == b->cap) {
        b->cap = b->cap ? 2 * b->cap : 1024;
        b->v = (rec_t *)realloc(b->v, b->cap * sizeof(rec_t));
    }
    rec_t *r = &b->v[b->n++];
    r->a.tx = tx; r->a.el = el; r->a.ray = ray; r->a.event = ev; r->a.t = t; r->a.amp = amp;
    r->order = ((uint64_t)(uint32_t)tx << 32) | ray;
    r->seq = seq;
}

static int rec_cmp(const void *pa, const void *pb)
{
    const rec_t *a = (const rec_t *)pa, *b = (const rec_t *)pb;
    if (a->order != b->order) return a->order < b->order ? -1 : 1;
    if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
    return 0;
}

typedef struct {
    uint32_t i;
    int k;
    uint32_t seq;
    abuf_t *buf;
    or_stats st;
} ray_job;

/* ----------------------------------------------------- transducer sampling */

/* Events of scatterer j seen from the ray segment starting at o (segment b):
 * connection to one random element (MC) or to every element (expectation). */
static void scatter_event(const ctx_t *C, ray_job *J, int j, double t_ca, double t, double w,
                          int med, int b)
{
    const float *s = &C->sc->scat[4 * j];
    double p[3] = {s[0], s[1], s[2]};
    int n_el = C->ar->n_el;
    int e_lo = 0, e_hi = n_el;
    double pick_w = 1.0;
    if (C->cfg->mode == OR_MODE_MC) {
        uint32_t x[4];
        draw(C->cfg->seed, J->i, (uint32_t)J->k, 2u | ((uint32_t)b << 8), (uint32_t)j, x);
        int e = (int)((((uint64_t)(x[0] >> 8)) * (uint64_t)n_el) >> 24);
        e_lo = e; e_hi = e + 1;
        pick_w = (double)n_el;               /* 1 / p(element) */
    }
    for (int e = e_lo; e < e_hi; ++e) {
        double ce[3], ne[3];
        elem_frame(C, e, ce, ne);
        double v[3] = {ce[0] - p[0], ce[1] - p[1], ce[2] - p[2]};
        double D = sqrt(dot3(v, v));
        double alpha = acos(-dot3(v, ne) / D);               /* to the element normal */
        double fd = or_directivity(alpha, C->am, C->ac);   /* Eq. 13 */
        if (!(fd > 0.0)) continue;
        J->st.connections++;
        double tc, ac;
        double fac = connection_to(C, p, med, -1, ce, &tc, &ac);
        if (fac == 0.0) continue;
        double t_arr = t + t_ca * C->slow[med] + tc;
        if (t_arr > C->t_last) continue;
        double amp = w * exp(-C->a[med] * t_ca) * (double)s[3] * pick_w * fd * fac * exp(-ac);
        push(J->buf, J->k, e, J->i, ((uint32_t)b << 24) | (uint32_t)j, t_arr, amp, J->seq++);
        J->st.arrivals++;
    }
}

/* All scatterers within r_s of the open segment o + t d, 0 < t < seg. */
static void segment_scatterers(const ctx_t *C, ray_job *J, const double o[3], const double d[3],
                               double seg, double t, double w, int med, int b)
{
    const or_scene *sc = C->sc;
    double r2 = (double)sc->r_s * sc->r_s;
    for (int j = 0; j < sc->n_scat; ++j) {
        const float *s = &sc->scat[4 * j];
        double v[3] = {s[0] - o[0], s[1] - o[1], s[2] - o[2]};
        double t_ca = dot3(v, d);
        if (!(t_ca > 0.0 && t_ca < seg)) continue;
        double q[3] = {v[0] - t_ca * d[0], v[1] - t_ca * d[1], v[2] - t_ca * d[2]};
        if (!(dot3(q, q) < r2)) continue;
        J->st.candidates++;
        scatter_event(C, J, j, t_ca, t, w, med, b);
    }
}

/* Transducer sampling at a rough vertex p on boundary `hit` (d incident, n the
 * normal facing the incident side; med / m2 the near / far media): connection to
 * a uniformly drawn element centre, balance-heuristic weight against the BSDF
 * sampling of the same direction. */
static void rough_nee(const ctx_t *C, ray_job *J, const double p[3], const double d[3], const double n[3],
                      int hit, int med, int m2, double t, double w, int b)
{
    int n_el = C->ar->n_el;
    uint32_t x[4];
    draw(C->cfg->seed, J->i, (uint32_t)J->k, 4u | ((uint32_t)b << 8), 0u, x);
    int e = (int)((((uint64_t)(x[0] >> 8)) * (uint64_t)n_el) >> 24);
    double ce[3], ne[3];
    elem_frame(C, e, ce, ne);
    double v[3] = {ce[0] - p[0], ce[1] - p[1], ce[2] - p[2]};
    double D = sqrt(dot3(v, v));
    double o[3] = {v[0] / D, v[1] / D, v[2] / D};
    double cos_e = -dot3(o, ne);                           /* at the element, to its normal */
    double fd = or_directivity(acos(cos_e), C->am, C->ac);  /* Eq. 13 */
    if (!(fd > 0.0)) return;
    double pdf_bsdf;
    double f = or_rough_eval(d, n, o, C->alpha_b[hit], C->c[med], C->Z[med], C->c[m2], C->Z[m2], &pdf_bsdf);
    if (!(f > 0.0)) return;
    J->st.connections++;
    double tc, ac;
    double fac = connection_to(C, p, dot3(o, n) > 0.0 ? med : m2, hit, ce, &tc, &ac);
    if (fac == 0.0) return;
    double t_arr = t + tc;
    if (t_arr > C->t_last) return;
    double omega = C->pitch * C->H * cos_e / (D * D);    /* element solid angle seen from p */
    double p_nee = 1.0 / ((double)n_el * omega);
    double amp = w * f * fd * fac * exp(-ac) / (p_nee + pdf_bsdf);
    push(J->buf, J->k, e, J->i, 0x80000000u | ((uint32_t)b << 24) | (uint32_t)(hit + 1), t_arr, amp, J->seq++);
    J->st.arrivals++;
}

/* BSDF sampling at a rough vertex: microfacet normal, smooth branch about it,
 * Walter's weight.  Updates d, w, med; writes the branch (0 reflect, 1 transmit,
 * 2 total internal reflection) and the solid-angle density of the new direction.
 * Returns 0, or OR_END_ROUGH if the sample is not admissible. */
static int rough_scatter(const ctx_t *C, ray_job *J, double d[3], const double n[3], double alpha,
                         int *med, int m2, double *w, int b, int *branch, double *pdf)
{
    double cos_i = -dot3(d, n);
    uint32_t x[4];
    draw(C->cfg->seed, J->i, (uint32_t)J->k, 3u | ((uint32_t)b << 8), 0u, x);
    double m[3];
    or_ggx_sample(n, alpha, u24(x[0]), u24(x[1]), m);
    double c_im = -dot3(d, m), mn = dot3(m, n);
    if (!(c_im > 0.0)) return OR_END_ROUGH;
    double c1 = C->c[*med], c2 = C->c[m2];
    double dr[3], dt[3], r, R;
    int tir = or_interface(d, m, c1, C->Z[*med], c2, C->Z[m2], dr, dt, &r, &R);
    double o[3], fac, pb, jac;
    int to_far = 0;
    if (tir) {
        *branch = 2; memcpy(o, dr, sizeof o); fac = 1.0; pb = 1.0; jac = 1.0 / (4.0 * c_im);
    } else {
        uint32_t y[4];
        draw(C->cfg->seed, J->i, (uint32_t)J->k, 1u | ((uint32_t)b << 8), 0u, y);
        if (u24(y[0]) < R) {                                   /* reflect if y < A_r^2 */
            *branch = 0; memcpy(o, dr, sizeof o); fac = r / R; pb = R; jac = 1.0 / (4.0 * c_im);
        } else {
            *branch = 1; memcpy(o, dt, sizeof o); fac = sqrt(1.0 - R) / (1.0 - R); pb = 1.0 - R;
            double om = dot3(o, m), den = c_im / c1 + om / c2;
            jac = -om / (c2 * c2 * den * den);
            to_far = 1;
        }
    }
    double on = dot3(o, n);
    if (to_far ? !(on < 0.0) : !(on > 0.0)) return OR_END_ROUGH;
    double G = or_ggx_g1(cos_i, alpha) * or_ggx_g1(fabs(on), alpha);
    *w *= fac * c_im * G / (cos_i * mn);
    *pdf = or_ggx_d(mn, alpha) * mn * jac * pb;
    memcpy(d, o, sizeof o);
    if (to_far) *med = m2;
    return 0;
}

/* ------------------------------------------------------------ primary path */

/* Follows one primary ray (and, in expectation mode, both branches of every
 * interaction).  Returns the termination reason; *h accumulates the path hash. */
static int follow(const ctx_t *C, ray_job *J, double o[3], double d[3], double t, double w,
                  int med, int b, double L, int prev, uint64_t *h)
{
    const or_scene *sc = C->sc;
    const or_array *ar = C->ar;
    const or_trace_cfg *cfg = C->cfg;
    int mis = 0;                  /* the path left a rough vertex with smooth transmissions since */
    double mis_p[3] = {0.0, 0.0, 0.0}, mis_pdf = 0.0;
    for (int guard = 0; guard < OR_MAX_SEG; ++guard) {
        double th;
        int hit = nearest_boundary(C, o, d, prev, 1, &th);
        double seg = th;
        int clipped = 0;
        if (L + seg > (double)cfg->max_path) { seg = (double)cfg->max_path - L; clipped = 1; }
        J->st.segments++;
        if (sc->n_scat > 0) segment_scatterers(C, J, o, d, seg, t, w, med, b);
        /* advance along the segment: time of flight and attenuation */
        t += seg * C->slow[med];
        w *= exp(-C->a[med] * seg);
        L += seg;
        for (int q = 0; q < 3; ++q) o[q] += seg * d[q];
        if (clipped) return OR_END_PATH;
        if (hit == C->esc) return OR_END_ARRAY_MISS;
        if (hit == C->top) {
            int e = -1;
            if (C->R > 0.0) {   /* on the probe's cylinder: the element whose arc holds the hit */
                double ph = atan2(o[0], o[2] + C->R);
                double u = (ph - C->phi0) / C->dphi + 0.5;
                if (fabs(o[1]) <= 0.5 * C->H && u >= 0.0 && u < (double)ar->n_el) e = (int)floor(u);
            } else {
                o[2] = 0.0;
                double xl = C->x0 - 0.5 * C->pitch;
                if (fabs(o[1]) <= 0.5 * C->H && o[0] >= xl && o[0] < xl + ar->n_el * C->pitch) {
                    e = (int)floor((o[0] - xl) / C->pitch);
                    if (e > ar->n_el - 1) e = ar->n_el - 1;
                }
            }
            if (e >= 0) {
                double ce[3], ne[3];
                elem_frame(C, e, ce, ne);
                double fd = or_directivity(acos(-dot3(d, ne)), C->am, C->ac);
                if (fd > 0.0 && t <= C->t_last) {
                    double wa = w * fd;
                    if (mis && !cfg->rough_bsdf_only) {   /* balance heuristic against transducer sampling */
                        double v[3] = {ce[0] - mis_p[0], ce[1] - mis_p[1], ce[2] - mis_p[2]};
                        double D2 = dot3(v, v);
                        double omega = C->pitch * C->H * (-dot3(v, ne) / sqrt(D2)) / D2;
                        if (omega > 0.0) wa *= mis_pdf / (mis_pdf + 1.0 / ((double)ar->n_el * omega));
                    }
                    push(J->buf, J->k, e, J->i, 0x80000000u | ((uint32_t)b << 24), t, wa, J->seq++);
                    J->st.arrivals++;
                }
                return OR_END_APERTURE;
            }
            return OR_END_ARRAY_MISS;
        }
        if (hit == C->bot) return OR_END_BOTTOM;
        if (hit < sc->n_bnd && sc->bnd_kind[hit] == OR_PLANE_Z) o[2] = sc->bnd_p[4 * hit];
        if (t > C->t_last) return OR_END_TIME;
        if (b >= cfg->max_bounces) return OR_END_MAXB;
        /* interaction (Eqs. 7-11) */
        double n_out[3], dr[3], dt[3], r, R;
        outward_normal(C, hit, o, n_out);
        int m2 = far_medium(C, hit, d, n_out);
        if (C->alpha_b[hit] > 0.0) {   /* rough boundary (Eq. 12) */
            double nn[3] = {n_out[0], n_out[1], n_out[2]};
            if (dot3(d, nn) > 0.0) { nn[0] = -nn[0]; nn[1] = -nn[1]; nn[2] = -nn[2]; }
            if (!cfg->rough_bsdf_only) rough_nee(C, J, o, d, nn, hit, med, m2, t, w, b);
            J->st.interactions++;
            int branch = 0;
            double pdf = 0.0;
            int end = rough_scatter(C, J, d, nn, C->alpha_b[hit], &med, m2, &w, b, &branch, &pdf);
            if (end) return end;
            mis = 1;
            memcpy(mis_p, o, sizeof mis_p);
            mis_pdf = pdf;
            *h = fnv(*h, 0x10000u | ((uint32_t)hit << 4) | (uint32_t)branch);
            b += 1;
            prev = hit;
            continue;
        }
        int tir = or_interface(d, n_out, C->c[med], C->Z[med], C->c[m2], C->Z[m2], dr, dt, &r, &R);
        /* the branch is drawn with the sampling media (the same media unless overridden) */
        double drs[3], dts[3], rs = r, Rs = R;
        int tir_s = tir;
        if (sc->med_sampling)
            tir_s = or_interface(d, n_out, C->cs[med], C->Zs[med], C->cs[m2], C->Zs[m2], drs, dts, &rs, &Rs);
        J->st.interactions++;
        int branch;
        if (tir_s && cfg->mode == OR_MODE_MC) {
            branch = 2;
            memcpy(d, dr, sizeof dr);
        } else if (tir) {
            branch = 2;
            memcpy(d, dr, sizeof dr);
        } else if (cfg->mode == OR_MODE_MC) {
            uint32_t x[4];
            draw(cfg->seed, J->i, (uint32_t)J->k, 1u | ((uint32_t)b << 8), 0u, x);
            if (u24(x[0]) < Rs) {           /* reflect if y < A_r^2 */
                branch = 0;
                w *= r / Rs;
                memcpy(d, dr, sizeof dr);
            } else {
                branch = 1;
                w *= sqrt(1.0 - R) / (1.0 - Rs);
                memcpy(d, dt, sizeof dt);
                med = m2;
            }
        } else {
            /* expectation: the reflected branch is followed recursively with
             * amplitude r, the transmitted one continues here with sqrt(1-R) */
            branch = 1;
            if (r != 0.0) {
                double o2[3] = {o[0], o[1], o[2]};
                uint64_t h2 = 0;
                follow(C, J, o2, dr, t, w * r, med, b + 1, L, hit, &h2);
            }
            w *= sqrt(1.0 - R);
            memcpy(d, dt, sizeof dt);
            med = m2;
        }
        if (branch != 1) mis = 0;   /* a smooth reflection: transducer sampling cannot produce this path */
        *h = fnv(*h, 0x10000u | ((uint32_t)hit << 4) | (uint32_t)branch);
        b += 1;
        prev = hit;
    }
    return OR_END_PATH;
}

/* Ray emission (Sec. 2.3, Eq. 6) followed by traversal. */
static uint64_t trace_ray(const ctx_t *C, ray_job *J)
{
    const or_array *ar = C->ar;
    const int sa = C->kind[J->k] == OR_TX_SYNTHETIC;
    int e = sa ? (int)C->vx[J->k] : (int)(J->i % (uint32_t)ar->n_el);
    uint32_t x[4];
    draw(C->cfg->seed, J->i, (uint32_t)J->k, 0u, 0u, x);
    double o[3] = {elem_x(C, e) + (u24(x[0]) - 0.5) * C->pitch, (u24(x[1]) - 0.5) * C->H, 0.0};
    double nrm[3] = {0.0, 0.0, 1.0};              /* normal at the emission point */
    if (C->R > 0.0) {                              /* a point of the element's arc face */
        double ph = C->phi0 + ((double)e + u24(x[0]) - 0.5) * C->dphi;
        nrm[0] = sin(ph); nrm[2] = cos(ph);
        o[0] = C->R * nrm[0]; o[2] = C->R * (nrm[2] - 1.0);
    }
    double d[3] = {C->sin_t[J->k], 0.0, C->cos_t[J->k]};
    if (sa) {                                      /* at a uniform angle to the face normal */
        double th = ((double)(x[2] >> 8) + 0.5) * 0x1p-24 * OR_PI - 0.5 * OR_PI;
        double st = sin(th), ct = cos(th);
        d[0] = nrm[0] * ct + nrm[2] * st; d[1] = 0.0; d[2] = nrm[2] * ct - nrm[0] * st;
    } else if (C->kind[J->k] != OR_TX_PLANE) {   /* along the line from the virtual source / toward the focus */
        double sg = C->kind[J->k] == OR_TX_DIVERGING ? 1.0 : -1.0;
        double dx = sg * (o[0] - C->vx[J->k]), dz = sg * (o[2] - C->vz[J->k]);
        double l = sqrt(dx * dx + dz * dz);
        d[0] = dx / l; d[1] = 0.0; d[2] = dz / l;
    }
    double t = C->delay[J->k * ar->n_el + e];
    double w = dot3(d, nrm) / (double)C->cfg->n_rays;   /* Eq. 6: cosine to the face normal over N */
    if (!(w > 0.0)) {                              /* aimed into the probe: no ray */
        J->st.rays++;
        return fnv(OR_FNV_OFFSET, 0x20000u | (uint32_t)OR_END_ARRAY_MISS);
    }
    uint64_t h = OR_FNV_OFFSET;
    int reason = follow(C, J, o, d, t, w, C->sc->med_array, 0, 0.0, -1, &h);
    J->st.rays++;
    return fnv(h, 0x20000u | (uint32_t)reason);
}

static int setup(ctx_t *C, const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg)
{
    memset(C, 0, sizeof *C);
    C->sc = sc; C->ar = ar; C->cfg = cfg;
    int nm = sc->n_med;
    C->c = (double *)malloc(sizeof(double) * 6 * nm);
    C->Z = C->c + nm; C->a = C->Z + nm; C->slow = C->a + nm; C->cs = C->slow + nm; C->Zs = C->cs + nm;
    for (int m = 0; m < nm; ++m) {
        C->c[m] = sc->med[4 * m + 0];
        C->Z[m] = sc->med[4 * m + 1];
        C->a[m] = or_np_per_m(sc->med[4 * m + 2], ar->f0);
        C->slow[m] = (double)ar->fs / C->c[m];
        C->cs[m] = sc->med_sampling ? sc->med_sampling[4 * m + 0] : C->c[m];
        C->Zs[m] = sc->med_sampling ? sc->med_sampling[4 * m + 1] : C->Z[m];
    }
    int nt = cfg ? cfg->n_tx : 0;
    C->delay = (double *)malloc(sizeof(double) * ((size_t)nt * ar->n_el + 4 * (size_t)nt + 1));
    C->sin_t = C->delay + (size_t)nt * ar->n_el;
    C->cos_t = C->sin_t + nt;
    C->vx = C->cos_t + nt;
    C->vz = C->vx + nt;
    C->kind = (int *)malloc(sizeof(int) * (size_t)(nt + 1));
    C->pitch = ar->pitch;
    C->H = ar->elev_h;
    C->x0 = -0.5 * (double)(ar->n_el - 1) * C->pitch;
    C->R = ar->radius > 0.0f ? (double)ar->radius : 0.0;
    C->dphi = C->R > 0.0 ? C->pitch / C->R : 0.0;
    C->phi0 = -0.5 * (double)(ar->n_el - 1) * C->dphi;
    for (int k = 0; k < nt; ++k) {
        double th = cfg->angles ? cfg->angles[k] : 0.0;
        C->kind[k] = cfg->tx_kind ? cfg->tx_kind[k] : OR_TX_PLANE;
        C->vx[k] = cfg->tx_kind ? cfg->tx_x[k] : 0.0;
        C->vz[k] = cfg->tx_kind ? cfg->tx_z[k] : 0.0;
        C->sin_t[k] = sin(th);
        C->cos_t[k] = cos(th);
        /* path length from the wave's reference to element e: plane wave: x_e sin(theta);
         * diverging: distance from the virtual source; focused: minus the distance to the
         * focus.  Each element fires when the wavefront through the first-firing element
         * reaches it. */
        double mn = INFINITY, *len = (double *)malloc(sizeof(double) * (size_t)ar->n_el);
        for (int e = 0; e < ar->n_el; ++e) {
            double ce[3], ne[3];
            elem_frame(C, e, ce, ne);
            double dx = ce[0] - C->vx[k], dz = ce[2] - C->vz[k];
            if (C->kind[k] == OR_TX_PLANE) len[e] = ce[0] * C->sin_t[k] + ce[2] * C->cos_t[k];
            else if (C->kind[k] == OR_TX_SYNTHETIC) len[e] = 0.0;   /* the one element fires at t = 0 */
            else if (C->kind[k] == OR_TX_DIVERGING) len[e] = sqrt(dx * dx + dz * dz);
            else len[e] = -sqrt(dx * dx + dz * dz);
            if (len[e] < mn) mn = len[e];
        }
        for (int e = 0; e < ar->n_el; ++e)
            C->delay[k * ar->n_el + e] = (len[e] - mn) / (double)ar->c_bf * (double)ar->fs;
        free(len);
    }
    double s = (double)ar->n_cycles / (4.0 * (double)ar->f0);
    C->K = (double)ar->tcut_sigmas * s * (double)ar->fs;
    C->t_last = (double)(ar->n_s - 1) + C->K;
    C->am = (double)ar->alpha_m_deg * OR_PI / 180.0;
    C->ac = (double)ar->alpha_c_deg * OR_PI / 180.0;
    C->top = sc->n_bnd;
    C->bot = sc->n_bnd + 1;
    C->esc = sc->n_bnd + 2;
    C->tri0 = sc->n_bnd + 3;
    C->alpha_b = (double *)calloc((size_t)C->tri0 + (size_t)sc->n_tri, sizeof(double));   /* by hit id */
    for (int p = 0; p < sc->n_bnd + sc->n_tri; ++p) {
        const int32_t *m = p < sc->n_bnd ? &sc->bnd_med[2 * p] : &sc->tri_med[2 * (p - sc->n_bnd)];
        double a0 = sc->med[4 * m[0] + 3], a1 = sc->med[4 * m[1] + 3];
        C->alpha_b[p < sc->n_bnd ? p : C->tri0 + (p - sc->n_bnd)] = a0 > a1 ? a0 : a1;
    }
    return 0;
}

static void teardown(ctx_t *C)
{
    free(C->c);
    free(C->delay);
    free(C->alpha_b);
    free(C->kind);
}

static int scene_is_rough(const or_scene *sc)
{
    for (int m = 0; m < sc->n_med; ++m)
        if (sc->med[4 * m + 3] != 0.0f) return 1;
    return 0;
}

int64_t or_trace(const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg,
                 or_arrival *out, int64_t cap, uint64_t *topo, or_stats *st, int n_threads)
{
    if (!sc || !ar || !cfg || cfg->n_tx <= 0 || cfg->n_rays == 0 || cfg->n_rays > 0xFFFFFFFFull ||
        cfg->mix < 0 || cfg->mix > 1 ||
        cfg->n_rays * (cfg->mix ? (uint64_t)cfg->n_tx : 1u) > 0xFFFFFFFFull || cfg->ray_end < cfg->ray_begin ||
        cfg->ray_end > cfg->n_rays * (cfg->mix ? (uint64_t)cfg->n_tx : 1u) || ar->n_el <= 0 ||
        cfg->max_bounces < 0 || cfg->max_bounces > 127 || sc->n_scat > (1 << 24))
        return -1;
    for (int m = 0; m < sc->n_med; ++m)
        if (!(sc->med[4 * m + 3] >= 0.0f && sc->med[4 * m + 3] <= 4.0f)) return -1;
    if (sc->n_tri < 0 || sc->n_tri > (1 << 22) || (sc->n_tri > 0 && (!sc->tri || !sc->tri_med))) return -1;
    for (int q = 0; q < sc->n_tri; ++q) {
        const int32_t *m = &sc->tri_med[2 * q];
        if (m[0] < 0 || m[0] >= sc->n_med || m[1] < 0 || m[1] >= sc->n_med) return -1;
        const float *v = &sc->tri[9 * q];
        double e1[3] = {(double)v[3] - v[0], (double)v[4] - v[1], (double)v[5] - v[2]};
        double e2[3] = {(double)v[6] - v[0], (double)v[7] - v[1], (double)v[8] - v[2]}, n[3];
        cross3(e1, e2, n);
        if (!(dot3(n, n) > 0.0)) return -1;      /* degenerate triangle */
    }
    if (!(ar->radius >= 0.0f) || (ar->radius > 0.0f && !((double)ar->n_el * ar->pitch < 3.0 * ar->radius)))
        return -1;   /* convex: the aperture spans less than about 170 degrees */
    if (cfg->tx_kind) {
        if (!cfg->tx_x || !cfg->tx_z) return -1;
        for (int k = 0; k < cfg->n_tx; ++k) {
            int kd = cfg->tx_kind[k];
            if (kd == OR_TX_DIVERGING ? !(cfg->tx_z[k] < 0.0f) : kd == OR_TX_FOCUSED ? !(cfg->tx_z[k] > 0.0f)
                : kd == OR_TX_SYNTHETIC ? !(cfg->tx_x[k] >= 0.0f && cfg->tx_x[k] < (float)ar->n_el &&
                                            cfg->tx_x[k] == floorf(cfg->tx_x[k]))
                : kd != OR_TX_PLANE)
                return -1;
        }
    }
    /* rough boundaries: Monte Carlo mode with the media deciding their own branches */
    if (scene_is_rough(sc) && (cfg->mode != OR_MODE_MC || sc->med_sampling)) return -1;
    ctx_t C;
    setup(&C, sc, ar, cfg);
    uint64_t n_sub = cfg->ray_end - cfg->ray_begin;
    int64_t total = (int64_t)(n_sub * (cfg->mix ? 1u : (uint64_t)cfg->n_tx));
    if (n_threads <= 0) n_threads = 1;
    abuf_t *bufs = (abuf_t *)calloc((size_t)n_threads, sizeof(abuf_t));
    or_stats *sts = (or_stats *)calloc((size_t)n_threads, sizeof(or_stats));
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t g = 0; g < total; ++g) {
            ray_job J;
            memset(&J, 0, sizeof J);
            J.k = (int)(g / (int64_t)n_sub);
            J.i = (uint32_t)(cfg->ray_begin + (uint64_t)(g % (int64_t)n_sub));
            if (cfg->mix) {   /* the ray's transmit, uniform over n_tx, from counter (i, 0, EMIT, 1) */
                uint32_t y[4];
                draw(cfg->seed, J.i, 0u, 0u, 1u, y);
                J.k = (int)(((uint64_t)(y[0] >> 8) * (uint64_t)cfg->n_tx) >> 24);
            }
            J.buf = &bufs[tid];
            uint64_t h = trace_ray(&C, &J);
            if (topo) topo[g] = h;
            sts[tid].rays += J.st.rays;
            sts[tid].segments += J.st.segments;
            sts[tid].interactions += J.st.interactions;
            sts[tid].candidates += J.st.candidates;
            sts[tid].connections += J.st.connections;
            sts[tid].arrivals += J.st.arrivals;
        }
    }
    size_t n = 0;
    for (int q = 0; q < n_threads; ++q) n += bufs[q].n;
    rec_t *all = (rec_t *)malloc((n ? n : 1) * sizeof(rec_t));
    size_t pos = 0;
    for (int q = 0; q < n_threads; ++q) {
        if (bufs[q].n) memcpy(all + pos, bufs[q].v, bufs[q].n * sizeof(rec_t));
        pos += bufs[q].n;
        free(bufs[q].v);
    }
    qsort(all, n, sizeof(rec_t), rec_cmp);
    for (size_t q = 0; q < n && (int64_t)q < cap; ++q) out[q] = all[q].a;
    if (st) {
        memset(st, 0, sizeof *st);
        for (int q = 0; q < n_threads; ++q) {
            st->rays += sts[q].rays; st->segments += sts[q].segments;
            st->interactions += sts[q].interactions; st->candidates += sts[q].candidates;
            st->connections += sts[q].connections; st->arrivals += sts[q].arrivals;
        }
    }
    free(all);
    free(bufs);
    free(sts);
    teardown(&C);
    return (int64_t)n;
}

double or_connection(const or_scene *sc, const or_array *ar, const double p[3], int32_t med,
                     double x_e, double *t_samples, double *atten_np)
{
    or_trace_cfg cfg;
    memset(&cfg, 0, sizeof cfg);
    ctx_t C;
    setup(&C, sc, ar, &cfg);
    double t = 0.0, a = 0.0;
    double fac = connection(&C, p, med, x_e, &t, &a);
    teardown(&C);
    *t_samples = t;
    *atten_np = a;
    return fac;
}

/* ------------------------------------------------------- signal chain */

void or_deposit(const or_array *ar, int32_t n_tx, const or_arrival *arr, int64_t n_arr,
                double *rf, double *quad)
{
    double s_n = (double)ar->n_cycles / (4.0 * (double)ar->f0) * (double)ar->fs; /* s in samples */
    double K = (double)ar->tcut_sigmas * s_n;
    double om = 2.0 * OR_PI * (double)ar->f0 / (double)ar->fs;              /* rad per sample */
    for (int64_t q = 0; q < n_arr; ++q) {
        const or_arrival *a = &arr[q];
        if (a->tx < 0 || a->tx >= n_tx || a->el < 0 || a->el >= ar->n_el) continue;
        double *row_r = rf + ((size_t)a->tx * ar->n_el + a->el) * ar->n_s;
        double *row_q = quad + ((size_t)a->tx * ar->n_el + a->el) * ar->n_s;
        long n0 = (long)ceil(a->t - K), n1 = (long)floor(a->t + K);
        if (n0 < 0) n0 = 0;
        if (n1 > ar->n_s - 1) n1 = ar->n_s - 1;
        for (long n = n0; n <= n1; ++n) {
            double tau = (double)n - a->t;
            double g = exp(-tau * tau / (2.0 * s_n * s_n));
            row_r[n] += a->amp * g * sin(om * tau);
            row_q[n] -= a->amp * g * cos(om * tau);
        }
    }
}

void or_beamform(const or_array *ar, int32_t n_tx, const float *angles,
                 const double *rf, const double *quad,
                 const float *x_px, int32_t nx, const float *z_px, int32_t nz,
                 double *img_re, double *img_im, int n_threads)
{
    or_beamform_tx(ar, n_tx, angles, NULL, NULL, NULL, rf, quad, x_px, nx, z_px, nz, img_re, img_im, n_threads);
}

void or_beamform_tx(const or_array *ar, int32_t n_tx, const float *angles, const int32_t *tx_kind,
                    const float *tx_x, const float *tx_z, const double *rf, const double *quad,
                    const float *x_px, int32_t nx, const float *z_px, int32_t nz,
                    double *img_re, double *img_im, int n_threads)
{
    int n_el = ar->n_el, n_s = ar->n_s;
    double c = ar->c_bf, fs = ar->fs;
    ctx_t G;                 /* element centres only */
    memset(&G, 0, sizeof G);
    G.pitch = ar->pitch;
    G.x0 = -0.5 * (double)(n_el - 1) * G.pitch;
    G.R = ar->radius > 0.0f ? (double)ar->radius : 0.0;
    G.dphi = G.R > 0.0 ? G.pitch / G.R : 0.0;
    G.phi0 = -0.5 * (double)(n_el - 1) * G.dphi;
    double *cx = (double *)malloc(sizeof(double) * 2 * (size_t)n_el), *cz = cx + n_el;
    for (int e = 0; e < n_el; ++e) {
        double ce[3], ne[3];
        elem_frame(&G, e, ce, ne);
        cx[e] = ce[0]; cz[e] = ce[2];
    }
    if (n_threads <= 0) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 4)
#endif
    for (int iz = 0; iz < nz; ++iz) {
        for (int ix = 0; ix < nx; ++ix) {
            double x = x_px[ix], z = z_px[iz];
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < n_tx; ++k) {
                int kd = tx_kind ? tx_kind[k] : OR_TX_PLANE;
                double st = sin((double)angles[k]), ct = cos((double)angles[k]);
                double vx = tx_kind ? tx_x[k] : 0.0, vz = tx_kind ? tx_z[k] : 0.0;
                double mn = INFINITY, mx = -INFINITY;
                for (int e = 0; e < n_el; ++e) {
                    if (kd == OR_TX_SYNTHETIC) break;
                    double v = kd == OR_TX_PLANE ? cx[e] * st + cz[e] * ct
                                                 : sqrt((cx[e] - vx) * (cx[e] - vx) + (cz[e] - vz) * (cz[e] - vz));
                    if (v < mn) mn = v;
                    if (v > mx) mx = v;
                }
                double t_tx;
                if (kd == OR_TX_SYNTHETIC) {                         /* from the firing element */
                    int f = (int)vx;
                    t_tx = sqrt((x - cx[f]) * (x - cx[f]) + (z - cz[f]) * (z - cz[f])) / c;
                } else if (kd == OR_TX_PLANE) {
                    t_tx = (x * st + z * ct - mn) / c;               /* plane wave reaches the pixel */
                } else if (kd == OR_TX_DIVERGING) {                  /* from the virtual source */
                    t_tx = (sqrt((x - vx) * (x - vx) + (z - vz) * (z - vz)) - mn) / c;
                } else {                                             /* through the focus at mx / c */
                    double r = sqrt((x - vx) * (x - vx) + (z - vz) * (z - vz));
                    t_tx = (mx + (z >= vz ? r : -r)) / c;
                }
                for (int e = 0; e < n_el; ++e) {
                    double dx = x - cx[e], dz = z - cz[e];
                    double t_rx = sqrt(dz * dz + dx * dx) / c;      /* echo back to element e */
                    double tau = (t_tx + t_rx) * fs;
                    if (tau < 0.0 || tau > (double)(n_s - 1)) continue;
                    long i0 = (long)floor(tau);
                    double f = tau - (double)i0;
                    long i1 = i0 + 1 < n_s ? i0 + 1 : i0;
                    const double *rr = rf + ((size_t)k * n_el + e) * n_s;
                    const double *qq = quad + ((size_t)k * n_el + e) * n_s;
                    sr += rr[i0] * (1.0 - f) + rr[i1] * f;
                    si += qq[i0] * (1.0 - f) + qq[i1] * f;
                }
            }
            img_re[(size_t)iz * nx + ix] = sr;
            img_im[(size_t)iz * nx + ix] = si;
        }
    }
    free(cx);
}

void or_envelope_log(const double *img_re, const double *img_im, int64_t n_px,
                     double dyn_range_db, double *env, double *db)
{
    double mx = 0.0;
    for (int64_t q = 0; q < n_px; ++q) {
        env[q] = sqrt(img_re[q] * img_re[q] + img_im[q] * img_im[q]);
        if (env[q] > mx) mx = env[q];
    }
    for (int64_t q = 0; q < n_px; ++q) {
        double v = (mx > 0.0 && env[q] > 0.0) ? 20.0 * log10(env[q] / mx) : -dyn_range_db;
        db[q] = v < -dyn_range_db ? -dyn_range_db : v;
    }
}

/* ==================================================================== *
 * Pathwise gradient with FP64 dual numbers (forward mode).              *
 * Parameters: index 3m + 0 = c_m, 3m + 1 = Z_m, 3m + 2 = alpha_m.       *
 * The path is the Monte Carlo path of trace_ray; branch decisions and   *
 * the branch probabilities dividing the weights are held at their       *
 * values (they carry no derivative), everything else is differentiated, *
 * including hit distances, normals and refracted directions.            *
 * ==================================================================== */

#define OR_NP 12

typedef struct { double v, d[OR_NP]; } dnum;
typedef struct { dnum x, y, z; } dvec;

static dnum dn_c(double v) { dnum r; r.v = v; memset(r.d, 0, sizeof r.d); return r; }
static dnum dn_add(dnum a, dnum b) { for (int q = 0; q < OR_NP; ++q) a.d[q] += b.d[q]; a.v += b.v; return a; }
static dnum dn_sub(dnum a, dnum b) { for (int q = 0; q < OR_NP; ++q) a.d[q] -= b.d[q]; a.v -= b.v; return a; }
static dnum dn_scale(dnum a, double s) { for (int q = 0; q < OR_NP; ++q) a.d[q] *= s; a.v *= s; return a; }
static dnum dn_mul(dnum a, dnum b)
{
    dnum r;
    r.v = a.v * b.v;
    for (int q = 0; q < OR_NP; ++q) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
    return r;
}
static dnum dn_div(dnum a, dnum b)
{
    dnum r;
    r.v = a.v / b.v;
    for (int q = 0; q < OR_NP; ++q) r.d[q] = (a.d[q] - r.v * b.d[q]) / b.v;
    return r;
}
static dnum dn_sqrt(dnum a)
{
    dnum r;
    r.v = sqrt(a.v);
    for (int q = 0; q < OR_NP; ++q) r.d[q] = a.d[q] / (2.0 * r.v);
    return r;
}
static dnum dn_exp(dnum a)
{
    dnum r;
    r.v = exp(a.v);
    for (int q = 0; q < OR_NP; ++q) r.d[q] = a.d[q] * r.v;
    return r;
}
static dnum dn_acos(dnum a)
{
    dnum r;
    r.v = acos(a.v);
    double s = -1.0 / sqrt(1.0 - a.v * a.v);
    for (int q = 0; q < OR_NP; ++q) r.d[q] = a.d[q] * s;
    return r;
}
static dvec dv_c(double x, double y, double z) { dvec r = {dn_c(x), dn_c(y), dn_c(z)}; return r; }
static dvec dv_add(dvec a, dvec b) { dvec r = {dn_add(a.x, b.x), dn_add(a.y, b.y), dn_add(a.z, b.z)}; return r; }
static dvec dv_sub(dvec a, dvec b) { dvec r = {dn_sub(a.x, b.x), dn_sub(a.y, b.y), dn_sub(a.z, b.z)}; return r; }
static dvec dv_smul(dnum s, dvec a) { dvec r = {dn_mul(s, a.x), dn_mul(s, a.y), dn_mul(s, a.z)}; return r; }
static dnum dv_dot(dvec a, dvec b) { return dn_add(dn_add(dn_mul(a.x, b.x), dn_mul(a.y, b.y)), dn_mul(a.z, b.z)); }
static dvec dv_unit(dvec a)
{
    dnum l = dn_sqrt(dv_dot(a, a));
    dvec r = {dn_div(a.x, l), dn_div(a.y, l), dn_div(a.z, l)};
    return r;
}
static void dv_val(dvec a, double out[3]) { out[0] = a.x.v; out[1] = a.y.v; out[2] = a.z.v; }

typedef struct {
    const ctx_t *C;
    dnum *c, *Z, *a, *slow;         /* media as dual numbers */
    const double *g_rf, *g_q;
    double grad[OR_NP];
    double *grad_amp;               /* thread-private [n_scat] */
    double s_n, K, om;              /* pulse width (samples), half-width, rad per sample */
} gctx_t;

/* dL/d amplitude and dL/d time of one arrival, from dL/dA over its taps. */
static void arrival_sens(const gctx_t *G, int k, int e, double t, double amp, double *g_amp, double *g_t)
{
    const or_array *ar = G->C->ar;
    const double *gr = G->g_rf + ((size_t)k * ar->n_el + e) * ar->n_s;
    const double *gq = G->g_q + ((size_t)k * ar->n_el + e) * ar->n_s;
    long n0 = (long)ceil(t - G->K), n1 = (long)floor(t + G->K);
    if (n0 < 0) n0 = 0;
    if (n1 > ar->n_s - 1) n1 = ar->n_s - 1;
    double sa = 0.0, st = 0.0;
    for (long n = n0; n <= n1; ++n) {
        double tau = (double)n - t;
        double g = exp(-tau * tau / (2.0 * G->s_n * G->s_n));
        double sn = sin(G->om * tau), cs = cos(G->om * tau);
        double p_re = g * sn, p_im = -g * cs;
        double dp_re = g * (G->om * cs - tau / (G->s_n * G->s_n) * sn);   /* d/dtau */
        double dp_im = g * (G->om * sn + tau / (G->s_n * G->s_n) * cs);
        sa += gr[n] * p_re + gq[n] * p_im;
        st -= amp * (gr[n] * dp_re + gq[n] * dp_im);                      /* d/dt = -d/dtau */
    }
    *g_amp = sa;
    *g_t = st;
}

static void accumulate(gctx_t *G, int k, int e, dnum t, dnum amp_wo_a, double a_j, int j)
{
    double g_amp, g_t;
    double amp = amp_wo_a.v * a_j;
    arrival_sens(G, k, e, t.v, amp, &g_amp, &g_t);
    for (int q = 0; q < OR_NP; ++q) G->grad[q] += g_amp * a_j * amp_wo_a.d[q] + g_t * t.d[q];
    if (j >= 0) G->grad_amp[j] += g_amp * amp_wo_a.v;
}

/* Dual hit distance along o + t d for primitive `hit` (chosen on values). */
static dnum dual_hit(const gctx_t *G, int hit, dvec o, dvec d, int skip)
{
    const ctx_t *C = G->C;
    if (hit == C->top) return dn_div(dn_scale(o.z, -1.0), d.z);
    if (hit == C->bot) return dn_div(dn_sub(dn_c(C->sc->z_max), o.z), d.z);
    const float *q = &C->sc->bnd_p[4 * hit];
    int kind = C->sc->bnd_kind[hit];
    if (kind == OR_PLANE_Z) return dn_div(dn_sub(dn_c(q[0]), o.z), d.z);
    if (kind == OR_SPHERE) {
        dvec oc = dv_sub(o, dv_c(q[0], q[1], q[2]));
        dnum b = dv_dot(oc, d);
        if (hit == skip) return dn_scale(b, -2.0);
        dvec f = dv_sub(oc, dv_smul(b, d));
        dnum s = dn_sqrt(dn_sub(dn_c((double)q[3] * q[3]), dv_dot(f, f)));
        dnum t = dn_sub(dn_scale(b, -1.0), s);
        if (!(t.v > OR_TMIN)) t = dn_add(dn_scale(b, -1.0), s);
        return t;
    }
    dnum ocx = dn_sub(o.x, dn_c(q[0])), ocz = dn_sub(o.z, dn_c(q[1]));
    dnum a = dn_add(dn_mul(d.x, d.x), dn_mul(d.z, d.z));
    dnum b = dn_div(dn_add(dn_mul(ocx, d.x), dn_mul(ocz, d.z)), a);
    if (hit == skip) return dn_scale(b, -2.0);
    dnum fx = dn_sub(ocx, dn_mul(b, d.x)), fz = dn_sub(ocz, dn_mul(b, d.z));
    dnum disc = dn_div(dn_sub(dn_c((double)q[2] * q[2]), dn_add(dn_mul(fx, fx), dn_mul(fz, fz))), a);
    dnum s = dn_sqrt(disc);
    dnum t = dn_sub(dn_scale(b, -1.0), s);
    if (!(t.v > OR_TMIN)) t = dn_add(dn_scale(b, -1.0), s);
    return t;
}

static dvec dual_normal(const gctx_t *G, int p, dvec h)
{
    const float *q = &G->C->sc->bnd_p[4 * p];
    int kind = G->C->sc->bnd_kind[p];
    if (kind == OR_PLANE_Z) return dv_c(0.0, 0.0, 1.0);
    if (kind == OR_SPHERE) return dv_unit(dv_sub(h, dv_c(q[0], q[1], q[2])));
    dvec v = {dn_sub(h.x, dn_c(q[0])), dn_c(0.0), dn_sub(h.z, dn_c(q[1]))};
    return dv_unit(v);
}

/* Connection ray p -> element centre with dual factors, time and attenuation
 * (its geometry does not depend on the parameters). */
static dnum dual_connection(const gctx_t *G, const double p[3], int med, double x_e, dnum *t_out, dnum *att_out)
{
    const ctx_t *C = G->C;
    double o[3] = {p[0], p[1], p[2]};
    double w[3] = {x_e - p[0], -p[1], -p[2]};
    double rem = sqrt(dot3(w, w));
    w[0] /= rem; w[1] /= rem; w[2] /= rem;
    dnum fac = dn_c(1.0), t = dn_c(0.0), att = dn_c(0.0);
    int m = med, skip = -1;
    for (int it = 0; it < OR_MAX_CROSS; ++it) {
        double th;
        int hit = nearest_boundary(C, o, w, skip, 0, &th);
        if (hit < 0 || th >= rem) {
            t = dn_add(t, dn_scale(G->slow[m], rem));
            att = dn_add(att, dn_scale(G->a[m], rem));
            break;
        }
        t = dn_add(t, dn_scale(G->slow[m], th));
        att = dn_add(att, dn_scale(G->a[m], th));
        double h[3] = {o[0] + th * w[0], o[1] + th * w[1], o[2] + th * w[2]};
        if (hit < C->sc->n_bnd && C->sc->bnd_kind[hit] == OR_PLANE_Z) h[2] = C->sc->bnd_p[4 * hit];
        double n_out[3];
        outward_normal(C, hit, h, n_out);
        int m2 = far_medium(C, hit, w, n_out);
        double ci = fabs(dot3(w, n_out));
        dnum eta = dn_div(G->c[m2], G->c[m]);
        dnum k = dn_sub(dn_c(1.0), dn_mul(dn_mul(eta, eta), dn_c(1.0 - ci * ci)));
        if (k.v < 0.0) return dn_c(0.0);
        dnum ct = dn_sqrt(k);
        dnum num = dn_sub(dn_scale(G->Z[m2], ci), dn_mul(G->Z[m], ct));
        dnum den = dn_add(dn_scale(G->Z[m2], ci), dn_mul(G->Z[m], ct));
        dnum r = dn_div(num, den);
        fac = dn_mul(fac, dn_sqrt(dn_sub(dn_c(1.0), dn_mul(r, r))));
        m = m2;
        o[0] = h[0]; o[1] = h[1]; o[2] = h[2];
        rem -= th;
        skip = hit;
    }
    *t_out = t;
    *att_out = att;
    return fac;
}

static dnum dual_directivity(const ctx_t *C, dnum cos_a)
{
    double al = acos(cos_a.v);
    if (al > C->ac) return dn_c(0.0);
    if (al > C->am) return dn_scale(dn_sub(dn_c(C->ac), dn_acos(cos_a)), 1.0 / (C->ac - C->am));
    return dn_c(1.0);
}

static void grad_ray(gctx_t *G, uint32_t i, int k)
{
    const ctx_t *C = G->C;
    const or_scene *sc = C->sc;
    const or_array *ar = C->ar;
    const or_trace_cfg *cfg = C->cfg;
    int e = (int)(i % (uint32_t)ar->n_el);
    uint32_t x[4];
    draw(cfg->seed, i, (uint32_t)k, 0u, 0u, x);
    dvec o = dv_c(elem_x(C, e) + (u24(x[0]) - 0.5) * C->pitch, (u24(x[1]) - 0.5) * C->H, 0.0);
    dvec d = dv_c(C->sin_t[k], 0.0, C->cos_t[k]);
    dnum t = dn_c(C->delay[k * ar->n_el + e]);
    dnum w = dn_c(C->cos_t[k] / (double)cfg->n_rays);
    dnum L = dn_c(0.0);
    int med = sc->med_array, b = 0, prev = -1;
    double r2 = (double)sc->r_s * sc->r_s;
    for (int guard = 0; guard < OR_MAX_SEG; ++guard) {
        double ov[3], dv[3], th;
        dv_val(o, ov);
        dv_val(d, dv);
        int hit = nearest_boundary(C, ov, dv, prev, 1, &th);
        dnum seg = hit >= 0 ? dual_hit(G, hit, o, d, prev) : dn_c(th);
        int clipped = 0;
        if (L.v + seg.v > (double)cfg->max_path) { seg = dn_sub(dn_c(cfg->max_path), L); clipped = 1; }
        /* scatterer events on the segment */
        double ov2[3], dv2[3];
        dv_val(o, ov2);
        dv_val(d, dv2);
        for (int j = 0; j < sc->n_scat; ++j) {
            const float *s = &sc->scat[4 * j];
            /* candidate test on values (as in segment_scatterers), dual only for candidates */
            double vv0[3] = {s[0] - ov2[0], s[1] - ov2[1], s[2] - ov2[2]};
            double tv = dot3(vv0, dv2);
            if (!(tv > 0.0 && tv < seg.v)) continue;
            double qv[3] = {vv0[0] - tv * dv2[0], vv0[1] - tv * dv2[1], vv0[2] - tv * dv2[2]};
            if (!(dot3(qv, qv) < r2)) continue;
            dvec v = dv_sub(dv_c(s[0], s[1], s[2]), o);
            dnum tca = dv_dot(v, d);
            draw(cfg->seed, i, (uint32_t)k, 2u | ((uint32_t)b << 8), (uint32_t)j, x);
            int e2 = (int)((((uint64_t)(x[0] >> 8)) * (uint64_t)ar->n_el) >> 24);
            double xe = elem_x(C, e2);
            double p[3] = {s[0], s[1], s[2]};
            double vv[3] = {xe - p[0], -p[1], -p[2]};
            double D = sqrt(dot3(vv, vv));
            double fd = or_directivity(acos(-vv[2] / D), C->am, C->ac);
            if (!(fd > 0.0)) continue;
            dnum tc, ac;
            dnum fac = dual_connection(G, p, med, xe, &tc, &ac);
            if (fac.v == 0.0) continue;
            dnum ta = dn_add(dn_add(t, dn_mul(tca, G->slow[med])), tc);
            if (ta.v > C->t_last) continue;
            dnum amp = dn_mul(dn_mul(w, dn_exp(dn_scale(dn_mul(G->a[med], tca), -1.0))),
                              dn_mul(dn_scale(fac, (double)ar->n_el * fd), dn_exp(dn_scale(ac, -1.0))));
            accumulate(G, k, e2, ta, amp, (double)s[3], j);
        }
        /* advance */
        t = dn_add(t, dn_mul(seg, G->slow[med]));
        w = dn_mul(w, dn_exp(dn_scale(dn_mul(G->a[med], seg), -1.0)));
        L = dn_add(L, seg);
        o = dv_add(o, dv_smul(seg, d));
        if (clipped) return;
        if (hit == C->top) {
            o.z = dn_c(0.0);
            double xl = C->x0 - 0.5 * C->pitch;
            if (fabs(o.y.v) <= 0.5 * C->H && o.x.v >= xl && o.x.v < xl + ar->n_el * C->pitch) {
                int el = (int)floor((o.x.v - xl) / C->pitch);
                if (el > ar->n_el - 1) el = ar->n_el - 1;
                dnum fd = dual_directivity(C, dn_scale(d.z, -1.0));
                if (fd.v > 0.0 && t.v <= C->t_last) accumulate(G, k, el, t, dn_mul(w, fd), 1.0, -1);
            }
            return;
        }
        if (hit == C->bot || hit < 0) return;
        if (sc->bnd_kind[hit] == OR_PLANE_Z) o.z = dn_c(sc->bnd_p[4 * hit]);
        if (t.v > C->t_last) return;
        if (b >= cfg->max_bounces) return;
        /* interaction: same decisions as trace_ray, derivatives of everything else */
        dvec n_out = dual_normal(G, hit, o);
        double nv[3], dvv[3];
        dv_val(n_out, nv);
        dv_val(d, dvv);
        int out_side = dot3(dvv, nv) > 0.0;
        int m2 = out_side ? sc->bnd_med[2 * hit + 1] : sc->bnd_med[2 * hit];
        dvec n = out_side ? dv_smul(dn_c(-1.0), n_out) : n_out;
        dnum ci = dn_scale(dv_dot(n, d), -1.0);
        dvec dr = dv_unit(dv_add(d, dv_smul(dn_scale(ci, 2.0), n)));
        dnum eta = dn_div(G->c[m2], G->c[med]);
        dnum kk = dn_sub(dn_c(1.0), dn_mul(dn_mul(eta, eta), dn_sub(dn_c(1.0), dn_mul(ci, ci))));
        double d_r[3], d_t[3], rr, RR;
        int tir = or_interface(dvv, nv, C->c[med], C->Z[med], C->c[m2], C->Z[m2], d_r, d_t, &rr, &RR);
        if (tir) {
            d = dr;
        } else {
            draw(cfg->seed, i, (uint32_t)k, 1u | ((uint32_t)b << 8), 0u, x);
            dnum ct = dn_sqrt(kk);
            dnum num = dn_sub(dn_mul(G->Z[m2], ci), dn_mul(G->Z[med], ct));
            dnum den = dn_add(dn_mul(G->Z[m2], ci), dn_mul(G->Z[med], ct));
            dnum r = dn_div(num, den);
            double Rv = r.v * r.v;
            if (u24(x[0]) < Rv) {
                w = dn_mul(w, dn_scale(r, 1.0 / Rv));
                d = dr;
            } else {
                w = dn_mul(w, dn_scale(dn_sqrt(dn_sub(dn_c(1.0), dn_mul(r, r))), 1.0 / (1.0 - Rv)));
                dvec tv = dv_add(dv_smul(eta, d), dv_smul(dn_sub(dn_mul(eta, ci), ct), n));
                d = dv_unit(tv);
                med = m2;
            }
        }
        b += 1;
        prev = hit;
    }
}

int or_grad(const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg, const double *g_rf,
            const double *g_q, double *grad_media, double *grad_amp, int n_threads)
{
    if (!sc || !ar || !cfg || !g_rf || !g_q || !grad_media || sc->n_med > 4 || cfg->mode != OR_MODE_MC ||
        cfg->ray_end > cfg->n_rays || cfg->ray_end < cfg->ray_begin || sc->med_sampling || scene_is_rough(sc) ||
        ar->radius != 0.0f || cfg->tx_kind || cfg->mix || sc->n_tri)
        return -1;
    ctx_t C;
    setup(&C, sc, ar, cfg);
    int nm = sc->n_med;
    dnum c[4], Z[4], a[4], slow[4];
    double k_a = (double)ar->f0 * 1e-6 * 100.0 / (20.0 * log10(exp(1.0)));
    for (int m = 0; m < nm; ++m) {
        c[m] = dn_c(C.c[m]); c[m].d[3 * m + 0] = 1.0;
        Z[m] = dn_c(C.Z[m]); Z[m].d[3 * m + 1] = 1.0;
        dnum alpha = dn_c(sc->med[4 * m + 2]); alpha.d[3 * m + 2] = 1.0;
        a[m] = dn_scale(alpha, k_a);
        slow[m] = dn_div(dn_c((double)ar->fs), c[m]);
    }
    if (n_threads <= 0) n_threads = 1;
    uint64_t n_sub = cfg->ray_end - cfg->ray_begin;
    int64_t total = (int64_t)(n_sub * (uint64_t)cfg->n_tx);
    double s_n = (double)ar->n_cycles / (4.0 * (double)ar->f0) * (double)ar->fs;
    double *g_all = (double *)calloc((size_t)n_threads * OR_NP, sizeof(double));
    double *ga_all = (double *)calloc((size_t)n_threads * (size_t)(sc->n_scat > 0 ? sc->n_scat : 1), sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        gctx_t G;
        memset(&G, 0, sizeof G);
        G.C = &C;
        G.c = c; G.Z = Z; G.a = a; G.slow = slow;
        G.g_rf = g_rf; G.g_q = g_q;
        G.grad_amp = ga_all + (size_t)tid * (size_t)(sc->n_scat > 0 ? sc->n_scat : 1);
        G.s_n = s_n;
        G.K = (double)ar->tcut_sigmas * s_n;
        G.om = 2.0 * OR_PI * (double)ar->f0 / (double)ar->fs;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t g = 0; g < total; ++g) {
            int k = (int)(g / (int64_t)n_sub);
            uint32_t i = (uint32_t)(cfg->ray_begin + (uint64_t)(g % (int64_t)n_sub));
            grad_ray(&G, i, k);
        }
        for (int q = 0; q < OR_NP; ++q) g_all[(size_t)tid * OR_NP + q] = G.grad[q];
    }
    for (int q = 0; q < 3 * nm; ++q) {
        double s = 0.0;
        for (int th = 0; th < n_threads; ++th) s += g_all[(size_t)th * OR_NP + q];
        grad_media[q] = s;
    }
    if (grad_amp)
        for (int j = 0; j < sc->n_scat; ++j) {
            double s = 0.0;
            for (int th = 0; th < n_threads; ++th) s += ga_all[(size_t)th * sc->n_scat + j];
            grad_amp[j] = s;
        }
    free(g_all);
    free(ga_all);
    teardown(&C);
    return 0;
}
