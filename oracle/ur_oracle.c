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
    double *delay;              /* [n_tx][n_el] transmit delays in samples */
    double *sin_t, *cos_t;      /* per transmit */
    double x0, pitch, H;        /* centre of element 0, pitch, elevation height */
    double K, t_last;           /* pulse half-width; latest useful arrival time (samples) */
    double am, ac;              /* directivity angles (rad) */
    int top, bot;               /* ids of the terminal planes */
} ctx_t;

static double elem_x(const ctx_t *C, int e) { return C->x0 + (double)e * C->pitch; }

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
    if (terminals) {
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
    return dot3(d, n_out) > 0.0 ? C->sc->bnd_med[2 * p + 1] : C->sc->bnd_med[2 * p];
}

/* Connection (secondary) ray: straight from p to the element centre. */
static double connection(const ctx_t *C, const double p[3], int med, double x_e,
                         double *t_samples, double *atten)
{
    double o[3] = {p[0], p[1], p[2]};
    double w[3] = {x_e - p[0], -p[1], -p[2]};
    double rem = sqrt(dot3(w, w));
    w[0] /= rem; w[1] /= rem; w[2] /= rem;
    double fac = 1.0, t = 0.0, att = 0.0;
    int m = med, skip = -1;
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
        if (C->sc->bnd_kind[hit] == OR_PLANE_Z) h[2] = C->sc->bnd_p[4 * hit];
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
        double xe = elem_x(C, e);
        double v[3] = {xe - p[0], -p[1], -p[2]};
        double D = sqrt(dot3(v, v));
        double alpha = acos(-v[2] / D);
        double fd = or_directivity(alpha, C->am, C->ac);   /* Eq. 13 */
        if (!(fd > 0.0)) continue;
        J->st.connections++;
        double tc, ac;
        double fac = connection(C, p, med, xe, &tc, &ac);
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

/* ------------------------------------------------------------ primary path */

/* Follows one primary ray (and, in expectation mode, both branches of every
 * interaction).  Returns the termination reason; *h accumulates the path hash. */
static int follow(const ctx_t *C, ray_job *J, double o[3], double d[3], double t, double w,
                  int med, int b, double L, int prev, uint64_t *h)
{
    const or_scene *sc = C->sc;
    const or_array *ar = C->ar;
    const or_trace_cfg *cfg = C->cfg;
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
        if (hit == C->top) {
            o[2] = 0.0;
            double xl = C->x0 - 0.5 * C->pitch;
            if (fabs(o[1]) <= 0.5 * C->H && o[0] >= xl && o[0] < xl + ar->n_el * C->pitch) {
                int e = (int)floor((o[0] - xl) / C->pitch);
                if (e > ar->n_el - 1) e = ar->n_el - 1;
                double fd = or_directivity(acos(-d[2]), C->am, C->ac);
                if (fd > 0.0 && t <= C->t_last) {
                    push(J->buf, J->k, e, J->i, 0x80000000u | ((uint32_t)b << 24), t, w * fd, J->seq++);
                    J->st.arrivals++;
                }
                return OR_END_APERTURE;
            }
            return OR_END_ARRAY_MISS;
        }
        if (hit == C->bot) return OR_END_BOTTOM;
        if (sc->bnd_kind[hit] == OR_PLANE_Z) o[2] = sc->bnd_p[4 * hit];
        if (t > C->t_last) return OR_END_TIME;
        if (b >= cfg->max_bounces) return OR_END_MAXB;
        /* interaction (Eqs. 7-11) */
        double n_out[3], dr[3], dt[3], r, R;
        outward_normal(C, hit, o, n_out);
        int m2 = far_medium(C, hit, d, n_out);
        int tir = or_interface(d, n_out, C->c[med], C->Z[med], C->c[m2], C->Z[m2], dr, dt, &r, &R);
        J->st.interactions++;
        int branch;
        if (tir) {
            branch = 2;
            memcpy(d, dr, sizeof dr);
        } else if (cfg->mode == OR_MODE_MC) {
            uint32_t x[4];
            draw(cfg->seed, J->i, (uint32_t)J->k, 1u | ((uint32_t)b << 8), 0u, x);
            if (u24(x[0]) < R) {            /* reflect if y < A_r^2 */
                branch = 0;
                w *= r / R;
                memcpy(d, dr, sizeof dr);
            } else {
                branch = 1;
                w *= sqrt(1.0 - R) / (1.0 - R);
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
    int e = (int)(J->i % (uint32_t)ar->n_el);
    uint32_t x[4];
    draw(C->cfg->seed, J->i, (uint32_t)J->k, 0u, 0u, x);
    double o[3] = {elem_x(C, e) + (u24(x[0]) - 0.5) * C->pitch, (u24(x[1]) - 0.5) * C->H, 0.0};
    double d[3] = {C->sin_t[J->k], 0.0, C->cos_t[J->k]};
    double t = C->delay[J->k * ar->n_el + e];
    double w = C->cos_t[J->k] / (double)C->cfg->n_rays;
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
    C->c = (double *)malloc(sizeof(double) * 4 * nm);
    C->Z = C->c + nm; C->a = C->Z + nm; C->slow = C->a + nm;
    for (int m = 0; m < nm; ++m) {
        C->c[m] = sc->med[4 * m + 0];
        C->Z[m] = sc->med[4 * m + 1];
        C->a[m] = or_np_per_m(sc->med[4 * m + 2], ar->f0);
        C->slow[m] = (double)ar->fs / C->c[m];
    }
    int nt = cfg ? cfg->n_tx : 0;
    C->delay = (double *)malloc(sizeof(double) * ((size_t)nt * ar->n_el + 2 * (size_t)nt + 1));
    C->sin_t = C->delay + (size_t)nt * ar->n_el;
    C->cos_t = C->sin_t + nt;
    C->pitch = ar->pitch;
    C->H = ar->elev_h;
    C->x0 = -0.5 * (double)(ar->n_el - 1) * C->pitch;
    for (int k = 0; k < nt; ++k) {
        double th = cfg->angles[k];
        C->sin_t[k] = sin(th);
        C->cos_t[k] = cos(th);
        /* plane-wave transmit delays: each element fires when the steered
         * wavefront through the first-firing element reaches it */
        double mn = INFINITY;
        for (int e = 0; e < ar->n_el; ++e) {
            double v = elem_x(C, e) * C->sin_t[k];
            if (v < mn) mn = v;
        }
        for (int e = 0; e < ar->n_el; ++e)
            C->delay[k * ar->n_el + e] = (elem_x(C, e) * C->sin_t[k] - mn) / (double)ar->c_bf * (double)ar->fs;
    }
    double s = (double)ar->n_cycles / (4.0 * (double)ar->f0);
    C->K = (double)ar->tcut_sigmas * s * (double)ar->fs;
    C->t_last = (double)(ar->n_s - 1) + C->K;
    C->am = (double)ar->alpha_m_deg * OR_PI / 180.0;
    C->ac = (double)ar->alpha_c_deg * OR_PI / 180.0;
    C->top = sc->n_bnd;
    C->bot = sc->n_bnd + 1;
    return 0;
}

static void teardown(ctx_t *C)
{
    free(C->c);
    free(C->delay);
}

int64_t or_trace(const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg,
                 or_arrival *out, int64_t cap, uint64_t *topo, or_stats *st, int n_threads)
{
    if (!sc || !ar || !cfg || cfg->ray_end < cfg->ray_begin || cfg->ray_end > cfg->n_rays ||
        cfg->n_rays == 0 || cfg->n_rays > 0xFFFFFFFFull || ar->n_el <= 0 || cfg->n_tx <= 0 ||
        cfg->max_bounces < 0 || cfg->max_bounces > 127 || sc->n_scat > (1 << 24))
        return -1;
    ctx_t C;
    setup(&C, sc, ar, cfg);
    uint64_t n_sub = cfg->ray_end - cfg->ray_begin;
    int64_t total = (int64_t)(n_sub * (uint64_t)cfg->n_tx);
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
    int n_el = ar->n_el, n_s = ar->n_s;
    double pitch = ar->pitch, c = ar->c_bf, fs = ar->fs;
    double x0 = -0.5 * (double)(n_el - 1) * pitch;
    if (n_threads <= 0) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(n_threads) schedule(dynamic, 4)
#endif
    for (int iz = 0; iz < nz; ++iz) {
        for (int ix = 0; ix < nx; ++ix) {
            double x = x_px[ix], z = z_px[iz];
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < n_tx; ++k) {
                double st = sin((double)angles[k]), ct = cos((double)angles[k]);
                double mn = INFINITY;
                for (int e = 0; e < n_el; ++e) {
                    double v = (x0 + e * pitch) * st;
                    if (v < mn) mn = v;
                }
                double t_tx = (x * st + z * ct - mn) / c;           /* plane wave reaches the pixel */
                for (int e = 0; e < n_el; ++e) {
                    double dx = x - (x0 + e * pitch);
                    double t_rx = sqrt(z * z + dx * dx) / c;        /* echo back to element e */
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
