/*
 * FP64 CPU oracle for full-path Monte Carlo acoustic ray tracing of plane-wave
 * ultrasound (UltraRay, arXiv 2501.05828).
 *
 * TEST INFRASTRUCTURE ONLY.  This tree is the slow, obviously-correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * entry point and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library and never calls it.
 *
 * Every routine takes the method's steps in the paper's order:
 *   ray emission            Sec. 2.3 "Ray Emission", Eq. 6
 *   traversal / interaction Sec. 2.3 "Ray Traversal", Eqs. 7-11
 *   transducer sampling     Sec. 2.3 "Transducer Sampling", Eq. 13
 *   pulse / signal chain    Sec. 2.3 "Phase Calculation and Signal Processing", Eq. 14
 * Scatterers and attenuation are not part of the paper's method (Sec. 5 lists
 * them as future work); the readings used for them are stated in the .c file.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), keyed per ray/event.
 *
 * Inputs are float32 (the exact values the GPU receives); all arithmetic is
 * double precision.  Brute force everywhere: no acceleration structure.
 */
#ifndef UR_ORACLE_H
#define UR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_PLANE_Z = 0, OR_SPHERE = 1, OR_CYL_Y = 2 };
enum { OR_TX_PLANE = 0, OR_TX_DIVERGING = 1, OR_TX_FOCUSED = 2, OR_TX_SYNTHETIC = 3 };
enum { OR_MODE_MC = 0, OR_MODE_EXPECT = 1 };
enum { OR_END_APERTURE = 1, OR_END_ARRAY_MISS = 2, OR_END_BOTTOM = 3,  /* 2: missed the aperture or escaped past a convex probe */
       OR_END_PATH = 4, OR_END_TIME = 5, OR_END_MAXB = 6, OR_END_ROUGH = 7 };

typedef struct {
    int32_t n_med;
    const float *med;        /* [n_med][4]: c (m/s), Z (MRayl), alpha (dB/cm/MHz), GGX roughness in
                                [0, 4] (a boundary takes the larger of its two media; 0: smooth) */
    int32_t n_bnd;
    const int32_t *bnd_kind; /* OR_PLANE_Z: z = p0.  OR_SPHERE: centre p0..p2, radius p3.
                                OR_CYL_Y: axis parallel to y through (x = p0, z = p1), radius p2 */
    const float *bnd_p;      /* [n_bnd][4] */
    const int32_t *bnd_med;  /* [n_bnd][2]: medium on the negative side (z < p0, or inside),
                                medium on the positive side (z > p0, or outside) */
    int32_t med_array;       /* medium in contact with the array plane z = 0 */
    float z_max;             /* absorbing plane z = z_max */
    int32_t n_scat;
    const float *scat;       /* [n_scat][4]: x, y, z (m), amplitude */
    float r_s;               /* scatterer capture radius (m) */
    const float *med_sampling; /* nullable [n_med][4]: c, Z used for the Monte Carlo branch decisions
                                  and the branch probabilities in the weights (default: med) */
    int32_t n_tri;           /* triangle-mesh boundaries (0 <= n_tri <= 2^22); triangle t has hit id
                                n_bnd + 3 + t (after the terminal planes) */
    const float *tri;        /* [n_tri][9]: vertices v0, v1, v2 (m) */
    const int32_t *tri_med;  /* [n_tri][2]: medium behind the triangle (negative side of its normal
                                (v1 - v0) x (v2 - v0)), medium in front */
} or_scene;

typedef struct {
    int32_t n_el;
    float pitch, elev_h, f0, fs;
    int32_t n_s;
    float n_cycles, alpha_m_deg, alpha_c_deg, c_bf, tcut_sigmas;
    float radius;            /* 0: linear array on z = 0; > 0: convex array, elements on the arc of this
                                radius about (0, 0, -radius), centres `pitch` apart along the arc */
} or_array;

typedef struct {
    int32_t n_tx;
    const float *angles;     /* [n_tx] steering angles (rad) */
    uint64_t n_rays;         /* N: rays per transmit */
    uint64_t ray_begin, ray_end; /* trace only rays i in [ray_begin, ray_end) of each transmit */
    uint64_t seed;
    int32_t max_bounces;
    float max_path;          /* m */
    int32_t mode;            /* OR_MODE_MC or OR_MODE_EXPECT (smooth scenes only) */
    int32_t rough_bsdf_only; /* 0: transducer sampling at rough boundaries, balance heuristic with the
                                direct aperture hits (the method); 1: BSDF sampling alone (for tests) */
    const int32_t *tx_kind;  /* nullable [n_tx]: OR_TX_* per transmit (default: plane waves of angles[]) */
    const float *tx_x, *tx_z;/* [n_tx] with tx_kind: virtual source (diverging, z < 0) or focus
                                (focused, z > 0) in the xz plane (m); synthetic aperture: tx_x is the
                                index of the one element that fires (an integer value), tx_z unused */
    int32_t mix;             /* 0: n_rays rays per transmit, ray_begin/ray_end index each transmit's rays.
                                1: n_tx * n_rays rays in all, each drawing its transmit (Sec. 2.3);
                                ray_begin/ray_end index that one sequence and topo is [ray_end - ray_begin] */
} or_trace_cfg;

typedef struct {
    int32_t tx, el;
    uint32_t ray, event;     /* event: bits 24..30 = segment index b; scatter arrivals: bits 0..23 =
                                scatterer index; aperture arrivals: bit31 set, bits 0..23 = 0;
                                transducer sampling at rough boundary p: bit31 set, bits 0..23 = p + 1 */
    double t;                /* arrival time in samples */
    double amp;
} or_arrival;

typedef struct {
    uint64_t rays, segments, interactions, candidates, connections, arrivals;
} or_stats;

/* Philox4x32-10 block: out = philox(ctr, key). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Traces rays [ray_begin, ray_end) of every transmit.  Writes up to `cap` arrivals
 * (sorted by tx, ray, emission order) and returns the total number produced
 * (a return value > cap means the buffer was too small; re-run with more room).
 * topo (nullable): [n_tx][ray_end - ray_begin] FNV-1a path hashes (MC mode).
 * Returns -1 on invalid arguments. */
int64_t or_trace(const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg,
                 or_arrival *out, int64_t cap, uint64_t *topo, or_stats *st, int n_threads);

/* Eq. 14 deposit of arrivals into the analytic channel data A = rf + j quad
 * ([n_tx][n_el][n_s], accumulated, not cleared). */
void or_deposit(const or_array *ar, int32_t n_tx, const or_arrival *arr, int64_t n_arr,
                double *rf, double *quad);

/* Plane-wave delay-and-sum with coherent compounding over all transmits.
 * x_px[nx], z_px[nz] pixel coordinates (m); img_re/img_im [nz][nx]. */
void or_beamform(const or_array *ar, int32_t n_tx, const float *angles,
                 const double *rf, const double *quad,
                 const float *x_px, int32_t nx, const float *z_px, int32_t nz,
                 double *img_re, double *img_im, int n_threads);

/* The same with transmit kinds (tx_kind, tx_x, tx_z nullable as in or_trace_cfg): the
 * transmit delay of a diverging wave is the distance from its virtual source, that of a
 * focused wave the arrival of the converging then diverging wave through its focus, that
 * of a synthetic-aperture transmit the distance from the firing element's centre. */
void or_beamform_tx(const or_array *ar, int32_t n_tx, const float *angles, const int32_t *tx_kind,
                    const float *tx_x, const float *tx_z, const double *rf, const double *quad,
                    const float *x_px, int32_t nx, const float *z_px, int32_t nz,
                    double *img_re, double *img_im, int n_threads);

/* Envelope |I|, normalisation by its maximum, 20 log10, clip at -dyn_range_db. */
void or_envelope_log(const double *img_re, const double *img_im, int64_t n_px,
                     double dyn_range_db, double *env, double *db);

/* Pathwise gradient (forward mode, FP64 dual numbers) of L with respect to the
 * media parameters (c, Z, alpha of every medium, n_med <= 4) and the scatterer
 * amplitudes, for the Monte Carlo estimate of or_trace (MC mode) with the branch
 * decisions and branch probabilities held fixed.  g_rf, g_q = dL/d rf,
 * dL/d quad [n_tx][n_el][n_s].  grad_media[n_med][3] (c, Z, alpha) and
 * grad_amp[n_scat] are overwritten.  Returns 0, or -1 on invalid arguments. */
int or_grad(const or_scene *sc, const or_array *ar, const or_trace_cfg *cfg, const double *g_rf,
            const double *g_q, double *grad_media, double *grad_amp, int n_threads);

/* ---- single-step routines exposed for the closed-form tests ---- */

/* Boundary interaction (Eqs. 7-11 with the acoustic readings): incident unit
 * direction d, normal n (either orientation), media (c1, Z1) -> (c2, Z2).
 * Returns 1 on total internal reflection (r = 1), else 0.  Outputs reflected and
 * transmitted directions, the pressure reflection coefficient r and R = r^2. */
int or_interface(const double d[3], const double n[3], double c1, double Z1,
                 double c2, double Z2, double d_r[3], double d_t[3],
                 double *r, double *R);

/* Eq. 12: GGX density of microfacet normals at cos_m = n.h (0 for cos_m <= 0). */
double or_ggx_d(double cos_m, double alpha);

/* Smith masking G1 of GGX for a direction at cosine c > 0 to the macro normal. */
double or_ggx_g1(double c, double alpha);

/* Microfacet normal m with density D(m)(m.n) about the unit normal n, from two
 * uniforms in [0, 1). */
void or_ggx_sample(const double n[3], double alpha, double xi1, double xi2, double m[3]);

/* Rough-boundary scattering from incident direction d (unit; n = unit macro
 * normal on the incident side) into direction o: returns f(i, o) |o.n| in the
 * amplitude form, writes the solid-angle density of o under the method's
 * sampling (microfacet normal, then the reflect-if-y < R branch). */
double or_rough_eval(const double d[3], const double n[3], const double o[3], double alpha,
                     double c1, double Z1, double c2, double Z2, double *pdf);

/* Receive directivity Eq. 13; alpha in radians. */
double or_directivity(double alpha, double alpha_m, double alpha_c);

/* Analytic transmit pulse at lag tau (s): returns real part, writes imaginary part. */
double or_pulse(double tau, double f0, double n_cycles, double *imag);

/* Amplitude attenuation in Np/m for alpha (dB/cm/MHz) at f0 (Hz). */
double or_np_per_m(double alpha_db_cm_mhz, double f0);

/* Straight connection from p to element centre (x_e, 0, 0) starting in medium
 * `med` (Sec. 2.3 "Transducer Sampling").  Returns the product of the
 * transmission factors (0 if blocked by total internal reflection); writes the
 * travel time in samples and the summed attenuation exponent. */
double or_connection(const or_scene *sc, const or_array *ar, const double p[3], int32_t med,
                     double x_e, double *t_samples, double *atten_np);

#ifdef __cplusplus
}
#endif
#endif
