/*
 * ultraray.h - C ABI of the GB300 (sm_103a) full-path acoustic ray tracer.
 *
 * Implements the simulation pipeline of UltraRay (Duelmer et al., "UltraRay:
 * Introducing Full-Path Ray Tracing in Physics-Based Ultrasound Simulation",
 * arXiv 2501.05828):
 *   plane-wave ray emission with per-element transmit delays   Sec. 2.3 "Ray Emission", Eq. 6
 *   traversal: reflection / refraction at tissue boundaries     Sec. 2.3 "Ray Traversal", Eqs. 7-11
 *   transducer sampling (connection rays, receive directivity) Sec. 2.3 "Transducer Sampling", Eq. 13
 *   pulse shaping of the recorded time-pressure signals         Sec. 2.3 "Phase Calculation ...", Eq. 14
 *   delay-and-sum beamforming, envelope, log compression        same paragraph (last sentences)
 * The Monte Carlo estimators are those of Sec. 2.2 (Eqs. 4-5).  Point scatterers
 * and attenuation, which the paper names as future work (Sec. 5), are included:
 * every scatterer within a capture radius r_s of a primary-ray segment casts a
 * connection ray to a uniformly chosen element centre.
 *
 * Conventions shared by every entry point
 *  - Units: metres, seconds, m/s, MRayl (only impedance ratios matter),
 *    attenuation in dB/cm/MHz evaluated at the centre frequency.
 *  - Coordinates: the array lies in the plane z = 0 along x, centred on x = 0,
 *    elements of width `pitch` (no kerf) and elevation height `elev_h` along y;
 *    +z points into the body.
 *  - Pointers: every input pointer may be host or device memory (the library
 *    copies what it needs).  Output buffers may be host or device memory too;
 *    device outputs are written in place on the context's stream, host outputs
 *    are staged through library-owned device memory.  The caller owns all
 *    buffers it passes; the library owns the scene copy, the scatterer grid,
 *    the arrival queues and every other scratch buffer it allocates.
 *  - Streams: all work is issued on the stream given to ur_create.  Calls that
 *    return data sizes or statistics synchronise that stream.
 *  - Errors: no exception crosses the ABI.  Every call returns a ur_status;
 *    ur_last_error gives a message for the last failing call on that context.
 *    A context is used by one host thread at a time.
 */
#ifndef ULTRARAY_H
#define ULTRARAY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ur_ctx ur_ctx;

typedef enum {
    UR_OK = 0,
    UR_ERR_INVALID_ARG = 1,  /* an argument is out of range or inconsistent */
    UR_ERR_CUDA = 2,         /* a CUDA runtime call failed (message in ur_last_error) */
    UR_ERR_OOM = 3,          /* device allocation failed */
    UR_ERR_OVERFLOW = 4,     /* a caller-sized buffer was too small (required size reported) */
    UR_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
    UR_ERR_STATE = 6         /* scene, array or transmits not set before use */
} ur_status;

enum { UR_PLANE_Z = 0, UR_SPHERE = 1, UR_CYL_Y = 2 };

/* One tissue type.  c: sound speed (m/s); Z: acoustic impedance (MRayl);
 * alpha: amplitude attenuation (dB/cm/MHz, applied at the array's f0);
 * roughness: GGX parameter of the microfacet boundaries of Sec. 2.3 (Eq. 12),
 * in [0, 4]; a boundary takes the larger roughness of its two media, 0 keeps it
 * smooth (specular).  At a rough boundary the microfacet normal is sampled from
 * D(m)(m.n) and the smooth branch is taken about it (Walter et al. 2007
 * weights), and a secondary ray goes to a random element centre; these returns
 * and the direct aperture hits of the same paths are combined by the balance
 * heuristic (event word bit 31 | b << 24 | boundary + 1).  The adjoint and frozen
 * sampling media need smooth boundaries. */
typedef struct {
    float c, Z, alpha_db_cm_mhz, roughness;
} ur_medium;

/* One analytic boundary between two media (Sec. 2.3 "Ray Traversal").
 *   UR_PLANE_Z: the plane z = p[0]; med_neg lies at z < p[0], med_pos at z > p[0].
 *   UR_SPHERE:  centre (p[0], p[1], p[2]), radius p[3]; med_neg inside, med_pos outside.
 *   UR_CYL_Y:   infinite cylinder with axis parallel to y through (x = p[0], z = p[1]),
 *               radius p[2]; med_neg inside, med_pos outside. */
typedef struct {
    int32_t kind;
    int32_t med_neg, med_pos;
    float p[4];
} ur_boundary;

/* Transducer (Sec. 2.3 "Ray Emission"; parameters of Sec. 4).  Linear
 * (radius = 0): n_el elements at x_e = (e - (n_el-1)/2) pitch on z = 0, normal +z.
 * Convex (radius R > 0): element centres `pitch` apart along the arc of radius R
 * about (0, 0, -R), apex at the origin, normals radial (opening angle
 * n_el pitch / R, below about 170 degrees); the probe is the cylinder inside the
 * arc, returning rays are received where they meet it and rays passing beside it
 * end at z = -R; boundaries must stay out of the probe.  f0 centre frequency (Hz);
 * fs sampling frequency (Hz); n_s samples per channel; n_cycles sets the pulse
 * width s = n_cycles/(4 f0) of Eq. 14; alpha_m_deg / alpha_c_deg are the
 * main-beam and cutoff angles of Eq. 13 (equal values give a step);
 * c_bf is the sound speed used for transmit delays and beamforming;
 * tcut_sigmas truncates the pulse at |tau| <= tcut_sigmas * s (5 recommended). */
typedef struct {
    int32_t n_el;
    float pitch, elev_h, f0, fs;
    int32_t n_s;
    float n_cycles, alpha_m_deg, alpha_c_deg, c_bf, tcut_sigmas;
    float radius;            /* 0: linear array; > 0: convex array of this radius (m) */
} ur_array;

/* Counters of one trace call. */
typedef struct {
    uint64_t rays;          /* primary rays emitted */
    uint64_t segments;      /* straight primary-ray segments traced */
    uint64_t interactions;  /* boundary interactions (reflect / transmit / TIR) */
    uint64_t candidates;    /* scatterer events (scatterer within r_s of a segment) */
    uint64_t connections;   /* connection rays traced (events that pass the directivity) */
    uint64_t arrivals;      /* arrivals deposited into the channel data */
} ur_stats;

/* Per-arrival and per-path records for verification (all device pointers,
 * each array holds `capacity` entries).  An arrival's time in samples is
 * t_hi + t_lo; row = transmit * n_el + element; event: bits 24..30 the number
 * of boundary interactions before the event, and bit 31 set with bits 0..23 = 0
 * for a primary ray crossing the aperture, bit 31 clear with bits 0..23 the
 * scatterer index for scatterer events, bit 31 set with bits 0..23 = boundary
 * index + 1 for the secondary ray of a rough boundary.  path_hash (nullable,
 * [n_tx][n_rays]) is a 64-bit FNV-1a hash of each primary path's interaction
 * sequence and termination reason (7: a rough-boundary sample left on the wrong
 * side of the surface). */
typedef struct {
    uint64_t capacity;
    uint64_t count;          /* out: arrivals produced */
    uint32_t *ray, *event, *row;
    float *t_hi, *t_lo, *amp;
    uint64_t *path_hash;
} ur_debug;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (cudaStreamLegacy for the legacy default stream; NULL: the context creates
 * and owns a non-blocking stream).  Graph capture needs a non-default stream.
 * Errors: UR_ERR_INVALID_ARG (out == NULL, bad device), UR_ERR_CUDA. */
ur_status ur_create(ur_ctx **out, int device, void *cuda_stream);

/* Release the context and every device buffer it owns (synchronises its stream). */
ur_status ur_destroy(ur_ctx *ctx);

/* Message describing the last failing call on ctx ("" if none); valid until the next call. */
const char *ur_last_error(const ur_ctx *ctx);

/* Scene of Sec. 2.3 "Ray Traversal": media table (n_med <= 16), analytic
 * boundaries (n_bnd <= 16, media indices in [0, n_med)), the medium touching
 * the array plane, an absorbing plane z = z_max, and n_scat point scatterers
 * scat_xyza[n_scat][4] = (x, y, z, amplitude) with capture radius r_s > 0.
 * Copies everything and builds the scatterer grid on the device.  This is
 * scene slot 0, the one ur_trace uses.
 * Errors: UR_ERR_INVALID_ARG, UR_ERR_OOM, UR_ERR_CUDA. */
ur_status ur_scene_upload(ur_ctx *ctx, const ur_medium *media, int n_med,
                          const ur_boundary *bnd, int n_bnd, int med_array, float z_max,
                          const float *scat_xyza, int n_scat, float r_s);

/* Same as ur_scene_upload for scene slot `slot` in [0, 16): a context holds up
 * to 16 scenes that a batch traces together (simultaneous acquisition events,
 * Sec. 2.3 "Ray Emission"). */
ur_status ur_scene_upload_slot(ur_ctx *ctx, int slot, const ur_medium *media, int n_med,
                               const ur_boundary *bnd, int n_bnd, int med_array, float z_max,
                               const float *scat_xyza, int n_scat, float r_s);

/* Triangle-mesh boundaries of scene slot `slot` (the paper's bone is a CT-derived
 * mesh, Sec. 4), replacing any set before; an upload of the slot clears them.
 * tri[n_tri][9] = vertices v0, v1, v2 (m); tri_med[n_tri][2] = medium behind the
 * triangle (negative side of its normal (v1 - v0) x (v2 - v0)) and in front.  A
 * triangle is an interface like the analytic boundaries (Eqs. 7-11; GGX with the
 * rougher medium's roughness, Eq. 12) with that unit normal; a ray leaving it does not
 * meet it again.  Triangle t has hit id n_bnd + 3 + t in path hashes and debug
 * events.  Host or device arrays; 0 <= n_tri <= 2^22 (0 removes the mesh).  A bounding
 * volume hierarchy is built on the host; scenes with triangles are traced by the
 * extended tracer and refused by the adjoint.
 * Errors: UR_ERR_STATE (no scene in the slot), UR_ERR_INVALID_ARG (non-finite or
 * degenerate triangles, media out of range), UR_ERR_OOM, UR_ERR_CUDA. */
ur_status ur_scene_set_triangles(ur_ctx *ctx, int slot, const float *tri, const int32_t *tri_med, int n_tri);

/* Transducer description (Sec. 2.3 "Ray Emission").  1 <= n_el <= 4096,
 * 16 <= n_s <= 8192, positive geometry and frequencies, 0 <= alpha_m <= alpha_c < 90.
 * Errors: UR_ERR_INVALID_ARG. */
ur_status ur_set_array(ur_ctx *ctx, const ur_array *arr);

/* Plane-wave transmits (Sec. 2.3, Fig. 3): steering angles in radians,
 * |angle| < 60 deg, 1 <= n_tx <= 65536.  Element e of transmit k fires at
 * (x_e sin(a_k) - min_e' x_e' sin(a_k)) / c_bf.
 * Errors: UR_ERR_INVALID_ARG, UR_ERR_STATE (array not set). */
ur_status ur_set_plane_waves(ur_ctx *ctx, const float *angles_rad, int n_tx);

/* Transmit kinds (Sec. 2.3 "Ray Emission": planar, diverging or focused
 * wavefronts made by element delays).  A transmit is
 *   UR_TX_PLANE:     steering angle `angle` (rad, |angle| < 60 deg), as ur_set_plane_waves;
 *   UR_TX_DIVERGING: virtual source (x, 0, z) behind the array (z < 0): element e fires at
 *                    (|c_e - v| - min_e' |c_e' - v|) / c_bf and its rays leave along the line
 *                    from v through the emission point;
 *   UR_TX_FOCUSED:   focus (x, 0, z) in front of the array (z > 0): element e fires at
 *                    (max_e' |c_e' - f| - |c_e - f|) / c_bf and its rays head for f;
 *   UR_TX_SYNTHETIC: synthetic aperture (Sec. 1): element x (an integer value in [0, n_el))
 *                    alone fires, at t = 0; every ray of the transmit leaves a uniform point
 *                    of its face at an angle to its normal drawn uniformly in (-pi/2, pi/2)
 *                    from the ray's emission counter (third word).
 * Directions lie in the xz plane (the delays act laterally); the emission weight is the
 * cosine to the element normal over the rays of the transmit (Eq. 6).  ur_beamform uses
 * the matching transmit delays (synthetic aperture: distance from the firing element's
 * centre).  Host or device array of n_tx entries, 1 <= n_tx <= 65536.  The adjoint,
 * ur_beamform_noalloc and frozen sampling media take plane waves (and linear arrays) only.
 * Errors: UR_ERR_INVALID_ARG, UR_ERR_STATE (array not set). */
enum { UR_TX_PLANE = 0, UR_TX_DIVERGING = 1, UR_TX_FOCUSED = 2, UR_TX_SYNTHETIC = 3 };
typedef struct {
    int32_t kind;
    float angle;     /* UR_TX_PLANE */
    float x, z;      /* UR_TX_DIVERGING: virtual source; UR_TX_FOCUSED: focus (m);
                        UR_TX_SYNTHETIC: x = index of the firing element */
} ur_transmit;
ur_status ur_set_transmits(ur_ctx *ctx, const ur_transmit *tx, int n_tx);

/* Per-ray transmit mixing (Sec. 2.3: rays of different acquisition events leave
 * together, each with a randomly selected transmit).  With enabled = 1, ur_trace and
 * ur_trace_debug trace one sequence of n_tx * n_rays_per_tx rays (below 2^32); ray i
 * draws its transmit k = ((x0 >> 8) * n_tx) >> 24 from x = Philox(counter (i, 0, 0, 1))
 * and is from then on ray i of transmit k (emission counter (i, k, 0, 0), weight over
 * n_rays_per_tx, the expected rays per transmit).  Path hashes are indexed by i alone.
 * enabled = 0 (the default) traces n_rays_per_tx rays of each transmit.  Batches are not
 * affected; the adjoint and frozen sampling media refuse mixing.
 * Errors: UR_ERR_INVALID_ARG (enabled not 0 or 1). */
ur_status ur_set_transmit_mixing(ur_ctx *ctx, int enabled);

/* Trace n_rays_per_tx primary rays for every transmit (Eqs. 4-11, 13) and
 * deposit the pulse-shaped arrivals (Eq. 14) into the analytic channel data
 * rf + j quad, both [n_tx][n_el][n_s] float32 (overwritten).  Ray i of
 * transmit k leaves element i mod n_el at a uniformly random point of its
 * face; all randomness is Philox4x32-10 keyed by (seed, i, k, event), so the
 * result is a pure function of the arguments.  max_bounces <= 127 boundary
 * interactions per path, max_path_m total path length.  st may be NULL.
 * Errors: UR_ERR_STATE, UR_ERR_INVALID_ARG, UR_ERR_OOM, UR_ERR_CUDA. */
ur_status ur_trace(ur_ctx *ctx, uint64_t n_rays_per_tx, uint64_t seed, int max_bounces,
                   float max_path_m, float *rf, float *quad, ur_stats *st);

/* ur_trace plus the arrival list and per-path hashes for verification.
 * dbg->count receives the number of arrivals; UR_ERR_OVERFLOW if it exceeds
 * dbg->capacity (rf/quad are still complete). */
ur_status ur_trace_debug(ur_ctx *ctx, uint64_t n_rays_per_tx, uint64_t seed, int max_bounces,
                         float max_path_m, float *rf, float *quad, ur_stats *st, ur_debug *dbg);

/* Plane-wave delay-and-sum with coherent compounding over all transmits
 * (Sec. 2.3, last paragraph): pixel (x_px[ix], z_px[iz]) sums, over transmits
 * k and elements e, the analytic channel data linearly interpolated at
 * tau = [x sin a_k + z cos a_k - min_e x_e sin a_k + sqrt(z^2 + (x - x_e)^2)] fs / c_bf.
 * Outputs (each nullable, [nz][nx], x fastest): iq complex image as float
 * pairs, env = |iq|, db = max(20 log10(env / max env), -dyn_range_db).
 * nx, nz in [1, 16384].  Errors: UR_ERR_STATE, UR_ERR_INVALID_ARG, UR_ERR_CUDA. */
ur_status ur_beamform(ur_ctx *ctx, const float *rf, const float *quad,
                      const float *x_px, int nx, const float *z_px, int nz, float dyn_range_db,
                      float *iq, float *env, float *db);

/* ---- differentiation (the paper builds on a differentiable renderer and names
 * gradient-based optimisation as the goal, Sec. 1 and Sec. 3) ---- */

/* Replace the media of a scene slot without re-uploading its geometry
 * (n_med must match).  `sampling` (nullable) sets the media that decide the
 * Monte Carlo branches and the branch probabilities in the weights; by default
 * they are the media themselves.  Holding them fixed while `media` moves gives
 * the estimator whose derivative ur_trace_adjoint returns. */
ur_status ur_scene_set_media(ur_ctx *ctx, int slot, const ur_medium *media, int n_med, const ur_medium *sampling);

/* Replace the scatterer amplitudes of a scene slot (n_scat must match). */
ur_status ur_scene_set_amplitudes(ur_ctx *ctx, int slot, const float *amp, int n_scat);

/* Path-replay adjoint of ur_trace on scene slot 0 (at most 4 media): given
 * g_rf = dL/d rf and g_quad = dL/d quad ([n_tx][n_el][n_s], host or device),
 * replays every ray from its Philox stream with the same branch decisions and
 * returns dL/d(c, Z, alpha) of each medium in grad_media[n_med][3] and
 * dL/d(amplitude) of each scatterer in grad_amp[n_scat] (nullable).  The
 * derivative runs through hit distances, normals, refracted directions,
 * reflection/transmission factors, attenuation and times of flight (primary
 * and connection rays); branch probabilities dividing the weights are held
 * fixed (detached sampling), as are the branch decisions.  Synchronous. */
ur_status ur_trace_adjoint(ur_ctx *ctx, uint64_t n_rays_per_tx, uint64_t seed, int max_bounces,
                           float max_path_m, const float *g_rf, const float *g_quad,
                           float *grad_media, float *grad_amp);

/* ---- learned denoiser of the channel data ----
 * The paper names neural-network integration as a goal of a differentiable
 * simulator (Abstract); this library adds a small network that maps the
 * channel data of a low-ray-count trace to that of a high-ray-count trace.
 * Architecture: 4-level 2D U-Net over one transmit's channel data viewed as an
 * n_el x n_s image with 2 channels (rf, quad): two 3x3 convolutions with ReLU
 * per level, 2x2 average pooling, nearest upsampling and skip concatenation,
 * widths w, 2w, 4w, 8w, and a 1x1 head added to the input (residual).  BF16
 * weights and activations, FP32 accumulation on the tensor cores, FP32 master
 * weights and Adam.  The loss is the mean squared error of the normalised
 * channel data (channel data / scale). */
typedef struct ur_nn ur_nn;

/* Network for images of n_el x n_s (multiples of 8), up to max_batch frames,
 * width w = 32 (widths 32-256, about 2M parameters), He-initialised from seed. */
ur_status ur_nn_create(ur_nn **out, int device, void *cuda_stream, int max_batch, int n_el, int n_s, int width,
                       uint64_t seed);
ur_status ur_nn_destroy(ur_nn *nn);
const char *ur_nn_last_error(const ur_nn *nn);

/* Number of parameters of the packed FP32 vector: per convolution l (order
 * e1a e1b e2a e2b e3a e3b e4a e4b d3a d3b d2a d2b d1a d1b) the weights
 * [9 taps][c_out][c_in] (the first convolution's c_in padded to 32 with zero
 * weights beyond the 2 real channels) then the bias [c_out], each tensor
 * starting at a multiple of 8 entries; then the head [2][w] and its bias [2]. */
ur_status ur_nn_param_count(const ur_nn *nn, uint64_t *n);

/* Number of kernels the network has enqueued since ur_nn_create (every
 * convolution is one launch; memsets and copies are not counted). */
ur_status ur_nn_launch_count(const ur_nn *nn, uint64_t *n);

/* Copy the parameters out (get, nullable) and/or in (set, nullable; resets Adam). */
ur_status ur_nn_params(ur_nn *nn, float *get, const float *set);

/* Normalisation: the network sees channel data / scale. */
ur_status ur_nn_set_scale(ur_nn *nn, float scale);

/* Denoise `batch` frames: rf, quad [batch][n_el][n_s] -> out_rf, out_quad (same
 * layout).  Each pointer may be device or host memory (host buffers are staged
 * through device copies on the network's stream; pinned memory keeps the copies
 * asynchronous).  Synchronises the stream before returning.
 * Errors: UR_ERR_INVALID_ARG (batch outside 1..max_batch, null pointers),
 * UR_ERR_TIMEOUT (a convolution pipeline wait gave up), UR_ERR_CUDA. */
ur_status ur_nn_forward(ur_nn *nn, const float *rf, const float *quad, int batch, float *out_rf, float *out_quad);

/* One training step on `batch` pairs (inputs rf, quad; targets t_rf, t_quad;
 * host or device, as for ur_nn_forward): forward, loss, backward, then Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with learning rate lr
 * (lr = 0: no update).  loss (nullable, host) receives the loss; grad_out
 * (nullable, host or device, ur_nn_param_count floats) the parameter gradient
 * before the update.  Same errors as ur_nn_forward. */
ur_status ur_nn_train_step(ur_nn *nn, const float *rf, const float *quad, const float *t_rf, const float *t_quad,
                           int batch, float lr, float *loss, float *grad_out);

/* ---- batches: many (scene, transmit) items in one persistent launch ----
 * Rays of different transmits and scenes are independent (Sec. 2.3, "Ray
 * Emission": acquisition events can be simulated at the same time), so a
 * batch traces all its items in one launch of the persistent tracer, sorts and
 * deposits all arrivals in one pass, and beamforms one compounded image per
 * scene.  Item q: scene slot, index into the plane-wave table, n_rays rays,
 * and `stream`, the Philox counter word that keys its random numbers (ur_trace
 * uses stream = transmit index; distinct items should use distinct
 * (scene, stream) pairs). */
typedef struct {
    int32_t scene;
    int32_t tx;
    uint32_t stream;
    uint32_t reserved;
    uint64_t n_rays;
} ur_batch_item;

/* Validate the items, allocate every buffer a run needs (arrival queue of
 * arrival_capacity entries, 0 = estimate from earlier traces), upload the item
 * table and the image grid (x_px[nx], z_px[nz], host or device).  Must run
 * outside stream capture; it synchronises the stream.  Images are produced for
 * the scenes present, in increasing slot order.
 * Errors: UR_ERR_STATE (missing scene/array/transmits), UR_ERR_INVALID_ARG, UR_ERR_OOM. */
ur_status ur_batch_plan(ur_ctx *ctx, const ur_batch_item *items, int n_items, uint64_t arrival_capacity,
                        const float *x_px, int nx, const float *z_px, int nz);

/* Trace and deposit the planned batch into rf, quad [n_items][n_el][n_s]
 * (device memory).  Asynchronous, allocates nothing and may be captured into
 * a graph (ur_graph_begin).  If the queue overflows, ur_batch_status reports it. */
ur_status ur_batch_trace(ur_ctx *ctx, uint64_t seed, int max_bounces, float max_path_m, float *rf, float *quad);

/* Synchronise and report the last trace: arrivals produced and counters.
 * UR_ERR_OVERFLOW if the planned capacity was too small (re-plan larger). */
ur_status ur_batch_status(ur_ctx *ctx, uint64_t *n_arrivals, ur_stats *st);

/* Delay-and-sum of the planned batch: image i compounds all items of the i-th
 * scene present (outputs [n_images][nz][nx], device memory, each nullable).
 * Asynchronous and capturable. */
ur_status ur_batch_beamform(ur_ctx *ctx, const float *rf, const float *quad, float dyn_range_db,
                            float *iq, float *env, float *db);

/* CUDA-graph capture of the context's stream: calls between ur_graph_begin and
 * ur_graph_end (ur_batch_trace, ur_batch_beamform) are recorded, not run;
 * ur_graph_launch replays them.  Calls that synchronise or allocate fail with
 * UR_ERR_STATE while capturing. */
ur_status ur_graph_begin(ur_ctx *ctx);
ur_status ur_graph_end(ur_ctx *ctx);
ur_status ur_graph_launch(ur_ctx *ctx);

/* Scatterer-grid and launch tuning (0 fields keep the defaults).  Cell sizes in
 * metres along x (cell_xy), y (cell_y) and z (cell_z), applied at the next
 * ur_scene_upload.  Defaults: 8 r_s, 0.3 r_s and 60 r_s when every boundary is
 * a plane z = c or a cylinder along y (plane waves of a linear array then never
 * gain a y component, so thin y cells add few cell steps and hold fewer
 * scatterers); 3 r_s, 3 r_s and 40 r_s when the scene holds a sphere.  block (multiple of 32, <= 256), blocks_per_sm and
 * resolve_batch (1..32: the tracer finishes segments and starts rays once this
 * many lanes of a warp wait; default 20) apply at the next trace. */
typedef struct {
    float cell_xy, cell_z;
    int32_t block, blocks_per_sm, resolve_batch;
    float cell_y;
} ur_tuning;
ur_status ur_set_tuning(ur_ctx *ctx, const ur_tuning *t);

/* Autotuner: coordinate descent over the three grid cell sizes, resolve batch and CTAs
 * per SM, timing n_rays rays of transmit 0 of scene slot `scene` with CUDA
 * events; keeps the fastest setting (rebuilding every scene's grid) and
 * returns it in *best (nullable).  Synchronous. */
ur_status ur_autotune(ur_ctx *ctx, int scene, uint64_t n_rays, uint64_t seed, int max_bounces,
                      float max_path_m, ur_tuning *best);

/* Device time per pipeline phase, measured with CUDA events recorded on the
 * context's stream around each phase's kernels while profiling is on.  While
 * profiling, every call synchronises the stream before returning. */
enum { UR_PHASE_GRID = 0, UR_PHASE_TRACE = 1, UR_PHASE_SORT = 2, UR_PHASE_DEPOSIT = 3,
       UR_PHASE_DAS = 4, UR_PHASE_LOG = 5, UR_PHASE_ADJOINT = 6, UR_N_PHASES = 8 };
typedef struct {
    double ms[UR_N_PHASES];          /* accumulated device milliseconds */
    uint64_t launches[UR_N_PHASES];  /* kernels launched */
    uint64_t calls[UR_N_PHASES];     /* times the phase ran */
} ur_profile;

/* on != 0 clears the accumulators and starts profiling; on == 0 stops it. */
ur_status ur_set_profiling(ur_ctx *ctx, int on);

/* Copy the accumulators (valid whether or not profiling is still on). */
ur_status ur_get_profile(ur_ctx *ctx, ur_profile *out);

/* Allocation-free variant of ur_beamform (the paper has no counterpart).
 *
 * Some callers cannot let a library call cudaMalloc: real-time acquisition
 * loops that forbid allocation after start-up (cudaMalloc can synchronise the
 * device and stall a frame by milliseconds), hosts that hand all of the GPU's
 * memory to their own pool up front (a library allocation would fail or
 * fragment that pool), and plug-ins inside frameworks that own every device
 * buffer themselves.  This entry point computes exactly what ur_beamform
 * computes (same kernels) but allocates nothing: its scratch (transmit tables,
 * pixel coordinates, the envelope maximum and, when env is NULL, the envelope)
 * lives in a fixed device array of UR_NOALLOC_SCRATCH_BYTES (4.5 MiB) that
 * every GPU loading the library holds until the process exits.
 *
 * Requirements: the context's array and transmits are set (UR_ERR_STATE
 * otherwise), the transmits are plane waves and the array is linear
 * (UR_ERR_INVALID_ARG otherwise); rf, quad and every non-NULL output are
 * device memory of the context's GPU (or managed memory; UR_ERR_INVALID_ARG
 * otherwise); x_px / z_px may be host or device memory.  Limits:
 * n_tx <= UR_NOALLOC_MAX_TX, nx, nz <= UR_NOALLOC_MAX_AXIS, and
 * nx * nz <= UR_NOALLOC_MAX_PIXELS when env is NULL; larger requests return
 * UR_ERR_INVALID_ARG without launching work.  The first call on a device looks
 * up the scratch's device address (once per device).  All calls share the one
 * scratch array, which keeps the last call's contents (the envelope maximum is
 * cleared by each call): calls whose work overlaps on the GPU (for example on
 * two streams) race and must be serialised by the caller.  A CUDA error left
 * pending by earlier work is reported as UR_ERR_CUDA and not cleared.
 * Works asynchronously on the context's stream; reports errors through the
 * status only (ur_last_error is not updated). */
#define UR_NOALLOC_MAX_TX 1024
#define UR_NOALLOC_MAX_AXIS 8192
#define UR_NOALLOC_MAX_PIXELS (1 << 20)
#define UR_NOALLOC_SCRATCH_BYTES (4608 * 1024)
ur_status ur_beamform_noalloc(ur_ctx *ctx, const float *rf, const float *quad,
                              const float *x_px, int nx, const float *z_px, int nz, float dyn_range_db,
                              float *iq, float *env, float *db);

/* Wait for all work on the context's stream and report asynchronous errors. */
ur_status ur_sync(ur_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ULTRARAY_H */
