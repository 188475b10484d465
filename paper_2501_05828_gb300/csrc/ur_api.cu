// C ABI of the acoustic ray tracer (declared in include/ultraray.h): argument
// validation, device buffers owned by the context, derived constants (media
// slowness, transmit delays, directivity cosines), the launch sequence
// trace -> sort -> deposit and delay-and-sum -> log compression, batches of
// (scene, transmit) items in one persistent launch, CUDA-graph capture of a
// batch, and the tracer autotuner.
#include "ultraray.h"
#include "ur_device.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Fail {
    ur_status code;
    std::string msg;
};

[[noreturn]] void fail(ur_status code, const std::string &msg) { throw Fail{code, msg}; }

void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? UR_ERR_OOM : UR_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

ur::ff split(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr double kPi = 3.14159265358979323846;
constexpr uint32_t kChunk = 4096;      // most arrivals per deposit work item
constexpr uint32_t kChunkMin = 512;    // fewest (work items are sized for several deposit waves)

// One uploaded scene: host copies of media and boundaries, device scatterers and grid.
// Default scatterer-grid cell sizes (x, y, z) in units of the capture radius
// r_s.  The tracer walks columns in x and y; z cells only index each column's
// references by depth (a visit reads the z cells within r_s of the depths it
// spans).  Plane waves of a linear array travel in the xz plane, and smooth
// planes z = c and cylinders along y keep them there (their normals have no y
// component), so in such scenes thin y columns hold few scatterers and cost no
// steps.  Rough boundaries scatter part of the rays out of the plane (wider y
// columns), and spheres and triangle meshes turn every ray in 3D (square
// columns).  Measured on the layered frame (smooth: 10.6 ms at 6 x 0.3 x 4 r_s),
// its rough-bone version (17.7 ms at 4 x 2 x 4 against 20.0 at 6 x 0.3 x 4) and
// the paper-settings and mesh-bone acquisitions (9.1 and 23.9 ms at 6 x 6 x 4
// against 10.9 and 26.6 at 3 x 3 x 5).
constexpr float kCellSlab[3] = {6.f, 0.3f, 4.f};
constexpr float kCellRough[3] = {4.f, 2.f, 4.f};
constexpr float kCellIso[3] = {6.f, 6.f, 4.f};
// Fine columns (x, y, z in r_s) for exactly vertical segments (every 0-degree plane-wave ray until
// it meets a tilted boundary, and every normal-incidence echo): such a segment stays in one
// column, so narrow columns cost it no steps and hold (0.5 + 2)^2 / pi = 2x the scatterers of
// its capture tube, against (6 + 2) (0.3 + 2) / pi = 5.9x in the default columns of a planar
// scene.  83 % of the layered frame's reference tests came from such segments.
constexpr float kCellFine[3] = {0.5f, 0.5f, 10.f};
constexpr double kFineMaxCells = (double)(1u << 24);
constexpr int kResolveBatch = 20;   // default: lanes that must wait before a tracer warp resolves segments

struct SceneData {
    bool ok = false;
    uint64_t version = 0;              // changes with every upload and media change (paths may change)
    std::vector<ur_medium> media;
    std::vector<ur_medium> sampling;   // media deciding Monte Carlo branches (same as media unless overridden)
    std::vector<ur_boundary> bnd;
    int med_array = 0;
    float z_max = 0.f;
    int n_scat = 0;
    float r_s = 1e-4f;
    float g_rm = 0.f;
    float cell_req[3] = {0.f, 0.f, 0.f};   // cell sizes the grid was built for (before any enlargement)
    float3 g_lo{}, g_h{}, g_inv_h{};
    int3 g_dim{};
    DevBuf scat, amp, refs, cell_count, cell_start, cell_fill, scan_tmp, bbox;
    // fine columns for exactly vertical segments (same build, narrow x-y cells)
    DevBuf f_refs, f_cell_count, f_cell_start, f_cell_fill;
    float3 f_lo{}, f_h{}, f_inv_h{};
    int3 f_dim{};
    bool f_built = false;
    int n_tri = 0;                     // triangle-mesh boundaries (ur_scene_set_triangles)
    DevBuf bvh, tri, tri_nrm;
};

}  // namespace

struct ur_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    unsigned long long *host_scratch = nullptr;  // pinned, 64 words

    SceneData scenes[ur::kMaxScenes];

    // array and plane-wave table
    bool array_ok = false;
    ur_array arr{};
    std::vector<float> angles;              // plane-wave angle per transmit (0 for the other kinds)
    std::vector<int> tx_kinds;              // UR_TX_* per transmit
    std::vector<float> tx_vx, tx_vz;        // virtual source / focus (synthetic aperture: element) per transmit
    bool tx_dirty = true;
    bool mix_tx = false;                    // ur_trace: each ray draws its transmit
    ur::MixP mix{};                         // ray order of the last mixed trace (list null: none)
    DevBuf mix_list, mix_bins;
    DevBuf adj_order, adj_keys;        // arrivals of the adjoint in path-shape order, and that sort's counts
    DevBuf delay, tx_sin, tx_cos, tx_m, tx_kind, elem_xz;

    // work items of the last trace or batch plan
    std::vector<ur::ItemP> items;
    std::vector<ur_batch_item> batch_items;
    uint64_t n_slots = 0;
    DevBuf items_dev;

    // trace buffers
    DevBuf arrivals, arr_dbg, sorted, counters, row_count, row_fill, row_off, work, n_work;
    uint64_t arr_cap = 0;
    double arr_per_ray = 0.5;

    // images
    DevBuf stage_rf, stage_quad, pix, stage_iq, stage_env, stage_db, env_max, img_lists;

    // adjoint
    DevBuf adj_grad, adj_amp, adj_g;
    // (ray, event) words of the last ur_trace's arrivals (recorded once an adjoint has been asked
    // for) and the settings they were traced with
    bool want_rec = false;
    uint64_t versions = 0;
    struct MaskKey {
        bool valid = false;
        uint64_t seed = 0, n_rays = 0, scene_version = 0, n_slots = 0;
        int max_b = 0;
        float max_path = 0.f;
        std::vector<float> angles;
        bool operator==(const MaskKey &o) const {
            return valid && o.valid && seed == o.seed && n_rays == o.n_rays && scene_version == o.scene_version &&
                   n_slots == o.n_slots && max_b == o.max_b && max_path == o.max_path && angles == o.angles;
        }
    } rec_key;

    // batch plan
    bool batch_ok = false;
    uint64_t batch_cap = 0;
    int batch_nx = 0, batch_nz = 0, batch_images = 0;
    std::vector<int> batch_image_scene;
    DevBuf batch_pix, batch_lists, batch_env, batch_max;

    // stream capture into a CUDA graph
    bool capturing = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;

    ur_tuning tune{};

    // per-phase CUDA-event profiling
    bool prof = false;
    cudaEvent_t ev0[UR_N_PHASES] = {}, ev1[UR_N_PHASES] = {};
    ur_profile acc{};
    bool pending[UR_N_PHASES] = {};

    bool profiling() const { return prof && !capturing; }
    void phase_begin(int p) {
        if (!profiling()) return;
        if (!ev0[p]) {
            ck(cudaEventCreate(&ev0[p]), "cudaEventCreate");
            ck(cudaEventCreate(&ev1[p]), "cudaEventCreate");
        }
        ck(cudaEventRecord(ev0[p], stream), "cudaEventRecord");
    }
    void phase_end(int p, int kernels) {
        if (!profiling()) return;
        ck(cudaEventRecord(ev1[p], stream), "cudaEventRecord");
        pending[p] = true;
        acc.launches[p] += (uint64_t)kernels;
        acc.calls[p] += 1;
    }
    // after a stream synchronisation: fold finished phases into the accumulators
    void phase_collect() {
        if (!profiling()) return;
        for (int p = 0; p < UR_N_PHASES; ++p)
            if (pending[p]) {
                float ms = 0.f;
                ck(cudaEventElapsedTime(&ms, ev0[p], ev1[p]), "cudaEventElapsedTime");
                acc.ms[p] += ms;
                pending[p] = false;
            }
    }
    void prof_sync() {
        if (!profiling()) return;
        ck(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
        phase_collect();
    }
    void no_capture(const char *what) {
        if (capturing) fail(UR_ERR_STATE, std::string(what) + " cannot run while the stream is being captured");
    }

    void grow(DevBuf &b, size_t bytes) {
        if (bytes <= b.bytes && b.p) return;
        if (capturing) fail(UR_ERR_STATE, "a buffer would have to grow during stream capture: plan the batch first");
        if (b.p) {
            ck(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
            ck(cudaFree(b.p), "cudaFree");
            b.p = nullptr;
            b.bytes = 0;
        }
        const size_t want = std::max<size_t>(bytes, 256);
        ck(cudaMalloc(&b.p, want), "cudaMalloc");
        b.bytes = want;
    }
    void release(DevBuf &b) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    void set_device() { ck(cudaSetDevice(device), "cudaSetDevice"); }
};

namespace {

template <class F>
ur_status guarded(ur_ctx *c, F &&f) {
    if (!c) return UR_ERR_INVALID_ARG;
    try {
        c->err.clear();
        f();
        return UR_OK;
    } catch (const Fail &e) {
        c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        c->err = "host allocation failed";
        return UR_ERR_OOM;
    } catch (...) {
        c->err = "unexpected host exception";
        return UR_ERR_CUDA;
    }
}

// Transmit tables: per-element delays, and per transmit the delay-and-sum constants
// (plane wave: sin, cos, min_e x_e sin; diverging / focused wave: x, z of the virtual
// source / focus and the smallest / largest element distance to it).
void prepare_transmits(ur_ctx *c) {
    if (!c->tx_dirty) return;
    c->no_capture("preparing transmit tables");
    const int nt = (int)c->angles.size(), ne = c->arr.n_el;
    std::vector<ur::ff> delay((size_t)nt * ne), s(nt), co(nt), m(nt);
    const double pitch = c->arr.pitch, x0 = -0.5 * (double)(ne - 1) * pitch;
    std::vector<double> len(ne), cx(ne), cz(ne);   // element centres: linear, or on the convex arc
    const double R = c->arr.radius, dphi = R > 0.0 ? pitch / R : 0.0, phi0 = -0.5 * (double)(ne - 1) * dphi;
    for (int e = 0; e < ne; ++e) {
        cx[e] = R > 0.0 ? R * std::sin(phi0 + e * dphi) : x0 + e * pitch;
        cz[e] = R > 0.0 ? R * (std::cos(phi0 + e * dphi) - 1.0) : 0.0;
    }
    std::vector<int> das_kind(c->tx_kinds);
    for (int k = 0; k < nt; ++k) {
        int kind = c->tx_kinds[k];
        double vx = c->tx_vx[k], vz = c->tx_vz[k];
        if (kind == UR_TX_SYNTHETIC) {   // to the delay-and-sum, a wave diverging from the element's centre
            if (!(vx < (double)ne)) fail(UR_ERR_INVALID_ARG, "a synthetic-aperture transmit names an element past the array");
            const int f = (int)vx;
            vx = cx[f];
            vz = cz[f];
            das_kind[k] = UR_TX_DIVERGING;
        }
        const double th = c->angles[k];
        const double sn = std::sin(th), cs = std::cos(th);
        // path from the wave's reference to element e: c_e . (sin, cos) (plane), |c_e - v|
        // (diverging), -|c_e - f| (focused); each element fires when the wavefront through the
        // first-firing element reaches it
        double mn = INFINITY;
        for (int e = 0; e < ne; ++e) {
            const double r = std::sqrt((cx[e] - vx) * (cx[e] - vx) + (cz[e] - vz) * (cz[e] - vz));
            len[e] = kind == UR_TX_PLANE ? cx[e] * sn + cz[e] * cs
                   : kind == UR_TX_SYNTHETIC ? 0.0   // the one element fires at t = 0
                   : kind == UR_TX_DIVERGING ? r : -r;
            mn = std::min(mn, len[e]);
        }
        for (int e = 0; e < ne; ++e)
            delay[(size_t)k * ne + e] = split((len[e] - mn) / (double)c->arr.c_bf * (double)c->arr.fs);
        s[k] = split(kind == UR_TX_PLANE ? sn : vx);
        co[k] = split(kind == UR_TX_PLANE ? cs : vz);
        m[k] = split(kind == UR_TX_FOCUSED ? -mn : mn);
    }
    if (R > 0.0) {   // element centres for the convex delay-and-sum
        std::vector<ur::ff> exz(2 * (size_t)ne);
        for (int e = 0; e < ne; ++e) {
            exz[2 * e] = split(cx[e]);
            exz[2 * e + 1] = split(cz[e]);
        }
        c->grow(c->elem_xz, sizeof(ur::ff) * exz.size());
        ck(cudaMemcpyAsync(c->elem_xz.p, exz.data(), sizeof(ur::ff) * exz.size(), cudaMemcpyHostToDevice, c->stream),
           "copy element centres");
        ck(cudaStreamSynchronize(c->stream), "element centres");
    }
    c->grow(c->tx_kind, sizeof(int) * std::max(nt, 1));
    ck(cudaMemcpyAsync(c->tx_kind.p, das_kind.data(), sizeof(int) * nt, cudaMemcpyHostToDevice, c->stream),
       "copy kinds");
    c->grow(c->delay, sizeof(ur::ff) * delay.size());
    c->grow(c->tx_sin, sizeof(ur::ff) * nt);
    c->grow(c->tx_cos, sizeof(ur::ff) * nt);
    c->grow(c->tx_m, sizeof(ur::ff) * nt);
    ck(cudaMemcpyAsync(c->delay.p, delay.data(), sizeof(ur::ff) * delay.size(), cudaMemcpyHostToDevice, c->stream), "copy delay");
    ck(cudaMemcpyAsync(c->tx_sin.p, s.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy sin");
    ck(cudaMemcpyAsync(c->tx_cos.p, co.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy cos");
    ck(cudaMemcpyAsync(c->tx_m.p, m.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy m");
    ck(cudaStreamSynchronize(c->stream), "sync transmit tables");  // host vectors go out of scope
    c->tx_dirty = false;
}

// Default cell size along axis a (0 x, 1 y, 2 z) for a scene, in metres.
// Planar scenes: no sphere and no triangles (plane waves of a linear array keep to the xz plane
// at their smooth boundaries, and travel vertically at 0 degrees).
bool planar_scene(const SceneData &sd) {
    bool planar = sd.n_tri == 0;
    for (const ur_boundary &b : sd.bnd) planar &= b.kind != UR_SPHERE;
    return planar;
}

bool rough_scene(const SceneData &sd) {
    bool rough = false;
    for (const ur_boundary &b : sd.bnd)
        rough |= sd.media[b.med_neg].roughness > 0.f || sd.media[b.med_pos].roughness > 0.f;
    return rough;
}

float default_cell(const SceneData &sd, int a) {
    return (!planar_scene(sd) ? kCellIso : rough_scene(sd) ? kCellRough : kCellSlab)[a] * sd.r_s;
}

// Fine columns serve the plane-wave tracer's vertical segments: smooth planar scenes only (rough
// boundaries, spheres and triangles run the extended tracers, which keep to the usual columns).
bool wants_fine(const SceneData &sd) { return planar_scene(sd) && !rough_scene(sd); }

void build_grid(ur_ctx *c, SceneData &sd, const float *src);

// Rebuild a scene's grid when its default cells changed (triangles or roughness set after the
// upload) and no tuning overrides them, or when triangles decide whether it has fine columns.
void regrid_if_default_changed(ur_ctx *c, SceneData &sd) {
    if (sd.n_scat == 0) return;
    const float want[3] = {c->tune.cell_xy > 0.f ? c->tune.cell_xy : default_cell(sd, 0),
                           c->tune.cell_y > 0.f ? c->tune.cell_y : default_cell(sd, 1),
                           c->tune.cell_z > 0.f ? c->tune.cell_z : default_cell(sd, 2)};
    if (want[0] != sd.cell_req[0] || want[1] != sd.cell_req[1] || want[2] != sd.cell_req[2] ||
        sd.f_built != wants_fine(sd))
        build_grid(c, sd, nullptr);
}

// Build (or rebuild) a scene's scatterer grid; src == nullptr reuses the device copy.
void build_grid(ur_ctx *c, SceneData &sd, const float *src) {
    const int n = sd.n_scat;
    if (src) {
        c->grow(sd.scat, sizeof(float4) * n);
        c->grow(sd.amp, sizeof(float) * n);
        ck(cudaMemcpyAsync(sd.scat.p, src, sizeof(float4) * n, cudaMemcpyDefault, c->stream), "copy scatterers");
    }
    c->grow(sd.bbox, 6 * sizeof(unsigned int));
    const unsigned int init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    ck(cudaMemcpyAsync(sd.bbox.p, init, sizeof init, cudaMemcpyHostToDevice, c->stream), "init bbox");
    c->phase_begin(UR_PHASE_GRID);
    ur::launch_bbox((const float4 *)sd.scat.p, n, (float *)sd.bbox.p, c->stream);
    c->phase_end(UR_PHASE_GRID, 1);
    ck(cudaGetLastError(), "bbox kernel");
    unsigned int *hb = (unsigned int *)c->host_scratch;
    ck(cudaMemcpyAsync(hb, sd.bbox.p, sizeof init, cudaMemcpyDeviceToHost, c->stream), "read bbox");
    ck(cudaStreamSynchronize(c->stream), "bbox sync");
    c->phase_collect();
    float lo[3], hi[3];
    for (int a = 0; a < 6; ++a) {
        unsigned int u = hb[a];
        u = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
        float f;
        std::memcpy(&f, &u, 4);
        (a < 3 ? lo[a] : hi[a - 3]) = f;
    }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a])) fail(UR_ERR_INVALID_ARG, "scatterer coordinates must be finite");
    // capture box margin: r_s plus a relative and absolute slack far above FP32 rounding
    const float r_m = sd.r_s * 1.001f + 1e-7f;
    float h_x = c->tune.cell_xy > 0.f ? c->tune.cell_xy : default_cell(sd, 0);
    float h_y = c->tune.cell_y > 0.f ? c->tune.cell_y : default_cell(sd, 1);
    float h_z = c->tune.cell_z > 0.f ? c->tune.cell_z : default_cell(sd, 2);
    sd.cell_req[0] = h_x;
    sd.cell_req[1] = h_y;
    sd.cell_req[2] = h_z;
    int3 dim;
    for (;;) {
        dim.x = std::max(1, (int)std::ceil((hi[0] - lo[0] + 2.f * r_m) / h_x));
        dim.y = std::max(1, (int)std::ceil((hi[1] - lo[1] + 2.f * r_m) / h_y));
        dim.z = std::max(1, (int)std::ceil((hi[2] - lo[2] + 2.f * r_m) / h_z));
        if ((double)dim.x * dim.y * dim.z <= (double)(1u << 26)) break;
        h_x *= 1.5f;
        h_y *= 1.5f;
        h_z *= 1.5f;
    }
    sd.g_rm = r_m;
    sd.g_lo = make_float3(lo[0] - r_m, lo[1] - r_m, lo[2] - r_m);
    sd.g_h = make_float3(h_x, h_y, h_z);
    sd.g_inv_h = make_float3(1.f / h_x, 1.f / h_y, 1.f / h_z);
    sd.g_dim = dim;
    // the fine columns over the same box
    float f_x = kCellFine[0] * sd.r_s, f_y = kCellFine[1] * sd.r_s, f_z = kCellFine[2] * sd.r_s;
    int3 fdim;
    for (;;) {
        fdim.x = std::max(1, (int)std::ceil((hi[0] - lo[0] + 2.f * r_m) / f_x));
        fdim.y = std::max(1, (int)std::ceil((hi[1] - lo[1] + 2.f * r_m) / f_y));
        fdim.z = std::max(1, (int)std::ceil((hi[2] - lo[2] + 2.f * r_m) / f_z));
        if ((double)fdim.x * fdim.y * fdim.z <= kFineMaxCells) break;
        f_x *= 1.5f;
        f_y *= 1.5f;
        f_z *= 1.5f;
    }
    sd.f_lo = sd.g_lo;
    sd.f_h = make_float3(f_x, f_y, f_z);
    sd.f_inv_h = make_float3(1.f / f_x, 1.f / f_y, 1.f / f_z);
    sd.f_dim = fdim;
    const uint32_t n_cells = (uint32_t)dim.x * dim.y * dim.z;
    const uint32_t f_cells = (uint32_t)fdim.x * fdim.y * fdim.z;
    c->grow(sd.scan_tmp, sizeof(uint32_t) * (std::max(n_cells, f_cells) / 4096 + 4));
    struct One {
        DevBuf *count, *start, *fill, *refs;
        float3 lo, inv_h;
        int3 dim;
        uint32_t n_cells;
    } grids[2] = {{&sd.cell_count, &sd.cell_start, &sd.cell_fill, &sd.refs, sd.g_lo, sd.g_inv_h, dim, n_cells},
                  {&sd.f_cell_count, &sd.f_cell_start, &sd.f_cell_fill, &sd.f_refs, sd.f_lo, sd.f_inv_h, fdim, f_cells}};
    ur::GridBuildP G[2];
    sd.f_built = wants_fine(sd);
    const int n_grids = sd.f_built ? 2 : 1;
    c->phase_begin(UR_PHASE_GRID);
    for (int q = 0; q < n_grids; ++q) {
        const One &o = grids[q];
        c->grow(*o.count, sizeof(uint32_t) * (o.n_cells + 1));
        c->grow(*o.start, sizeof(uint32_t) * (o.n_cells + 1));
        c->grow(*o.fill, sizeof(uint32_t) * (o.n_cells + 1));
        ck(cudaMemsetAsync(o.count->p, 0, sizeof(uint32_t) * (o.n_cells + 1), c->stream), "memset counts");
        ck(cudaMemsetAsync(o.fill->p, 0, sizeof(uint32_t) * (o.n_cells + 1), c->stream), "memset fill");
        G[q] = ur::GridBuildP{};
        G[q].scat = (const float4 *)sd.scat.p;
        G[q].n_scat = n;
        G[q].r_m = r_m;
        G[q].lo = o.lo;
        G[q].inv_h = o.inv_h;
        G[q].dim = o.dim;
        G[q].cell_count = (uint32_t *)o.count->p;
        G[q].cell_start = (uint32_t *)o.start->p;
        G[q].cell_fill = (uint32_t *)o.fill->p;
        G[q].amp = (float *)sd.amp.p;
        ur::launch_grid_count(G[q], c->stream);
        ck(cudaGetLastError(), "grid count kernel");
        ur::launch_scan_u32(G[q].cell_count, G[q].cell_start, (uint32_t *)sd.scan_tmp.p, o.n_cells, c->stream);
        ck(cudaGetLastError(), "scan kernel");
        ck(cudaMemcpyAsync(hb + q, G[q].cell_start + o.n_cells, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream),
           "read refs");
    }
    c->phase_end(UR_PHASE_GRID, 4 * n_grids);
    ck(cudaStreamSynchronize(c->stream), "grid sync");
    c->phase_collect();
    const uint32_t n_refs[2] = {((uint32_t *)hb)[0], ((uint32_t *)hb)[1]};
    c->phase_begin(UR_PHASE_GRID);
    for (int q = 0; q < n_grids; ++q) {
        c->grow(*grids[q].refs, sizeof(float4) * std::max<uint32_t>(n_refs[q], 1));
        G[q].refs = (float4 *)grids[q].refs->p;
        ur::launch_grid_fill(G[q], c->stream);
        ck(cudaGetLastError(), "grid fill kernel");
    }
    c->phase_end(UR_PHASE_GRID, n_grids);
    c->prof_sync();
}

void upload_scene(ur_ctx *c, int slot, const ur_medium *media, int n_med, const ur_boundary *bnd, int n_bnd,
                  int med_array, float z_max, const float *scat_xyza, int n_scat, float r_s) {
    c->set_device();
    c->no_capture("ur_scene_upload");
    if (slot < 0 || slot >= ur::kMaxScenes) fail(UR_ERR_INVALID_ARG, "scene slot must be in [0, 16)");
    SceneData &sd = c->scenes[slot];
    sd.ok = false;
    sd.n_tri = 0;   // a new scene starts without triangles
    c->batch_ok = false;
    if (!media || n_med < 1 || n_med > ur::kMaxMed) fail(UR_ERR_INVALID_ARG, "n_med must be in [1, 16]");
    if (n_bnd < 0 || n_bnd > ur::kMaxBnd || (n_bnd > 0 && !bnd)) fail(UR_ERR_INVALID_ARG, "n_bnd must be in [0, 16]");
    if (med_array < 0 || med_array >= n_med) fail(UR_ERR_INVALID_ARG, "med_array out of range");
    if (!(z_max > 0.f) || !std::isfinite(z_max)) fail(UR_ERR_INVALID_ARG, "z_max must be positive");
    if (n_scat < 0 || n_scat >= (1 << 24)) fail(UR_ERR_INVALID_ARG, "n_scat must be in [0, 2^24)");
    if (n_scat > 0 && (!scat_xyza || !(r_s > 0.f) || !std::isfinite(r_s)))
        fail(UR_ERR_INVALID_ARG, "scatterers need a pointer and a positive capture radius");
    std::vector<ur_medium> M(media, media + n_med);
    for (const ur_medium &m : M) {
        if (!(m.c > 0.f) || !(m.Z > 0.f) || !(m.alpha_db_cm_mhz >= 0.f) || !std::isfinite(m.c) || !std::isfinite(m.Z))
            fail(UR_ERR_INVALID_ARG, "media need c > 0, Z > 0, alpha >= 0");
        if (!(m.roughness >= 0.f && m.roughness <= 4.f)) fail(UR_ERR_INVALID_ARG, "roughness must be in [0, 4]");
    }
    std::vector<ur_boundary> Bv(bnd, bnd + n_bnd);
    for (const ur_boundary &b : Bv) {
        if (b.kind < UR_PLANE_Z || b.kind > UR_CYL_Y) fail(UR_ERR_INVALID_ARG, "unknown boundary kind");
        if (b.med_neg < 0 || b.med_neg >= n_med || b.med_pos < 0 || b.med_pos >= n_med)
            fail(UR_ERR_INVALID_ARG, "boundary media out of range");
        for (float v : b.p)
            if (!std::isfinite(v)) fail(UR_ERR_INVALID_ARG, "boundary parameters must be finite");
        if (b.kind == UR_PLANE_Z && !(b.p[0] > 0.f && b.p[0] < z_max))
            fail(UR_ERR_INVALID_ARG, "planes must lie strictly between the array and z_max");
        if (b.kind == UR_SPHERE && !(b.p[3] > 0.f)) fail(UR_ERR_INVALID_ARG, "sphere radius must be positive");
        if (b.kind == UR_CYL_Y && !(b.p[2] > 0.f)) fail(UR_ERR_INVALID_ARG, "cylinder radius must be positive");
    }
    sd.media = M;
    sd.sampling = M;
    sd.bnd = Bv;
    sd.med_array = med_array;
    sd.z_max = z_max;
    sd.n_scat = n_scat;
    sd.r_s = n_scat > 0 ? r_s : 1e-4f;
    if (n_scat > 0) {
        build_grid(c, sd, scat_xyza);
    } else {
        sd.g_dim = make_int3(1, 1, 1);
        sd.g_lo = make_float3(0.f, 0.f, 0.f);
        sd.g_h = make_float3(1.f, 1.f, 1.f);
        sd.g_inv_h = make_float3(1.f, 1.f, 1.f);
        c->grow(sd.cell_start, 2 * sizeof(uint32_t));
        ck(cudaMemsetAsync(sd.cell_start.p, 0, 2 * sizeof(uint32_t), c->stream), "memset cells");
    }
    sd.ok = true;
    sd.version = ++c->versions;
}

// Bounding volume hierarchy over a scene's triangles, built on the host: each node takes the
// split of lowest surface-area cost (MacDonald & Booth 1990) among 16 centroid bins per axis,
// or stays a leaf when that costs more than testing its triangles; where median splits from
// then on would reach the traversal stack's depth, a node splits at the median centroid
// instead, so the depth stays within the stack.
// Boxes are padded outward so that FP32 slab tests cannot cut off a triangle's edge.  Device
// layout: see ur::SceneP (bvh, tri in leaf order, tri_nrm by triangle id).
struct MeshBuild {
    std::vector<float4> bvh, tri, nrm;
};

void build_mesh(const float *v, const int32_t *med, int n, int n_med, MeshBuild &B) {
    std::vector<double> cen(3 * (size_t)n);
    B.nrm.resize(n);
    for (int t = 0; t < n; ++t) {
        const float *p = v + 9 * (size_t)t;
        for (int q = 0; q < 9; ++q)
            if (!std::isfinite(p[q])) fail(UR_ERR_INVALID_ARG, "triangle vertices must be finite");
        if (med[2 * t] < 0 || med[2 * t] >= n_med || med[2 * t + 1] < 0 || med[2 * t + 1] >= n_med)
            fail(UR_ERR_INVALID_ARG, "triangle media out of range");
        const double e1[3] = {(double)p[3] - p[0], (double)p[4] - p[1], (double)p[5] - p[2]};
        const double e2[3] = {(double)p[6] - p[0], (double)p[7] - p[1], (double)p[8] - p[2]};
        const double nx = e1[1] * e2[2] - e1[2] * e2[1], ny = e1[2] * e2[0] - e1[0] * e2[2],
                     nz = e1[0] * e2[1] - e1[1] * e2[0];
        const double l = std::sqrt(nx * nx + ny * ny + nz * nz);
        if (!(l > 0.0)) fail(UR_ERR_INVALID_ARG, "degenerate triangle");
        int bits = med[2 * t] | (med[2 * t + 1] << 8);
        float wf;
        std::memcpy(&wf, &bits, 4);
        B.nrm[t] = make_float4((float)(nx / l), (float)(ny / l), (float)(nz / l), wf);
        for (int a = 0; a < 3; ++a) cen[3 * t + a] = ((double)p[a] + p[3 + a] + p[6 + a]) / 3.0;
    }
    std::vector<int> idx(n);
    for (int t = 0; t < n; ++t) idx[t] = t;
    struct Node { double lo[3], hi[3]; int a, b; };
    struct Task { int node, begin, end, depth; };
    std::vector<Node> nodes(1);
    std::vector<Task> todo{{0, 0, n, 1}};
    int depth = 0;
    while (!todo.empty()) {
        const Task k = todo.back();
        todo.pop_back();
        depth = std::max(depth, k.depth);
        Node &N = nodes[k.node];
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int a = 0; a < 3; ++a) {
            N.lo[a] = INFINITY;
            N.hi[a] = -INFINITY;
        }
        for (int q = k.begin; q < k.end; ++q) {
            const float *p = v + 9 * (size_t)idx[q];
            for (int a = 0; a < 3; ++a) {
                for (int c3 = 0; c3 < 3; ++c3) {
                    N.lo[a] = std::min(N.lo[a], (double)p[3 * c3 + a]);
                    N.hi[a] = std::max(N.hi[a], (double)p[3 * c3 + a]);
                }
                clo[a] = std::min(clo[a], cen[3 * idx[q] + a]);
                chi[a] = std::max(chi[a], cen[3 * idx[q] + a]);
            }
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
        const int cnt = k.end - k.begin;
        if (cnt <= 2 || !(chi[axis] > clo[axis])) {   // leaf
            N.a = k.begin;
            N.b = cnt;
            continue;
        }
        int mid = -1;
        int need = 0;   // levels a median split of this node would still add
        while ((1 << need) < cnt) ++need;
        if (k.depth + need + 2 < ur::kBvhStack) {   // binned surface-area heuristic
            constexpr int nb = 16;
            auto area = [](const double *lo, const double *hi) {
                const double x = hi[0] - lo[0], y = hi[1] - lo[1], z = hi[2] - lo[2];
                return x * y + y * z + z * x;
            };
            double best = INFINITY;
            int best_axis = -1, best_split = 0;
            for (int a = 0; a < 3; ++a) {
                if (!(chi[a] > clo[a])) continue;
                const double scale = nb / (chi[a] - clo[a]);
                int bc[nb] = {};
                double blo[nb][3], bhi[nb][3];
                for (int q = 0; q < nb; ++q)
                    for (int c3 = 0; c3 < 3; ++c3) {
                        blo[q][c3] = INFINITY;
                        bhi[q][c3] = -INFINITY;
                    }
                for (int q = k.begin; q < k.end; ++q) {
                    const int t = idx[q];
                    const int bin = std::min(nb - 1, (int)((cen[3 * t + a] - clo[a]) * scale));
                    ++bc[bin];
                    const float *p = v + 9 * (size_t)t;
                    for (int c3 = 0; c3 < 3; ++c3)
                        for (int vv = 0; vv < 3; ++vv) {
                            blo[bin][c3] = std::min(blo[bin][c3], (double)p[3 * vv + c3]);
                            bhi[bin][c3] = std::max(bhi[bin][c3], (double)p[3 * vv + c3]);
                        }
                }
                double rarea[nb];   // area and count of bins split+1 .. nb-1
                int rcnt[nb];
                double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
                int c = 0;
                for (int q = nb - 1; q > 0; --q) {
                    for (int c3 = 0; c3 < 3; ++c3) {
                        lo[c3] = std::min(lo[c3], blo[q][c3]);
                        hi[c3] = std::max(hi[c3], bhi[q][c3]);
                    }
                    c += bc[q];
                    rarea[q - 1] = c ? area(lo, hi) : 0.0;
                    rcnt[q - 1] = c;
                }
                for (int c3 = 0; c3 < 3; ++c3) {
                    lo[c3] = INFINITY;
                    hi[c3] = -INFINITY;
                }
                c = 0;
                for (int q = 0; q < nb - 1; ++q) {
                    for (int c3 = 0; c3 < 3; ++c3) {
                        lo[c3] = std::min(lo[c3], blo[q][c3]);
                        hi[c3] = std::max(hi[c3], bhi[q][c3]);
                    }
                    c += bc[q];
                    if (c == 0 || rcnt[q] == 0) continue;
                    const double cost = area(lo, hi) * c + rarea[q] * rcnt[q];
                    if (cost < best) {
                        best = cost;
                        best_axis = a;
                        best_split = q;
                    }
                }
            }
            // a node visit costs about one triangle test: stay a leaf if splitting does not pay
            const double leaf_cost = area(N.lo, N.hi) * cnt;
            if (best_axis < 0 || (cnt <= 4 && best + area(N.lo, N.hi) >= leaf_cost)) {
                N.a = k.begin;
                N.b = cnt;
                continue;
            }
            const double scale = nb / (chi[best_axis] - clo[best_axis]);
            const auto it = std::partition(idx.begin() + k.begin, idx.begin() + k.end, [&](int t) {
                return std::min(nb - 1, (int)((cen[3 * t + best_axis] - clo[best_axis]) * scale)) <= best_split;
            });
            mid = (int)(it - idx.begin());
        }
        if (mid <= k.begin || mid >= k.end) {   // median split
            mid = (k.begin + k.end) / 2;
            std::nth_element(idx.begin() + k.begin, idx.begin() + mid, idx.begin() + k.end,
                             [&](int x, int y) { return cen[3 * x + axis] < cen[3 * y + axis]; });
        }
        const int left = (int)nodes.size();
        nodes[k.node].a = left;   // N may move when nodes grows
        nodes[k.node].b = 0;
        nodes.resize(nodes.size() + 2);
        todo.push_back({left, k.begin, mid, k.depth + 1});
        todo.push_back({left + 1, mid, k.end, k.depth + 1});
    }
    if (depth >= ur::kBvhStack) fail(UR_ERR_INVALID_ARG, "triangle hierarchy deeper than the traversal stack");
    B.bvh.resize(2 * nodes.size());
    for (size_t q = 0; q < nodes.size(); ++q) {
        const Node &N = nodes[q];
        float f[2][3];
        for (int a = 0; a < 3; ++a) {
            const double pad = 1e-7 + 1e-6 * std::max(std::fabs(N.lo[a]), std::fabs(N.hi[a]));
            f[0][a] = std::nextafter((float)(N.lo[a] - pad), -INFINITY);
            f[1][a] = std::nextafter((float)(N.hi[a] + pad), INFINITY);
        }
        float wa, wb;
        std::memcpy(&wa, &N.a, 4);
        std::memcpy(&wb, &N.b, 4);
        B.bvh[2 * q] = make_float4(f[0][0], f[0][1], f[0][2], wa);
        B.bvh[2 * q + 1] = make_float4(f[1][0], f[1][1], f[1][2], wb);
    }
    B.tri.resize(3 * (size_t)n);
    for (int q = 0; q < n; ++q) {
        const int t = idx[q];
        const float *p = v + 9 * (size_t)t;
        float wt;
        std::memcpy(&wt, &t, 4);
        B.tri[3 * q] = make_float4(p[0], p[1], p[2], wt);
        B.tri[3 * q + 1] = make_float4((float)((double)p[3] - p[0]), (float)((double)p[4] - p[1]),
                                       (float)((double)p[5] - p[2]), 0.f);
        B.tri[3 * q + 2] = make_float4((float)((double)p[6] - p[0]), (float)((double)p[7] - p[1]),
                                       (float)((double)p[8] - p[2]), 0.f);
    }
}

void fill_scene(const ur_ctx *c, const SceneData &sd, ur::SceneP &S) {
    const ur_array &A = c->arr;
    S.n_med = (int)sd.media.size();
    S.n_bnd = (int)sd.bnd.size();
    S.med_array = sd.med_array;
    S.z_max = sd.z_max;
    const double np_per_db = std::log(10.0) / 20.0;
    for (int m = 0; m < S.n_med; ++m) {
        const ur_medium &M = sd.media[m];
        S.med[m].c = M.c;
        S.med[m].Z = M.Z;
        S.med[m].a = (float)((double)M.alpha_db_cm_mhz * ((double)A.f0 * 1e-6) * 100.0 * np_per_db);
        S.med[m].slow = split((double)A.fs / (double)M.c);
        S.cs[m] = sd.sampling[m].c;
        S.Zs[m] = sd.sampling[m].Z;
    }
    S.split_sampling = 0;
    for (int m = 0; m < S.n_med; ++m)
        if (S.cs[m] != S.med[m].c || S.Zs[m] != S.med[m].Z) S.split_sampling = 1;
    for (int b = 0; b < S.n_bnd; ++b) {
        S.bnd[b].kind = sd.bnd[b].kind;
        S.bnd[b].med_neg = sd.bnd[b].med_neg;
        S.bnd[b].med_pos = sd.bnd[b].med_pos;
        S.bnd[b].alpha = std::max(sd.media[sd.bnd[b].med_neg].roughness, sd.media[sd.bnd[b].med_pos].roughness);
        for (int q = 0; q < 4; ++q) S.bnd[b].p[q] = sd.bnd[b].p[q];
    }
    S.n_tri = sd.n_tri;
    S.tri_base = S.n_bnd + 3;
    S.bvh = (const float4 *)sd.bvh.p;
    S.tri = (const float4 *)sd.tri.p;
    S.tri_nrm = (const float4 *)sd.tri_nrm.p;
    for (int m = 0; m < S.n_med; ++m) S.rough[m] = sd.media[m].roughness;
    S.n_scat = sd.n_scat;
    S.r2 = sd.r_s * sd.r_s;
    S.g_rm = sd.g_rm;
    S.g_lo = sd.g_lo;
    S.g_h = sd.g_h;
    S.g_inv_h = sd.g_inv_h;
    S.g_dim = sd.g_dim;
    S.refs = (const float4 *)sd.refs.p;
    S.cell_start = (const uint32_t *)sd.cell_start.p;
    S.f_lo = sd.f_lo;
    S.f_inv_h = sd.f_inv_h;
    S.f_dim = sd.f_dim;
    S.f_refs = sd.n_scat > 0 && sd.f_built ? (const float4 *)sd.f_refs.p : nullptr;
    S.f_cell_start = (const uint32_t *)sd.f_cell_start.p;
    S.amp = (const float *)sd.amp.p;
    S.scat = (const float4 *)sd.scat.p;
}

// Items -> slot ranges (element-major, padded to the tracer's pool size) and hash offsets.
// mix_rays > 0: item 0 holds the slots of one sequence of mix_rays rays that draw their
// item (transmit mixing); the other items hold none and every item's hashes start at 0.
void set_items(ur_ctx *c, const std::vector<ur_batch_item> &in, uint64_t mix_rays = 0) {
    c->no_capture("setting work items");
    const int n_el = c->arr.n_el;
    std::vector<ur::ItemP> it(in.size());
    uint64_t slot = 0, hash = 0;
    for (size_t q = 0; q < in.size(); ++q) {
        const ur_batch_item &b = in[q];
        ur::ItemP &I = it[q];
        I.slot_begin = slot;
        I.hash_begin = hash;
        I.n_rays = (uint32_t)b.n_rays;
        I.rays_per_el = (uint32_t)((b.n_rays + (uint64_t)n_el - 1) / (uint64_t)n_el);
        I.scene = b.scene;
        I.angle = b.tx;
        I.stream = b.stream;
        const double th = c->angles[b.tx];
        I.sin_t = (float)std::sin(th);
        I.cos_t = (float)std::cos(th);
        I.kind = c->tx_kinds[b.tx];
        I.vx = c->tx_vx[b.tx];
        I.vz = c->tx_vz[b.tx];
        I.inv_n = (float)(1.0 / (double)b.n_rays);
        const uint64_t s = (uint64_t)I.rays_per_el * (uint64_t)n_el;
        slot += (s + ur::kTracePool - 1) / ur::kTracePool * ur::kTracePool;
        hash += b.n_rays;
    }
    if (mix_rays > 0) {
        const uint32_t per_el = (uint32_t)((mix_rays + (uint64_t)n_el - 1) / (uint64_t)n_el);
        slot = ((uint64_t)per_el * (uint64_t)n_el + ur::kTracePool - 1) / ur::kTracePool * ur::kTracePool;
        for (size_t q = 0; q < it.size(); ++q) {
            it[q].slot_begin = q == 0 ? 0 : slot;
            it[q].hash_begin = 0;
        }
        it[0].n_rays = (uint32_t)mix_rays;
        it[0].rays_per_el = per_el;
    }
    c->items = it;
    c->n_slots = slot;
    c->grow(c->items_dev, sizeof(ur::ItemP) * std::max<size_t>(it.size(), 1));
    ck(cudaMemcpyAsync(c->items_dev.p, c->items.data(), sizeof(ur::ItemP) * it.size(), cudaMemcpyHostToDevice, c->stream),
       "copy items");
    ck(cudaStreamSynchronize(c->stream), "items sync");
}

void validate_items(ur_ctx *c, const ur_batch_item *items, int n) {
    if (!items || n < 1 || n > 65536) fail(UR_ERR_INVALID_ARG, "n_items must be in [1, 65536]");
    for (int q = 0; q < n; ++q) {
        const ur_batch_item &b = items[q];
        if (b.scene < 0 || b.scene >= ur::kMaxScenes || !c->scenes[b.scene].ok)
            fail(UR_ERR_STATE, "batch item refers to a scene slot that holds no scene");
        if (b.tx < 0 || b.tx >= (int)c->angles.size()) fail(UR_ERR_INVALID_ARG, "batch item transmit out of range");
        if (b.n_rays == 0 || b.n_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "n_rays must be in [1, 2^32)");
    }
}

ur::TraceP make_trace_params(ur_ctx *c, uint64_t seed, int max_b, float max_path) {
    ur::TraceP P{};
    const ur_array &A = c->arr;
    int n_scenes = 0;
    for (const ur::ItemP &I : c->items) n_scenes = std::max(n_scenes, I.scene + 1);
    P.n_scenes = n_scenes;
    for (int s = 0; s < n_scenes; ++s)
        if (c->scenes[s].ok) fill_scene(c, c->scenes[s], P.S[s]);
    P.n_el = A.n_el;
    P.n_s = A.n_s;
    P.pitch = A.pitch;
    P.H = A.elev_h;
    P.x_first = (float)(-0.5 * (double)(A.n_el - 1) * (double)A.pitch);
    P.radius = A.radius;
    P.dphi = A.radius > 0.f ? (float)((double)A.pitch / (double)A.radius) : 0.f;
    P.phi0 = (float)(-0.5 * (double)(A.n_el - 1) * (double)P.dphi);
    const double s_samples = (double)A.n_cycles / (4.0 * (double)A.f0) * (double)A.fs;
    P.K = (float)((double)A.tcut_sigmas * s_samples);
    P.t_last = (float)((double)(A.n_s - 1) + (double)P.K);
    const double am = (double)A.alpha_m_deg * kPi / 180.0, ac = (double)A.alpha_c_deg * kPi / 180.0;
    P.am = (float)am;
    P.ac = (float)ac;
    P.t2am = (float)(std::tan(am) * std::tan(am));
    P.t2ac = (float)(std::tan(ac) * std::tan(ac));
    P.items = (const ur::ItemP *)c->items_dev.p;
    P.n_items = (int)c->items.size();
    P.n_slots = c->n_slots;
    P.delay = (const ur::ff *)c->delay.p;
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.max_b = max_b;
    P.max_path = max_path;
    P.resolve_batch = c->tune.resolve_batch > 0 ? c->tune.resolve_batch : kResolveBatch;
    c->grow(c->counters, 8 * sizeof(unsigned long long));
    unsigned long long *cnt = (unsigned long long *)c->counters.p;
    P.arr_count = cnt;
    P.stats = cnt + 1;
    P.next_slot = cnt + 7;
    return P;
}

void check_ready(ur_ctx *c) {
    if (!c->scenes[0].ok) fail(UR_ERR_STATE, "no scene uploaded");
    if (!c->array_ok) fail(UR_ERR_STATE, "array not set");
    if (c->angles.empty()) fail(UR_ERR_STATE, "no transmits set");
}

void check_trace_args(int max_b, float max_path) {
    if (max_b < 0 || max_b > 127) fail(UR_ERR_INVALID_ARG, "max_bounces must be in [0, 127]");
    if (!(max_path > 0.f) || !std::isfinite(max_path)) fail(UR_ERR_INVALID_ARG, "max_path_m must be positive");
}

int trace_grid(ur_ctx *c, bool dbg) {
    const int block = c->tune.block > 0 ? c->tune.block : 256;
    const int per_sm = c->tune.blocks_per_sm > 0 ? c->tune.blocks_per_sm : ur::trace_occupancy(block, dbg);
    return std::max(1, c->sms * per_sm);
}

// Arrival queue and sort buffers for `cap` arrivals and the current items.
void size_trace_buffers(ur_ctx *c, uint64_t cap, bool dbg) {
    const uint64_t n_rows = (uint64_t)c->items.size() * c->arr.n_el;
    if (cap > c->arr_cap) {
        c->grow(c->arrivals, sizeof(uint4) * cap);
        c->arr_cap = cap;
    }
    if (dbg) c->grow(c->arr_dbg, sizeof(uint2) * c->arr_cap);
    c->grow(c->sorted, sizeof(float4) * c->arr_cap);
    c->grow(c->row_count, sizeof(uint32_t) * n_rows);
    c->grow(c->row_fill, sizeof(uint32_t) * n_rows);
    c->grow(c->row_off, sizeof(uint32_t) * (n_rows + 1));
    c->grow(c->work, sizeof(uint4) * (n_rows + c->arr_cap / kChunkMin + 16));
    c->grow(c->n_work, sizeof(uint32_t));
}

void launch_trace_kernel(ur_ctx *c, ur::TraceP &P, bool dbg, uint2 *arr_dbg) {
    c->rec_key.valid = false;   // the arrival buffers are about to change
    P.arr = (uint4 *)c->arrivals.p;
    P.arr_dbg = (dbg || P.record) ? arr_dbg : nullptr;
    P.arr_cap = c->arr_cap;
    ck(cudaMemsetAsync(P.arr_count, 0, 8 * sizeof(unsigned long long), c->stream), "memset counters");
    c->phase_begin(UR_PHASE_TRACE);
    if (P.mix_list) ck(ur::launch_mix_plan(c->mix, c->sms, c->stream), "mixed ray order");
    bool point_waves = P.mix_tx > 0, emit = P.mix_tx > 0;   // other transmit kinds and mixing: extended tracer
    for (const ur::ItemP &it : c->items) {
        point_waves = point_waves || it.kind != UR_TX_PLANE;
        emit = emit || it.kind == UR_TX_SYNTHETIC;
    }
    bool split = false;
    for (int q = 0; q < P.n_scenes; ++q) split = split || P.S[q].split_sampling != 0;
    if (split && (point_waves || P.radius > 0.f))
        fail(UR_ERR_INVALID_ARG, "frozen sampling media need plane-wave transmits without mixing on a linear array");
    ur::launch_trace(P, dbg, c->tune.block > 0 ? c->tune.block : 256, trace_grid(c, dbg), c->stream, point_waves, emit);
    ck(cudaGetLastError(), "trace kernel launch");
    c->phase_end(UR_PHASE_TRACE, P.mix_list ? 4 : 1);
}

// Sort the arrival queue by row and deposit the pulses (asynchronous).
void launch_binning(ur_ctx *c, float *d_rf, float *d_q) {
    const uint64_t n_rows = (uint64_t)c->items.size() * c->arr.n_el;
    const size_t out_elems = (size_t)n_rows * c->arr.n_s;
    ck(cudaMemsetAsync(d_rf, 0, sizeof(float) * out_elems, c->stream), "memset rf");
    ck(cudaMemsetAsync(d_q, 0, sizeof(float) * out_elems, c->stream), "memset quad");
    ur::BinP B{};
    B.arr = (const uint4 *)c->arrivals.p;
    B.arr_count = (const unsigned long long *)c->counters.p;
    B.arr_cap = c->arr_cap;
    B.n_rows = (int)n_rows;
    B.n_s = c->arr.n_s;
    B.chunk = kChunk;
    B.chunk_min = kChunkMin;
    B.target_items = (uint32_t)(c->sms * 4 * 8);   // 8 waves of the deposit grid
    B.max_items = (uint32_t)(n_rows + c->arr_cap / kChunkMin + 16);
    B.priv_rows = ur::bin_sort_smem((int)n_rows) > 0;
    B.row_count = (uint32_t *)c->row_count.p;
    B.row_fill = (uint32_t *)c->row_fill.p;
    B.row_off = (uint32_t *)c->row_off.p;
    B.items = (uint4 *)c->work.p;
    B.n_items = (uint32_t *)c->n_work.p;
    B.sorted = (float4 *)c->sorted.p;
    B.rf = d_rf;
    B.quad = d_q;
    const double s_samples = (double)c->arr.n_cycles / (4.0 * (double)c->arr.f0) * (double)c->arr.fs;
    B.K = (float)((double)c->arr.tcut_sigmas * s_samples);
    B.inv_2s2_log2e = (float)(1.4426950408889634 / (2.0 * s_samples * s_samples));
    B.phase_per_sample = (float)(2.0 * (double)c->arr.f0 / (double)c->arr.fs);
    B.rot32_s = (float)std::sin(kPi * 32.0 * (double)B.phase_per_sample);
    B.rot32_c = (float)std::cos(kPi * 32.0 * (double)B.phase_per_sample);
    ck(cudaMemsetAsync(B.row_count, 0, sizeof(uint32_t) * n_rows, c->stream), "memset rows");
    ck(cudaMemsetAsync(B.row_fill, 0, sizeof(uint32_t) * n_rows, c->stream), "memset rows");
    c->phase_begin(UR_PHASE_SORT);
    ur::launch_bin_sort(B, c->sms, c->stream);
    ck(cudaGetLastError(), "sort kernels");
    c->phase_end(UR_PHASE_SORT, 3);
    c->phase_begin(UR_PHASE_DEPOSIT);
    ur::launch_bin_deposit(B, c->sms, c->stream);
    ck(cudaGetLastError(), "deposit kernel");
    c->phase_end(UR_PHASE_DEPOSIT, 1);
}

void read_stats(const unsigned long long *h, ur_stats *st) {
    if (!st) return;
    st->rays = h[1];
    st->segments = h[2];
    st->interactions = h[3];
    st->candidates = h[4];
    st->connections = h[5];
    st->arrivals = h[6];
}

ur_ctx::MaskKey trace_key(const ur_ctx *c, uint64_t seed, uint64_t n_rays, int max_b, float max_path) {
    ur_ctx::MaskKey k;
    k.valid = true;
    k.seed = seed;
    k.n_rays = n_rays;
    k.scene_version = c->scenes[0].version;
    k.n_slots = c->n_slots;
    k.max_b = max_b;
    k.max_path = max_path;
    k.angles = c->angles;
    return k;
}

void do_trace(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path, float *rf, float *quad,
              ur_stats *st, ur_debug *dbg) {
    c->set_device();
    c->no_capture("ur_trace");
    check_ready(c);
    if (n_rays == 0 || n_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "n_rays_per_tx must be in [1, 2^32)");
    check_trace_args(max_b, max_path);
    if (!rf || !quad) fail(UR_ERR_INVALID_ARG, "rf and quad are required");
    prepare_transmits(c);
    const int n_tx = (int)c->angles.size(), n_el = c->arr.n_el, n_s = c->arr.n_s;
    const uint64_t mix_rays = c->mix_tx ? n_rays * (uint64_t)n_tx : 0;
    if (mix_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "with transmit mixing n_tx * n_rays_per_tx must be below 2^32");
    const uint64_t n_rows = (uint64_t)n_tx * n_el;
    if (n_rows > (1ull << 26)) fail(UR_ERR_INVALID_ARG, "n_tx * n_el too large");
    const size_t out_elems = (size_t)n_rows * n_s;
    const bool dbg_on = dbg != nullptr;
    if (dbg_on && dbg->path_hash && !is_device_ptr(dbg->path_hash)) fail(UR_ERR_INVALID_ARG, "debug arrays must be device memory");
    std::vector<ur_batch_item> items(n_tx);
    for (int k = 0; k < n_tx; ++k) items[k] = ur_batch_item{0, k, (uint32_t)k, 0u, n_rays};
    set_items(c, items, mix_rays);
    c->batch_ok = false;
    ur::TraceP P = make_trace_params(c, seed, max_b, max_path);
    P.mix_tx = mix_rays > 0 ? n_tx : 0;
    if (mix_rays > 0) {   // counting sort of the mixed sequence by (drawn transmit, element)
        bool per_el = false;
        const int bins = ur::mix_bins(n_tx, n_el, &per_el);
        if (bins > 0) {
            c->grow(c->mix_list, sizeof(uint32_t) * mix_rays);
            c->grow(c->mix_bins, sizeof(uint32_t) * 3 * (size_t)bins);
            ur::MixP &M = c->mix;
            M.key = P.key;
            M.n_rays = (uint32_t)mix_rays;
            M.n_tx = (uint32_t)n_tx;
            M.n_el = (uint32_t)n_el;
            M.n_bins = (uint32_t)bins;
            M.per_element = per_el;
            M.count = (uint32_t *)c->mix_bins.p;
            M.offset = M.count + bins;
            M.fill = M.offset + bins;
            M.list = (uint32_t *)c->mix_list.p;
            P.mix_list = M.list;
        }
    }
    P.path_hash = dbg_on ? (unsigned long long *)dbg->path_hash : nullptr;
    // (ray, event) of each arrival, for ur_trace_adjoint (which refuses mixed traces)
    const bool record = c->want_rec && !dbg_on && mix_rays == 0;
    P.record = record ? 1 : 0;

    const double want = c->arr_per_ray * (double)n_rays * (double)n_tx * 1.25 + 4096.0;
    uint64_t cap = std::max<uint64_t>(c->arr_cap, (uint64_t)want);
    unsigned long long *h = c->host_scratch;
    for (int attempt = 0;; ++attempt) {
        size_trace_buffers(c, cap, dbg_on || record);
        launch_trace_kernel(c, P, dbg_on, (uint2 *)c->arr_dbg.p);
        ck(cudaMemcpyAsync(h, P.arr_count, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream), "read count");
        ck(cudaStreamSynchronize(c->stream), "trace kernel");
        c->phase_collect();
        const uint64_t n_arr = h[0];
        c->arr_per_ray = std::max(1e-3, (double)n_arr / ((double)n_rays * (double)n_tx));
        if (n_arr <= c->arr_cap) break;
        if (attempt == 2) fail(UR_ERR_OVERFLOW, "arrival queue kept overflowing");
        cap = (uint64_t)((double)n_arr * 1.1) + 4096;
    }
    const uint64_t n_arr = h[0];
    read_stats(h, st);
    if (record) c->rec_key = trace_key(c, seed, n_rays, max_b, max_path);

    const bool rf_dev = is_device_ptr(rf), q_dev = is_device_ptr(quad);
    float *d_rf = rf, *d_q = quad;
    if (!rf_dev) {
        c->grow(c->stage_rf, sizeof(float) * out_elems);
        d_rf = (float *)c->stage_rf.p;
    }
    if (!q_dev) {
        c->grow(c->stage_quad, sizeof(float) * out_elems);
        d_q = (float *)c->stage_quad.p;
    }
    launch_binning(c, d_rf, d_q);
    if (dbg_on) {
        dbg->count = n_arr;
        ur::DebugOut D{dbg->ray, dbg->event, dbg->row, dbg->t_hi, dbg->t_lo, dbg->amp, dbg->capacity};
        if (D.cap > 0) {
            if (!D.ray || !D.event || !D.row || !D.t_hi || !D.t_lo || !D.amp)
                fail(UR_ERR_INVALID_ARG, "debug arrays must all be set when capacity > 0");
            ur::launch_unpack_debug((const uint4 *)c->arrivals.p, (const uint2 *)c->arr_dbg.p,
                                    (const unsigned long long *)c->counters.p, c->arr_cap, D, c->stream);
            ck(cudaGetLastError(), "unpack kernel");
        }
    }
    if (!rf_dev) ck(cudaMemcpyAsync(rf, d_rf, sizeof(float) * out_elems, cudaMemcpyDeviceToHost, c->stream), "copy rf");
    if (!q_dev) ck(cudaMemcpyAsync(quad, d_q, sizeof(float) * out_elems, cudaMemcpyDeviceToHost, c->stream), "copy quad");
    if (!rf_dev || !q_dev || dbg_on) ck(cudaStreamSynchronize(c->stream), "trace outputs");
    c->prof_sync();
    if (dbg_on && n_arr > dbg->capacity) fail(UR_ERR_OVERFLOW, "debug capacity smaller than the arrival count");
}

// Delay-and-sum constants shared by every beamforming call.
ur::ImageP image_params(ur_ctx *c) {
    ur::ImageP I{};
    I.n_el = c->arr.n_el;
    I.n_s = c->arr.n_s;
    I.q = split((double)c->arr.fs / (double)c->arr.c_bf);
    I.x_first = split(-0.5 * (double)(c->arr.n_el - 1) * (double)c->arr.pitch);
    I.pitch = c->arr.pitch;
    I.tx_sin = (const ur::ff *)c->tx_sin.p;
    I.tx_cos = (const ur::ff *)c->tx_cos.p;
    I.tx_m = (const ur::ff *)c->tx_m.p;
    I.tx_kind = (const int *)c->tx_kind.p;
    I.elem_xz = c->arr.radius > 0.f ? (const ur::ff *)c->elem_xz.p : nullptr;
    return I;
}

}  // namespace

namespace ur {
bool ctx_view(const ur_ctx *c, CtxView *v) {
    if (!c || !c->array_ok || c->angles.empty()) return false;
    v->device = c->device;
    v->stream = (void *)c->stream;
    v->arr = c->arr;
    v->n_tx = (int)c->angles.size();
    v->angles = c->angles.data();
    v->plane_waves = true;
    for (int k : c->tx_kinds) v->plane_waves = v->plane_waves && k == UR_TX_PLANE;
    v->linear = c->arr.radius == 0.f;
    return true;
}
}  // namespace ur

extern "C" {

ur_status ur_create(ur_ctx **out, int device, void *cuda_stream) {
    if (!out) return UR_ERR_INVALID_ARG;
    *out = nullptr;
    ur_ctx *c = new (std::nothrow) ur_ctx();
    if (!c) return UR_ERR_OOM;
    ur_status st = guarded(c, [&] {
        int n = 0;
        ck(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
        if (device < 0 || device >= n) fail(UR_ERR_INVALID_ARG, "bad device index");
        c->device = device;
        c->set_device();
        ck(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device), "SM count");
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
        } else {
            ck(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            c->own_stream = true;
        }
        ck(cudaMallocHost(&c->host_scratch, 64 * sizeof(unsigned long long)), "cudaMallocHost");
    });
    if (st != UR_OK) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return st;
    }
    *out = c;
    return UR_OK;
}

ur_status ur_destroy(ur_ctx *c) {
    if (!c) return UR_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (c->capturing) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(c->stream, &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    cudaStreamSynchronize(c->stream);
    for (SceneData &sd : c->scenes) {
        DevBuf *bs[] = {&sd.scat, &sd.amp, &sd.refs, &sd.cell_count, &sd.cell_start, &sd.cell_fill, &sd.scan_tmp, &sd.bbox,
                        &sd.bvh, &sd.tri, &sd.tri_nrm, &sd.f_refs, &sd.f_cell_count, &sd.f_cell_start, &sd.f_cell_fill};
        for (DevBuf *b : bs) c->release(*b);
    }
    DevBuf *all[] = {&c->delay, &c->tx_sin, &c->tx_cos, &c->tx_m, &c->tx_kind, &c->elem_xz, &c->items_dev, &c->arrivals, &c->arr_dbg, &c->sorted,
                     &c->counters, &c->row_count, &c->row_fill, &c->row_off, &c->work, &c->n_work, &c->stage_rf,
                     &c->stage_quad, &c->pix, &c->stage_iq, &c->stage_env, &c->stage_db, &c->env_max, &c->img_lists,
                     &c->batch_pix, &c->batch_lists, &c->batch_env, &c->batch_max, &c->adj_grad, &c->adj_amp,
                     &c->adj_g, &c->mix_list, &c->mix_bins, &c->adj_order, &c->adj_keys};
    for (DevBuf *b : all) c->release(*b);
    for (int p = 0; p < UR_N_PHASES; ++p) {
        if (c->ev0[p]) cudaEventDestroy(c->ev0[p]);
        if (c->ev1[p]) cudaEventDestroy(c->ev1[p]);
    }
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->host_scratch) cudaFreeHost(c->host_scratch);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return UR_OK;
}

const char *ur_last_error(const ur_ctx *c) { return c ? c->err.c_str() : "null context"; }

ur_status ur_scene_upload(ur_ctx *c, const ur_medium *media, int n_med, const ur_boundary *bnd, int n_bnd,
                          int med_array, float z_max, const float *scat_xyza, int n_scat, float r_s) {
    return guarded(c, [&] { upload_scene(c, 0, media, n_med, bnd, n_bnd, med_array, z_max, scat_xyza, n_scat, r_s); });
}

ur_status ur_scene_upload_slot(ur_ctx *c, int slot, const ur_medium *media, int n_med, const ur_boundary *bnd,
                               int n_bnd, int med_array, float z_max, const float *scat_xyza, int n_scat, float r_s) {
    return guarded(c, [&] { upload_scene(c, slot, media, n_med, bnd, n_bnd, med_array, z_max, scat_xyza, n_scat, r_s); });
}

ur_status ur_scene_set_media(ur_ctx *c, int slot, const ur_medium *media, int n_med, const ur_medium *sampling) {
    return guarded(c, [&] {
        c->no_capture("ur_scene_set_media");
        if (slot < 0 || slot >= ur::kMaxScenes || !c->scenes[slot].ok) fail(UR_ERR_STATE, "scene slot holds no scene");
        SceneData &sd = c->scenes[slot];
        if (!media || n_med != (int)sd.media.size()) fail(UR_ERR_INVALID_ARG, "n_med must match the uploaded scene");
        std::vector<ur_medium> M(media, media + n_med), Ms = M;
        if (sampling) Ms.assign(sampling, sampling + n_med);
        bool rough = false;
        for (int q = 0; q < n_med; ++q) {
            for (const ur_medium *m : {&M[q], &Ms[q]})
                if (!(m->c > 0.f) || !(m->Z > 0.f) || !(m->alpha_db_cm_mhz >= 0.f) ||
                    !(m->roughness >= 0.f && m->roughness <= 4.f))
                    fail(UR_ERR_INVALID_ARG, "media need c > 0, Z > 0, alpha >= 0, roughness in [0, 4]");
            rough = rough || M[q].roughness != 0.f;
        }
        if (sampling && rough) fail(UR_ERR_INVALID_ARG, "frozen sampling media need smooth boundaries");
        sd.media = M;
        sd.sampling = Ms;
        sd.version = ++c->versions;
        c->set_device();
        regrid_if_default_changed(c, sd);
    });
}

ur_status ur_scene_set_triangles(ur_ctx *c, int slot, const float *tri, const int32_t *tri_med, int n_tri) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_scene_set_triangles");
        if (slot < 0 || slot >= ur::kMaxScenes || !c->scenes[slot].ok) fail(UR_ERR_STATE, "scene slot holds no scene");
        if (n_tri < 0 || n_tri > ur::kMaxTri) fail(UR_ERR_INVALID_ARG, "n_tri must be in [0, 2^22]");
        if (n_tri > 0 && (!tri || !tri_med)) fail(UR_ERR_INVALID_ARG, "triangles need vertices and media");
        SceneData &sd = c->scenes[slot];
        c->batch_ok = false;
        if (n_tri == 0) {
            sd.n_tri = 0;
            sd.version = ++c->versions;
            regrid_if_default_changed(c, sd);
            return;
        }
        std::vector<float> v(9 * (size_t)n_tri);
        std::vector<int32_t> m(2 * (size_t)n_tri);
        ck(cudaMemcpy(v.data(), tri, sizeof(float) * v.size(), cudaMemcpyDefault), "copy triangles");
        ck(cudaMemcpy(m.data(), tri_med, sizeof(int32_t) * m.size(), cudaMemcpyDefault), "copy triangle media");
        MeshBuild B;
        build_mesh(v.data(), m.data(), n_tri, (int)sd.media.size(), B);
        c->grow(sd.bvh, sizeof(float4) * B.bvh.size());
        c->grow(sd.tri, sizeof(float4) * B.tri.size());
        c->grow(sd.tri_nrm, sizeof(float4) * B.nrm.size());
        ck(cudaMemcpyAsync(sd.bvh.p, B.bvh.data(), sizeof(float4) * B.bvh.size(), cudaMemcpyHostToDevice, c->stream),
           "copy hierarchy");
        ck(cudaMemcpyAsync(sd.tri.p, B.tri.data(), sizeof(float4) * B.tri.size(), cudaMemcpyHostToDevice, c->stream),
           "copy triangles");
        ck(cudaMemcpyAsync(sd.tri_nrm.p, B.nrm.data(), sizeof(float4) * B.nrm.size(), cudaMemcpyHostToDevice,
                           c->stream), "copy normals");
        ck(cudaStreamSynchronize(c->stream), "triangles");
        sd.n_tri = n_tri;
        sd.version = ++c->versions;
        regrid_if_default_changed(c, sd);
    });
}

ur_status ur_scene_set_amplitudes(ur_ctx *c, int slot, const float *amp, int n_scat) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_scene_set_amplitudes");
        if (slot < 0 || slot >= ur::kMaxScenes || !c->scenes[slot].ok) fail(UR_ERR_STATE, "scene slot holds no scene");
        SceneData &sd = c->scenes[slot];
        if (n_scat != sd.n_scat || (n_scat > 0 && !amp)) fail(UR_ERR_INVALID_ARG, "n_scat must match the uploaded scene");
        if (n_scat == 0) return;
        ck(cudaMemcpy2DAsync((char *)sd.scat.p + 12, sizeof(float4), amp, sizeof(float), sizeof(float), (size_t)n_scat,
                             cudaMemcpyDefault, c->stream), "copy amplitudes");
        ck(cudaMemcpyAsync(sd.amp.p, amp, sizeof(float) * n_scat, cudaMemcpyDefault, c->stream), "copy amplitudes");
        ck(cudaStreamSynchronize(c->stream), "amplitudes");
    });
}

ur_status ur_set_array(ur_ctx *c, const ur_array *a) {
    return guarded(c, [&] {
        c->no_capture("ur_set_array");
        if (!a) fail(UR_ERR_INVALID_ARG, "array is NULL");
        const ur_array &A = *a;
        if (A.n_el < 1 || A.n_el > 4096) fail(UR_ERR_INVALID_ARG, "n_el must be in [1, 4096]");
        if (A.n_s < 16 || A.n_s > ur::kMaxNs) fail(UR_ERR_INVALID_ARG, "n_s must be in [16, 8192]");
        if (!(A.pitch > 0.f) || !(A.elev_h > 0.f) || !(A.f0 > 0.f) || !(A.fs > 0.f) || !(A.n_cycles > 0.f) ||
            !(A.c_bf > 0.f) || !(A.tcut_sigmas > 0.f) || !std::isfinite(A.pitch) || !std::isfinite(A.fs))
            fail(UR_ERR_INVALID_ARG, "array geometry, frequencies, cycles, c_bf and tcut must be positive");
        if (!(A.alpha_m_deg >= 0.f) || !(A.alpha_c_deg >= A.alpha_m_deg) || !(A.alpha_c_deg < 90.f))
            fail(UR_ERR_INVALID_ARG, "need 0 <= alpha_m <= alpha_c < 90 degrees");
        const double K = (double)A.tcut_sigmas * (double)A.n_cycles / (4.0 * (double)A.f0) * (double)A.fs;
        if (K > 2048.0) fail(UR_ERR_INVALID_ARG, "pulse longer than 2048 samples");
        if (!(A.radius >= 0.f) || !std::isfinite(A.radius) ||
            (A.radius > 0.f && !((double)A.n_el * A.pitch < 3.0 * (double)A.radius)))
            fail(UR_ERR_INVALID_ARG, "radius must be 0 (linear) or a convex radius with an opening below 170 degrees");
        c->arr = A;
        c->array_ok = true;
        c->tx_dirty = true;
        c->batch_ok = false;
    });
}

ur_status ur_set_plane_waves(ur_ctx *c, const float *angles_rad, int n_tx) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_set_plane_waves");
        if (!c->array_ok) fail(UR_ERR_STATE, "set the array before the transmits");
        if (!angles_rad || n_tx < 1 || n_tx > 65536) fail(UR_ERR_INVALID_ARG, "n_tx must be in [1, 65536]");
        std::vector<float> a(n_tx);
        ck(cudaMemcpy(a.data(), angles_rad, sizeof(float) * n_tx, cudaMemcpyDefault), "copy angles");
        for (float v : a)
            if (!(std::fabs(v) < (float)(kPi / 3.0))) fail(UR_ERR_INVALID_ARG, "|angle| must be below 60 degrees");
        c->angles = a;
        c->tx_kinds.assign(n_tx, UR_TX_PLANE);
        c->tx_vx.assign(n_tx, 0.f);
        c->tx_vz.assign(n_tx, 0.f);
        c->tx_dirty = true;
        c->batch_ok = false;
    });
}

ur_status ur_set_transmits(ur_ctx *c, const ur_transmit *tx, int n_tx) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_set_transmits");
        if (!c->array_ok) fail(UR_ERR_STATE, "set the array before the transmits");
        if (!tx || n_tx < 1 || n_tx > 65536) fail(UR_ERR_INVALID_ARG, "n_tx must be in [1, 65536]");
        std::vector<ur_transmit> t(n_tx);
        ck(cudaMemcpy(t.data(), tx, sizeof(ur_transmit) * n_tx, cudaMemcpyDefault), "copy transmits");
        std::vector<float> a(n_tx, 0.f), vx(n_tx, 0.f), vz(n_tx, 0.f);
        std::vector<int> kinds(n_tx);
        for (int k = 0; k < n_tx; ++k) {
            const ur_transmit &q = t[k];
            if (q.kind == UR_TX_PLANE) {
                if (!(std::fabs(q.angle) < (float)(kPi / 3.0))) fail(UR_ERR_INVALID_ARG, "|angle| must be below 60 degrees");
                a[k] = q.angle;
            } else if (q.kind == UR_TX_DIVERGING || q.kind == UR_TX_FOCUSED) {
                if (!std::isfinite(q.x) || !std::isfinite(q.z)) fail(UR_ERR_INVALID_ARG, "transmit points must be finite");
                if (q.kind == UR_TX_DIVERGING && !(q.z < 0.f))
                    fail(UR_ERR_INVALID_ARG, "a diverging wave's virtual source lies behind the array (z < 0)");
                if (q.kind == UR_TX_FOCUSED && !(q.z > 0.f))
                    fail(UR_ERR_INVALID_ARG, "a focused wave's focus lies in front of the array (z > 0)");
                vx[k] = q.x;
                vz[k] = q.z;
            } else if (q.kind == UR_TX_SYNTHETIC) {
                if (!(q.x >= 0.f && q.x < (float)c->arr.n_el && q.x == std::floor(q.x)))
                    fail(UR_ERR_INVALID_ARG, "a synthetic-aperture transmit names an element index in [0, n_el)");
                vx[k] = q.x;
            } else {
                fail(UR_ERR_INVALID_ARG, "unknown transmit kind");
            }
            kinds[k] = q.kind;
        }
        c->angles = a;
        c->tx_kinds = kinds;
        c->tx_vx = vx;
        c->tx_vz = vz;
        c->tx_dirty = true;
        c->batch_ok = false;
    });
}

ur_status ur_set_transmit_mixing(ur_ctx *c, int enabled) {
    return guarded(c, [&] {
        if (enabled != 0 && enabled != 1) fail(UR_ERR_INVALID_ARG, "enabled must be 0 or 1");
        c->mix_tx = enabled == 1;
    });
}

ur_status ur_trace(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path, float *rf, float *quad,
                   ur_stats *st) {
    return guarded(c, [&] { do_trace(c, n_rays, seed, max_b, max_path, rf, quad, st, nullptr); });
}

ur_status ur_trace_debug(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path, float *rf,
                         float *quad, ur_stats *st, ur_debug *dbg) {
    return guarded(c, [&] {
        if (!dbg) fail(UR_ERR_INVALID_ARG, "debug struct is NULL");
        do_trace(c, n_rays, seed, max_b, max_path, rf, quad, st, dbg);
    });
}

ur_status ur_beamform(ur_ctx *c, const float *rf, const float *quad, const float *x_px, int nx, const float *z_px,
                      int nz, float dyn_range_db, float *iq, float *env, float *db) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_beamform");
        if (!c->array_ok) fail(UR_ERR_STATE, "array not set");
        if (c->angles.empty()) fail(UR_ERR_STATE, "no transmits set");
        if (!rf || !quad || !x_px || !z_px) fail(UR_ERR_INVALID_ARG, "rf, quad and pixel coordinates are required");
        if (nx < 1 || nz < 1 || nx > 16384 || nz > 16384) fail(UR_ERR_INVALID_ARG, "nx, nz must be in [1, 16384]");
        if (!iq && !env && !db) fail(UR_ERR_INVALID_ARG, "no output requested");
        if (db && !(dyn_range_db > 0.f)) fail(UR_ERR_INVALID_ARG, "dyn_range_db must be positive");
        prepare_transmits(c);
        const int n_tx = (int)c->angles.size(), n_el = c->arr.n_el, n_s = c->arr.n_s;
        const size_t n_in = (size_t)n_tx * n_el * n_s, n_px = (size_t)nx * nz;
        const float *d_rf = rf, *d_q = quad;
        if (!is_device_ptr(rf)) {
            c->grow(c->stage_rf, sizeof(float) * n_in);
            ck(cudaMemcpyAsync(c->stage_rf.p, rf, sizeof(float) * n_in, cudaMemcpyHostToDevice, c->stream), "copy rf in");
            d_rf = (const float *)c->stage_rf.p;
        }
        if (!is_device_ptr(quad)) {
            c->grow(c->stage_quad, sizeof(float) * n_in);
            ck(cudaMemcpyAsync(c->stage_quad.p, quad, sizeof(float) * n_in, cudaMemcpyHostToDevice, c->stream), "copy quad in");
            d_q = (const float *)c->stage_quad.p;
        }
        c->grow(c->pix, sizeof(float) * (nx + nz));
        ck(cudaMemcpyAsync(c->pix.p, x_px, sizeof(float) * nx, cudaMemcpyDefault, c->stream), "copy x");
        ck(cudaMemcpyAsync((float *)c->pix.p + nx, z_px, sizeof(float) * nz, cudaMemcpyDefault, c->stream), "copy z");
        const bool iq_dev = iq && is_device_ptr(iq), env_dev = env && is_device_ptr(env), db_dev = db && is_device_ptr(db);
        float2 *d_iq = nullptr;
        if (iq) {
            if (iq_dev) {
                d_iq = (float2 *)iq;
            } else {
                c->grow(c->stage_iq, sizeof(float2) * n_px);
                d_iq = (float2 *)c->stage_iq.p;
            }
        }
        float *d_env;
        if (env_dev) {
            d_env = env;
        } else {
            c->grow(c->stage_env, sizeof(float) * n_px);
            d_env = (float *)c->stage_env.p;
        }
        float *d_db = nullptr;
        if (db) {
            if (db_dev) {
                d_db = db;
            } else {
                c->grow(c->stage_db, sizeof(float) * n_px);
                d_db = (float *)c->stage_db.p;
            }
        }
        c->grow(c->env_max, sizeof(unsigned int));
        ck(cudaMemsetAsync(c->env_max.p, 0, sizeof(unsigned int), c->stream), "memset max");
        ur::ImageP I = image_params(c);
        I.rf = d_rf;
        I.quad = d_q;
        I.n_tx = n_tx;
        I.x_px = (const float *)c->pix.p;
        I.z_px = (const float *)c->pix.p + nx;
        I.nx = nx;
        I.nz = nz;
        I.iq = d_iq;
        I.env = d_env;
        I.db = d_db;
        I.env_max = (unsigned int *)c->env_max.p;
        I.dyn_range_db = dyn_range_db;
        I.n_images = 1;
        c->phase_begin(UR_PHASE_DAS);
        ur::launch_das(I, c->stream);
        ck(cudaGetLastError(), "das kernel");
        c->phase_end(UR_PHASE_DAS, 1);
        if (db) {
            c->phase_begin(UR_PHASE_LOG);
            ur::launch_log(I, c->stream);
            ck(cudaGetLastError(), "log kernel");
            c->phase_end(UR_PHASE_LOG, 1);
        }
        bool sync = false;
        if (iq && !iq_dev) {
            ck(cudaMemcpyAsync(iq, d_iq, sizeof(float2) * n_px, cudaMemcpyDeviceToHost, c->stream), "copy iq");
            sync = true;
        }
        if (env && !env_dev) {
            ck(cudaMemcpyAsync(env, d_env, sizeof(float) * n_px, cudaMemcpyDeviceToHost, c->stream), "copy env");
            sync = true;
        }
        if (db && !db_dev) {
            ck(cudaMemcpyAsync(db, d_db, sizeof(float) * n_px, cudaMemcpyDeviceToHost, c->stream), "copy db");
            sync = true;
        }
        if (sync || !is_device_ptr(rf) || !is_device_ptr(quad)) ck(cudaStreamSynchronize(c->stream), "beamform outputs");
        c->prof_sync();
    });
}

// ------------------------------------------------------------------ adjoint

// A forward trace that keeps (ray, event) of every arrival (queue grown until it fits).
void record_arrivals(ur_ctx *c, ur::TraceP P, uint64_t n_rays, int n_tx) {
    P.record = 1;
    P.path_hash = nullptr;
    const double want = c->arr_per_ray * (double)n_rays * (double)n_tx * 1.25 + 4096.0;
    uint64_t cap = std::max<uint64_t>(c->arr_cap, (uint64_t)want);
    unsigned long long *h = c->host_scratch;
    for (int attempt = 0;; ++attempt) {
        size_trace_buffers(c, cap, true);
        launch_trace_kernel(c, P, false, (uint2 *)c->arr_dbg.p);
        ck(cudaMemcpyAsync(h, P.arr_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream), "read count");
        ck(cudaStreamSynchronize(c->stream), "recording trace");
        c->phase_collect();
        const uint64_t n_arr = h[0];
        c->arr_per_ray = std::max(1e-3, (double)n_arr / ((double)n_rays * (double)n_tx));
        if (n_arr <= c->arr_cap) break;
        if (attempt == 2) fail(UR_ERR_OVERFLOW, "arrival queue kept overflowing");
        cap = (uint64_t)((double)n_arr * 1.1) + 4096;
    }
}

ur_status ur_trace_adjoint(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path, const float *g_rf,
                           const float *g_quad, float *grad_media, float *grad_amp) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_trace_adjoint");
        check_ready(c);
        if (n_rays == 0 || n_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "n_rays_per_tx must be in [1, 2^32)");
        check_trace_args(max_b, max_path);
        if (!g_rf || !g_quad || !grad_media) fail(UR_ERR_INVALID_ARG, "g_rf, g_quad and grad_media are required");
        const SceneData &sd = c->scenes[0];
        const int n_med = (int)sd.media.size();
        if (n_med > ur::kAdjMed) fail(UR_ERR_INVALID_ARG, "the adjoint supports scenes with at most 4 media");
        for (const ur_medium &m : sd.media)
            if (m.roughness != 0.f) fail(UR_ERR_INVALID_ARG, "the adjoint supports smooth boundaries only");
        for (int k : c->tx_kinds)
            if (k != UR_TX_PLANE) fail(UR_ERR_INVALID_ARG, "the adjoint supports plane-wave transmits only");
        if (c->mix_tx) fail(UR_ERR_INVALID_ARG, "the adjoint does not support transmit mixing");
        if (sd.n_tri > 0) fail(UR_ERR_INVALID_ARG, "the adjoint supports analytic boundaries only");
        if (c->arr.radius != 0.f) fail(UR_ERR_INVALID_ARG, "the adjoint supports linear arrays only");
        prepare_transmits(c);
        const int n_tx = (int)c->angles.size();
        std::vector<ur_batch_item> items(n_tx);
        for (int k = 0; k < n_tx; ++k) items[k] = ur_batch_item{0, k, (uint32_t)k, 0u, n_rays};
        set_items(c, items);
        c->batch_ok = false;
        const size_t n_out = (size_t)n_tx * c->arr.n_el * c->arr.n_s;
        const float *d_g[2] = {g_rf, g_quad};
        if (!is_device_ptr(g_rf) || !is_device_ptr(g_quad)) {
            c->grow(c->adj_g, 2 * sizeof(float) * n_out);
            for (int q = 0; q < 2; ++q) {
                float *dst = (float *)c->adj_g.p + q * n_out;
                ck(cudaMemcpyAsync(dst, q ? g_quad : g_rf, sizeof(float) * n_out, cudaMemcpyDefault, c->stream), "copy g");
                d_g[q] = dst;
            }
        }
        ur::AdjP A{};
        A.T = make_trace_params(c, seed, max_b, max_path);
        A.g_rf = d_g[0];
        A.g_q = d_g[1];
        c->grow(c->adj_grad, sizeof(double) * 3 * ur::kAdjMed);
        ck(cudaMemsetAsync(c->adj_grad.p, 0, sizeof(double) * 3 * ur::kAdjMed, c->stream), "memset grad");
        A.grad = (double *)c->adj_grad.p;
        if (grad_amp && sd.n_scat > 0) {
            c->grow(c->adj_amp, sizeof(float) * sd.n_scat);
            ck(cudaMemsetAsync(c->adj_amp.p, 0, sizeof(float) * sd.n_scat, c->stream), "memset grad_amp");
            A.grad_amp = (float *)c->adj_amp.p;
        }
        const ur_array &Ar = c->arr;
        const double s_n = (double)Ar.n_cycles / (4.0 * (double)Ar.f0) * (double)Ar.fs;
        A.K = (float)((double)Ar.tcut_sigmas * s_n);
        A.inv_2s2 = (float)(1.0 / (2.0 * s_n * s_n));
        A.inv_s2 = (float)(1.0 / (s_n * s_n));
        A.half_cycles = (float)(2.0 * (double)Ar.f0 / (double)Ar.fs);
        A.om = (float)(2.0 * kPi * (double)Ar.f0 / (double)Ar.fs);
        A.fs = Ar.fs;
        A.k_alpha = (float)((double)Ar.f0 * 1e-6 * 100.0 * std::log(10.0) / 20.0);
        // only paths that deposit have a gradient: the arrivals of the matching forward trace name them
        if (!(c->rec_key == trace_key(c, seed, n_rays, max_b, max_path))) {
            record_arrivals(c, A.T, n_rays, n_tx);
            c->rec_key = trace_key(c, seed, n_rays, max_b, max_path);
        }
        c->want_rec = true;   // later ur_trace calls record as they go
        A.arr = (const uint4 *)c->arrivals.p;
        A.rec = (const uint2 *)c->arr_dbg.p;
        A.n_arr = (const unsigned long long *)c->counters.p;
        A.arr_cap = c->arr_cap;
        c->grow(c->adj_order, sizeof(uint32_t) * std::max<uint64_t>(c->arr_cap, 1));
        c->grow(c->adj_keys, sizeof(uint32_t) * 3 * ur::kAdjKeys);
        A.order = (uint32_t *)c->adj_order.p;
        A.key_count = (uint32_t *)c->adj_keys.p;
        c->phase_begin(UR_PHASE_ADJOINT);
        ur::launch_adjoint(A, c->sms, c->stream);
        ck(cudaGetLastError(), "adjoint kernel");
        c->phase_end(UR_PHASE_ADJOINT, 4);
        double g[3 * ur::kAdjMed];
        ck(cudaMemcpyAsync(c->host_scratch, c->adj_grad.p, sizeof g, cudaMemcpyDeviceToHost, c->stream), "read grad");
        ck(cudaStreamSynchronize(c->stream), "adjoint");
        c->phase_collect();
        std::memcpy(g, c->host_scratch, sizeof g);
        float gf[3 * ur::kAdjMed];
        for (int q = 0; q < 3 * n_med; ++q) gf[q] = (float)g[q];
        ck(cudaMemcpy(grad_media, gf, sizeof(float) * 3 * n_med, cudaMemcpyDefault), "write grad_media");
        if (grad_amp && sd.n_scat > 0)
            ck(cudaMemcpy(grad_amp, c->adj_amp.p, sizeof(float) * sd.n_scat, cudaMemcpyDefault), "write grad_amp");
    });
}

// ------------------------------------------------------------------ batches

ur_status ur_batch_plan(ur_ctx *c, const ur_batch_item *items, int n_items, uint64_t arrival_capacity,
                        const float *x_px, int nx, const float *z_px, int nz) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_batch_plan");
        c->batch_ok = false;
        if (!c->array_ok) fail(UR_ERR_STATE, "array not set");
        if (c->angles.empty()) fail(UR_ERR_STATE, "no transmits set");
        validate_items(c, items, n_items);
        if ((uint64_t)n_items * c->arr.n_el > (1ull << 26)) fail(UR_ERR_INVALID_ARG, "n_items * n_el too large");
        if (!x_px || !z_px || nx < 1 || nz < 1 || nx > 16384 || nz > 16384)
            fail(UR_ERR_INVALID_ARG, "pixel coordinates with 1 <= nx, nz <= 16384 are required");
        prepare_transmits(c);
        c->batch_items.assign(items, items + n_items);
        set_items(c, c->batch_items);
        double rays = 0.0;
        for (int q = 0; q < n_items; ++q) rays += (double)items[q].n_rays;
        const uint64_t cap = arrival_capacity ? arrival_capacity : (uint64_t)(c->arr_per_ray * rays * 1.5 + 4096.0);
        size_trace_buffers(c, cap, false);
        c->batch_cap = c->arr_cap;
        // images: one per scene present, in slot order, compounding that scene's items
        std::vector<int> lists, begin, angle(n_items), scenes;
        for (int s = 0; s < ur::kMaxScenes; ++s) {
            std::vector<int> mine;
            for (int q = 0; q < n_items; ++q)
                if (items[q].scene == s) mine.push_back(q);
            if (mine.empty()) continue;
            scenes.push_back(s);
            begin.push_back((int)lists.size());
            lists.insert(lists.end(), mine.begin(), mine.end());
        }
        begin.push_back((int)lists.size());
        for (int q = 0; q < n_items; ++q) angle[q] = items[q].tx;
        std::vector<int> packed;
        packed.insert(packed.end(), lists.begin(), lists.end());
        packed.insert(packed.end(), begin.begin(), begin.end());
        packed.insert(packed.end(), angle.begin(), angle.end());
        c->grow(c->batch_lists, sizeof(int) * packed.size());
        ck(cudaMemcpyAsync(c->batch_lists.p, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice, c->stream),
           "copy image lists");
        c->batch_images = (int)scenes.size();
        c->batch_image_scene = scenes;
        c->batch_nx = nx;
        c->batch_nz = nz;
        c->grow(c->batch_pix, sizeof(float) * (nx + nz));
        ck(cudaMemcpyAsync(c->batch_pix.p, x_px, sizeof(float) * nx, cudaMemcpyDefault, c->stream), "copy x");
        ck(cudaMemcpyAsync((float *)c->batch_pix.p + nx, z_px, sizeof(float) * nz, cudaMemcpyDefault, c->stream), "copy z");
        c->grow(c->batch_env, sizeof(float) * (size_t)c->batch_images * nx * nz);
        c->grow(c->batch_max, sizeof(unsigned int) * c->batch_images);
        c->grow(c->counters, 8 * sizeof(unsigned long long));
        ck(cudaStreamSynchronize(c->stream), "batch plan");
        c->batch_ok = true;
    });
}

ur_status ur_batch_trace(ur_ctx *c, uint64_t seed, int max_b, float max_path, float *rf, float *quad) {
    return guarded(c, [&] {
        c->set_device();
        if (!c->batch_ok) fail(UR_ERR_STATE, "no batch planned (ur_batch_plan)");
        check_trace_args(max_b, max_path);
        if (!rf || !quad || !is_device_ptr(rf) || !is_device_ptr(quad))
            fail(UR_ERR_INVALID_ARG, "batch rf and quad must be device memory");
        if (c->items.size() != c->batch_items.size() || c->arr_cap < c->batch_cap)
            fail(UR_ERR_STATE, "the batch plan was replaced by another trace: plan again");
        ur::TraceP P = make_trace_params(c, seed, max_b, max_path);
        launch_trace_kernel(c, P, false, nullptr);
        launch_binning(c, rf, quad);
        c->prof_sync();
    });
}

ur_status ur_batch_status(ur_ctx *c, uint64_t *n_arrivals, ur_stats *st) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_batch_status");
        if (!c->counters.p) fail(UR_ERR_STATE, "no trace has run");
        unsigned long long *h = c->host_scratch;
        ck(cudaMemcpyAsync(h, c->counters.p, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream),
           "read counters");
        ck(cudaStreamSynchronize(c->stream), "batch status");
        if (n_arrivals) *n_arrivals = h[0];
        read_stats(h, st);
        if (h[0] > c->arr_cap) fail(UR_ERR_OVERFLOW, "arrival capacity exceeded: plan with a larger capacity");
    });
}

ur_status ur_batch_beamform(ur_ctx *c, const float *rf, const float *quad, float dyn_range_db, float *iq, float *env,
                            float *db) {
    return guarded(c, [&] {
        c->set_device();
        if (!c->batch_ok) fail(UR_ERR_STATE, "no batch planned (ur_batch_plan)");
        if (!rf || !quad || !is_device_ptr(rf) || !is_device_ptr(quad))
            fail(UR_ERR_INVALID_ARG, "batch rf and quad must be device memory");
        if (!iq && !env && !db) fail(UR_ERR_INVALID_ARG, "no output requested");
        if ((iq && !is_device_ptr(iq)) || (env && !is_device_ptr(env)) || (db && !is_device_ptr(db)))
            fail(UR_ERR_INVALID_ARG, "batch outputs must be device memory");
        if (db && !(dyn_range_db > 0.f)) fail(UR_ERR_INVALID_ARG, "dyn_range_db must be positive");
        const int n_items = (int)c->batch_items.size();
        const int *lists = (const int *)c->batch_lists.p;
        ck(cudaMemsetAsync(c->batch_max.p, 0, sizeof(unsigned int) * c->batch_images, c->stream), "memset max");
        ur::ImageP I = image_params(c);
        I.rf = rf;
        I.quad = quad;
        I.n_tx = n_items;
        I.img_items = lists;
        I.img_begin = lists + n_items;
        I.item_angle = lists + n_items + c->batch_images + 1;
        I.n_images = c->batch_images;
        I.x_px = (const float *)c->batch_pix.p;
        I.z_px = (const float *)c->batch_pix.p + c->batch_nx;
        I.nx = c->batch_nx;
        I.nz = c->batch_nz;
        I.iq = (float2 *)iq;
        I.env = env ? env : (float *)c->batch_env.p;
        I.db = db;
        I.env_max = (unsigned int *)c->batch_max.p;
        I.dyn_range_db = dyn_range_db;
        c->phase_begin(UR_PHASE_DAS);
        ur::launch_das(I, c->stream);
        ck(cudaGetLastError(), "das kernel");
        c->phase_end(UR_PHASE_DAS, 1);
        if (db) {
            c->phase_begin(UR_PHASE_LOG);
            ur::launch_log(I, c->stream);
            ck(cudaGetLastError(), "log kernel");
            c->phase_end(UR_PHASE_LOG, 1);
        }
        c->prof_sync();
    });
}

ur_status ur_graph_begin(ur_ctx *c) {
    return guarded(c, [&] {
        c->set_device();
        if (c->capturing) fail(UR_ERR_STATE, "already capturing");
        ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        c->capturing = true;
    });
}

ur_status ur_graph_end(ur_ctx *c) {
    return guarded(c, [&] {
        c->set_device();
        if (!c->capturing) fail(UR_ERR_STATE, "not capturing");
        c->capturing = false;
        cudaGraph_t g = nullptr;
        ck(cudaStreamEndCapture(c->stream, &g), "cudaStreamEndCapture");
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->graph = g;
        c->graph_exec = nullptr;
        ck(cudaGraphInstantiate(&c->graph_exec, g, 0), "cudaGraphInstantiate");
    });
}

ur_status ur_graph_launch(ur_ctx *c) {
    return guarded(c, [&] {
        c->set_device();
        if (!c->graph_exec) fail(UR_ERR_STATE, "no graph captured");
        c->no_capture("ur_graph_launch");
        c->rec_key.valid = false;   // the captured traces overwrite the arrival buffers
        ck(cudaGraphLaunch(c->graph_exec, c->stream), "cudaGraphLaunch");
    });
}

// ------------------------------------------------------------------ autotuner

ur_status ur_autotune(ur_ctx *c, int scene, uint64_t n_rays, uint64_t seed, int max_b, float max_path,
                      ur_tuning *best_out) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_autotune");
        if (scene < 0 || scene >= ur::kMaxScenes || !c->scenes[scene].ok) fail(UR_ERR_STATE, "scene slot holds no scene");
        if (!c->array_ok || c->angles.empty()) fail(UR_ERR_STATE, "array and transmits must be set");
        if (n_rays == 0 || n_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "n_rays must be in [1, 2^32)");
        check_trace_args(max_b, max_path);
        prepare_transmits(c);
        c->batch_ok = false;
        SceneData &sd = c->scenes[scene];
        const bool prof_was = c->prof;
        c->prof = false;
        cudaEvent_t e0, e1;
        ck(cudaEventCreate(&e0), "cudaEventCreate");
        ck(cudaEventCreate(&e1), "cudaEventCreate");
        std::vector<ur_batch_item> items(1, ur_batch_item{scene, 0, 0u, 0u, n_rays});
        set_items(c, items);
        const ur_tuning base = c->tune;
        // device time of one trace of n_rays rays with tuning t (grid rebuilt when its cells change)
        auto measure = [&](const ur_tuning &t) {
            const bool regrid = sd.n_scat > 0 && (t.cell_xy != c->tune.cell_xy || t.cell_y != c->tune.cell_y ||
                                                  t.cell_z != c->tune.cell_z);
            c->tune = t;
            if (regrid) build_grid(c, sd, nullptr);
            ur::TraceP P = make_trace_params(c, seed, max_b, max_path);
            size_trace_buffers(c, (uint64_t)(c->arr_per_ray * (double)n_rays * 1.5) + 4096, false);
            float best = INFINITY;
            for (int rep = 0; rep < 3; ++rep) {
                launch_trace_kernel(c, P, false, nullptr);
                ck(cudaEventRecord(e0, c->stream), "event");
                launch_trace_kernel(c, P, false, nullptr);
                ck(cudaEventRecord(e1, c->stream), "event");
                ck(cudaEventSynchronize(e1), "event sync");
                float ms = 0.f;
                ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
                best = std::min(best, ms);
            }
            ck(cudaMemcpy(c->host_scratch, c->counters.p, sizeof(unsigned long long), cudaMemcpyDeviceToHost), "count");
            c->arr_per_ray = std::max(1e-3, (double)c->host_scratch[0] / (double)n_rays);
            return best;
        };
        ur_tuning cur = base;
        const float r = sd.r_s;
        if (cur.cell_xy <= 0.f) cur.cell_xy = default_cell(sd, 0);
        if (cur.cell_y <= 0.f) cur.cell_y = default_cell(sd, 1);
        if (cur.cell_z <= 0.f) cur.cell_z = default_cell(sd, 2);
        if (cur.resolve_batch <= 0) cur.resolve_batch = kResolveBatch;
        if (cur.blocks_per_sm <= 0) cur.blocks_per_sm = ur::trace_occupancy(256, false);
        float t_cur = measure(cur);
        // coordinate descent over the knobs
        const float z_mult[] = {2.f, 3.f, 5.f, 8.f, 12.f};
        const float xy_mult[] = {1.f, 1.5f, 2.f, 3.f, 4.f, 6.f};
        const float y_mult[] = {0.2f, 0.3f, 0.5f, 1.f, 2.f, 3.f};
        const int batches[] = {8, 12, 16, 20, 24};
        for (int pass = 0; pass < 2; ++pass) {
            for (float m : z_mult) {
                ur_tuning t = cur;
                t.cell_z = m * r;
                const float v = measure(t);
                if (v < t_cur) { t_cur = v; cur = t; }
            }
            for (float m : xy_mult) {
                ur_tuning t = cur;
                t.cell_xy = m * r;
                const float v = measure(t);
                if (v < t_cur) { t_cur = v; cur = t; }
            }
            for (float m : y_mult) {
                ur_tuning t = cur;
                t.cell_y = m * r;
                const float v = measure(t);
                if (v < t_cur) { t_cur = v; cur = t; }
            }
            for (int b : batches) {
                ur_tuning t = cur;
                t.resolve_batch = b;
                const float v = measure(t);
                if (v < t_cur) { t_cur = v; cur = t; }
            }
            for (int bps = 2; bps <= 4; ++bps) {
                ur_tuning t = cur;
                t.blocks_per_sm = bps;
                const float v = measure(t);
                if (v < t_cur) { t_cur = v; cur = t; }
            }
        }
        c->tune = cur;
        if (sd.n_scat > 0) build_grid(c, sd, nullptr);
        for (int s = 0; s < ur::kMaxScenes; ++s)
            if (s != scene && c->scenes[s].ok && c->scenes[s].n_scat > 0) build_grid(c, c->scenes[s], nullptr);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->prof = prof_was;
        if (best_out) *best_out = cur;
    });
}

ur_status ur_set_tuning(ur_ctx *c, const ur_tuning *t) {
    return guarded(c, [&] {
        if (!t) fail(UR_ERR_INVALID_ARG, "tuning is NULL");
        if (t->cell_xy < 0.f || t->cell_y < 0.f || t->cell_z < 0.f || t->block < 0 || t->block > 256 || (t->block % 32) != 0 ||
            t->blocks_per_sm < 0 || t->blocks_per_sm > 64 || t->resolve_batch < 0 || t->resolve_batch > 32)
            fail(UR_ERR_INVALID_ARG, "tuning values out of range (block must be a multiple of 32, <= 256)");
        c->tune = *t;
    });
}

ur_status ur_set_profiling(ur_ctx *c, int on) {
    return guarded(c, [&] {
        c->set_device();
        if (c->prof) c->prof_sync();
        c->prof = on != 0;
        if (c->prof) {
            c->acc = ur_profile{};
            for (bool &p : c->pending) p = false;
        }
    });
}

ur_status ur_get_profile(ur_ctx *c, ur_profile *out) {
    return guarded(c, [&] {
        if (!out) fail(UR_ERR_INVALID_ARG, "out is NULL");
        *out = c->acc;
    });
}

ur_status ur_sync(ur_ctx *c) {
    return guarded(c, [&] {
        c->set_device();
        c->no_capture("ur_sync");
        ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        ck(cudaGetLastError(), "asynchronous error");
    });
}

}  // extern "C"
