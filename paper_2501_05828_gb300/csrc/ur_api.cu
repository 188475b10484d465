// C ABI of the acoustic ray tracer (declared in include/ultraray.h): argument
// validation, device buffers owned by the context, derived constants (media
// slowness, transmit delays, directivity cosines) and the launch sequence
// trace -> bin -> deposit and delay-and-sum -> log compression.
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

struct Status {
    ur_status code;
    std::string msg;
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

}  // namespace

struct ur_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    unsigned long long *host_scratch = nullptr;  // pinned, 64 words

    // scene (host copies; derived per trace because attenuation and slowness depend on the array)
    bool scene_ok = false;
    std::vector<ur_medium> media;
    std::vector<ur_boundary> bnd;
    int med_array = 0;
    float z_max = 0.f;
    int n_scat = 0;
    float r_s = 0.f;
    float3 g_lo{}, g_h{}, g_inv_h{};
    int3 g_dim{};
    DevBuf scat, amp, refs, cell_count, cell_start, cell_fill, scan_tmp, bbox;

    // array and transmits
    bool array_ok = false;
    ur_array arr{};
    std::vector<float> angles;
    bool tx_dirty = true;
    DevBuf txdir, delay, tx_sin, tx_cos, tx_m;

    // trace buffers
    DevBuf arrivals, arr_dbg, sorted, counters, row_count, row_fill, row_off, items, n_items;
    uint64_t arr_cap = 0;
    double arr_per_ray = 0.5;

    // staging for host-side inputs/outputs
    DevBuf stage_rf, stage_quad, pix, stage_iq, stage_env, stage_db, env_max;

    ur_tuning tune{};

    // per-phase CUDA-event profiling
    bool prof = false;
    cudaEvent_t ev0[UR_N_PHASES] = {}, ev1[UR_N_PHASES] = {};
    ur_profile acc{};
    bool pending[UR_N_PHASES] = {};

    void phase_begin(int p) {
        if (!prof) return;
        if (!ev0[p]) {
            ck(cudaEventCreate(&ev0[p]), "cudaEventCreate");
            ck(cudaEventCreate(&ev1[p]), "cudaEventCreate");
        }
        ck(cudaEventRecord(ev0[p], stream), "cudaEventRecord");
    }
    void phase_end(int p, int kernels) {
        if (!prof) return;
        ck(cudaEventRecord(ev1[p], stream), "cudaEventRecord");
        pending[p] = true;
        acc.launches[p] += (uint64_t)kernels;
        acc.calls[p] += 1;
    }
    // after a stream synchronisation: fold finished phases into the accumulators
    void phase_collect() {
        if (!prof) return;
        for (int p = 0; p < UR_N_PHASES; ++p)
            if (pending[p]) {
                float ms = 0.f;
                ck(cudaEventElapsedTime(&ms, ev0[p], ev1[p]), "cudaEventElapsedTime");
                acc.ms[p] += ms;
                pending[p] = false;
            }
    }
    void prof_sync() {
        if (!prof) return;
        ck(cudaStreamSynchronize(stream), "cudaStreamSynchronize");
        phase_collect();
    }

    void grow(DevBuf &b, size_t bytes) {
        if (bytes <= b.bytes && b.p) return;
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

// Transmit tables: direction (sin, cos), per-element delays, DAS constants.
void prepare_transmits(ur_ctx *c) {
    if (!c->tx_dirty) return;
    const int nt = (int)c->angles.size(), ne = c->arr.n_el;
    std::vector<float2> dir(nt);
    std::vector<ur::ff> delay((size_t)nt * ne), s(nt), co(nt), m(nt);
    const double pitch = c->arr.pitch, x0 = -0.5 * (double)(ne - 1) * pitch;
    for (int k = 0; k < nt; ++k) {
        const double th = c->angles[k];
        const double sn = std::sin(th), cs = std::cos(th);
        dir[k] = make_float2((float)sn, (float)cs);
        double mn = INFINITY;
        for (int e = 0; e < ne; ++e) mn = std::min(mn, (x0 + e * pitch) * sn);
        for (int e = 0; e < ne; ++e)
            delay[(size_t)k * ne + e] = split(((x0 + e * pitch) * sn - mn) / (double)c->arr.c_bf * (double)c->arr.fs);
        s[k] = split(sn);
        co[k] = split(cs);
        m[k] = split(mn);
    }
    c->grow(c->txdir, sizeof(float2) * nt);
    c->grow(c->delay, sizeof(ur::ff) * delay.size());
    c->grow(c->tx_sin, sizeof(ur::ff) * nt);
    c->grow(c->tx_cos, sizeof(ur::ff) * nt);
    c->grow(c->tx_m, sizeof(ur::ff) * nt);
    ck(cudaMemcpyAsync(c->txdir.p, dir.data(), sizeof(float2) * nt, cudaMemcpyHostToDevice, c->stream), "copy txdir");
    ck(cudaMemcpyAsync(c->delay.p, delay.data(), sizeof(ur::ff) * delay.size(), cudaMemcpyHostToDevice, c->stream), "copy delay");
    ck(cudaMemcpyAsync(c->tx_sin.p, s.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy sin");
    ck(cudaMemcpyAsync(c->tx_cos.p, co.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy cos");
    ck(cudaMemcpyAsync(c->tx_m.p, m.data(), sizeof(ur::ff) * nt, cudaMemcpyHostToDevice, c->stream), "copy m");
    ck(cudaStreamSynchronize(c->stream), "sync transmit tables");  // host vectors go out of scope
    c->tx_dirty = false;
}

void build_grid(ur_ctx *c, const float *scat_xyza) {
    const int n = c->n_scat;
    c->grow(c->scat, sizeof(float4) * n);
    c->grow(c->amp, sizeof(float) * n);
    ck(cudaMemcpyAsync(c->scat.p, scat_xyza, sizeof(float4) * n, cudaMemcpyDefault, c->stream), "copy scatterers");
    c->grow(c->bbox, 6 * sizeof(unsigned int));
    const unsigned int init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
    ck(cudaMemcpyAsync(c->bbox.p, init, sizeof init, cudaMemcpyHostToDevice, c->stream), "init bbox");
    c->phase_begin(UR_PHASE_GRID);
    ur::launch_bbox((const float4 *)c->scat.p, n, (float *)c->bbox.p, c->stream);
    c->phase_end(UR_PHASE_GRID, 1);
    ck(cudaGetLastError(), "bbox kernel");
    unsigned int *hb = (unsigned int *)c->host_scratch;
    ck(cudaMemcpyAsync(hb, c->bbox.p, sizeof init, cudaMemcpyDeviceToHost, c->stream), "read bbox");
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
    const float r_m = c->r_s * 1.001f + 1e-7f;
    float h_xy = c->tune.cell_xy > 0.f ? c->tune.cell_xy : 3.f * c->r_s;
    float h_z = c->tune.cell_z > 0.f ? c->tune.cell_z : 40.f * c->r_s;
    int3 dim;
    for (int tries = 0;; ++tries) {
        dim.x = std::max(1, (int)std::ceil((hi[0] - lo[0] + 2.f * r_m) / h_xy));
        dim.y = std::max(1, (int)std::ceil((hi[1] - lo[1] + 2.f * r_m) / h_xy));
        dim.z = std::max(1, (int)std::ceil((hi[2] - lo[2] + 2.f * r_m) / h_z));
        if ((double)dim.x * dim.y * dim.z <= (double)(1u << 26)) break;
        h_xy *= 1.5f;
        h_z *= 1.5f;
    }
    c->g_lo = make_float3(lo[0] - r_m, lo[1] - r_m, lo[2] - r_m);
    c->g_h = make_float3(h_xy, h_xy, h_z);
    c->g_inv_h = make_float3(1.f / h_xy, 1.f / h_xy, 1.f / h_z);
    c->g_dim = dim;
    const uint32_t n_cells = (uint32_t)dim.x * dim.y * dim.z;
    c->grow(c->cell_count, sizeof(uint32_t) * (n_cells + 1));
    c->grow(c->cell_start, sizeof(uint32_t) * (n_cells + 1));
    c->grow(c->cell_fill, sizeof(uint32_t) * (n_cells + 1));
    c->grow(c->scan_tmp, sizeof(uint32_t) * (n_cells / 4096 + 4));
    ck(cudaMemsetAsync(c->cell_count.p, 0, sizeof(uint32_t) * (n_cells + 1), c->stream), "memset counts");
    ck(cudaMemsetAsync(c->cell_fill.p, 0, sizeof(uint32_t) * (n_cells + 1), c->stream), "memset fill");
    ur::GridBuildP G{};
    G.scat = (const float4 *)c->scat.p;
    G.n_scat = n;
    G.r_m = r_m;
    G.lo = c->g_lo;
    G.inv_h = c->g_inv_h;
    G.dim = dim;
    G.cell_count = (uint32_t *)c->cell_count.p;
    G.cell_start = (uint32_t *)c->cell_start.p;
    G.cell_fill = (uint32_t *)c->cell_fill.p;
    G.amp = (float *)c->amp.p;
    c->phase_begin(UR_PHASE_GRID);
    ur::launch_grid_count(G, c->stream);
    ck(cudaGetLastError(), "grid count kernel");
    ur::launch_scan_u32(G.cell_count, G.cell_start, (uint32_t *)c->scan_tmp.p, n_cells, c->stream);
    ck(cudaGetLastError(), "scan kernel");
    c->phase_end(UR_PHASE_GRID, 4);
    ck(cudaMemcpyAsync(hb, G.cell_start + n_cells, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream), "read refs");
    ck(cudaStreamSynchronize(c->stream), "grid sync");
    c->phase_collect();
    const uint32_t n_refs = hb[0];
    c->grow(c->refs, sizeof(float4) * std::max<uint32_t>(n_refs, 1));
    G.refs = (float4 *)c->refs.p;
    c->phase_begin(UR_PHASE_GRID);
    ur::launch_grid_fill(G, c->stream);
    ck(cudaGetLastError(), "grid fill kernel");
    c->phase_end(UR_PHASE_GRID, 1);
    c->prof_sync();
}

ur::TraceP make_trace_params(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path) {
    ur::TraceP P{};
    const ur_array &A = c->arr;
    ur::SceneP &S = P.S;
    S.n_med = (int)c->media.size();
    S.n_bnd = (int)c->bnd.size();
    S.med_array = c->med_array;
    S.z_max = c->z_max;
    const double np_per_db = std::log(10.0) / 20.0;
    for (int m = 0; m < S.n_med; ++m) {
        const ur_medium &M = c->media[m];
        S.med[m].c = M.c;
        S.med[m].Z = M.Z;
        S.med[m].a = (float)((double)M.alpha_db_cm_mhz * ((double)A.f0 * 1e-6) * 100.0 * np_per_db);
        S.med[m].slow = split((double)A.fs / (double)M.c);
    }
    for (int b = 0; b < S.n_bnd; ++b) {
        S.bnd[b].kind = c->bnd[b].kind;
        S.bnd[b].med_neg = c->bnd[b].med_neg;
        S.bnd[b].med_pos = c->bnd[b].med_pos;
        for (int q = 0; q < 4; ++q) S.bnd[b].p[q] = c->bnd[b].p[q];
    }
    S.n_scat = c->n_scat;
    S.r2 = c->r_s * c->r_s;
    S.g_lo = c->g_lo;
    S.g_h = c->g_h;
    S.g_inv_h = c->g_inv_h;
    S.g_dim = c->g_dim;
    S.refs = (const float4 *)c->refs.p;
    S.cell_start = (const uint32_t *)c->cell_start.p;
    S.amp = (const float *)c->amp.p;
    S.scat = (const float4 *)c->scat.p;
    P.n_el = A.n_el;
    P.n_s = A.n_s;
    P.pitch = A.pitch;
    P.H = A.elev_h;
    P.x_first = (float)(-0.5 * (double)(A.n_el - 1) * (double)A.pitch);
    const double s_samples = (double)A.n_cycles / (4.0 * (double)A.f0) * (double)A.fs;
    P.K = (float)((double)A.tcut_sigmas * s_samples);
    P.t_last = (float)((double)(A.n_s - 1) + (double)P.K);
    const double am = (double)A.alpha_m_deg * kPi / 180.0, ac = (double)A.alpha_c_deg * kPi / 180.0;
    P.am = (float)am;
    P.ac = (float)ac;
    P.cos_am = (float)std::cos(am);
    P.cos_ac = (float)std::cos(ac);
    P.n_tx = (int)c->angles.size();
    P.txdir = (const float2 *)c->txdir.p;
    P.delay = (const ur::ff *)c->delay.p;
    P.n_rays = (uint32_t)n_rays;
    P.rays_per_el = (uint32_t)((n_rays + (uint64_t)A.n_el - 1) / (uint64_t)A.n_el);
    P.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    P.max_b = max_b;
    P.max_path = max_path;
    P.inv_n = (float)(1.0 / (double)n_rays);
    P.resolve_batch = c->tune.resolve_batch > 0 ? c->tune.resolve_batch : 16;
    return P;
}

void check_ready(ur_ctx *c) {
    if (!c->scene_ok) fail(UR_ERR_STATE, "no scene uploaded");
    if (!c->array_ok) fail(UR_ERR_STATE, "array not set");
    if (c->angles.empty()) fail(UR_ERR_STATE, "no transmits set");
}

void do_trace(ur_ctx *c, uint64_t n_rays, uint64_t seed, int max_b, float max_path, float *rf, float *quad,
              ur_stats *st, ur_debug *dbg) {
    c->set_device();
    check_ready(c);
    if (n_rays == 0 || n_rays > 0xFFFFFFFFull) fail(UR_ERR_INVALID_ARG, "n_rays_per_tx must be in [1, 2^32)");
    if (max_b < 0 || max_b > 127) fail(UR_ERR_INVALID_ARG, "max_bounces must be in [0, 127]");
    if (!(max_path > 0.f) || !std::isfinite(max_path)) fail(UR_ERR_INVALID_ARG, "max_path_m must be positive");
    if (!rf || !quad) fail(UR_ERR_INVALID_ARG, "rf and quad are required");
    prepare_transmits(c);
    const int n_tx = (int)c->angles.size(), n_el = c->arr.n_el, n_s = c->arr.n_s;
    const uint64_t n_rows = (uint64_t)n_tx * n_el;
    if (n_rows > (1ull << 26)) fail(UR_ERR_INVALID_ARG, "n_tx * n_el too large");
    const size_t out_elems = (size_t)n_rows * n_s;
    const bool dbg_on = dbg != nullptr;
    if (dbg_on && dbg->path_hash && !is_device_ptr(dbg->path_hash)) fail(UR_ERR_INVALID_ARG, "debug arrays must be device memory");

    ur::TraceP P = make_trace_params(c, n_rays, seed, max_b, max_path);
    // counters: [0] arrival count, [1..6] stats
    c->grow(c->counters, 8 * sizeof(unsigned long long));
    unsigned long long *cnt = (unsigned long long *)c->counters.p;
    P.arr_count = cnt;
    P.stats = cnt + 1;
    P.next_slot = cnt + 7;
    P.path_hash = dbg_on ? (unsigned long long *)dbg->path_hash : nullptr;

    const int block = c->tune.block > 0 ? c->tune.block : 256;
    const int per_sm = c->tune.blocks_per_sm > 0 ? c->tune.blocks_per_sm : ur::trace_occupancy(block, dbg_on);
    const int grid = std::max(1, c->sms * per_sm);

    const double want = c->arr_per_ray * (double)n_rays * (double)n_tx * 1.25 + 4096.0;
    uint64_t cap = std::max<uint64_t>(c->arr_cap, (uint64_t)want);
    unsigned long long *h = c->host_scratch;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if (cap > c->arr_cap) {
            c->grow(c->arrivals, sizeof(uint4) * cap);
            if (dbg_on) c->grow(c->arr_dbg, sizeof(uint2) * cap);
            c->arr_cap = cap;
        }
        if (dbg_on && c->arr_dbg.bytes < sizeof(uint2) * c->arr_cap) c->grow(c->arr_dbg, sizeof(uint2) * c->arr_cap);
        P.arr = (uint4 *)c->arrivals.p;
        P.arr_dbg = dbg_on ? (uint2 *)c->arr_dbg.p : nullptr;
        P.arr_cap = c->arr_cap;
        ck(cudaMemsetAsync(cnt, 0, 8 * sizeof(unsigned long long), c->stream), "memset counters");
        c->phase_begin(UR_PHASE_TRACE);
        ur::launch_trace(P, dbg_on, block, grid, c->stream);
        ck(cudaGetLastError(), "trace kernel launch");
        c->phase_end(UR_PHASE_TRACE, 1);
        ck(cudaMemcpyAsync(h, cnt, 7 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream), "read count");
        ck(cudaStreamSynchronize(c->stream), "trace kernel");
        c->phase_collect();
        const uint64_t n_arr = h[0];
        c->arr_per_ray = std::max(1e-3, (double)n_arr / ((double)n_rays * (double)n_tx));
        if (n_arr <= c->arr_cap) break;
        cap = (uint64_t)((double)n_arr * 1.1) + 4096;
        if (attempt == 2) fail(UR_ERR_OVERFLOW, "arrival queue kept overflowing");
    }
    const uint64_t n_arr = h[0];
    if (st) {
        st->rays = h[1];
        st->segments = h[2];
        st->interactions = h[3];
        st->candidates = h[4];
        st->connections = h[5];
        st->arrivals = h[6];
    }

    // outputs: device in place, or staged for host buffers
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
    ck(cudaMemsetAsync(d_rf, 0, sizeof(float) * out_elems, c->stream), "memset rf");
    ck(cudaMemsetAsync(d_q, 0, sizeof(float) * out_elems, c->stream), "memset quad");

    ur::BinP B{};
    B.arr = (const uint4 *)c->arrivals.p;
    B.arr_count = cnt;
    B.arr_cap = c->arr_cap;
    B.n_rows = (int)n_rows;
    B.n_s = n_s;
    B.chunk = 4096;
    B.max_items = (uint32_t)(n_rows + n_arr / B.chunk + 16);
    c->grow(c->row_count, sizeof(uint32_t) * n_rows);
    c->grow(c->row_fill, sizeof(uint32_t) * n_rows);
    c->grow(c->row_off, sizeof(uint32_t) * (n_rows + 1));
    c->grow(c->items, sizeof(uint4) * B.max_items);
    c->grow(c->n_items, sizeof(uint32_t));
    c->grow(c->sorted, sizeof(float4) * std::max<uint64_t>(n_arr, 1));
    B.row_count = (uint32_t *)c->row_count.p;
    B.row_fill = (uint32_t *)c->row_fill.p;
    B.row_off = (uint32_t *)c->row_off.p;
    B.items = (uint4 *)c->items.p;
    B.n_items = (uint32_t *)c->n_items.p;
    B.sorted = (float4 *)c->sorted.p;
    B.rf = d_rf;
    B.quad = d_q;
    const double s_samples = (double)c->arr.n_cycles / (4.0 * (double)c->arr.f0) * (double)c->arr.fs;
    B.K = P.K;
    B.inv_2s2 = (float)(1.0 / (2.0 * s_samples * s_samples));
    B.phase_per_sample = (float)(2.0 * (double)c->arr.f0 / (double)c->arr.fs);
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

    if (dbg_on) {
        dbg->count = n_arr;
        ur::DebugOut D{dbg->ray, dbg->event, dbg->row, dbg->t_hi, dbg->t_lo, dbg->amp, dbg->capacity};
        if (D.cap > 0) {
            if (!D.ray || !D.event || !D.row || !D.t_hi || !D.t_lo || !D.amp)
                fail(UR_ERR_INVALID_ARG, "debug arrays must all be set when capacity > 0");
            ur::launch_unpack_debug((const uint4 *)c->arrivals.p, (const uint2 *)c->arr_dbg.p, cnt, c->arr_cap, D,
                                    c->stream);
            ck(cudaGetLastError(), "unpack kernel");
        }
    }
    if (!rf_dev) ck(cudaMemcpyAsync(rf, d_rf, sizeof(float) * out_elems, cudaMemcpyDeviceToHost, c->stream), "copy rf");
    if (!q_dev) ck(cudaMemcpyAsync(quad, d_q, sizeof(float) * out_elems, cudaMemcpyDeviceToHost, c->stream), "copy quad");
    if (!rf_dev || !q_dev || dbg_on) ck(cudaStreamSynchronize(c->stream), "trace outputs");
    c->prof_sync();
    if (dbg_on && n_arr > dbg->capacity) fail(UR_ERR_OVERFLOW, "debug capacity smaller than the arrival count");
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
    cudaStreamSynchronize(c->stream);
    DevBuf *all[] = {&c->scat, &c->amp, &c->refs, &c->cell_count, &c->cell_start, &c->cell_fill, &c->scan_tmp,
                     &c->bbox, &c->txdir, &c->delay, &c->tx_sin, &c->tx_cos, &c->tx_m, &c->arrivals, &c->arr_dbg,
                     &c->sorted, &c->counters, &c->row_count, &c->row_fill, &c->row_off, &c->items, &c->n_items,
                     &c->stage_rf, &c->stage_quad, &c->pix, &c->stage_iq, &c->stage_env, &c->stage_db, &c->env_max};
    for (DevBuf *b : all) c->release(*b);
    for (int p = 0; p < UR_N_PHASES; ++p) {
        if (c->ev0[p]) cudaEventDestroy(c->ev0[p]);
        if (c->ev1[p]) cudaEventDestroy(c->ev1[p]);
    }
    if (c->host_scratch) cudaFreeHost(c->host_scratch);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return UR_OK;
}

const char *ur_last_error(const ur_ctx *c) { return c ? c->err.c_str() : "null context"; }

ur_status ur_scene_upload(ur_ctx *c, const ur_medium *media, int n_med, const ur_boundary *bnd, int n_bnd,
                          int med_array, float z_max, const float *scat_xyza, int n_scat, float r_s) {
    return guarded(c, [&] {
        c->set_device();
        c->scene_ok = false;
        if (!media || n_med < 1 || n_med > ur::kMaxMed) fail(UR_ERR_INVALID_ARG, "n_med must be in [1, 16]");
        if (n_bnd < 0 || n_bnd > ur::kMaxBnd || (n_bnd > 0 && !bnd)) fail(UR_ERR_INVALID_ARG, "n_bnd must be in [0, 32]");
        if (med_array < 0 || med_array >= n_med) fail(UR_ERR_INVALID_ARG, "med_array out of range");
        if (!(z_max > 0.f) || !std::isfinite(z_max)) fail(UR_ERR_INVALID_ARG, "z_max must be positive");
        if (n_scat < 0 || n_scat >= (1 << 24)) fail(UR_ERR_INVALID_ARG, "n_scat must be in [0, 2^24)");
        if (n_scat > 0 && (!scat_xyza || !(r_s > 0.f) || !std::isfinite(r_s)))
            fail(UR_ERR_INVALID_ARG, "scatterers need a pointer and a positive capture radius");
        std::vector<ur_medium> M(media, media + n_med);
        for (const ur_medium &m : M) {
            if (!(m.c > 0.f) || !(m.Z > 0.f) || !(m.alpha_db_cm_mhz >= 0.f) || !std::isfinite(m.c) || !std::isfinite(m.Z))
                fail(UR_ERR_INVALID_ARG, "media need c > 0, Z > 0, alpha >= 0");
            if (m.roughness != 0.f) fail(UR_ERR_INVALID_ARG, "rough (GGX) boundaries are not supported: roughness must be 0");
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
        c->media = M;
        c->bnd = Bv;
        c->med_array = med_array;
        c->z_max = z_max;
        c->n_scat = n_scat;
        c->r_s = n_scat > 0 ? r_s : 1e-4f;
        if (n_scat > 0) {
            build_grid(c, scat_xyza);
        } else {
            c->g_dim = make_int3(1, 1, 1);
            c->g_lo = make_float3(0.f, 0.f, 0.f);
            c->g_h = make_float3(1.f, 1.f, 1.f);
            c->g_inv_h = make_float3(1.f, 1.f, 1.f);
            c->grow(c->cell_start, 2 * sizeof(uint32_t));
            ck(cudaMemsetAsync(c->cell_start.p, 0, 2 * sizeof(uint32_t), c->stream), "memset cells");
        }
        c->scene_ok = true;
    });
}

ur_status ur_set_array(ur_ctx *c, const ur_array *a) {
    return guarded(c, [&] {
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
        c->arr = A;
        c->array_ok = true;
        c->tx_dirty = true;
    });
}

ur_status ur_set_plane_waves(ur_ctx *c, const float *angles_rad, int n_tx) {
    return guarded(c, [&] {
        c->set_device();
        if (!c->array_ok) fail(UR_ERR_STATE, "set the array before the transmits");
        if (!angles_rad || n_tx < 1 || n_tx > 65536) fail(UR_ERR_INVALID_ARG, "n_tx must be in [1, 65536]");
        std::vector<float> a(n_tx);
        ck(cudaMemcpy(a.data(), angles_rad, sizeof(float) * n_tx, cudaMemcpyDefault), "copy angles");
        for (float v : a)
            if (!(std::fabs(v) < (float)(kPi / 3.0))) fail(UR_ERR_INVALID_ARG, "|angle| must be below 60 degrees");
        c->angles = a;
        c->tx_dirty = true;
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
        ur::ImageP I{};
        I.rf = d_rf;
        I.quad = d_q;
        I.n_tx = n_tx;
        I.n_el = n_el;
        I.n_s = n_s;
        I.x_px = (const float *)c->pix.p;
        I.z_px = (const float *)c->pix.p + nx;
        I.nx = nx;
        I.nz = nz;
        I.q = split((double)c->arr.fs / (double)c->arr.c_bf);
        I.x_first = split(-0.5 * (double)(n_el - 1) * (double)c->arr.pitch);
        I.pitch = c->arr.pitch;
        I.tx_sin = (const ur::ff *)c->tx_sin.p;
        I.tx_cos = (const ur::ff *)c->tx_cos.p;
        I.tx_m = (const ur::ff *)c->tx_m.p;
        I.iq = d_iq;
        I.env = d_env;
        I.db = d_db;
        I.env_max = (unsigned int *)c->env_max.p;
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

ur_status ur_set_tuning(ur_ctx *c, const ur_tuning *t) {
    return guarded(c, [&] {
        if (!t) fail(UR_ERR_INVALID_ARG, "tuning is NULL");
        if (t->cell_xy < 0.f || t->cell_z < 0.f || t->block < 0 || t->block > 256 || (t->block % 32) != 0 ||
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
        ck(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        ck(cudaGetLastError(), "asynchronous error");
    });
}

}  // extern "C"
