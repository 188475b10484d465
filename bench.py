#!/usr/bin/env python3
"""Throughput of the full simulation chain on the 128-element layered phantom.

One step = one RF frame: 1e7 primary rays of one 0-degree plane wave traced
through skin / fat / muscle / bone cylinder with 50k point scatterers
(emission, reflection/refraction, transducer sampling, aperture returns),
pulse deposit into [1 x 128 x 3200] analytic channel data, delay-and-sum to a
512 x 256 image, envelope and log compression.  Metric: rays/s (RF frames/s
alongside).  Inputs are resident in HBM before the timed region; L2 is
flushed (256 MiB write, untimed) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same frame.  Under torchrun every rank simulates its own frame
(independent seeds, no collective on the data path): weak scaling.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rays/s and RF frames/s at 128 elements"
UNIT = "rays/s"
WORKLOAD = ("layered phantom: 128 el, pitch 0.3 mm, f0 5 MHz, fs 40 MHz, 0-deg plane wave, skin/fat/muscle + "
            "bone cylinder r=6 mm, 50k scatterers, 1e7 rays/frame, 8 bounces, 3200 samples, DAS 512x256, 60 dB")

# Algorithmic floating-point operations per unit of work the tracer counts, taken
# from the FP64 oracle's own steps on the layered phantom (2 planes, 1 cylinder,
# 2 terminal planes): every add, subtract, multiply, divide and square root is 1,
# every exp / sin / cos / acos is 1, comparisons and integer work (Philox, element
# indices) are 0.  Independent of the GPU's search structure (no reference tests,
# no grid steps).
#   segment:      nearest boundary (2 planes x 2, cylinder 21, terminal 2) + advance
#                 (time 2, attenuation 3, path length 1, position 6, clip 1)      = 40
#   interaction:  medium side 5 + Eqs. 7-11 (cos_i 5, orientation 5, reflected
#                 direction 7 + normalise 9, eta 1, k 5, sqrt 1, transmitted 11 +
#                 normalise 9, r 7, R 1) + branch weight and uniform 6             = 72
#   scatterer event: tube test (v 3, t_ca 5, offset 6, |offset|^2 5) + element
#                 centre 2, direction 3, distance 6, angle 7, directivity 1      = 38
#   connection:   direction 12 + per boundary crossed 105 (nearest 25, time 2,
#                 attenuation 2, point 6, side 5, Eqs. 7-11 61, sqrt(1-R) 3,
#                 remaining 1) x 1.8 crossings (skin/fat and fat/muscle planes
#                 above a scatterer uniform in depth) + last leg 29 + arrival
#                 time 3 and amplitude 10                                         = 243
#   pulse tap (Eq. 14): tau 1, Gaussian 3, phase 1, sin 1, cos 1, amp g 1,
#                 rf 2, quad 2                                                    = 12
FLOPS_PER_SEGMENT = 40
FLOPS_PER_INTERACTION = 72
FLOPS_PER_CANDIDATE = 38
FLOPS_PER_CONNECTION = 243
FLOPS_PER_TAP = 12
FP32_LANES_PER_SM = 128

# DRAM traffic of the tracer kernel (dram__bytes_read.sum + dram__bytes_write.sum) and its warp
# instructions (smsp__inst_executed.sum), from one single-pass ncu capture of the benchmarked
# 1e7-ray launch, per primary ray; valid only while the tracer sources hash to `src_sha`.
TRACE_TRAFFIC = {"src_sha": "1b78d85b6f5ad132", "bytes_per_ray": 5.548, "warp_inst_per_ray": 428.6}


def tracer_sha():
    """Hash of the tracer kernel's sources and of the default grid cells (which set its traffic)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2501_05828_gb300", "csrc")
    for f in ("ur_trace.cu", "ur_device.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "ur_api.cu"), "rb") as fh:
        h.update(b"".join(l for l in fh if l.startswith(b"constexpr float kCell")))
    return h.hexdigest()[:16]


def taps_per_arrival(arr):
    s = arr["n_cycles"] / (4.0 * arr["f0"]) * arr["fs"]
    return 2 * int(arr["tcut_sigmas"] * s) + 1


def trace_flops(stats):
    return (stats["segments"] * FLOPS_PER_SEGMENT + stats["interactions"] * FLOPS_PER_INTERACTION
            + stats["candidates"] * FLOPS_PER_CANDIDATE + stats["connections"] * FLOPS_PER_CONNECTION)


def algorithmic_flops(stats, arr):
    return trace_flops(stats) + stats["arrivals"] * taps_per_arrival(arr) * FLOPS_PER_TAP


def issue_slots(rays, t_launch, n_sm, sm_mhz):
    """What bounds the tracer: warp instructions it issues (captured per ray with ncu, same source
    hash as the traffic) against 4 schedulers x 1 instruction per clock per SM.  Implementation
    work, not the method's arithmetic: reported beside the algorithmic ALU roofline."""
    got = TRACE_TRAFFIC["warp_inst_per_ray"] * rays / t_launch
    peak = n_sm * 4 * sm_mhz * 1e6
    return {"achieved_warp_inst_per_s": got, "peak_warp_inst_per_s": peak, "frac": got / peak,
            "peak_note": "%d SMs x 4 schedulers x 1 warp instruction per clock x %.0f MHz" % (n_sm, sm_mhz)}


# Shared-memory float atomics: ncu counts two data-stage wavefronts per 32-lane ATOMS
# (l1tex__data_pipe_lsu_wavefronts_mem_shared_op_atom / smsp__inst_executed_op_shared_atom = 2.00
# on k_bin_deposit), so the unit completes at most 16 lane atomics per SM per clock.
SHARED_ATOMIC_LANES_PER_CLOCK = 16


def binning_roofline(st, arr, phase_ms, alu_peak, peaks, n_sm, sm_mhz):
    """Binning of one frame: the deposit kernel against the FP32 ALU peak (FLOPS_PER_TAP per
    pulse tap), its shared-memory atomics against the atomic unit's 16 lanes per SM per clock,
    and the counting sort's algorithmic bytes (arrival read by count and scatter, sorted write)
    against HBM."""
    taps = st["arrivals"] * taps_per_arrival(arr)
    t_dep = phase_ms.get("deposit", float("nan")) * 1e-3
    t_sort = phase_ms.get("sort", float("nan")) * 1e-3
    ach = taps * FLOPS_PER_TAP / t_dep / 1e12
    atom_peak = n_sm * SHARED_ATOMIC_LANES_PER_CLOCK * sm_mhz * 1e6
    sort_bytes = st["arrivals"] * 48
    hbm = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "alu", "kernel": "k_bin_deposit", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": ach / alu_peak, "traffic": None, "algorithmic_flops_per_launch": taps * FLOPS_PER_TAP,
            "deposit_ms_per_launch": t_dep * 1e3,
            "shared_atomics": {"achieved_per_s": 2 * taps / t_dep, "peak_per_s": atom_peak,
                               "frac": 2 * taps / t_dep / atom_peak,
                               "peak_note": "%d SMs x %d lane atomics x %.0f MHz (two data-stage wavefronts per "
                                            "32-lane float atomic, ncu)" % (n_sm, SHARED_ATOMIC_LANES_PER_CLOCK, sm_mhz)},
            "sort": {"bound": "hbm", "kernels": "k_bin_count + k_bin_plan + k_bin_scatter",
                     "algorithmic_bytes": sort_bytes, "achieved": sort_bytes / t_sort / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": sort_bytes / t_sort / 1e9 / hbm, "ms": t_sort * 1e3,
                     "peak_note": "hbm_gbs of measured"}}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=None):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_index is not None:
            cmd += ["-i", str(gpu_index)]
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        pmax = max(r[2] for r in rows)
        loaded = [r for r in rows if r[2] >= 0.5 * pmax] or rows
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in loaded for n, v in zip(names, r[3][1:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": pmax, "samples": len(rows), "samples_under_load": len(loaded), "reasons": reasons}


# ------------------------------------------------------------------ ranks
class Ranks:
    """One process per GPU under torchrun: process group, barrier and max over
    ranks.  Every rank simulates its own replica (weak scaling); there is no
    data-path collective, only the timing reduction."""

    def __init__(self, rank, world, local_rank, backend="nccl"):
        import torch
        self.torch, self.rank, self.world = torch, rank, world
        self.cuda = backend == "nccl"
        self.device = torch.device("cuda", local_rank) if self.cuda else torch.device("cpu")
        self.dist = None
        if world > 1:
            import torch.distributed as dist
            if self.cuda:
                dist.init_process_group("nccl", device_id=self.device)
            else:
                dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()
        if self.cuda:
            self.torch.cuda.synchronize(self.device)

    def max(self, x):
        """Maximum of a float over ranks (the slowest rank's time)."""
        if not self.dist:
            return float(x)
        t = self.torch.tensor([float(x)], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units all ranks processed per second of the slowest rank."""
    return units_per_rank * world / seconds_max


# ------------------------------------------------------------------ CPU oracle
def oracle_rate(w, target_s, threads=None):
    """FP64 oracle on a bounded sample of the frame (rays 0..n-1 of every transmit): returns
    (rays/s, rays per transmit in the sample, seconds, threads)."""
    import numpy as np
    import oracle
    threads = threads or (os.cpu_count() or 1)
    t0 = time.perf_counter()
    tx = w.get("transmits")   # (kind, x, z) of other transmit kinds (the oracle's form)
    mix = bool(w.get("mix"))  # with transmit mixing the sample is rays 0 .. n * n_tx - 1 of the one sequence
    n_tx = len(np.atleast_1d(w["angles"]))
    per = n_tx if mix else 1
    n_probe = min(4096, w["n_rays"])
    oracle.simulate(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"], w["x_px"],
                    w["z_px"], w["dyn_range_db"], w["max_path"], 0, n_probe * per, threads=threads, transmits=tx,
                    mix=mix)
    probe = time.perf_counter() - t0
    n = int(min(w["n_rays"], max(1024, n_probe * target_s / max(probe, 1e-3))))
    t0 = time.perf_counter()
    oracle.simulate(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"], w["x_px"],
                    w["z_px"], w["dyn_range_db"], w["max_path"], 0, n * per, threads=threads, transmits=tx, mix=mix)
    dt = time.perf_counter() - t0
    return n * n_tx / dt, n, dt, threads


def run_reference(args, rank):
    if rank != 0:
        return
    import phantoms
    w = phantoms.layered()
    threads = os.cpu_count() or 1
    per_step = max(0.5, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    rate, n, _, _ = oracle_rate(w, per_step, threads)
    import oracle
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.simulate(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"], w["x_px"],
                        w["z_px"], w["dyn_range_db"], w["max_path"], 0, n, threads=threads)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    step = sum(times) / len(times)
    value = n / step
    sample = "first %d of the frame's 1e7 rays (ray indices 0..%d), full chain incl. deposit and 512x256 DAS" % (n, n - 1)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# ------------------------------------------------------------------ GPU
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2501_05828_gb300 as ur
    import phantoms

    torch.cuda.set_device(local_rank)
    R = Ranks(rank, world, local_rank)
    dev = R.device
    w = frame_workload(args)
    if args.rays:
        w["n_rays"] = args.rays
    seed = w["seed"] + rank
    N, A = w["n_rays"], w["array"]
    n_tx = len(w["angles"])
    sim = ur.Simulator(local_rank)
    sim.load(w)
    shape = (n_tx, A["n_el"], A["n_s"])
    rf = torch.empty(shape, dtype=torch.float32, device=dev)
    quad = torch.empty(shape, dtype=torch.float32, device=dev)
    nx, nz = w["x_px"].size, w["z_px"].size
    x_d = torch.from_numpy(w["x_px"]).to(dev)
    z_d = torch.from_numpy(w["z_px"]).to(dev)
    env = torch.empty((nz, nx), dtype=torch.float32, device=dev)
    db = torch.empty((nz, nx), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    last = {}

    def step():
        _, _, st = sim.trace(N, seed, w["max_bounces"], w["max_path"], rf=rf, quad=quad, stats=True)
        sim.beamform(rf, quad, x_d, z_d, w["dyn_range_db"], iq=None, env=env, db=db)
        last["stats"] = st

    barrier = R.barrier

    for _ in range(args.warmup):
        step()
    barrier()
    sim.set_profiling(True)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        step()
        ev[k][1].record()
    barrier()
    clk = clocks.stop() if clocks else None
    prof = sim.profile()
    sim.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    ms_max = R.max(ms)
    value = whole_job_rate(N * n_tx, world, ms_max * 1e-3)

    # ---- roofline of the dominant kernel (the tracer) ----
    st = last["stats"]
    trace_ms, trace_launches, trace_calls = prof["trace"]
    t_launch = trace_ms / max(trace_calls, 1) * 1e-3
    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = trace_flops(st) / t_launch / 1e12
    traffic = None
    if args.workload == "layered" and TRACE_TRAFFIC and TRACE_TRAFFIC.get("src_sha") == tracer_sha():
        traffic = TRACE_TRAFFIC["bytes_per_ray"] * N
    launches = sum(v[1] for v in prof.values())
    phase_ms = {k: v[0] / max(v[2], 1) for k, v in prof.items() if v[2]}

    # ---- end to end through the C ABI with host buffers ----
    sc_host = torch.from_numpy(w["scene"]["scatterers"]).pin_memory()
    x_h = torch.from_numpy(w["x_px"]).pin_memory()
    z_h = torch.from_numpy(w["z_px"]).pin_memory()
    db_h = torch.empty((nz, nx), dtype=torch.float32).pin_memory()
    s = w["scene"]
    h2d = sc_host.numel() * 4 + x_h.numel() * 4 + z_h.numel() * 4 + len(s["media"]) * 16 + len(s["boundaries"]) * 28 + 4
    d2h = db_h.numel() * 4

    tri_h = s.get("triangles")   # a new scene upload clears the triangles: set them again (BVH on the host)
    if tri_h is not None:
        h2d += tri_h[0].size * 4 + tri_h[1].size * 4

    def e2e_step():
        sim.upload_scene(s["media"], s["boundaries"], s["med_array"], s["z_max"], sc_host, s["r_s"])
        if tri_h is not None:
            sim.set_triangles(tri_h[0], tri_h[1])
        sim.trace(N, seed, w["max_bounces"], w["max_path"], rf=rf, quad=quad)
        sim.beamform(rf, quad, x_h, z_h, w["dyn_range_db"], iq=None, env=None, db=db_h)
        torch.cuda.synchronize()

    n_e2e = 0 if args.skip_e2e else max(3, min(args.steps, 20))
    e2e_s = float("nan")
    if n_e2e:
        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        barrier()
        e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = R.max(e2e_s)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": FRAME_WORKLOADS[args.workload], "rays_per_step": N * n_tx, "transmits": n_tx, "n_el": A["n_el"], "n_s": A["n_s"],
                       "image": "%dx%d" % (nx, nz), "l2": "flushed before every timed step (256 MiB write, untimed)",
                       "parallelism": "replicas: one frame per GPU"},
            "frames_per_s": whole_job_rate(n_tx, world, ms_max * 1e-3),
            "acquisitions_per_s": whole_job_rate(1, world, ms_max * 1e-3),
            "phase_ms": phase_ms,
            "roofline": {"bound": "alu",
                         "kernel": "k_trace" + (" (extended instantiation: rough boundaries, transmit kinds other "
                                                "than plane waves, transmit mixing, convex arrays, triangle meshes)" if args.workload != "layered" else ""),
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_note": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (sm_max_mhz)" % (
                             props.multi_processor_count, FP32_LANES_PER_SM, sm_mhz),
                         "trace_ms_per_launch": t_launch * 1e3,
                         "algorithmic_flops_per_launch": trace_flops(st),
                         "issue_slots": issue_slots(N * n_tx, t_launch, props.multi_processor_count, sm_mhz)
                         if traffic is not None else None},
            "roofline_binning": binning_roofline(st, A, phase_ms, peak, peaks, props.multi_processor_count, sm_mhz),
            "stats_per_frame": st,
            "gpu_launches": launches,
            "e2e": {"value": whole_job_rate(N * n_tx, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "path": "ur_scene_upload(pinned host scatterers, grid build) + ur_trace + ur_beamform(db -> pinned host)"},
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            rate, n, dt, thr = oracle_rate(w, args.cpu_seconds)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                    "sample": "rays 0..%d of each of the %d transmits (%.1f s), trace + deposit + "
                                              "512x256 DAS + log" % (n - 1, n_tx, dt)}
        print(json.dumps(line), flush=True)
    sim.close()
    R.close()


ROUGH_WORKLOAD = WORKLOAD + "; bone boundary rough (GGX roughness 0.5, the paper's bone value)"
PAPER_WORKLOAD = ("paper settings (Sec. 4) on a synthetic vertebra stand-in: 128 el, 5 MHz, fs 50 MHz, 5 cycles, "
                  "4 mm elevation, 2-deg directivity, 25 plane waves -30..30 deg x 512k rays (12.8M rays per "
                  "acquisition), 10 bounces, 20 cm paths; water around a rough bone sphere (r 10 mm, 45 mm) and two "
                  "rough bone cylinders (GGX 0.5), 20k scatterers in the bone; DAS of all 25 transmits to 512x256, "
                  "90 dB")
DIVERGING_WORKLOAD = ("layered phantom imaged with 9 diverging waves: virtual sources 10 mm behind the array at "
                      "x = -12..12 mm, 1.11M rays each (1e7 rays per acquisition), compounded DAS to 512x256, 60 dB")
CONVEX_WORKLOAD = PAPER_WORKLOAD.replace("128 el,", "128 el on a 70-deg convex arc (R 50 mm, the paper's probe),", 1)
SYNTHETIC_WORKLOAD = ("layered phantom imaged by synthetic aperture: 16 transmits, each firing one element (every "
                      "8th, 4..124) at t = 0, 625k rays each at uniform angles to the element normal (1e7 rays per "
                      "acquisition), compounded DAS to 512x256, 60 dB")
MIXED_WORKLOAD = PAPER_WORKLOAD.replace("25 plane waves -30..30 deg x 512k rays (12.8M rays per acquisition)",
                                        "25 plane waves -30..30 deg, 12.8M rays per acquisition, each drawing its "
                                        "plane wave (per-ray transmit mixing)", 1)
MESH_WORKLOAD = PAPER_WORKLOAD.replace("a rough bone sphere (r 10 mm, 45 mm) and two rough bone cylinders (GGX 0.5)",
                                       "rough bone (GGX 0.5) as triangle meshes: an icosphere body (r 10 mm, 45 mm, "
                                       "5120 triangles) and two closed 96-sided prisms along elevation (768 "
                                       "triangles), traced through a BVH", 1)
FRAME_WORKLOADS = {"layered": WORKLOAD, "rough": ROUGH_WORKLOAD, "paper": PAPER_WORKLOAD,
                   "diverging": DIVERGING_WORKLOAD, "convex": CONVEX_WORKLOAD, "synthetic": SYNTHETIC_WORKLOAD,
                   "mixed": MIXED_WORKLOAD, "mesh": MESH_WORKLOAD}


def frame_workload(args):
    """The phantom of a frame workload: layered (default), rough or paper."""
    import phantoms
    if args.workload == "mesh":
        return phantoms.paper_mesh_like()
    if args.workload in ("paper", "convex", "mixed"):
        w = phantoms.paper_like(convex=args.workload == "convex")
        w["mix"] = args.workload == "mixed"
        return w
    w = phantoms.layered()
    if args.workload == "synthetic":
        import numpy as np
        els = np.arange(4, w["array"]["n_el"], 8)
        w["angles"] = np.zeros(els.size, np.float32)
        w["transmits"] = [(3, float(e), 0.0) for e in els]   # (synthetic aperture, element, unused)
        w["n_rays"] = 10_000_000 // els.size
        return w
    if args.workload == "diverging":
        import numpy as np
        xs = np.linspace(-12e-3, 12e-3, 9)
        w["angles"] = np.zeros(xs.size, np.float32)
        w["transmits"] = [(1, float(x), -10e-3) for x in xs]   # (diverging, virtual source x, z)
        w["n_rays"] = 10_000_000 // xs.size
        return w
    if args.workload == "rough":
        s = dict(w["scene"])
        med = [list(m) for m in s["media"]]
        med[3][3] = 0.5                      # bone: the rough cylinder
        s["media"] = [tuple(m) for m in med]
        w["scene"] = s
    return w


BATCH_WORKLOAD = ("batched: 8 jittered layered phantoms (skin +-1 mm, fat +-2 mm, bone r U(3,10) mm, 10k-200k "
                  "scatterers) x 31 plane waves -15..15 deg, log-uniform 1e6-3e7 rays per transmit, one persistent "
                  "launch replayed as a CUDA graph, per-scene coherent compounding to 512x256, 60 dB")


def run_batched(args, rank, world, local_rank):
    """All 248 (scene, transmit) items traced, deposited and beamformed per step
    through one captured CUDA graph."""
    import torch

    import paper_2501_05828_gb300 as ur
    import phantoms

    torch.cuda.set_device(local_rank)
    R = Ranks(rank, world, local_rank)
    dev = R.device
    side = torch.cuda.Stream(dev)
    scenes = [phantoms.batched_variant(s) for s in range(1, 9)]
    scale = args.batch_scale
    with torch.cuda.stream(side):
        sim = ur.Simulator(local_rank)
        w0 = scenes[0]
        sim.set_array(w0["array"])
        sim.set_plane_waves(w0["angles"])
        for slot, w in enumerate(scenes):
            s = w["scene"]
            sim.upload_scene(s["media"], s["boundaries"], s["med_array"], s["z_max"], s["scatterers"], s["r_s"], slot)
        items = [(slot, k, max(1, int(w["n_rays"] * scale)), (slot << 16) | k)
                 for slot, w in enumerate(scenes) for k in range(len(w["angles"]))]
        total_rays = sum(it[2] for it in items)
        sim.batch_plan(items, w0["x_px"], w0["z_px"], capacity=int(0.35 * total_rays) + 4096)
        n_items = len(items)
        A = w0["array"]
        rf = torch.empty((n_items, A["n_el"], A["n_s"]), dtype=torch.float32, device=dev)
        quad = torch.empty_like(rf)
        db = torch.empty((len(scenes), w0["z_px"].size, w0["x_px"].size), dtype=torch.float32, device=dev)
        seed = rank
        for _ in range(args.warmup):
            sim.batch_trace(seed, 8, 0.2, rf=rf, quad=quad)
            sim.batch_beamform(rf, quad, 60.0, db=db)
        n_arr, st = sim.batch_status()
        # one profiled direct run for the tracer's own launch time
        sim.set_profiling(True)
        sim.batch_trace(seed, 8, 0.2, rf=rf, quad=quad)
        sim.batch_beamform(rf, quad, 60.0, db=db)
        prof = sim.profile()
        sim.set_profiling(False)
        side.synchronize()
        sim.graph_begin()
        sim.batch_trace(seed, 8, 0.2, rf=rf, quad=quad)
        sim.batch_beamform(rf, quad, 60.0, db=db)
        sim.graph_end()
        sim.graph_launch()
        side.synchronize()
        R.barrier()
        clocks = ClockSampler(local_rank) if rank == 0 else None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(side)
            sim.graph_launch()
            ev[k][1].record(side)
        side.synchronize()
        R.barrier()
        clk = clocks.stop() if clocks else None
        n_arr2, _ = sim.batch_status()

        # ---- end to end through the C ABI: scenes from pinned host memory, plan, trace, images to host
        sc_host = [torch.from_numpy(w["scene"]["scatterers"]).pin_memory() for w in scenes]
        x_h = torch.from_numpy(w0["x_px"]).pin_memory()
        z_h = torch.from_numpy(w0["z_px"]).pin_memory()
        db_h = torch.empty(tuple(db.shape), dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * 4 + len(w["scene"]["media"]) * 16 + len(w["scene"]["boundaries"]) * 28
                  for t, w in zip(sc_host, scenes)) + x_h.numel() * 4 + z_h.numel() * 4 + n_items * 24
        d2h = db_h.numel() * 4

        def e2e_step():
            for slot, (w, sc) in enumerate(zip(scenes, sc_host)):
                s = w["scene"]
                sim.upload_scene(s["media"], s["boundaries"], s["med_array"], s["z_max"], sc, s["r_s"], slot)
            sim.batch_plan(items, x_h, z_h, capacity=int(0.35 * total_rays) + 4096)
            sim.batch_trace(seed, 8, 0.2, rf=rf, quad=quad)
            sim.batch_beamform(rf, quad, 60.0, db=db)
            db_h.copy_(db, non_blocking=True)
            side.synchronize()

        n_e2e = 0 if args.skip_e2e else max(1, min(args.steps, 3))
        e2e_s = float("nan")
        if n_e2e:
            e2e_step()
            R.barrier()
            t0 = time.perf_counter()
            for _ in range(n_e2e):
                e2e_step()
            R.barrier()
            e2e_s = (time.perf_counter() - t0) / n_e2e
        e2e_s = R.max(e2e_s)
    ms = R.max(sum(a.elapsed_time(b) for a, b in ev) / args.steps)
    trace_ms = prof["trace"][0] / max(prof["trace"][2], 1)
    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    achieved = trace_flops(st) / (trace_ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": METRIC, "value": whole_job_rate(total_rays, world, ms * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "items": n_items, "rays_per_step": total_rays,
                       "ray_scale": scale, "l2": "flushed before every timed step (256 MiB write, untimed)"},
            "frames_per_s": whole_job_rate(n_items, world, ms * 1e-3),
            "images_per_s": whole_job_rate(len(scenes), world, ms * 1e-3),
            "arrivals_per_step": n_arr2, "stats_per_step": st,
            "phase_ms_direct_run": {k: v[0] / max(v[2], 1) for k, v in prof.items() if v[2]},
            "roofline": {"bound": "alu",
                         "kernel": "k_trace" + (" (extended instantiation: rough boundaries, transmit kinds other "
                                                "than plane waves, transmit mixing, convex arrays, triangle meshes)" if args.workload != "layered" else ""),
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "trace_ms_per_launch": trace_ms},
            "gpu_launches": 7 * args.steps, "clocks": clk,
            "e2e": {"value": whole_job_rate(total_rays, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "path": "8 x ur_scene_upload_slot (pinned host scatterers, grid builds) + ur_batch_plan + "
                            "ur_batch_trace + ur_batch_beamform, 8 dB images to pinned host"}}
        if world == 1 and not args.no_cpu_baseline:
            w = dict(scenes[0])
            w["angles"] = scenes[0]["angles"][15:16]
            rate, n, dt, thr = oracle_rate(w, args.cpu_seconds)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                    "sample": "rays 0..%d of scene seed 1's 0-degree transmit (%.1f s), trace + "
                                              "deposit + 512x256 DAS + log" % (n - 1, dt)}
        print(json.dumps(line), flush=True)
    sim.close()
    R.close()


def oracle_adjoint_rate(w, tgt_media, target_s, threads=None):
    """FP64 oracle forward + pathwise gradient on a bounded sample of the frame's rays:
    returns (rays/s, rays in sample, seconds, threads).  The target channel data of the
    sample is computed first and not timed, as on the GPU side."""
    import numpy as np
    import oracle
    threads = threads or (os.cpu_count() or 1)
    wt = dict(w["scene"])
    wt["media"] = [tuple(float(v) for v in m) for m in tgt_media]
    n_tx = len(np.atleast_1d(w["angles"]))

    def run(n, timed_scene):
        arr, _, _ = oracle.trace(timed_scene, w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"],
                                 w["max_path"], 0, n, threads=threads)
        return oracle.deposit(w["array"], n_tx, arr)

    def step(n, t_rf, t_q):
        rf, q = run(n, w["scene"])
        oracle.grad(w["scene"], w["array"], w["angles"], w["n_rays"], w["seed"], w["max_bounces"], 2 * (rf - t_rf),
                    2 * (q - t_q), w["max_path"], 0, n, threads=threads)

    n = 2048
    t_rf, t_q = run(n, wt)
    t0 = time.perf_counter()
    step(n, t_rf, t_q)
    probe = time.perf_counter() - t0
    n = int(max(1024, min(w["n_rays"], n * target_s / max(probe, 1e-3))))
    t_rf, t_q = run(n, wt)
    t0 = time.perf_counter()
    step(n, t_rf, t_q)
    dt = time.perf_counter() - t0
    return n * len(np.atleast_1d(w["angles"])) / dt, n, dt, threads


def run_adjoint(args, rank, world, local_rank):
    """Differentiation workload: forward trace of the layered frame against a target simulated
    with speeds +2 %, impedances +5 %, attenuation +10 % (same seed), then the path-replay
    adjoint for the gradient w.r.t. 4 media x (c, Z, alpha) and 50k scatterer amplitudes."""
    import numpy as np
    import torch

    import paper_2501_05828_gb300 as ur
    import phantoms

    torch.cuda.set_device(local_rank)
    R = Ranks(rank, world, local_rank)
    dev = R.device
    w = phantoms.layered()
    N = w["n_rays"] if not args.rays else args.rays
    seed = w["seed"] + rank
    sim = ur.Simulator(local_rank)
    sim.load(w)
    med0 = np.array(w["scene"]["media"], np.float32)
    tgt_med = med0.astype(np.float64).copy()
    tgt_med[:, 0] *= 1.02
    tgt_med[:, 1] *= 1.05
    tgt_med[:, 2] *= 1.10
    sim.set_media(tgt_med.astype(np.float32))
    trf, tq = sim.trace(N, seed, w["max_bounces"], w["max_path"])
    sim.set_media(med0)
    n_scat = len(w["scene"]["scatterers"])
    _, _, st = sim.trace(N, seed, w["max_bounces"], w["max_path"], stats=True)

    def step(t_rf=trf, t_q=tq):
        rf, q = sim.trace(N, seed, w["max_bounces"], w["max_path"])
        g_rf, g_q = 2 * (rf - t_rf), 2 * (q - t_q)
        return sim.trace_adjoint(N, seed, w["max_bounces"], g_rf, g_q, w["max_path"], n_med=len(med0),
                                 n_scat=n_scat)

    for _ in range(args.warmup):
        step()
    R.barrier()
    sim.set_profiling(True)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    R.barrier()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        gm, ga = step()
        ev[k][1].record()
    R.barrier()
    clk = clocks.stop() if clocks else None
    prof = sim.profile()
    sim.set_profiling(False)
    ms = R.max(sum(a.elapsed_time(b) for a, b in ev) / args.steps)
    per = {k: v[0] / max(v[2], 1) for k, v in prof.items() if v[2]}
    launches = sum(v[1] for v in prof.values())

    # ---- end to end: target channel data from pinned host memory, gradients back to host
    trf_h, tq_h = trf.cpu().pin_memory(), tq.cpu().pin_memory()
    h2d = (trf_h.numel() + tq_h.numel()) * 4
    d2h = (len(med0) * 3 + n_scat) * 4

    def e2e_step():
        t_rf = trf_h.to(dev, non_blocking=True)
        t_q = tq_h.to(dev, non_blocking=True)
        gm_d, ga_d = step(t_rf, t_q)
        return gm_d.cpu(), ga_d.cpu()

    n_e2e = 0 if args.skip_e2e else max(3, min(args.steps, 10))
    e2e_s = float("nan")
    if n_e2e:
        e2e_step()
        R.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            e2e_step()
        R.barrier()
        e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e_s = R.max(e2e_s)

    props = torch.cuda.get_device_properties(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    t_trace = per.get("trace", float("nan")) * 1e-3
    achieved = trace_flops(st) / t_trace / 1e12
    if rank == 0:
        line = {
            "metric": "rays/s of forward + gradient (path-replay adjoint)",
            "value": whole_job_rate(N, world, ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "differentiation: " + WORKLOAD, "rays_per_step": N, "parameters": 12 + n_scat,
                       "l2": "flushed before every timed step (256 MiB write, untimed)",
                       "parallelism": "replicas: one frame per GPU"},
            "phase_ms": per, "adjoint_over_trace": per.get("adjoint", 0.0) / max(per.get("trace", 1e-9), 1e-9),
            "roofline": {"bound": "alu", "kernel": "k_trace (recording arrivals for the adjoint)",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "peak_note": "%d SMs x %d FP32 lanes x 2 x %.0f MHz (sm_max_mhz)" % (
                             props.multi_processor_count, FP32_LANES_PER_SM, sm_mhz),
                         "trace_ms_per_launch": t_trace * 1e3, "algorithmic_flops_per_launch": trace_flops(st)},
            "gpu_launches": launches, "clocks": clk,
            "e2e": {"value": whole_job_rate(N, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                    "path": "target rf/quad from pinned host, ur_trace + loss gradient + ur_trace_adjoint, "
                            "gradients (12 + %d floats) to host" % n_scat},
            "grad_media_norm": float(gm.norm()), "grad_amp_norm": float(ga.norm())}
        if world == 1 and not args.no_cpu_baseline:
            rate, n, dt, thr = oracle_adjoint_rate(w, tgt_med, args.cpu_seconds)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                    "sample": "rays 0..%d of the frame (%.1f s): FP64 trace + deposit + pathwise "
                                              "gradient (dual numbers), target precomputed" % (n - 1, dt)}
        print(json.dumps(line), flush=True)
    sim.close()
    R.close()


DENOISER_WORKLOAD = ("denoiser: 4-level U-Net (widths 32-256, 1.95M parameters) on [128 x 3200] analytic channel "
                     "data, batch 8 pairs traced from jittered layered phantoms (1e6-ray input, 3e7-ray target), "
                     "BF16 weights/activations, FP32 accumulation, one step = forward + loss + backward + Adam")


def unet_forward_flops(batch, h, w, c=32):
    """Algorithmic multiply-adds x 2 of one forward pass (3x3 convolutions; the
    first sees its 2 real input channels)."""
    res = (1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 2, 2, 1, 1)
    cin = (2, c, c, 2 * c, 2 * c, 4 * c, 4 * c, 8 * c, 12 * c, 4 * c, 6 * c, 2 * c, 3 * c, c)
    cout = (c, c, 2 * c, 2 * c, 4 * c, 4 * c, 8 * c, 8 * c, 4 * c, 4 * c, 2 * c, 2 * c, c, c)
    return sum(2 * 9 * ci * co * batch * (h // r) * (w // r) for r, ci, co in zip(res, cin, cout))


def oracle_denoiser_rate(target_s):
    """FP64 reference U-Net: forward + backward on a 128 x 400 crop, scaled to
    [128 x 3200] samples/s."""
    import numpy as np
    from oracle import denoiser as D
    rng = np.random.default_rng(0)
    p = D.init_params(rng)
    x = rng.standard_normal((1, 128, 400, 2))
    t = rng.standard_normal((1, 128, 400, 2))
    n, t0 = 0, time.perf_counter()
    while True:
        y, cache = D.forward(p, x)
        _, g = D.mse(y, t)
        D.backward(p, cache, g)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return n / 8.0 / dt, n, dt


def run_denoiser(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2501_05828_gb300 as ur
    from paper_2501_05828_gb300 import denoise as dz
    import phantoms

    torch.cuda.set_device(local_rank)
    R = Ranks(rank, world, local_rank)
    dev = R.device
    B = 8
    sim = ur.Simulator(local_rank)
    xr, xq, tr, tq, _ = dz.make_pairs(sim, phantoms.batched_variant, range(1 + 8 * rank, 9 + 8 * rank), 1e6, 3e7)
    sim.close()
    H, W = int(xr.shape[1]), int(xr.shape[2])
    net = ur.Denoiser(local_rank, max_batch=B, n_el=H, n_s=W, width=32, seed=1)
    net.set_scale(dz.channel_scale(tr, tq))
    lr = 1e-4
    for _ in range(args.warmup):
        net.train_step(xr, xq, tr, tq, lr)
        net.forward(xr, xq)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    R.barrier()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = net.launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        loss = net.train_step(xr, xq, tr, tq, lr)
        ev[k][1].record()
        flush.zero_()
        fe[k][0].record()
        net.forward(xr, xq)
        fe[k][1].record()
    R.barrier()
    launches = net.launch_count() - launches0
    clk = clocks.stop() if clocks else None
    ms = R.max(sum(a.elapsed_time(b) for a, b in ev) / args.steps)
    ms_fwd = R.max(sum(a.elapsed_time(b) for a, b in fe) / args.steps)
    # end to end through the C ABI with pinned host buffers (inputs + targets in, loss out)
    hx = [t.cpu().pin_memory() for t in (xr, xq, tr, tq)]
    h2d = sum(t.numel() * 4 for t in hx)
    n_e2e = 0 if args.skip_e2e else max(3, min(args.steps, 20))
    e2e_ms = float("nan")
    if n_e2e:
        net.train_step(*hx, lr)
        R.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            net.train_step(*hx, lr)
        R.barrier()
        e2e_ms = (time.perf_counter() - t0) / n_e2e * 1e3
    e2e_ms = R.max(e2e_ms)
    F = unet_forward_flops(B, H, W)
    F_first = 2 * 9 * 2 * 32 * B * H * W
    train_flops = 3 * F - F_first           # forward, data gradients (none for the input), weight gradients
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    peak_burst = peaks.get("bf16_tflops", 1900.0)
    ach = train_flops / (ms * 1e-3) / 1e12
    ach_fwd = F / (ms_fwd * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": "denoiser training samples/s ([128 x 3200] channel data)", "value": whole_job_rate(B, world, ms * 1e-3),
            "unit": "samples/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": DENOISER_WORKLOAD, "batch": B, "n_el": H, "n_s": W,
                       "l2": "flushed before every timed call (256 MiB write, untimed)"},
            "inference_samples_per_s": whole_job_rate(B, world, ms_fwd * 1e-3), "ms_forward": ms_fwd, "loss": loss,
            "roofline": {"bound": "tensor", "kernel": "train step (tcgen05 convolutions + elementwise kernels)",
                         "achieved": ach, "peak": peak_sus, "unit": "TFLOP/s", "frac": ach / peak_sus,
                         "traffic": None, "peak_note": "bf16_tflops_sustained of measured",
                         "algorithmic_flops_per_step": train_flops,
                         "forward": {"achieved": ach_fwd, "peak": peak_burst, "frac": ach_fwd / peak_burst,
                                     "peak_note": "bf16_tflops (burst) of measured", "flops": F}},
            "gpu_launches": launches, "launches_per_step": launches / args.steps,
            "e2e": {"value": whole_job_rate(B, world, e2e_ms * 1e-3), "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": 8, "ms_per_step": e2e_ms,
                    "path": "ur_nn_train_step with pinned host inputs/targets (staged copies) and the loss to host"},
            "clocks": clk,
        }
        if world == 1 and not args.no_cpu_baseline:
            rate, n, dt = oracle_denoiser_rate(min(args.cpu_seconds, 20.0))
            line["cpu_baseline"] = {"value": rate, "unit": "samples/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                    "sample": "%d forward+backward passes of the FP64 reference on a 128x400 crop "
                                              "(1/8 sample) in %.1f s, numpy threads" % (n, dt)}
        print(json.dumps(line), flush=True)
    net.close()
    R.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (default: 150 layered, 5 batched, 30 adjoint, 30 denoiser)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rays", type=int, default=0, help="rays per frame override (profiling captures only)")
    ap.add_argument("--skip-e2e", action="store_true", help="omit the end-to-end leg (profiling captures only)")
    ap.add_argument("--workload", default="layered",
                    choices=("layered", "rough", "paper", "convex", "diverging", "synthetic", "mixed", "mesh", "batched",
                             "adjoint", "denoiser"))
    ap.add_argument("--batch-scale", type=float, default=1.0, help="scale of the batched workload's ray counts")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    args.warmup = max(3, args.warmup)
    if args.steps <= 0:
        args.steps = {"layered": 150, "rough": 60, "paper": 30, "convex": 30, "diverging": 60, "synthetic": 60,
                      "mixed": 30, "mesh": 30, "batched": 5, "adjoint": 30, "denoiser": 30}[args.workload]
    if args.impl == "reference":
        run_reference(args, rank)
    elif args.workload == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.workload == "adjoint":
        run_adjoint(args, rank, world, local_rank)
    elif args.workload == "denoiser":
        run_denoiser(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
