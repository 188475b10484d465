"""Comparison of the CUDA path's per-path and per-arrival records with the oracle's."""
import numpy as np

import oracle


def gpu_records(rec, n_el):
    """Debug tensors from Simulator.trace_debug -> structured numpy array like the oracle's."""
    row = rec["row"].cpu().numpy().view(np.uint32).astype(np.int64)
    out = np.zeros(row.size, oracle.ARRIVAL_DTYPE)
    out["tx"] = row // n_el
    out["el"] = row % n_el
    out["ray"] = rec["ray"].cpu().numpy().view(np.uint32)
    out["event"] = rec["event"].cpu().numpy().view(np.uint32)
    out["t"] = rec["t_hi"].cpu().numpy().astype(np.float64) + rec["t_lo"].cpu().numpy().astype(np.float64)
    out["amp"] = rec["amp"].cpu().numpy().astype(np.float64)
    return out


def _key(a):
    return (a["tx"].astype(np.uint64) << np.uint64(48)) ^ (a["ray"].astype(np.uint64) << np.uint64(16)) ^ \
        (a["event"].astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15))


def _sorted(a):
    o = np.lexsort((a["event"], a["ray"], a["tx"]))
    return a[o]


def compare(gpu_arr, orc_arr, gpu_hash=None, orc_hash=None, ray_begin=0, n_rays_sub=None, amp_floor=0.0):
    """Match arrivals by (transmit, ray, event); report path agreement and errors.

    amp_floor: amplitudes below amp_floor x the largest one are compared against that floor
    (relative error of tail arrivals).  Returns dict with: frac_paths (rays whose path hash
    and arrival set agree),
    bad_rays (set of (tx, ray)), max_dt (samples, matched arrivals), max_amp_rel,
    el_mismatch (matched arrivals on different elements), n_gpu, n_orc, n_matched."""
    g = _sorted(gpu_arr)
    o = _sorted(orc_arr)
    gk = np.stack([g["tx"].astype(np.int64), g["ray"].astype(np.int64), g["event"].astype(np.int64)], 1)
    ok = np.stack([o["tx"].astype(np.int64), o["ray"].astype(np.int64), o["event"].astype(np.int64)], 1)
    gv = gk.view([("a", np.int64), ("b", np.int64), ("c", np.int64)]).reshape(-1)
    ov = ok.view([("a", np.int64), ("b", np.int64), ("c", np.int64)]).reshape(-1)
    common, gi, oi = np.intersect1d(gv, ov, assume_unique=False, return_indices=True)
    only_g = np.setdiff1d(np.arange(g.size), gi)
    only_o = np.setdiff1d(np.arange(o.size), oi)
    bad = set(zip(g["tx"][only_g].tolist(), g["ray"][only_g].tolist()))
    bad |= set(zip(o["tx"][only_o].tolist(), o["ray"][only_o].tolist()))
    n_paths = None
    if gpu_hash is not None and orc_hash is not None:
        diff = np.argwhere(gpu_hash != orc_hash)
        for tx, r in diff.tolist():
            bad.add((tx, r + ray_begin))
        n_paths = orc_hash.size
    gm, om = g[gi], o[oi]
    dt = np.abs(gm["t"] - om["t"])
    floor = amp_floor * float(np.abs(om["amp"]).max()) if om.size else 0.0
    amp_rel = np.abs(gm["amp"] - om["amp"]) / np.maximum(np.maximum(np.abs(om["amp"]), floor), 1e-300)
    worst = int(np.argmax(amp_rel)) if amp_rel.size else -1
    wdt = int(np.argmax(dt)) if dt.size else -1
    res = {"bad_rays": bad, "n_gpu": int(g.size), "n_orc": int(o.size), "n_matched": int(common.size),
           "max_dt": float(dt.max()) if dt.size else 0.0,
           "dt_q99": float(np.quantile(dt, 0.99)) if dt.size else 0.0,
           "max_amp_rel": float(amp_rel.max()) if amp_rel.size else 0.0,
           "worst_amp": (hex(int(om["event"][worst])), int(om["ray"][worst]), float(om["amp"][worst]),
                         float(gm["amp"][worst])) if worst >= 0 else None,
           "worst_dt": (hex(int(om["event"][wdt])), int(om["tx"][wdt]), int(om["ray"][wdt]), float(om["t"][wdt]),
                        float(gm["t"][wdt])) if wdt >= 0 else None,
           "el_mismatch": int(np.sum(gm["el"] != om["el"]))}
    if n_paths:
        res["frac_paths"] = 1.0 - len(bad) / n_paths
    return res


def drop_rays(arr, bad):
    if not bad:
        return arr
    keys = set(bad)
    m = np.array([(int(t), int(r)) not in keys for t, r in zip(arr["tx"], arr["ray"])], bool)
    return arr[m]


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
