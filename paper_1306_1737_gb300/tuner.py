"""Autotuner for batches of boxes.

The boxes are split into size classes (equal numbers of boxes, by particle
count).  For every class and every candidate (cluster size C in {8, 4}, list
lifetime nstlist with its scaled list radius) the class's boxes are run
alone as one group for one horizon, captured in a CUDA graph, and timed with
CUDA events; the candidate with the least device time per frame wins the
class.  The winner is then also timed with the other prune intervals of
NSTPRUNES (each with its own prune radius, Sec. 2.3), and the fastest
interval is kept.  Winners are cached in a JSON file keyed by the GPU, the class's
sizes and the interaction parameters, so a later run with the same batch
skips the timing.  Classes that chose the same candidate are merged into one
group (one context).

The paper picks the cluster shape per architecture (Sec. 2.2, Table 1) and
the list lifetime from a buffer estimate (Sec. 2.3, Appendix); here both are
measured on the GPU at hand.  Each lifetime's list radius comes either from
scaling the configured buffer with sqrt(nstlist / nstlist0) or from the
Appendix's drift bound (nb_buffer_size).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from paper_1306_1737_gb300.batch import BatchRunner, GroupSpec, scaled_rlist

CLUSTER_SIZES = (8, 4)
NSTLISTS = (10, 20, 40)
NSTPRUNES = (2, 5, 10)


def _classes(counts, n_classes):
    order = np.argsort(counts, kind="stable")
    return [list(map(int, part)) for part in np.array_split(order, n_classes) if part.size]


def _key(gpu, counts, boxes, params, rlist0, nstlist0, nstprune, H):
    d = {"gpu": gpu, "counts": [int(c) for c in counts], "boxes": np.round(boxes, 6).tolist(),
         "elec": params["elec"], "rc": params["rc"], "beta": params.get("beta"), "rlist0": rlist0,
         "nstlist0": nstlist0, "nstprune": nstprune, "H": H,
         "candidates": [list(CLUSTER_SIZES), list(NSTLISTS), list(NSTPRUNES)]}
    return hashlib.sha1(json.dumps(d, sort_keys=True).encode()).hexdigest()[:16]


def time_group(spec, counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, params, nstprune,
               device, reps, rbb=0.0):
    """Device ms per frame of one group run alone (graph replays)."""
    import torch
    r = BatchRunner(counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, [spec], params, nstprune,
                    device=device, rbb=rbb)
    try:
        r.capture()
        r.replay()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            r.replay()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        for info in r.check():
            if info.status != 0:
                return float("inf")
        return float(np.median(ms)) / frames.shape[0]
    finally:
        r.close()


def particle_classes(q, types, mass):
    """[(count, mass, charge, LJ type)] of the distinct particle kinds."""
    keys = np.stack([np.asarray(types, np.float64), np.asarray(q, np.float64), np.asarray(mass, np.float64)], 1)
    uniq, cnt = np.unique(keys, axis=0, return_counts=True)
    return [(int(c), float(u[2]), float(u[1]), int(u[0])) for u, c in zip(uniq, cnt)]


def appendix_rlist(classes, c6c12, volume, params, nstlist, dt_ps=0.002, temperature=300.0, tolerance=None):
    """rc plus the buffer the Appendix's drift bound asks for over a list
    lifetime of (nstlist - 1) time steps; tolerance in kJ/mol/ps per particle
    (default 0.1 kB T per ns, the drift of the paper's Table 3)."""
    import paper_1306_1737_gb300 as nb
    if tolerance is None:
        tolerance = 0.1 * 0.0083144626 * temperature / 1000.0
    prm = nb.make_params(params["elec"], params["rc"], eps_rf=params.get("eps_rf", float("inf")),
                         beta=params.get("beta", 0.0))
    rb = nb.nb_buffer_size(classes, c6c12, volume, prm, max(nstlist - 1, 1) * dt_ps, temperature, tolerance)
    return params["rc"] + rb


def tune(counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, params, nstprune, rlist0, nstlist0,
         n_classes=4, reps=3, cache_path=None, device=0, log=None, rlist_rule="sqrt", mass=None,
         tolerance=None, rbb=0.0):
    """Returns (groups: list of GroupSpec, table: list of per-class results;
    a result key is "C/nstlist" at the configured prune interval or
    "C/nstlist/nstprune").

    rlist_rule: "sqrt" scales the configured buffer with sqrt(nstlist /
    nstlist0); "appendix" sizes it with the Appendix's drift bound (needs
    mass; candidates whose list radius reaches half a box edge are skipped)."""
    import torch
    counts = np.asarray(counts, dtype=np.int64)
    boxes = np.asarray(boxes, dtype=np.float64).reshape(-1, 3)
    H = int(frames.shape[0])
    gpu = torch.cuda.get_device_name(device)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    table = []
    choice = {}
    if rlist_rule == "appendix":
        if mass is None:
            raise ValueError("the appendix rule needs particle masses")
        pcls = particle_classes(q, types, mass)
        vol = float(np.prod(boxes, axis=1).sum())
        rlist_of = {nst: appendix_rlist(pcls, np.asarray(c6c12), vol, params, nst, tolerance=tolerance)
                    for nst in NSTLISTS}
    else:
        rlist_of = {nst: scaled_rlist(params["rc"], rlist0, nstlist0, nst) for nst in NSTLISTS}
    rule = rlist_rule if rlist_rule != "appendix" else f"appendix:{tolerance}"
    for cls in _classes(counts, n_classes):
        key = _key(gpu, counts[cls], boxes[cls], params, rlist0, nstlist0, nstprune, H) + rule + f"/rbb{rbb:g}"
        if key in cache:
            ent = cache[key]
            ent["cached"] = True
        else:
            times = {}
            for C in CLUSTER_SIZES:
                for nst in NSTLISTS:
                    if H % nst:
                        continue
                    if rlist_of[nst] >= 0.5 * float(boxes[cls].min()):
                        continue                    # list radius too large for these boxes
                    spec = GroupSpec(C, nst, rlist_of[nst], list(cls))
                    t = time_group(spec, counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, params,
                                   nstprune, device, reps, rbb=rbb)
                    times[f"{C}/{nst}"] = t
                    if log:
                        log(f"class {len(cls)} boxes {int(counts[cls].min())}-{int(counts[cls].max())} atoms: "
                            f"C={C} nstlist={nst}: {t:.4f} ms/frame")
            if not times:
                raise ValueError(f"no candidate fits the boxes of {int(counts[cls].min())}-"
                                 f"{int(counts[cls].max())} particles: a horizon of {H} frames needs an "
                                 f"nstlist in {NSTLISTS} dividing it, with a list radius below half the "
                                 f"smallest box edge {float(boxes[cls].min()):.4g} nm")
            best = min(times, key=times.get)
            if not np.isfinite(times[best]):
                raise RuntimeError("every candidate of a size class failed its device check")
            # second stage: other prune intervals for the winning shape and lifetime
            bC, bn = map(int, best.split("/"))
            for nsp in NSTPRUNES:
                if nsp == nstprune or nsp >= bn:
                    continue
                spec = GroupSpec(bC, bn, rlist_of[bn], list(cls), nstprune=nsp)
                t = time_group(spec, counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, params,
                               nstprune, device, reps, rbb=rbb)
                times[f"{bC}/{bn}/{nsp}"] = t
                if log:
                    log(f"class {len(cls)} boxes: C={bC} nstlist={bn} nstprune={nsp}: {t:.4f} ms/frame")
            best = min(times, key=times.get)
            ent = {"best": best, "ms_per_frame": times, "cached": False}
            cache[key] = {k: v for k, v in ent.items() if k != "cached"}
        parts = list(map(int, ent["best"].split("/")))
        C, nst = parts[0], parts[1]
        nsp = parts[2] if len(parts) > 2 else nstprune
        choice.setdefault((C, nst, nsp), []).extend(cls)
        table.append({"boxes": len(cls), "atoms_min": int(counts[cls].min()), "atoms_max": int(counts[cls].max()),
                      "best": ent["best"], "ms_per_frame": ent["ms_per_frame"], "cached": ent["cached"]})
    if cache_path:
        d = os.path.dirname(cache_path)
        if d:
            os.makedirs(d, exist_ok=True)
        with open(cache_path, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
    groups = [GroupSpec(C, nst, rlist_of[nst], sorted(b), nstprune=nsp) for (C, nst, nsp), b in sorted(choice.items())]
    return groups, table
