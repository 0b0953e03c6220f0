#!/usr/bin/env python
"""Benchmark of the cluster-pair non-bonded hot path on one GB300 per rank.

A step is one pair-list lifetime of the workload: grid the box
(nb_grid_put), build the buffered cluster-pair list (nb_pairlist_build), then
nstlist frames, each with new coordinates and one force evaluation
(nb_compute; energies and virial on the first and last frame; every nstprune
frames nb_prune_compute, which prunes the list in the same pass).  The
headline value is force evaluations per second over the whole job.  Default
workload: the 3,000,000-atom water box (10% of molecules re-typed among 8 LJ
types), Ewald real space rc 1.0 nm, beta 3.12 nm^-1, rlist 1.1 nm, nstlist
40, prune every 5; its line also carries a block for the 24,000-atom box
(nstlist 20) and one for the batch of 256 uneven boxes.

--impl reference times the FP64 CPU oracle (its cell-list tier, the same
pairs as the brute-force minimum-image loop) on the same workload and metric:
one force+energy evaluation per step.

Under torchrun each rank runs an independent replica of the workload on its
own GPU (the boxes share nothing); value = evaluations of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "force evals/s & pair interactions/s vs plain kernel, force err ≤1e-4 RMS"
UNIT = "force evals/s"
L2_FLUSH_BYTES = 512 << 20

# Algorithmic FP32 work per pair (paper, Tables 1-2: flops per pair of the
# analytical kernels): every listed pair costs a distance test (9 flops);
# pairs inside rc add the interaction (Ewald analytical 69, RF 40, minus the
# distance part).
FLOPS_DIST = 9
FLOPS_PAIR = {"ewald": 69, "rf": 40}


def workloads():
    from paper_1306_1737_gb300 import workloads as w
    return {
        "water24k": ("24,000-atom water box, Ewald, rc 1.0, rlist 1.1, nstlist 20, prune/5", w.config2),
        "water3m": ("3,000,000-atom water box + 8 LJ types (LB), Ewald, rlist 1.1, nstlist 40, prune/5",
                    w.config3),
        "water1536": ("1,536-atom water box, reaction field, rc 0.9, rlist 1.0", w.config1),
        "water1m": ("1,000,002-atom water box (profiling size), Ewald as the 3M box", water1m),
    }


def water1m():
    """A 1M-particle box with the 3M box's parameters, for profiler captures
    (working set above the 129 MB L2, device memory about 1.5 GB)."""
    from paper_1306_1737_gb300 import workloads as w
    b = w.water_box(333334, None, seed=1005, retype_frac=0.1, n_extra_types=8)
    return b, {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12, "nstlist": 40, "nstprune": 5,
               "comb": "lb"}


FORCE_SOURCES = ["paper_1306_1737_gb300/csrc/nb_force.cu", "paper_1306_1737_gb300/csrc/nb_internal.cuh",
                 "paper_1306_1737_gb300/csrc/nb_ewald_fit.h", "paper_1306_1737_gb300/csrc/nb_pair.cuh",
                 "paper_1306_1737_gb300/csrc/nb_mlp.cuh"]


def force_source_hash():
    """Hash of the force kernel's sources (a profile's counters apply only to
    the exact kernel they were taken on)."""
    import hashlib
    h = hashlib.sha1()
    for rel in FORCE_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:12]


def profiled_traffic(workload):
    """DRAM bytes per force-kernel launch from the committed ncu summary of
    this workload, or None when it was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"k_force8_{workload}.md")
    if not os.path.exists(path):
        return None
    src, traffic = None, None
    for line in open(path):
        if line.startswith("source-hash:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("dram-bytes-per-launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if src == force_source_hash() else None


def scaled_traffic(cluster_pairs):
    """DRAM bytes of a force launch over cluster_pairs cluster pairs, scaled
    from the 1M-box capture (the kernel reads each list entry and particle
    once, so its traffic is proportional to the cluster pairs), or None when
    that capture was taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "k_force8_water1m.md")
    t = profiled_traffic("water1m")
    if t is None:
        return None
    for line in open(path):
        if line.startswith("cluster-pairs-per-launch:"):
            return t * cluster_pairs / float(line.split(":", 1)[1])
    return None


def profiled_counters(workload):
    """ncu issue and FP32-pipe figures of the force kernel from the committed
    summary of this workload (None when taken on other kernel sources)."""
    path = os.path.join(ROOT, "profiles", f"k_force8_{workload}.md")
    if not os.path.exists(path):
        return None
    keys = {"source-hash": "src", "issue-active-pct": "issue_slots_busy_pct",
            "fma-pipe-cycles-active-pct": "fma_pipe_cycles_active_pct",
            "fp32-lane-ops-pct": "fp32_lane_ops_pct_of_issue_peak", "counters-from": "profile"}
    out = {}
    for line in open(path):
        k, _, v = line.partition(":")
        if k.strip() in keys:
            v = v.strip()
            try:
                v = float(v)
            except ValueError:
                pass
            out[keys[k.strip()]] = v
    if out.pop("src", None) != force_source_hash() or "issue_slots_busy_pct" not in out:
        return None
    return out


def peaks():
    p = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            p["hbm_gbs"] = float(d.get("hbm_gbs", p["hbm_gbs"]))
            p["sm_max_mhz"] = float(d.get("sm_max_mhz", p["sm_max_mhz"]))
            p["source"] = "measured"
        except Exception:
            pass
    return p


def device_uuid(dev):
    """'GPU-...' UUID of a torch CUDA device (None if torch does not expose it)."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


class ClockSampler:
    """SM clock and clock-event-reason samples of this GPU while the timed
    region runs: NVML (read-only queries through libnvidia-ml) every 50 ms in
    a thread (at 500 queries per second the driver calls delayed some of the
    host's own submissions), else nvidia-smi every 200 ms."""

    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap"}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.uuid = device_uuid(dev)
        self.proc = None
        self.path = None
        self.thread = None
        self.samples = []
        self.nvml = None
        self.handle = None
        try:
            import ctypes
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() == 0:
                h = ctypes.c_void_p()
                ok = self.uuid is not None and lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h)) == 0
                if ok:
                    self.nvml, self.handle = lib, h
        except Exception:
            self.nvml = None

    def _loop(self):
        import ctypes
        mhz = ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        getr = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop_flag:
            if self.nvml.nvmlDeviceGetClockInfo(self.handle, 1, ctypes.byref(mhz)) == 0 and \
                    getr(self.handle, ctypes.byref(reasons)) == 0:
                self.samples.append((mhz.value, reasons.value))
            time.sleep(0.05)

    def start(self):
        if self.nvml is not None:
            import threading
            self.stop_flag = False
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            sel = [f"--id={self.uuid}"] if self.uuid else []
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"] + sel,
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.thread is not None:
            import ctypes
            self.stop_flag = True
            self.thread.join(timeout=5)
            mx = ctypes.c_uint()
            smax = mx.value if self.nvml.nvmlDeviceGetMaxClockInfo(self.handle, 1, ctypes.byref(mx)) == 0 else None
            reasons = set()
            for _, r in self.samples:
                for bit, name in self.REASONS.items():
                    if r & bit:
                        reasons.add(name)
            out.update(sm_mhz=statistics.median([m for m, _ in self.samples]) if self.samples else None,
                       sm_max_mhz=smax, reasons=sorted(reasons), samples=len(self.samples), source="nvml")
            return out
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows), source="nvidia-smi")
        return out


def slowest_rank_seconds(seconds, dist=None, device=None):
    """The timed region's length on the slowest rank (every rank runs the
    same number of steps on its own replica; the job is done when the last
    rank is)."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_ranks, units_per_rank, seconds):
    """Units of all ranks per second of the slowest rank (weak scaling:
    each rank processes the same units)."""
    return n_ranks * units_per_rank / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


SAMPLE_ABOVE = 100_000   # larger boxes: the oracle evaluates a sample of particles


def oracle_eval(box, p, sel=None):
    import numpy as np
    import oracle
    prm = oracle.make_params(p["elec"], float(np.float32(p["rc"])), eps_rf=p.get("eps_rf", math.inf),
                             beta=p.get("beta", 0.0), comb=p.get("comb", "lb"))
    return oracle.forces_cells(box.xyz, box.q, box.types, box.sigma, box.eps, box.excl_off,
                               box.excl_idx, box.box, prm, sel=sel)


def oracle_unit(box, p, budget_s):
    """One timed unit of oracle work sized to about budget_s: a whole
    evaluation by the oracle's FP64 cell-list tier for small boxes, else the
    forces of a seeded particle sample (each against its cell neighbourhood).
    Returns (selection, fraction of one evaluation, text)."""
    import numpy as np
    if box.n <= SAMPLE_ABOVE:
        return None, 1.0, f"one FP64 cell-list force+energy evaluation of the {box.n}-particle box"
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    oracle_eval(box, p, sel=rng.choice(box.n, 64, replace=False))
    per_atom = (time.perf_counter() - t0) / 64
    k = int(max(64, min(box.n, budget_s / max(per_atom, 1e-9))))
    sel = rng.choice(box.n, k, replace=False)
    return sel, k / box.n, (f"FP64 cell-list forces of {k} seeded particles of the {box.n}-particle box "
                            f"= {k / box.n:.2e} of one evaluation")


def cpu_baseline(box, p, budget_s=15.0):
    """The oracle (its FP64 cell-list tier) on a bounded sample of the same
    workload, scaled to force evaluations per second."""
    import oracle
    sel, frac, what = oracle_unit(box, p, budget_s / 3)
    t0 = time.perf_counter()
    oracle_eval(box, p, sel)
    t1 = time.perf_counter() - t0
    n = max(1, min(20, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(n):
        oracle_eval(box, p, sel)
    dt = time.perf_counter() - t0
    return {"value": n * frac / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} x ({what}), FP64 OpenMP, after one untimed repetition"}


def run_reference_batch(args):
    """The oracle on the batch workload: each step is the seeded sample of
    batch_cpu_baseline, scaled to batch evaluations."""
    import oracle
    B, p = batch_workload()
    vals = [batch_cpu_baseline(B, p, budget_s=4.0) for _ in range(args.warmup + args.steps)][args.warmup:]
    value = len(vals) / sum(1.0 / v["value"] for v in vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": "batch256", "n_boxes": B.nbox, "n_atoms": int(B.n)},
        "cpu_baseline": {"value": value, "unit": BATCH_UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "each step: " + vals[0]["sample"]},
        "e2e": {"value": value, "unit": BATCH_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "batch256":
        return run_reference_batch(args)
    desc, fn = workloads()[args.workload]
    box, p = fn()
    import oracle
    sel, frac, what = oracle_unit(box, p, 5.0)
    for _ in range(args.warmup):
        oracle_eval(box, p, sel)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_eval(box, p, sel)
    dt = time.perf_counter() - t0
    value = args.steps * frac / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_dict(args, box, p, desc),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"each step: {what} (FP64, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(args, box, p, desc, workload=None):
    return {"workload": workload or args.workload, "description": desc, "n_atoms": int(box.n),
            "box_nm": [round(float(v), 6) for v in box.box], "elec": p["elec"], "rc_nm": p["rc"],
            "rlist_nm": p["rlist"], "beta_nm-1": p.get("beta"), "nstlist": p.get("nstlist", 1),
            "nstprune": p.get("nstprune", 0), "rbb_nm": args.rbb, "cluster": "8x8 cluster pairs (two 8x4 halves per warp), super-clusters of 2 i-clusters sharing a j-list",
            "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{args.gpus}",
            "launch": "each step captured once as a CUDA graph and replayed",
            "seed": int(box.seed)}


def surrogate_ab(nb, ctx, box, p, xs, F, stream, dev, steps=60000, reps=20):
    """The learned Ewald factor against the analytic kernel on the same list
    and GPU: train the network on the GPU (FP64 targets from the library),
    install it, and time force evaluations (forces only) of both kernels on
    the last frame; the surrogate's force error is taken against the
    analytic kernel's forces."""
    import numpy as np
    import torch
    from paper_1306_1737_gb300 import surrogate
    from paper_1306_1737_gb300 import workloads as w
    r = w.surrogate_samples(1 << 20, surrogate.R_MIN, surrogate.R_MAX, seed=1005)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    params, losses = surrogate.train(r, p["beta"], steps=steps, device=dev.index)
    train_s = time.perf_counter() - t0
    nb.nb_set_surrogate(ctx, params, surrogate.R_MIN, surrogate.R_MAX, stream)
    x = xs[-1]
    res = {}
    forces = {}
    for mode in ("ewald", "ewald_mlp"):
        prm = nb.make_params(mode, p["rc"], beta=p["beta"], want_energy=False)
        nb.nb_compute(ctx, prm, x, F, None, None, stream)
        torch.cuda.synchronize()
        forces[mode] = F.double().cpu().numpy()
        nb.nb_profile(ctx, True)
        nb.nb_profile_read(ctx)
        for _ in range(reps):
            nb.nb_compute(ctx, prm, None, F, None, None, stream)
        spans = [ms for kind, ms in nb.nb_profile_read(ctx) if kind == nb.NB_KERNEL_FORCE]
        nb.nb_profile(ctx, False)
        res[mode] = statistics.mean(spans)
    fa, fm = forces["ewald"], forces["ewald_mlp"]
    rms = float(np.sqrt((fa ** 2).sum(1).mean()))
    d = np.sqrt(((fm - fa) ** 2).sum(1))
    return {"network": "MLP 1-32-32-1 SiLU, layer 2 on BF16 mma.sync m16n8k16 (hi/lo split), FP32 accumulate",
            "train_steps": steps, "train_s": train_s, "final_minibatch_loss": float(losses[-1]),
            "force_ms_analytic": res["ewald"], "force_ms_surrogate": res["ewald_mlp"],
            "surrogate_over_analytic_time": res["ewald_mlp"] / res["ewald"],
            "max_dF_over_rms_vs_analytic": float(d.max() / rms), "rms_dF_over_rms_vs_analytic":
                float(np.sqrt((d ** 2).mean()) / rms)}


def compare_1x1(nb, ctx, box, p, x0, F, rlist, rprune, stream, reps=10, max_nbr=768):
    """The paper's comparison of cluster pairs with particle pairs (Table 3)
    on this GPU: on frame 0, the cluster kernel on the outer (rlist) list and
    on the pruned list, against a kernel with 4-16 lanes per particle on the
    full 1 x 1 Verlet list of the same radius; device times from CUDA-event
    spans; effective pairs are the distinct pairs inside rc per second."""
    import numpy as np
    import torch
    nb.nb_grid_put(ctx, x0, box.box, stream)
    nb.nb_pairlist_build(ctx, rlist, 0.0, torch.as_tensor(box.excl_off, device=x0.device),
                         torch.as_tensor(box.excl_idx, device=x0.device), stream)
    nbr = torch.empty((box.n, max_nbr), dtype=torch.int32, device=x0.device)
    cnt = torch.empty(box.n, dtype=torch.int32, device=x0.device)
    nb.nb_pairlist_1x1(ctx, rlist, max_nbr, nbr, cnt, stream)
    info_outer = nb.nb_check(ctx, stream)
    listed_1x1 = int(cnt.sum().item())
    prm = nb.make_params(p["elec"], p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                         want_energy=False)
    prm_e = nb.make_params(p["elec"], p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                           want_energy=True)

    def timed(fn, kind):
        fn()
        torch.cuda.synchronize()
        nb.nb_profile(ctx, True)
        nb.nb_profile_read(ctx)
        for _ in range(reps):
            fn()
        ms = [m for k, m in nb.nb_profile_read(ctx) if k == kind]
        nb.nb_profile(ctx, False)
        return statistics.mean(ms)

    t_1x1 = timed(lambda: nb.nb_compute_1x1(ctx, prm, None, nbr, cnt, max_nbr, F, stream), nb.NB_KERNEL_FORCE_1X1)
    t_outer = timed(lambda: nb.nb_compute(ctx, prm, None, F, None, None, stream), nb.NB_KERNEL_FORCE)
    nb.nb_compute(ctx, prm_e, None, F, None, None, stream)
    pairs_rc = int(nb.nb_check(ctx, stream).n_pairs_rc)
    nb.nb_prune(ctx, None, rprune, stream)
    t_pruned = timed(lambda: nb.nb_compute(ctx, prm, None, F, None, None, stream), nb.NB_KERNEL_FORCE)
    info_pruned = nb.nb_check(ctx, stream)
    del nbr
    return {"frame": 0, "rlist_nm": rlist, "r_prune_nm": rprune, "pairs_within_rc": pairs_rc,
            "kernel_1x1": {"ms": t_1x1, "listed_pairs": listed_1x1,
                           "pair_evaluations_per_s": listed_1x1 / (t_1x1 * 1e-3),
                           "effective_pairs_per_s": pairs_rc / (t_1x1 * 1e-3),
                           "note": "full list: each pair computed for both particles; 16, 8 or 4 lanes per particle"},
            "kernel_cluster_outer": {"ms": t_outer, "listed_pairs": int(info_outer.n_cluster_pairs) * 64,
                                     "pair_evaluations_per_s": int(info_outer.n_cluster_pairs) * 64 / (t_outer * 1e-3),
                                     "effective_pairs_per_s": pairs_rc / (t_outer * 1e-3)},
            "kernel_cluster_pruned": {"ms": t_pruned, "listed_pairs": int(info_pruned.n_cluster_pairs_pruned) * 64,
                                      "pair_evaluations_per_s":
                                          int(info_pruned.n_cluster_pairs_pruned) * 64 / (t_pruned * 1e-3),
                                      "effective_pairs_per_s": pairs_rc / (t_pruned * 1e-3)},
            "cluster_outer_over_1x1_speed": t_1x1 / t_outer,
            "cluster_pruned_over_1x1_speed": t_1x1 / t_pruned}


def tabulated_ab(nb, ctx, p, x, F, stream, reps=20):
    """The tabulated Ewald force factor against the fitted rational on the same
    list and frame: force-kernel times (CUDA-event spans) and the largest
    force difference relative to the RMS force."""
    import numpy as np
    import torch
    out, forces = {}, {}
    for mode in ("ewald", "ewald_tab"):
        prm = nb.make_params(mode, p["rc"], beta=p["beta"], want_energy=False)
        nb.nb_compute(ctx, prm, x, F, None, None, stream)
        torch.cuda.synchronize()
        forces[mode] = F.double().cpu().numpy()
        nb.nb_profile(ctx, True)
        nb.nb_profile_read(ctx)
        for _ in range(reps):
            nb.nb_compute(ctx, prm, None, F, None, None, stream)
        out[mode] = statistics.mean(m for k, m in nb.nb_profile_read(ctx) if k == nb.NB_KERNEL_FORCE)
        nb.nb_profile(ctx, False)
    fa, ft = forces["ewald"], forces["ewald_tab"]
    rms = float(np.sqrt((fa ** 2).sum(1).mean()))
    return {"force_ms_fitted": out["ewald"], "force_ms_tabulated": out["ewald_tab"],
            "tabulated_over_fitted_time": out["ewald_tab"] / out["ewald"],
            "max_dF_over_rms_vs_fitted": float(np.sqrt(((ft - fa) ** 2).sum(1)).max() / rms),
            "table": "2,048 intervals in (beta r)^2 on [0, 10], linear interpolation, shared memory"}


def pair_correlation(nb, ctx, box, x0, eo, ei, stream, rbb, r_max=1.0, nbins=400, reps=10):
    """The pair correlation analysis (Sec. 1, Sec. 2.3): per frame a fresh
    list at r_max (gridding + search, no pruning) and the histogram kernel
    with no cut-off conditional; device times from CUDA-event spans, the O-O
    g(r) first peak as a sanity figure."""
    import numpy as np
    import torch
    dev = x0.device
    nbox = 1
    h = torch.zeros((nbox, nbins + 1), dtype=torch.int64, device=dev)
    rl = float(np.float32(r_max))

    def frame(sel=(-1, -1)):
        nb.nb_grid_put(ctx, x0, box.box, stream)
        nb.nb_pairlist_build(ctx, rl, min(rbb, rl), eo, ei, stream)
        nb.nb_rdf(ctx, rl, nbins, sel[0], sel[1], 0, h, stream)

    frame()
    torch.cuda.synchronize()
    nb.nb_profile(ctx, True)
    nb.nb_profile_read(ctx)
    for _ in range(reps):
        frame()
    spans = nb.nb_profile_read(ctx)
    nb.nb_profile(ctx, False)
    ms = {k: statistics.mean(m for kind, m in spans if kind == v) for k, v in
          (("grid", nb.NB_KERNEL_GRID), ("search", nb.NB_KERNEL_SEARCH), ("rdf", nb.NB_KERNEL_RDF))}
    counts = h[0].cpu().numpy()
    info = nb.nb_check(ctx, stream)
    frame((0, 0))
    oo = h[0].cpu().numpy()[:nbins].astype(np.float64)
    n_o = int((box.types == 0).sum())
    dr = r_max / nbins
    shell = 4.0 * np.pi / 3.0 * dr ** 3 * ((np.arange(nbins) + 1) ** 3 - np.arange(nbins) ** 3)
    g_oo = oo * float(np.prod(box.box)) / (0.5 * n_o * (n_o - 1) * shell)
    binned = int(counts.sum())
    within = int(counts[:nbins].sum())
    frame_ms = ms["grid"] + ms["search"] + ms["rdf"]
    return {"r_max_nm": r_max, "nbins": nbins, "rbb_nm": min(rbb, rl),
            "list": "rebuilt every frame at r_max, no pruning; histogram kernel without a cut-off test",
            "kernel_ms": ms, "frame_ms": frame_ms,
            "listed_pairs_binned": binned, "pairs_within_r_max": within,
            "listed_pairs_per_s_rdf_kernel": binned / (ms["rdf"] * 1e-3),
            "pairs_within_r_max_per_s_frame": within / (frame_ms * 1e-3),
            "cluster_pairs": int(info.n_cluster_pairs),
            "oo_first_peak_nm": float((np.argmax(g_oo) + 0.5) * dr), "oo_first_peak_g": float(g_oo.max())}


def buffer_estimate(nb, box, p, nstlist, rlist, dt_ps=0.002, temperature=300.0):
    """The Appendix's drift bound for this workload's buffer and lifetime,
    and the buffer it asks for at the paper's 0.1 kB T/ns per particle."""
    import numpy as np
    from paper_1306_1737_gb300 import tuner
    cls = tuner.particle_classes(box.q, box.types, box.mass)
    table = nb.nb_lj_combine(box.sigma, box.eps)
    vol = float(np.prod(box.box))
    prm = nb.make_params(p["elec"], p["rc"], beta=p.get("beta", 0.0))
    t = max(nstlist - 1, 1) * dt_ps
    kt = 0.0083144626 * temperature
    tol = 0.1 * kt / 1000.0
    drift = nb.nb_buffer_drift(cls, table, vol, prm, rlist - p["rc"], t, temperature)
    return {"lifetime_ps": t, "temperature_K": temperature, "buffer_nm": rlist - p["rc"],
            "drift_bound_kT_per_ns_per_particle": drift / kt * 1000.0,
            "buffer_for_0.1_kT_per_ns_nm": nb.nb_buffer_size(cls, table, vol, prm, t, temperature, tol),
            "model": "free flight (sigma^2 = t^2 kB T (1/m1 + 1/m2)), an upper bound for rigid water"}


def init_ranks():
    """(dist or None, world size, rank, device) of this process; one GPU per rank."""
    import torch
    ws_n, rank, local = dist_env()
    if ws_n > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    return dist, ws_n, rank, torch.device("cuda", torch.cuda.current_device())


def run_ours(args):
    import paper_1306_1737_gb300 as nb
    dist, ws_n, rank, dev = init_ranks()
    nb.load()
    out = measure_box(args, args.workload, dist, ws_n, rank, dev, extras=True)
    if out is not None and args.sub_blocks and args.workload == "water3m":
        # the same path on the 24k box and on the batch of 256 boxes (this
        # rank's GPU only; the other ranks wait at the closing barrier)
        out["water24k"] = measure_box(args, "water24k", None, 1, 0, dev, extras=False)
        out["batch256"] = measure_batch(args, None, 1, 0, dev, sub=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


def measure_box(args, workload, dist, ws_n, rank, dev, extras=True):
    """One box workload: graph-replayed steps (the headline), per-kernel
    spans, the roofline of the force kernel, the end-to-end rate with host
    buffers, and (extras) the oracle baseline and the comparison blocks.
    Returns the JSON dict on rank 0, else None."""
    import numpy as np
    import torch

    import paper_1306_1737_gb300 as nb
    from paper_1306_1737_gb300 import workloads as w

    desc, fn = workloads()[workload]
    box, p = fn()
    nstlist = int(p.get("nstlist", 1))
    nstprune = int(p.get("nstprune", 0))
    rc, rlist = float(p["rc"]), float(p["rlist"])
    rprune = w.prune_radius(rc, rlist, nstprune) if nstprune else rlist
    elec = p["elec"]
    comb = nb.NB_COMB_LB if p.get("comb", "lb") == "lb" else nb.NB_COMB_GEOM

    cx = nb.Context(box.n, box.box, rlist, box.q, box.types, nb.nb_lj_combine(box.sigma, box.eps, comb),
                    device=dev.index)
    ctx = cx.ctx
    stream = torch.cuda.current_stream()
    # frame coordinates, resident in HBM before timing
    disp = w.frame_displacements(box.mass, max(nstlist - 1, 1), seed=2000 + box.seed)
    frames = np.empty((nstlist, box.n, 3), np.float32)
    frames[0] = box.xyz
    if nstlist > 1:
        frames[1:] = box.xyz[None] + np.cumsum(disp, axis=0)[: nstlist - 1]
    xs = torch.as_tensor(frames).to(dev)
    eo = torch.as_tensor(box.excl_off).to(dev)
    ei = torch.as_tensor(box.excl_idx).to(dev)
    F = torch.zeros((box.n, 3), dtype=torch.float32, device=dev)
    E = torch.zeros(2, dtype=torch.float64, device=dev)
    V = torch.zeros(9, dtype=torch.float64, device=dev)
    prm_e = nb.make_params(elec, rc, eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0), want_energy=True)
    prm_f = nb.make_params(elec, rc, eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0), want_energy=False)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rbb = rlist if args.rbb < 0 else args.rbb

    def energy_frame(f):
        return f == 0 or f == nstlist - 1

    def step(xdev):
        """One list lifetime on device frames xdev.  Launches go to the current
        stream (a capture stream while capturing)."""
        stream = torch.cuda.current_stream()
        x0 = xdev[0]
        nb.nb_grid_put(ctx, x0, box.box, stream)
        nb.nb_pairlist_build(ctx, rlist, rbb, eo, ei, stream)
        for f in range(nstlist):
            xf = xdev[f]
            prm = prm_e if energy_frame(f) else prm_f
            if nstprune and f % nstprune == 0 and (f > 0 or args.prune0):
                if args.fused_prune:
                    # prune while computing this frame's forces on the outer list
                    nb.nb_prune_compute(ctx, prm, xf if f > 0 else None, rprune, F, E, V, stream)
                else:
                    nb.nb_prune(ctx, xf if f > 0 else None, rprune, stream)
                    nb.nb_compute(ctx, prm, None, F, E, V, stream)
            else:
                nb.nb_compute(ctx, prm, xf if f > 0 else None, F, E, V, stream)

    efr = [energy_frame(f) for f in range(nstlist)]
    native_e2e = args.fused_prune and not args.prune0   # the schedule nb_run_frames runs

    def run_host(hx, hF, hE, hV, xbufs, Fbufs, Ebufs, Vbufs):
        """One list lifetime from pinned host frames to pinned host forces,
        energies and virial in one call (nb_run_frames: the same calls as
        step(), made by the library, with the transfers on a copy stream
        overlapping the neighbouring frames' kernels), its arguments
        marshalled once."""
        return nb.RunFrames(ctx, prm_f, hx, hF, xbufs, Fbufs, nbox=1, energy_frames=efr, e_host=hE, vir_host=hV,
                            e_dev=Ebufs, vir_dev=Vbufs, build=True, boxes=box.box, rlist=rlist, rbb=rbb,
                            excl_off=eo, excl_idx=ei, nstprune=nstprune, r_prune=rprune)

    def step_host(hx, hF, hE, xbufs, Fbufs, cs, ev):
        """One list lifetime from pinned host frames to pinned host forces
        through the same calls made from Python, with the transfers on a copy
        stream: frame f + 1's coordinates are copied in while frame f
        computes, and frame f's forces are read back while frame f + 1
        computes (two device buffers each, ordered by events).  For the
        schedules nb_run_frames does not run (a separate prune pass, a prune
        right after the build)."""
        main = torch.cuda.current_stream()
        x_ready, x_free, f_done, f_free = ev
        with torch.cuda.stream(cs):
            xbufs[0].copy_(hx[0], non_blocking=True)
            x_ready[0].record(cs)
        for f in range(nstlist):
            k = f % 2
            if f + 1 < nstlist:
                kn = (f + 1) % 2
                cs.wait_event(x_free[kn])          # frame f - 1 has read that buffer
                with torch.cuda.stream(cs):
                    xbufs[kn].copy_(hx[f + 1], non_blocking=True)
                    x_ready[kn].record(cs)
            main.wait_event(x_ready[k])
            main.wait_event(f_free[k])             # frame f - 2's forces are read back
            xf = xbufs[k]
            Fk = Fbufs[k]
            prm = prm_e if energy_frame(f) else prm_f
            if f == 0:
                nb.nb_grid_put(ctx, xf, box.box, main)
                nb.nb_pairlist_build(ctx, rlist, rbb, eo, ei, main)
            if nstprune and f % nstprune == 0 and (f > 0 or args.prune0):
                if args.fused_prune:
                    nb.nb_prune_compute(ctx, prm, xf if f > 0 else None, rprune, Fk, E, V, main)
                else:
                    nb.nb_prune(ctx, xf if f > 0 else None, rprune, main)
                    nb.nb_compute(ctx, prm, None, Fk, E, V, main)
            else:
                nb.nb_compute(ctx, prm, xf if f > 0 else None, Fk, E, V, main)
            x_free[k].record(main)
            f_done[k].record(main)
            cs.wait_event(f_done[k])
            with torch.cuda.stream(cs):
                hF[f].copy_(Fk, non_blocking=True)
                if energy_frame(f):
                    hE.copy_(E, non_blocking=True)
                f_free[k].record(cs)
        main.wait_stream(cs)

    # warm-up and a status check (capacity, coordinates)
    for _ in range(args.warmup):
        step(xs)
    info0 = nb.nb_check(ctx, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # launches of one step (counted on an eager step)
    launches0 = nb.nb_check(ctx, stream).n_launches
    step(xs)
    launches_per_step = nb.nb_check(ctx, stream).n_launches - launches0

    def capture():
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                step(xs)
        torch.cuda.current_stream().wait_stream(cs)
        torch.cuda.synchronize()
        return g

    # the step as one CUDA graph (all of its launches, no host work per kernel)
    graph = capture()
    # the same step with a pair of CUDA events around every hot-path kernel
    nb.nb_profile(ctx, True, keep=True)
    nb.nb_profile_read(ctx)
    graph_spans = capture()
    nb.nb_profile(ctx, False)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()

    # timed region: graph replays, device time per step with CUDA events
    step_ms = []
    sampler = ClockSampler(dev) if rank == 0 else None
    barrier()
    if sampler:
        sampler.start()
    gc_was = gc.isenabled()
    gc.disable()   # no collection pause between the start event and the replay
    for k in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph.replay()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    if gc_was:
        gc.enable()
    barrier()
    clocks = sampler.stop() if sampler else None
    info = nb.nb_check(ctx, stream)
    launches = launches_per_step * args.steps
    total_s = slowest_rank_seconds(sum(step_ms) / 1000.0, dist, dev)
    value = whole_job_rate(ws_n, args.steps * nstlist, total_s)

    # per-kernel device times: event spans inside replays of the same step
    # graph right after the timed region (L2 flushed before each)
    nb.nb_profile(ctx, True, keep=True)
    spans = []
    for k in range(3):
        flush.zero_()
        graph_spans.replay()
        torch.cuda.synchronize()
        spans.extend(nb.nb_profile_read(ctx))
    nb.nb_profile(ctx, False)

    # force-kernel roofline (FP32 ALU): algorithmic flops per launch / duration
    force_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_FORCE]
    prune_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_PRUNE]
    fprune_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_FORCE_PRUNE]
    final_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_FINALIZE]
    coords_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_COORDS]
    search_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_SEARCH]
    grid_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_GRID]
    pairs_outer = int(info.n_cluster_pairs) * 64
    pairs_pruned = int(info.n_cluster_pairs_pruned) * 64 if info.n_cluster_pairs_pruned >= 0 else pairs_outer
    # frames before the first prune, and fused prune frames, use the outer list
    prune_frames = [f for f in range(nstlist) if nstprune and f % nstprune == 0 and (f > 0 or args.prune0)]
    first_prune = prune_frames[0] if prune_frames else nstlist

    def listed_at(f):
        outer = f < first_prune or (args.fused_prune and f in prune_frames)
        return pairs_outer if outer else pairs_pruned
    listed_all = sum(listed_at(f) for f in range(nstlist)) / nstlist
    # the force-kernel spans: every frame but the fused prune frames (their own span kind)
    force_frames = [f for f in range(nstlist) if not (args.fused_prune and f in prune_frames)]
    listed = sum(listed_at(f) for f in force_frames) / len(force_frames)
    pairs_rc = int(info.n_pairs_rc)
    flops = FLOPS_DIST * listed + (FLOPS_PAIR[elec] - FLOPS_DIST) * pairs_rc
    t_force = statistics.mean(force_ms) / 1000.0 if force_ms else float("nan")
    pk = peaks()
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    fp32_peak = n_sm * 128 * 2 * pk["sm_max_mhz"] * 1e6
    achieved = flops / t_force
    roofline = {"bound": "alu", "kernel": "k_force8 (Ewald)" if elec == "ewald" else "k_force8 (RF)",
                "achieved": achieved / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": profiled_traffic(workload),
                "ncu": profiled_counters(workload),
                "traffic_unit": "bytes per launch (dram read + write, ncu)",
                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flops x {pk['sm_max_mhz']:.0f} MHz "
                               f"(max SM clock, {pk['source']})",
                "algorithmic_flops_per_launch": flops, "listed_pairs_per_launch": listed,
                "pairs_within_rc_per_launch": pairs_rc, "launch_ms": t_force * 1e3,
                "timing": "force-kernel spans: CUDA events recorded inside 3 replays of the timed step's "
                          "graph (captured with an event pair around every hot-path kernel), right after "
                          "the timed region"}

    out = None
    if rank == 0:
        # end to end through the C ABI with host buffers: H2D of each frame's
        # coordinates and D2H of each frame's forces (and energies) inside
        # the timed region
        hx = torch.as_tensor(frames).pin_memory()
        hF = torch.empty((nstlist, box.n, 3), dtype=torch.float32).pin_memory()
        xbufs = [torch.empty((box.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        Fbufs = [torch.empty((box.n, 3), dtype=torch.float32, device=dev) for _ in range(2)]
        cs = torch.cuda.Stream(device=dev)
        if native_e2e:
            hE = torch.zeros((nstlist, 1, 2), dtype=torch.float64).pin_memory()
            hV = torch.zeros((nstlist, 1, 9), dtype=torch.float64).pin_memory()
            Ebufs = [torch.empty((1, 2), dtype=torch.float64, device=dev) for _ in range(2)]
            Vbufs = [torch.empty((1, 9), dtype=torch.float64, device=dev) for _ in range(2)]
            run = run_host(hx, hF, hE, hV, xbufs, Fbufs, Ebufs, Vbufs)

            def host_step():
                run(torch.cuda.current_stream(), cs)
        else:
            hE = torch.empty(2, dtype=torch.float64).pin_memory()
            ev = tuple([torch.cuda.Event() for _ in range(2)] for _ in range(4))

            def host_step():
                step_host(hx, hF, hE, xbufs, Fbufs, cs, ev)
        for _ in range(2):
            host_step()
        torch.cuda.synchronize()
        e2e_ms = []
        e2e_sampler = ClockSampler(dev)
        e2e_sampler.start()
        gc_was = gc.isenabled()
        gc.disable()   # a collection pause of this process's heap would leave the GPU idle mid-step
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            host_step()
            torch.cuda.synchronize()
            e2e_ms.append(1000 * (time.perf_counter() - t0))
        if gc_was:
            gc.enable()
        e2e_clocks = e2e_sampler.stop()
        e2e_value = args.steps * nstlist / (sum(e2e_ms) / 1000.0)
        # forces read back by the last step against the device path's (same frames)
        Fd = F.double().cpu().numpy()
        e2e_check = float(np.sqrt(((hF[nstlist - 1].double().numpy() - Fd) ** 2).sum(1)).max()
                          / np.sqrt((Fd ** 2).sum(1).mean()))
        h2d = nstlist * box.n * 12
        # forces of every frame; energies (and with nb_run_frames the virial) of the energy frames
        d2h = nstlist * box.n * 12 + (sum(efr) * (16 + 72) if native_e2e else 16)
        ewald = elec == "ewald"
        cpu = cpu_baseline(box, p) if ws_n == 1 and extras else None
        surr = surrogate_ab(nb, ctx, box, p, xs, F, stream, dev) if ewald and args.surrogate and extras else None
        cmp11 = compare_1x1(nb, ctx, box, p, xs[0], F, rlist, rprune, stream) if args.compare_1x1 and extras \
            else None
        buf = buffer_estimate(nb, box, p, nstlist, rlist) if ewald and extras else None
        tab = tabulated_ab(nb, ctx, p, xs[0], F, stream) if ewald and extras else None
        pcf = pair_correlation(nb, ctx, box, xs[0], eo, ei, stream, rbb) if args.pair_correlation and extras \
            else None
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1000 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_dict(args, box, p, desc, workload),
            "pair_interactions_per_s": listed_all * nstlist * args.steps * ws_n / total_s,
            "effective_pair_interactions_per_s": pairs_rc * nstlist * args.steps * ws_n / total_s,
            "force_kernel": {"ms": t_force * 1e3, "listed_pairs_per_s": listed / t_force,
                             "pairs_within_rc_per_s": pairs_rc / t_force,
                             "effective_ratio": pairs_rc / listed if listed else None},
            "kernel_ms": {"grid": statistics.mean(grid_ms) if grid_ms else None,
                          "search": statistics.mean(search_ms) if search_ms else None,
                          "prune": statistics.mean(prune_ms) if prune_ms else None,
                          "force_prune": statistics.mean(fprune_ms) if fprune_ms else None,
                          "finalize": statistics.mean(final_ms) if final_ms else None,
                          "finalize_max": max(final_ms) if final_ms else None,
                          "set_coords": statistics.mean(coords_ms) if coords_ms else None,
                          "force": t_force * 1e3},
            "list": {"clusters": int(info.n_clusters), "superclusters": int(info.n_superclusters),
                     "ientries": int(info.n_ientries), "jentries": int(info.n_jentries),
                     "jentries_pruned": int(info.n_jentries_pruned),
                     "cluster_pairs": int(info.n_cluster_pairs),
                     "cluster_pairs_pruned": int(info.n_cluster_pairs_pruned), "r_prune_nm": rprune},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "pipeline": ("nb_run_frames, one call per list lifetime: " if native_e2e else
                                 "per-frame calls from Python: ") +
                                "each frame's coordinates copied in and forces read back on a copy stream, "
                                "overlapped with the neighbouring frames' kernels (two buffers each)",
                    "max_dF_over_rms_vs_device_path": e2e_check,
                    "step_ms_min_median_max": [min(e2e_ms), statistics.median(e2e_ms), max(e2e_ms)],
                    "step_ms": [round(t, 3) for t in e2e_ms],
                    "clocks": e2e_clocks},
            "surrogate": surr,
            "particle_pair_1x1": cmp11,
            "buffer_estimate": buf,
            "tabulated_ewald": tab,
            "pair_correlation": pcf,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "status": nb.status_name(info0.status),
        }
        if not extras:
            for k in ("cpu_baseline", "surrogate", "particle_pair_1x1", "buffer_estimate", "tabulated_ewald",
                      "pair_correlation"):
                del out[k]
    cx.close()
    del xs, flush
    torch.cuda.empty_cache()
    return out


BATCH_H = 40          # frames per batch step (a multiple of every tuned nstlist)
BATCH_UNIT = "batch force evals/s"


def batch_workload():
    from paper_1306_1737_gb300 import workloads as w
    B = w.batch_boxes(256, seed=1004)
    p = {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12, "nstlist": 20, "nstprune": 5}
    return B, p


def batch_frames(B, dev):
    """Device tensor [BATCH_H, n, 3]: a random walk of every box from its
    initial coordinates (seeded), drawn one frame at a time."""
    import torch
    from paper_1306_1737_gb300 import workloads as w
    fr = torch.empty((BATCH_H, B.n, 3), dtype=torch.float32, device=dev)
    for f, x in enumerate(w.frame_walk(B.xyz, B.mass, BATCH_H, seed=3004)):
        fr[f].copy_(torch.from_numpy(x))
    return fr


def batch_cpu_baseline(B, p, budget_s=15.0):
    """The oracle (FP64 cell-list tier) on a seeded sample: the forces of a
    seeded subset of particles in each of 8 seeded boxes; its cost per
    particle does not depend on the box size, so the sample is the fraction
    (sampled particles / all particles) of one batch evaluation."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(11)
    picks = rng.choice(B.nbox, 8, replace=False)
    b0 = B.members[int(picks[0])]
    t0 = time.perf_counter()
    oracle_eval(b0, p, sel=rng.choice(b0.n, min(256, b0.n), replace=False))
    per_atom = (time.perf_counter() - t0) / min(256, b0.n)
    m = int(max(64, budget_s / 8 / max(per_atom, 1e-9)))
    sels = [(B.members[int(k)], rng.choice(B.members[int(k)].n, min(m, B.members[int(k)].n), replace=False))
            for k in picks]
    work = sum(len(sel) for _, sel in sels)
    t0 = time.perf_counter()
    for b, sel in sels:
        oracle_eval(b, p, sel=sel)
    dt = time.perf_counter() - t0
    frac = work / B.n
    return {"value": frac / dt, "unit": BATCH_UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 cell-list forces of {work} seeded particles in 8 seeded boxes "
                      f"= {frac:.2e} of one batch evaluation"}


def run_batch(args):
    import paper_1306_1737_gb300 as nb
    dist, ws_n, rank, dev = init_ranks()
    nb.load()
    out = measure_batch(args, dist, ws_n, rank, dev)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)
    return 0


def measure_batch(args, dist, ws_n, rank, dev, sub=False):
    """The batch of 256 uneven boxes: tuned groups stepped in a CUDA graph,
    against one context for all boxes (graph) and one context per box
    (plain launches, one box after another).  sub: a block of another
    workload's line (no oracle baseline).  Returns the dict on rank 0."""
    import numpy as np
    import torch

    import paper_1306_1737_gb300 as nb
    from paper_1306_1737_gb300 import tuner
    from paper_1306_1737_gb300.batch import BatchRunner, GroupSpec

    B, p = batch_workload()
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    frames = batch_frames(B, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    common = (B.counts, B.boxes, B.q, B.types, c6c12, B.excl_off, B.excl_idx, frames)
    rc, rl0, nst0, nstprune = p["rc"], p["rlist"], p["nstlist"], p["nstprune"]

    def timed(fn, steps):
        ms = []
        gc_was = gc.isenabled()
        gc.disable()   # no collection pause between the start event and the launches
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        if gc_was:
            gc.enable()
        return ms

    def statuses(r):
        return [nb.status_name(i.status) for i in r.check()]

    # 1. autotuner (cached per GPU and batch)
    cache = os.path.join(ROOT, "paper_1306_1737_gb300", "_build", "tune_cache.json")
    t0 = time.perf_counter()
    groups, table = tuner.tune(*common, p, nstprune, rl0, nst0, cache_path=cache, device=dev.index,
                               rlist_rule=args.rlist_rule, mass=B.mass, rbb=args.rbb)
    tune_s = time.perf_counter() - t0

    # 2. tuned groups, graph
    tuned = BatchRunner(*common, groups, p, nstprune, device=dev.index, rbb=args.rbb)
    l0 = tuned.launches()
    tuned.step()
    torch.cuda.synchronize()
    launches_per_step = tuned.launches() - l0
    st_tuned = statuses(tuned)
    tuned.capture()
    for _ in range(args.warmup):
        tuned.replay()
    sampler = ClockSampler(dev) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ms_tuned = timed(tuned.replay, args.steps)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    total_s = slowest_rank_seconds(sum(ms_tuned) / 1000.0, dist, dev)
    value = whole_job_rate(ws_n, args.steps * BATCH_H, total_s)

    out = None
    if rank == 0:
        # 3. e2e through the API with host buffers (tuned groups, eager launches)
        host = []
        fr_cpu = frames.cpu()
        for g in tuned.groups:
            at = torch.as_tensor(g.atoms)
            hx = fr_cpu.index_select(1, at).contiguous().pin_memory()
            hf = torch.empty_like(hx).pin_memory()
            host.append((hx, hf))
        del fr_cpu
        tuned.step(host=host)
        torch.cuda.synchronize()
        e2e_ms = []
        e2e_sampler = ClockSampler(dev)
        e2e_sampler.start()
        gc_was = gc.isenabled()
        gc.disable()   # as for the single boxes
        for _ in range(max(1, min(args.steps, 5))):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            tuned.step(host=host)
            torch.cuda.synchronize()
            e2e_ms.append(1000 * (time.perf_counter() - t1))
        if gc_was:
            gc.enable()
        e2e_clocks = e2e_sampler.stop()
        e2e_value = len(e2e_ms) * BATCH_H / (sum(e2e_ms) / 1000.0)
        del host
    groups_info = [{"C": g.spec.C, "nstlist": g.spec.nstlist, "rlist_nm": round(g.spec.rlist, 4),
                    "nstprune": tuned.nstprune_of(g), "r_prune_nm": round(tuned.r_prune(g), 4),
                    "boxes": len(g.spec.boxes), "atoms": int(g.n)} for g in tuned.groups]
    per_box = {int(k): f"{g.spec.C}/{g.spec.nstlist}/{tuned.nstprune_of(g)}" for g in tuned.groups
               for k in g.spec.boxes}
    tuned.close()

    # 4. one context for all boxes (C = 8, nstlist 20, rlist 1.1), graph; its
    #    eager step gives the force kernel's launch times for the roofline
    one = BatchRunner(*common, [GroupSpec(8, nst0, rl0, list(range(B.nbox)))], p, nstprune, device=dev.index,
                      rbb=args.rbb)
    g1 = one.groups[0]
    nb.nb_profile(g1.cx.ctx, True)
    nb.nb_profile_read(g1.cx.ctx)
    one.step(concurrent=False)
    spans = nb.nb_profile_read(g1.cx.ctx)
    nb.nb_profile(g1.cx.ctx, False)
    info1 = nb.nb_check(g1.cx.ctx)
    one.capture(concurrent=False)
    for _ in range(args.warmup):
        one.replay()
    ms_one = timed(one.replay, args.steps)
    v_one = args.steps * BATCH_H / (sum(ms_one) / 1000.0)
    one.close()

    # 5. plain: one context per box, launches one box after another
    plain = BatchRunner(*common, [GroupSpec(8, nst0, rl0, [k]) for k in range(B.nbox)], p, nstprune,
                        device=dev.index, rbb=args.rbb)
    plain.step(concurrent=False)
    torch.cuda.synchronize()
    ms_plain = timed(lambda: plain.step(concurrent=False), max(1, min(args.steps, 3)))
    v_plain = len(ms_plain) * BATCH_H / (sum(ms_plain) / 1000.0)
    plain.close()

    if rank == 0:
        force_ms = [ms for kind, ms in spans if kind == nb.NB_KERNEL_FORCE]
        # force-kernel spans: every frame of a list lifetime but the prune
        # frames (fused force + prune, their own span kind); the frames before
        # the first prune use the outer list, the later ones the pruned list
        # (nb_check after the step reports the last list and prune)
        n_rc = int(info1.n_pairs_rc)
        outer = int(info1.n_cluster_pairs) * 64
        pruned = int(info1.n_cluster_pairs_pruned) * 64
        lf_force = [f for f in range(nst0) if not (nstprune and f > 0 and f % nstprune == 0)]
        n_out = sum(1 for f in lf_force if not nstprune or f < nstprune)
        listed = ((n_out * outer + (len(lf_force) - n_out) * pruned) / len(lf_force)) if pruned > 0 else outer
        flops = FLOPS_DIST * listed + (FLOPS_PAIR["ewald"] - FLOPS_DIST) * n_rc
        t_force = statistics.mean(force_ms) / 1000.0
        pk = peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak = n_sm * 128 * 2 * pk["sm_max_mhz"] * 1e6
        cpu = batch_cpu_baseline(B, p) if ws_n == 1 and not sub else None
        h2d = BATCH_H * B.n * 12
        out = {
            "metric": METRIC, "value": value, "unit": BATCH_UNIT, "n_gpus": ws_n, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1000 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch256",
                       "description": "256 water boxes, 1.5k-60k atoms log-uniform, Ewald rc 1.0, rlist 1.1 "
                                      "(scaled with nstlist), prune/5; a step = 40 frames of every box",
                       "n_boxes": B.nbox, "n_atoms": int(B.n), "frames_per_step": BATCH_H, "elec": "ewald",
                       "rc_nm": rc, "rlist_nm": rl0, "beta_nm-1": p["beta"], "nstlist": nst0, "nstprune": nstprune,
                       "l2": "flushed between timed steps (512 MiB write); inputs 2 GB > L2",
                       "parallelism": f"replicas x{ws_n}", "seed": 1004},
            "box_force_evals_per_s": value * B.nbox,
            "atom_force_evals_per_s": value * B.n,
            "batch": {"tuned_graph": value, "one_context_graph": v_one, "plain_per_box": v_plain,
                      "speedup_vs_plain": value / v_plain, "one_context_vs_plain": v_one / v_plain,
                      "groups": groups_info, "tuner_classes": table, "tuner_s": tune_s,
                      "per_box_choice": per_box},
            "roofline": {"bound": "alu", "kernel": "k_force8 (Ewald), one context for all 256 boxes",
                         "achieved": flops / t_force / 1e12, "peak": fp32_peak / 1e12, "unit": "TFLOP/s",
                         "frac": flops / t_force / fp32_peak, "traffic": scaled_traffic(listed / 64.0),
                         "traffic_note": "dram read + write per launch, scaled by cluster pairs from the 1M-box "
                                         "ncu capture (profiles/k_force8_water1m.md)",
                         "ncu": profiled_counters("water1m"), "listed_pairs_per_launch": listed,
                         "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flops x {pk['sm_max_mhz']:.0f} MHz "
                                        f"(max SM clock, {pk['source']})",
                         "algorithmic_flops_per_launch": flops, "launch_ms": t_force * 1e3},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": BATCH_UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                    "clocks": e2e_clocks},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
            "status": st_tuned[0] if len(set(st_tuned)) == 1 else st_tuned,
        }
    del frames, flush
    torch.cuda.empty_cache()
    return out


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rbb", type=float, default=0.8,
                    help="bounding-box distance below which the search skips the particle test (nm; <0: rlist; "
                         "0: the particle test always runs)")
    ap.add_argument("--prune0", action="store_true", help="also prune right after each list build")
    ap.add_argument("--rlist-rule", default="sqrt", choices=["sqrt", "appendix"],
                    help="batch tuner: list radius per lifetime by sqrt scaling or by the Appendix drift bound")
    ap.add_argument("--no-1x1", dest="compare_1x1", action="store_false",
                    help="skip the particle-pair (1 x 1) kernel comparison")
    ap.add_argument("--separate-prune", dest="fused_prune", action="store_false",
                    help="prune with the separate prune kernel instead of the fused force + prune pass")
    ap.add_argument("--no-rdf", dest="pair_correlation", action="store_false",
                    help="skip the pair correlation (g(r) histogram) measurement")
    ap.add_argument("--no-surrogate", dest="surrogate", action="store_false",
                    help="skip the learned Ewald factor A/B (Ewald workloads)")
    ap.add_argument("--no-sub-blocks", dest="sub_blocks", action="store_false",
                    help="water3m: skip the water24k and batch256 blocks of the line")
    ap.add_argument("--workload", default="water3m",
                    choices=["water24k", "water3m", "water1536", "water1m", "batch256"])
    return ap


def main():
    args = make_parser().parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch256":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
