"""Batched step over many independent boxes (argument marshalling and launch
order only; every computation runs in the library's kernels).

Boxes are split into groups; each group is one context (one cluster size C
and one list lifetime nstlist with its list radius), so every kernel of the
step covers all boxes of a group in one launch (Sec. 2.3: the GPU needs tens
of thousands of particles per launch to fill up; Sec. 4 reports the
drop-off for small systems).  A step is a horizon of H frames; group g
rebuilds its grid and list every nstlist_g frames (H a multiple of each),
prunes every nstprune_g frames in between (fused into that frame's force
pass) and evaluates forces every frame.
Groups run on their own CUDA streams, forked from and joined to the caller's
stream, so small groups overlap; the whole step can be captured once in a
CUDA graph and replayed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import paper_1306_1737_gb300 as nb


@dataclass
class GroupSpec:
    C: int                   # cluster size (4 or 8)
    nstlist: int             # frames per list lifetime
    rlist: float             # list radius (nm)
    boxes: list = field(default_factory=list)   # batch box indices
    nstprune: int | None = None   # frames between prunes (None: the runner's)


def scaled_rlist(rc: float, rlist0: float, nstlist0: int, nstlist: int) -> float:
    """List radius for another list lifetime: the buffer rlist0 - rc, chosen
    for nstlist0 frames, scaled by sqrt(nstlist / nstlist0) (the spread of a
    diffusive displacement grows with the square root of the time)."""
    return rc + (rlist0 - rc) * math.sqrt(nstlist / nstlist0)


def _subset_csr(excl_off, excl_idx, atom_off, boxes):
    """Exclusion CSR of the given boxes (batch-global partner indices mapped
    to the subset's indices)."""
    offs, idxs = [np.zeros(1, np.int64)], []
    base_e, base_a = 0, 0
    for k in boxes:
        a0, a1 = int(atom_off[k]), int(atom_off[k + 1])
        e0, e1 = int(excl_off[a0]), int(excl_off[a1])
        offs.append(excl_off[a0 + 1:a1 + 1].astype(np.int64) - e0 + base_e)
        idxs.append(excl_idx[e0:e1].astype(np.int64) - a0 + base_a)
        base_e += e1 - e0
        base_a += a1 - a0
    return (np.concatenate(offs).astype(np.int32),
            (np.concatenate(idxs) if idxs else np.zeros(0)).astype(np.int32))


class _Group:
    def __init__(self, spec, counts, boxes, atom_off, q, types, c6c12, excl_off, excl_idx, frames,
                 device, list_factor):
        import torch
        self.spec = spec
        idx = np.asarray(spec.boxes, dtype=np.int64)
        self.box_index = idx
        self.atoms = np.concatenate([np.arange(atom_off[k], atom_off[k + 1]) for k in idx]) \
            if idx.size else np.zeros(0, np.int64)
        dev = torch.device("cuda", device)
        self.cx = nb.Context(counts[idx], boxes[idx], spec.rlist, q[self.atoms], types[self.atoms], c6c12,
                             cluster_size=spec.C, device=device, list_factor=list_factor)
        self.boxes = np.ascontiguousarray(boxes[idx])
        eo, ei = _subset_csr(excl_off, excl_idx, atom_off, idx)
        self.excl_off = torch.as_tensor(eo, device=dev)
        self.excl_idx = torch.as_tensor(ei, device=dev)
        at = torch.as_tensor(self.atoms, device=dev)
        # this group's particles of every frame (gathered once, before any step)
        self.frames = frames.index_select(1, at).contiguous() if frames is not None else None
        n = int(self.atoms.size)
        self.n = n
        self.F = torch.zeros((n, 3), dtype=torch.float32, device=dev)
        self.E = torch.zeros((idx.size, 2), dtype=torch.float64, device=dev)
        self.V = torch.zeros((idx.size, 9), dtype=torch.float64, device=dev)
        self.stream = torch.cuda.Stream(device=dev)

    def close(self):
        self.cx.close()


class BatchRunner:
    """Groups of boxes stepped together over a horizon of H frames.

    frames: device tensor [H, n, 3] of the batch's coordinates per frame
    (batch order); counts/boxes: particles and edges per box; q, types,
    excl_off/excl_idx: batch arrays (exclusion partners batch-global)."""

    def __init__(self, counts, boxes, q, types, c6c12, excl_off, excl_idx, frames, groups,
                 params, nstprune, device=0, list_factor=0.0, rbb=0.0):
        import torch
        self.torch = torch
        self.rbb = float(rbb)   # Fig. 3's bounding-box shortcut radius of the list builds (nm)
        self.counts = np.asarray(counts, dtype=np.int64)
        self.boxes = np.asarray(boxes, dtype=np.float64).reshape(-1, 3)
        self.atom_off = np.concatenate([[0], np.cumsum(self.counts)])
        self.H = int(frames.shape[0])
        for g in groups:
            if self.H % g.nstlist:
                raise ValueError("the horizon must be a multiple of every group's nstlist")
        self.params = params
        self.nstprune = int(nstprune)
        self.groups = [_Group(g, self.counts, self.boxes, self.atom_off, np.asarray(q), np.asarray(types),
                              c6c12, np.asarray(excl_off), np.asarray(excl_idx), frames, device, list_factor)
                       for g in groups if g.boxes]
        self.graph = None

    def nstprune_of(self, g):
        return self.nstprune if g.spec.nstprune is None else int(g.spec.nstprune)

    def r_prune(self, g):
        from paper_1306_1737_gb300 import workloads as w
        nsp = self.nstprune_of(g)
        return w.prune_radius(self.params["rc"], g.spec.rlist, nsp) if nsp else g.spec.rlist

    def _frame_ops(self, g, f, x, stream, F=None):
        """Launches of group g at frame f (coordinates x, a device tensor;
        forces into F, default the group's buffer)."""
        p = self.params
        lf = f % g.spec.nstlist
        energy = f == 0 or f == self.H - 1
        prm = nb.make_params(p["elec"], p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                             want_energy=energy)
        ctx = g.cx.ctx
        F = g.F if F is None else F
        if lf == 0:
            nb.nb_grid_put(ctx, x, g.boxes, stream)
            rl = float(np.float32(g.spec.rlist))
            nb.nb_pairlist_build(ctx, rl, rl if self.rbb < 0 else min(self.rbb, rl), g.excl_off, g.excl_idx,
                                 stream)
            nb.nb_compute(ctx, prm, None, F, g.E, g.V, stream)
        elif self.nstprune_of(g) and lf % self.nstprune_of(g) == 0:
            # prune while computing this frame's forces on the outer list
            nb.nb_prune_compute(ctx, prm, x, float(np.float32(self.r_prune(g))), F, g.E, g.V, stream)
        else:
            nb.nb_compute(ctx, prm, x, F, g.E, g.V, stream)

    def step(self, concurrent=True, host=None):
        """One horizon of H frames for every group.  concurrent: each group
        on its own stream (forked from and joined to the current stream),
        else all groups one after another on the current stream.  host: per
        group (pinned frames [H, n_g, 3], pinned forces [H, n_g, 3]) -- each
        frame's coordinates are copied in and its forces copied out inside
        the step, on a copy stream per group and with two device buffers of
        each, so the transfers overlap the neighbouring frames' kernels."""
        torch = self.torch
        main = torch.cuda.current_stream()
        fork = torch.cuda.Event()
        fork.record(main)
        for gi, g in enumerate(self.groups):
            st = g.stream if concurrent else main
            if concurrent:
                st.wait_event(fork)
            with torch.cuda.stream(st):
                if host is None:
                    for f in range(self.H):
                        self._frame_ops(g, f, g.frames[f], st)
                else:
                    self._host_frames(g, host[gi], st)
            if concurrent:
                join = torch.cuda.Event()
                join.record(st)
                main.wait_event(join)

    def _host_frames(self, g, host, st):
        """The H frames of group g from pinned host frames to pinned host
        forces, one nb_run_frames call per list lifetime: frame f + 1's
        coordinates are copied in while frame f computes and frame f's forces
        are read back while frame f + 1 computes (copy stream, two buffers
        each, ordered by events the context owns)."""
        torch = self.torch
        hx, hf = host
        if not hasattr(g, "pipe"):
            dev = g.F.device
            g.pipe = {"cs": torch.cuda.Stream(device=dev),
                      "x": [torch.empty_like(g.F) for _ in range(2)],
                      "F": [torch.empty_like(g.F) for _ in range(2)]}
        cs, xb, Fb = g.pipe["cs"], g.pipe["x"], g.pipe["F"]
        p = self.params
        prm = nb.make_params(p["elec"], p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                             want_energy=False)
        rl = float(np.float32(g.spec.rlist))
        n_life = g.spec.nstlist
        nsp = self.nstprune_of(g)
        runs = g.pipe.setdefault("runs", {})   # marshalled arguments per host buffer and lifetime
        for f0 in range(0, self.H, n_life):
            key = (hx.data_ptr(), hf.data_ptr(), f0)
            if key not in runs:
                frames = range(f0, f0 + n_life)
                runs[key] = nb.RunFrames(g.cx.ctx, prm, hx[f0:f0 + n_life], hf[f0:f0 + n_life], xb, Fb,
                                         nbox=len(g.boxes), energy_frames=[f == 0 or f == self.H - 1 for f in frames],
                                         build=True, boxes=g.boxes, rlist=rl,
                                         rbb=rl if self.rbb < 0 else min(self.rbb, rl), excl_off=g.excl_off,
                                         excl_idx=g.excl_idx, nstprune=nsp, r_prune=float(np.float32(self.r_prune(g))))
            runs[key](st, cs)

    def capture(self, concurrent=True):
        """Capture one step in a CUDA graph (after an eager step has set up
        the box geometry and kernel attributes)."""
        torch = self.torch
        self.step(concurrent)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.step(concurrent)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def check(self):
        """nb_check of every group; returns the list of nb_info."""
        return [nb.nb_check(g.cx.ctx, g.stream) for g in self.groups]

    def launches(self):
        return sum(nb.nb_check(g.cx.ctx, g.stream).n_launches for g in self.groups)

    def close(self):
        for g in self.groups:
            g.close()
        self.groups = []
        self.graph = None
