"""Many boxes in one context: every kernel handles all boxes in one launch.

Per box, the batched result must equal what the oracle gives for that box
alone (forces within 1e-4 of the RMS force, energies and virial within 1e-5
relative), and the batched lists must hold exactly the cluster pairs that a
one-box context finds for the same box (counts equal per box).  An empty box
and boxes of very different sizes are part of the batch."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4
E_TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    return torch, torch.device("cuda", 0), nb


def _empty_like(b, L):
    return w.Box(xyz=np.zeros((0, 3), np.float32), q=np.zeros(0, np.float32),
                 types=np.zeros(0, np.int32), sigma=b.sigma.copy(), eps=b.eps.copy(),
                 mass=np.zeros(0), excl_off=np.zeros(1, np.int32), excl_idx=np.zeros(0, np.int32),
                 box=np.array([L, L, L]))


def _batch():
    sizes = [500, 1300, 620, 2400, 800]
    boxes = [w.water_box(m, None, seed=7000 + k) for k, m in enumerate(sizes)]
    boxes.insert(2, _empty_like(boxes[0], 2.6))
    return w.concat(boxes)


@pytest.mark.parametrize("C", [8, 4])
def test_batch_matches_single_boxes_and_oracle(env, C):
    torch, dev, nb = env
    B = _batch()
    rc, rl, beta, nstprune = 1.0, 1.1, 3.12, 5
    rlf = float(np.float32(rl))
    rp = float(np.float32(w.prune_radius(rc, rl, nstprune)))
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    prm = nb.make_params("ewald", rc, beta=beta)
    oprm = oracle.make_params("ewald", float(np.float32(rc)), beta=beta)
    disp = np.concatenate([w.frame_displacements(b.mass, nstprune, seed=8000 + k).sum(0)
                           if b.n else np.zeros((0, 3), np.float32)
                           for k, b in enumerate(B.members)]).astype(np.float32)
    x1 = (B.xyz + disp).astype(np.float32)

    cx = nb.Context(B.counts, B.boxes, rl, B.q, B.types, c6c12, cluster_size=C)
    try:
        ctx = cx.ctx
        nbx = B.nbox
        f = torch.zeros((B.n, 3), dtype=torch.float32, device=dev)
        e = torch.zeros((nbx, 2), dtype=torch.float64, device=dev)
        vir = torch.zeros((nbx, 9), dtype=torch.float64, device=dev)
        nb.nb_grid_put(ctx, torch.as_tensor(B.xyz, device=dev), B.boxes)
        nb.nb_pairlist_build(ctx, rlf, 0.0, torch.as_tensor(B.excl_off, device=dev),
                             torch.as_tensor(B.excl_idx, device=dev))
        nb.nb_check(ctx)
        outer = [nb.nb_box_info(ctx, k) for k in range(nbx)]
        nb.nb_compute(ctx, prm, None, f, e, vir)
        tot = nb.nb_check(ctx)
        assert tot.n_boxes == nbx and tot.n_atoms == B.n
        f0, e0, v0 = f.cpu().numpy().astype(np.float64), e.cpu().numpy(), vir.cpu().numpy()
        nb.nb_prune(ctx, torch.as_tensor(x1, device=dev), rp)
        nb.nb_check(ctx)
        pruned = [nb.nb_box_info(ctx, k) for k in range(nbx)]
        nb.nb_compute(ctx, prm, None, f, e, vir)
        nb.nb_check(ctx)
        f1, e1, v1 = f.cpu().numpy().astype(np.float64), e.cpu().numpy(), vir.cpu().numpy()
    finally:
        cx.close()

    off = B.offsets
    for k, b in enumerate(B.members):
        sl = slice(int(off[k]), int(off[k + 1]))
        assert outer[k].atom_offset == off[k] and outer[k].n_atoms == b.n
        if b.n == 0:
            assert outer[k].n_clusters == 0 and outer[k].n_cluster_pairs == 0
            assert np.all(e0[k] == 0.0) and np.all(v0[k] == 0.0)
            continue
        # the same box alone in a one-box context: identical list sizes
        one = nb.Context(b.n, b.box, rl, b.q, b.types, c6c12, cluster_size=C)
        try:
            nb.nb_grid_put(one.ctx, torch.as_tensor(b.xyz, device=dev), b.box)
            nb.nb_pairlist_build(one.ctx, rlf, 0.0, torch.as_tensor(b.excl_off, device=dev),
                                 torch.as_tensor(b.excl_idx, device=dev))
            i1 = nb.nb_check(one.ctx)
            nb.nb_prune(one.ctx, torch.as_tensor(x1[sl], device=dev), rp)
            i2 = nb.nb_check(one.ctx)
        finally:
            one.close()
        assert outer[k].n_clusters == i1.n_clusters
        assert outer[k].n_cluster_pairs == i1.n_cluster_pairs
        # (i-entry counts depend on how the search splits its work, the list's content does not)
        assert outer[k].n_jentries == i1.n_jentries
        assert outer[k].n_ientries >= (outer[k].n_jentries + 31) // 32
        assert pruned[k].n_cluster_pairs_pruned == i2.n_cluster_pairs_pruned
        assert pruned[k].n_jentries_pruned == i2.n_jentries_pruned
        # forces, energies and virial of this box against the oracle
        for x, fg, eg, vg in ((b.xyz, f0, e0, v0), (x1[sl], f1, e1, v1)):
            fo, eo, vo = oracle.forces_brute(x, b.q, b.types, b.sigma, b.eps, b.excl_off,
                                             b.excl_idx, b.box, oprm)
            rms = math.sqrt((fo ** 2).sum(1).mean())
            emax = np.sqrt(((fg[sl] - fo) ** 2).sum(1)).max() / rms
            assert emax < FORCE_TOL, (k, emax)
            assert np.abs(eg[k] - eo).max() / np.abs(eo).max() < E_TOL, (k, eg[k], eo)
            assert np.abs(vg[k].reshape(3, 3) - vo).max() / np.abs(vo).max() < E_TOL, k


def test_batch_box_change_and_errors(env):
    """Box edges may change between nb_grid_put calls within the planned
    capacity; a coordinate outside its own box's range is flagged for that
    box; a list radius above half of any box edge is refused."""
    torch, dev, nb = env
    boxes = [w.water_box(600, None, seed=7100), w.water_box(900, None, seed=7101)]
    B = w.concat(boxes)
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    cx = nb.Context(B.counts, B.boxes, 1.0, B.q, B.types, c6c12)
    try:
        ctx = cx.ctx
        x = torch.as_tensor(B.xyz, device=dev)
        nb.nb_grid_put(ctx, x, B.boxes * 1.01)
        nb.nb_check(ctx)
        bad = B.xyz.copy()
        bad[B.counts[0] + 7, 2] = 3.0 * B.boxes[1, 2]
        nb.nb_grid_put(ctx, torch.as_tensor(bad, device=dev), B.boxes)
        info = nb.nb_check(ctx, raise_on_error=False)
        assert info.status == nb.NB_ERR_COORD
        assert nb.nb_box_info(ctx, 1).flags & (1 << nb.NB_ERR_COORD)
        assert not nb.nb_box_info(ctx, 0).flags
        assert "box 1" in nb.nb_last_error(ctx)
        nb.nb_grid_put(ctx, x, B.boxes)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pairlist_build(ctx, float(0.5 * B.boxes[:, 0].min() + 0.01))
        assert ei.value.status == nb.NB_ERR_BOX
        with pytest.raises(nb.NbError) as ei:
            nb.nb_box_info(ctx, 2)
        assert ei.value.status == nb.NB_ERR_ARG
    finally:
        cx.close()


@pytest.mark.parametrize("rbb", [0.0, 0.8])
def test_batch_runner_groups_graph(env, rbb):
    """Two groups (C = 8 with nstlist 10 pruning every 2 frames, C = 4 with
    nstlist 20 pruning every 5) stepped over
    20 frames on their own streams and captured in a CUDA graph: after a
    replay, every box's last-frame forces and energies match the oracle.
    rbb: the lists' bounding-box shortcut radius (0.8 nm, as the bench)."""
    torch, dev, nb = env
    from paper_1306_1737_gb300.batch import BatchRunner, GroupSpec, scaled_rlist
    boxes = [w.water_box(m, None, seed=7200 + k) for k, m in enumerate([520, 900, 610, 1400])]
    B = w.concat(boxes)
    p = {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12}
    H = 20
    fr = torch.stack([torch.from_numpy(x) for x in w.frame_walk(B.xyz, B.mass, H, seed=7300)]).to(dev)
    groups = [GroupSpec(8, 10, scaled_rlist(1.0, 1.1, 20, 10), [0, 2], nstprune=2),
              GroupSpec(4, 20, 1.1, [1, 3])]
    r = BatchRunner(B.counts, B.boxes, B.q, B.types, nb.nb_lj_combine(B.sigma, B.eps), B.excl_off,
                    B.excl_idx, fr, groups, p, nstprune=5, rbb=rbb)
    try:
        r.capture()
        for g in r.groups:
            g.F.zero_()
            g.E.zero_()
        r.replay()
        torch.cuda.synchronize()
        assert all(i.status == 0 for i in r.check())
        xl = fr[H - 1].cpu().numpy()
        oprm = oracle.make_params("ewald", float(np.float32(1.0)), beta=3.12)
        off = B.offsets
        for g in r.groups:
            F = g.F.cpu().numpy().astype(np.float64)
            E = g.E.cpu().numpy()
            o = 0
            for j, k in enumerate(g.box_index):
                b = B.members[k]
                x = xl[int(off[k]):int(off[k + 1])]
                fo, eo, _ = oracle.forces_brute(x, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx,
                                                b.box, oprm)
                rms = math.sqrt((fo ** 2).sum(1).mean())
                emax = np.sqrt(((F[o:o + b.n] - fo) ** 2).sum(1)).max() / rms
                assert emax < FORCE_TOL, (k, emax)
                assert np.abs(E[j] - eo).max() / np.abs(eo).max() < E_TOL, (k, E[j], eo)
                o += b.n
    finally:
        r.close()


def test_batch_runner_host_pipeline(env):
    """The host path (frames copied in and forces read back on a copy stream,
    two device buffers each): every frame's forces read back into host memory
    match the oracle for that frame's coordinates, so no frame used a buffer
    still being filled or read a force buffer already reused."""
    torch, dev, nb = env
    from paper_1306_1737_gb300.batch import BatchRunner, GroupSpec
    boxes = [w.water_box(m, None, seed=7500 + k) for k, m in enumerate([600, 1100])]
    B = w.concat(boxes)
    p = {"elec": "ewald", "rc": 1.0, "rlist": 1.1, "beta": 3.12}
    H = 10
    frames = list(w.frame_walk(B.xyz, B.mass, H, seed=7600))
    fr = torch.stack([torch.from_numpy(x) for x in frames]).to(dev)
    r = BatchRunner(B.counts, B.boxes, B.q, B.types, nb.nb_lj_combine(B.sigma, B.eps), B.excl_off,
                    B.excl_idx, fr, [GroupSpec(8, 10, 1.1, [0, 1], nstprune=3)], p, nstprune=5)
    try:
        g = r.groups[0]
        at = torch.as_tensor(g.atoms)
        hx = fr.cpu().index_select(1, at).contiguous().pin_memory()
        hf = torch.zeros_like(hx).pin_memory()
        r.step(host=[(hx, hf)])
        torch.cuda.synchronize()
        assert all(i.status == 0 for i in r.check())
        oprm = oracle.make_params("ewald", float(np.float32(1.0)), beta=3.12)
        off = B.offsets
        for f in (0, 1, 3, 4, 8, 9):
            F = hf[f].numpy().astype(np.float64)
            o = 0
            for k in g.box_index:
                b = B.members[k]
                x = frames[f][int(off[k]):int(off[k + 1])]
                fo, _, _ = oracle.forces_brute(x, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
                rms = math.sqrt((fo ** 2).sum(1).mean())
                emax = np.sqrt(((F[o:o + b.n] - fo) ** 2).sum(1)).max() / rms
                assert emax < FORCE_TOL, (f, k, emax)
                o += b.n
    finally:
        r.close()
