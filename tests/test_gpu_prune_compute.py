"""Pruning fused into the force pass (nb_prune_compute) against the separate
prune kernel followed by a force evaluation (nb_prune + nb_compute).

The fused kernel tests the same FP32 distances against the same prune radius
and compacts the kept j-entries in the same order, so the pruned list it
writes must equal the separate prune kernel's bit for bit (i-entries,
j-words and masks), with the same per-box counts.  Its forces come from the
outer list instead of the pruned one: they must match the oracle within the
force tolerance, and the two-pass forces to summation-order rounding.  The
paths without a fused kernel (energies, 4-particle clusters) are checked the
same way."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4
ORDER_TOL = 1e-5   # two summation orders of the same FP32 pair forces, relative to the RMS force


@pytest.fixture(scope="module")
def gp():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    import gpu_path
    return gpu_path


def _pruned(gb):
    """Used part of the pruned list: per i-entry (q, s, j_begin, j_end) and
    the j-words and masks of its kept range."""
    info, ient, cj, masks, _ = gb.list_arrays(1)
    rows = []
    for e in range(ient.shape[0]):
        q, s, jb, je = (int(v) for v in ient[e])
        rows.append((q, s, jb, je, cj[jb:je].tobytes(), masks[:, jb:je].tobytes()))
    return info, rows


@pytest.mark.parametrize("C,mode,energy", [(8, "ewald", False), (8, "rf", False), (8, "ewald_tab", False),
                                           (8, "ewald", True), (4, "ewald", False)])
def test_fused_prune_equals_prune_then_compute(gp, C, mode, energy):
    import paper_1306_1737_gb300 as nb
    if mode == "rf":
        b, p = w.config1()
        p = dict(p, nstprune=5)
    else:
        b, p = w.config2()
    torch = gp.torch_dev()[0]
    gb = gp.GpuBox(b, p["rlist"], C=C)
    try:
        rl = float(np.float32(p["rlist"]))
        rp = float(np.float32(w.prune_radius(p["rc"], p["rlist"], p["nstprune"])))
        prm = nb.make_params(mode, p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                             want_energy=energy)
        gb.grid()
        gb.build(rl)
        x5 = list(w.frame_walk(b.xyz, b.mass, 6, seed=2500))[5]
        xd = torch.as_tensor(x5).to(gb.dev).contiguous()
        # two passes: prune kernel, then forces on the pruned list
        nb.nb_prune(gb.ctx, xd, rp)
        nb.nb_compute(gb.ctx, prm, None, gb.f, gb.e if energy else None, gb.vir if energy else None)
        nb.nb_check(gb.ctx)
        f_two = gb.f.cpu().numpy().astype(np.float64)
        e_two = gb.e.cpu().numpy().copy()
        info_two, rows_two = _pruned(gb)
        # one pass
        nb.nb_prune_compute(gb.ctx, prm, xd, rp, gb.f, gb.e if energy else None, gb.vir if energy else None)
        nb.nb_check(gb.ctx)
        f_one = gb.f.cpu().numpy().astype(np.float64)
        e_one = gb.e.cpu().numpy().copy()
        info_one, rows_one = _pruned(gb)
        # later evaluations use the pruned list written by the fused pass
        nb.nb_compute(gb.ctx, prm, None, gb.f, gb.e if energy else None, gb.vir if energy else None)
        nb.nb_check(gb.ctx)
        f_after = gb.f.cpu().numpy().astype(np.float64)
    finally:
        gb.close()
    assert info_one.n_jentries_pruned == info_two.n_jentries_pruned
    assert info_one.n_cluster_pairs_pruned == info_two.n_cluster_pairs_pruned
    assert rows_one == rows_two
    elec = "rf" if mode == "rf" else "ewald"
    oprm = oracle.make_params(elec, float(np.float32(p["rc"])), eps_rf=p.get("eps_rf", math.inf),
                              beta=p.get("beta", 0.0))
    fo, eo, _ = oracle.forces_cells(x5, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
    rms = math.sqrt((fo ** 2).sum(1).mean())
    for f in (f_one, f_two, f_after):
        emax = np.sqrt(((f - fo) ** 2).sum(1)).max() / rms
        assert emax < FORCE_TOL, emax
    assert np.sqrt(((f_one - f_two) ** 2).sum(1)).max() / rms < ORDER_TOL
    if energy:
        assert np.abs(e_one - e_two).max() <= 1e-6 * np.abs(e_two).max()
        assert np.abs(e_one - eo).max() / np.abs(eo).max() < 1e-5


def test_fused_prune_batch(gp):
    """Many boxes in one context: per-box pruned counts of the fused pass equal
    the prune kernel's."""
    import paper_1306_1737_gb300 as nb
    torch, dev = gp.torch_dev()
    sizes = [500, 1300, 620, 2400, 800]
    B = w.concat([w.water_box(m, None, seed=7300 + k) for k, m in enumerate(sizes)])
    rl, rp = float(np.float32(1.1)), float(np.float32(w.prune_radius(1.0, 1.1, 5)))
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    prm = nb.make_params("ewald", 1.0, beta=3.12, want_energy=False)
    x1 = np.concatenate([list(w.frame_walk(b.xyz, b.mass, 6, seed=7400 + k))[5]
                         for k, b in enumerate(B.members)]).astype(np.float32)
    cx = nb.Context(B.counts, B.boxes, rl, B.q, B.types, c6c12)
    try:
        ctx = cx.ctx
        f = torch.zeros((B.n, 3), dtype=torch.float32, device=dev)
        nb.nb_grid_put(ctx, torch.as_tensor(B.xyz, device=dev), B.boxes)
        nb.nb_pairlist_build(ctx, rl, 0.0, torch.as_tensor(B.excl_off, device=dev),
                             torch.as_tensor(B.excl_idx, device=dev))
        xd = torch.as_tensor(x1, device=dev)
        nb.nb_prune(ctx, xd, rp)
        nb.nb_check(ctx)
        two = [nb.nb_box_info(ctx, k) for k in range(B.nbox)]
        nb.nb_prune_compute(ctx, prm, xd, rp, f)
        nb.nb_check(ctx)
        one = [nb.nb_box_info(ctx, k) for k in range(B.nbox)]
        fg = f.cpu().numpy().astype(np.float64)
    finally:
        cx.close()
    off = B.offsets
    oprm = oracle.make_params("ewald", float(np.float32(1.0)), beta=3.12)
    for k, b in enumerate(B.members):
        assert one[k].n_jentries_pruned == two[k].n_jentries_pruned
        assert one[k].n_cluster_pairs_pruned == two[k].n_cluster_pairs_pruned
        sl = slice(int(off[k]), int(off[k + 1]))
        fo, _, _ = oracle.forces_brute(x1[sl], b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        rms = math.sqrt((fo ** 2).sum(1).mean())
        assert np.sqrt(((fg[sl] - fo) ** 2).sum(1)).max() / rms < FORCE_TOL


def test_prune_compute_errors(gp):
    import paper_1306_1737_gb300 as nb
    b, p = w.config1()
    gb = gp.GpuBox(b, p["rlist"])
    try:
        prm = nb.make_params("rf", p["rc"])
        with pytest.raises(nb.NbError) as ei:
            nb.nb_prune_compute(gb.ctx, prm, None, 0.95, gb.f)       # no grid or list yet
        assert ei.value.status == nb.NB_ERR_STATE
        gb.grid()
        gb.build(float(np.float32(p["rlist"])))
        for rp, st in ((0.0, nb.NB_ERR_ARG), (0.85, nb.NB_ERR_BOX), (1.3, nb.NB_ERR_BOX)):
            with pytest.raises(nb.NbError) as ei:
                nb.nb_prune_compute(gb.ctx, prm, None, rp, gb.f)    # rp <= 0, below rc, above half the box
            assert ei.value.status == st, rp
        nb.nb_check(gb.ctx)
    finally:
        gb.close()


def test_compute_radius_after_a_wide_prune(gp):
    """A prune at a radius above the list's keeps every listed pair; the list
    still holds only the pairs within rlist, so a cut-off between rlist and
    that prune radius is refused."""
    import paper_1306_1737_gb300 as nb
    b, p = w.config1()
    gb = gp.GpuBox(b, p["rlist"])
    try:
        gb.grid()
        gb.build(0.95)
        nb.nb_prune(gb.ctx, None, 1.2)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_compute(gb.ctx, nb.make_params("rf", 1.0), None, gb.f)
        assert ei.value.status == nb.NB_ERR_BOX
        nb.nb_compute(gb.ctx, nb.make_params("rf", 0.9), None, gb.f)
        nb.nb_check(gb.ctx)
    finally:
        gb.close()
