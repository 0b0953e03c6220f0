"""GPU parity against the FP64 oracle, through the C ABI.

Grid ordering and exclusion masks bit-exact; cluster-pair lists equal as
canonical key sets (keys whose minimum particle distance is within 1e-6 nm
of the list radius exempt); forces within 1e-4 of the RMS force (max over
particles); energies and virial reported and bounded by 1e-5 relative."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4   # max |dF| / RMS |F|  (required force accuracy)
EXEMPT_NM = 1e-6   # list keys this close to the threshold may differ
E_TOL = 1e-5       # relative error of FP64 totals of FP32 pair terms


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


def check_grid(g_gpu, g_or):
    assert g_gpu["info"].nx == g_or.nx and g_gpu["info"].ny == g_or.ny
    # super-clusters: runs of up to S consecutive clusters of each column
    S = g_gpu["info"].super_size
    want = []
    cs = g_or.col_clu_start
    for c in range(len(cs) - 1):
        for f in range(cs[c], cs[c + 1], S):
            want.append((f, min(S, cs[c + 1] - f)))
    assert [tuple(x) for x in g_gpu["sc_info"].tolist()] == want
    assert g_gpu["info"].n_clusters == g_or.nclu
    assert np.array_equal(g_gpu["col_clu_start"], g_or.col_clu_start)
    assert np.array_equal(g_gpu["col_of_atom"], g_or.col_of_atom)
    assert np.array_equal(g_gpu["atom_of_slot"], g_or.atom_of_slot)
    assert np.array_equal(g_gpu["slot_of_atom"], g_or.slot_of_atom)
    assert np.array_equal(g_gpu["type_slot"], g_or.type_slot)
    # bit-exact float data
    assert np.array_equal(g_gpu["xyzq"].view(np.uint32), g_or.xyzq.view(np.uint32))
    assert np.array_equal(g_gpu["bb"].view(np.uint32), g_or.bb.view(np.uint32))


def check_list(gb, g_or, pl_or, rlist, which=0, r_thresh=None, xyzq=None):
    """Compare the GPU list (which = 0 outer, 1 pruned) with the oracle's keys;
    differing keys must lie within EXEMPT_NM of the threshold (the list
    radius, or for the pruned list the prune radius under xyzq)."""
    gp_ = __import__("gpu_path")
    info, ient, cj, masks, sci = gb.list_arrays(which)
    keys_gpu, dup = gp_.canonical_keys(ient, cj, masks, sci)
    assert dup == 0
    keys_or = pl_or.key_mask()
    only_gpu = set(keys_gpu) - set(keys_or)
    only_or = set(keys_or) - set(keys_gpu)
    r = rlist if r_thresh is None else r_thresh
    for ks in (only_gpu, only_or):
        if ks:
            a = np.array([k[0] for k in ks], np.int32)
            b = np.array([k[1] for k in ks], np.int32)
            s = np.array([k[2] for k in ks], np.int32)
            if which == 0:
                dm, _ = oracle.key_distances(g_or, a, b, s, xyzq)
            else:
                _, dm = oracle.prune(g_or, oracle.PairList(a, b, s, np.zeros(a.size, np.uint64)),
                                     r, xyzq)
            assert np.all(np.abs(dm - r) < EXEMPT_NM), (len(ks), dm[np.abs(dm - r) >= EXEMPT_NM][:5])
    common = set(keys_gpu) & set(keys_or)
    bad = [k for k in common if keys_gpu[k] != keys_or[k]]
    assert not bad, bad[:5]
    # j-lists are chunked: each i-entry holds at most 32 j-entries
    assert np.all(ient[:, 3] - ient[:, 2] <= 32)
    # every stored j-entry interacts with at least one i-cluster
    lens = ient[:, 3] - ient[:, 2]
    used = np.concatenate([np.arange(b0, b1) for b0, b1 in ient[:, 2:4]]) if len(ient) else np.zeros(0, int)
    assert np.all((cj[used].astype(np.int64) & 0xFFFFFFFF) >> gp_.SUPER_SHIFT != 0)
    return len(keys_gpu), len(only_gpu) + len(only_or)


@pytest.mark.parametrize("C", [8, 4])
def test_config1_grid_list_forces_rf(gp, cfg1, C):
    b, p = cfg1
    gb = gp.GpuBox(b, p["rlist"], C=C)
    try:
        gb.grid()
        g_or = oracle.grid(b.xyz, b.q, b.types, b.box, C)
        check_grid(gb.grid_arrays(), g_or)
        rl = float(np.float32(p["rlist"]))
        gb.build(rl)
        pl = oracle.pairlist(g_or, rl, 0.0, b.excl_off, b.excl_idx)
        check_list(gb, g_or, pl, rl)
        import paper_1306_1737_gb300 as nb
        prm = nb.make_params("rf", p["rc"], eps_rf=math.inf)
        f, e, vir = gb.compute(prm)
        fo, eo, vo = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off,
                                         b.excl_idx, b.box, oracle.make_params("rf", float(np.float32(p["rc"]))))
        emax, erms, rms = gp.force_errors(f, fo)
        assert emax < FORCE_TOL, (emax, erms)
        assert np.abs(e - eo).max() / np.abs(eo).max() < E_TOL, (e, eo)
        assert np.abs(vir - vo).max() / np.abs(vo).max() < E_TOL, (vir, vo)
    finally:
        gb.close()


def test_config2_grid_list_prune_forces_ewald(gp, cfg2):
    b, p = cfg2
    gb = gp.GpuBox(b, p["rlist"])
    try:
        gb.grid()
        g_or = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
        check_grid(gb.grid_arrays(), g_or)
        rl = float(np.float32(p["rlist"]))
        gb.build(rl)
        pl = oracle.pairlist(g_or, rl, 0.0, b.excl_off, b.excl_idx)
        nkeys, nex = check_list(gb, g_or, pl, rl)
        assert nkeys > 0.9 * len(pl)
        import paper_1306_1737_gb300 as nb
        prm = nb.make_params("ewald", p["rc"], beta=p["beta"])
        oprm = oracle.make_params("ewald", float(np.float32(p["rc"])), beta=p["beta"])
        f, e, vir = gb.compute(prm)
        fo, eo, vo = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off,
                                         b.excl_idx, b.box, oprm)
        emax, erms, rms = gp.force_errors(f, fo)
        assert emax < FORCE_TOL, (emax, erms)
        assert np.abs(e - eo).max() / np.abs(eo).max() < E_TOL, (e, eo)
        assert np.abs(vir - vo).max() / np.abs(vo).max() < E_TOL
        # prune at a radius after moving the particles
        disp = w.frame_displacements(b.mass, 5, seed=2002).sum(0)
        x5 = b.xyz + disp
        rp = float(np.float32(w.prune_radius(p["rc"], p["rlist"], p["nstprune"])))
        gb.prune(rp, x5)
        x5s = oracle.slot_coords(g_or, x5)
        keep, dmin = oracle.prune(g_or, pl, rp, x5s)
        kept = oracle.PairList(pl.a[keep], pl.b[keep], pl.s[keep], pl.mask[keep])
        check_list(gb, g_or, kept, rl, which=1, r_thresh=rp, xyzq=x5s)
        f5, e5, v5 = gb.compute(prm)
        fo5, eo5, vo5 = oracle.forces_brute(x5, b.q, b.types, b.sigma, b.eps, b.excl_off,
                                            b.excl_idx, b.box, oprm)
        emax, erms, _ = gp.force_errors(f5, fo5)
        assert emax < FORCE_TOL, (emax, erms)
        assert np.abs(e5 - eo5).max() / np.abs(eo5).max() < E_TOL
    finally:
        gb.close()


def test_small_boxes_multiple_images(gp):
    # boxes barely above 2 rlist: cluster pairs in range under two shifts
    import paper_1306_1737_gb300 as nb
    for nmol, L, rl in ((70, 2.05, 1.0), (100, 1.45, 0.7)):
        b = w.water_box(nmol, L, seed=nmol)
        gb = gp.GpuBox(b, rl)
        try:
            gb.grid()
            g_or = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
            check_grid(gb.grid_arrays(), g_or)
            rlf = float(np.float32(rl))
            gb.build(rlf)
            pl = oracle.pairlist(g_or, rlf, 0.0, b.excl_off, b.excl_idx)
            check_list(gb, g_or, pl, rlf)
            rc = rl - 0.05
            f, e, vir = gb.compute(nb.make_params("ewald", rc, beta=3.12))
            fo, eo, vo = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off,
                                             b.excl_idx, b.box,
                                             oracle.make_params("ewald", float(np.float32(rc)), beta=3.12))
            emax, _, _ = gp.force_errors(f, fo)
            assert emax < FORCE_TOL
            assert np.abs(e - eo).max() / np.abs(eo).max() < E_TOL
        finally:
            gb.close()


def test_rbb_shortcut(gp, cfg1):
    b, p = cfg1
    gb = gp.GpuBox(b, p["rlist"])
    try:
        gb.grid()
        g_or = oracle.grid(b.xyz, b.q, b.types, b.box, 8)
        rl, rbb = float(np.float32(1.0)), float(np.float32(0.5))
        gb.build(rl, rbb)
        pl = oracle.pairlist(g_or, rl, rbb, b.excl_off, b.excl_idx)
        check_list(gb, g_or, pl, rl)
    finally:
        gb.close()


def test_error_paths(gp, cfg1):
    import paper_1306_1737_gb300 as nb
    b, p = cfg1
    gb = gp.GpuBox(b, 0.45)
    try:
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pairlist_build(gb.ctx, 1.0)
        assert ei.value.status == nb.NB_ERR_STATE
        gb.grid()
        with pytest.raises(nb.NbError) as ei:
            nb.nb_pairlist_build(gb.ctx, 1.3)      # >= L/2
        assert ei.value.status == nb.NB_ERR_BOX
        # list capacity sized for 0.45 nm, built at 1.2 nm: device overflow flag
        nb.nb_pairlist_build(gb.ctx, 1.2, 0.0, gb.excl_off, gb.excl_idx)
        info = nb.nb_check(gb.ctx, raise_on_error=False)
        assert info.status == nb.NB_ERR_CAPACITY
        # a coordinate outside [-L, 2L)
        bad = b.xyz.copy()
        bad[5, 1] = 3.5 * b.box[1]
        nb.nb_grid_put(gb.ctx, gb.torch.as_tensor(bad).to(gb.dev), b.box)
        info = nb.nb_check(gb.ctx, raise_on_error=False)
        assert info.status == nb.NB_ERR_COORD
        # flags are cleared by nb_check
        gb.grid()
        gb.build(0.45)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_compute(gb.ctx, nb.make_params("rf", 0.9), None, gb.f)   # rc > rlist
        assert ei.value.status == nb.NB_ERR_BOX
    finally:
        gb.close()


def test_config2_every_frame(gp, cfg2):
    """The benchmark's list lifetime on the 24,000-atom box: grid and list at
    frame 0, prune every 5 frames, forces and energies at each of the 20
    frames against the oracle's cell-list tier."""
    import paper_1306_1737_gb300 as nb
    b, p = cfg2
    gb = gp.GpuBox(b, p["rlist"])
    frames = list(w.frame_walk(b.xyz, b.mass, p["nstlist"], seed=2200))
    rp = float(np.float32(w.prune_radius(p["rc"], p["rlist"], p["nstprune"])))
    prm = nb.make_params("ewald", p["rc"], beta=p["beta"])
    oprm = oracle.make_params("ewald", float(np.float32(p["rc"])), beta=p["beta"])
    worst = 0.0
    try:
        gb.grid(frames[0])
        gb.build(float(np.float32(p["rlist"])))
        for f, x in enumerate(frames):
            if f > 0 and f % p["nstprune"] == 0:
                gb.prune(rp, x)
                fg, eg, vg = gb.compute(prm)
            else:
                fg, eg, vg = gb.compute(prm, x if f > 0 else None)
            fo, eo, vo = oracle.forces_cells(x, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
            emax, erms, _ = gp.force_errors(fg, fo)
            worst = max(worst, emax)
            assert emax < FORCE_TOL, (f, emax, erms)
            assert np.abs(eg - eo).max() / np.abs(eo).max() < E_TOL, (f, eg, eo)
            assert np.abs(vg - vo).max() / np.abs(vo).max() < E_TOL, f
    finally:
        gb.close()
    print(f"\nworst frame max|dF|/rms {worst:.2e}")


def test_no_missed_pairs_over_frames(gp):
    """Every particle pair inside rc is covered exactly once by the list in
    use (outer list, then the pruned lists) at every frame of a 20-frame
    lifetime: no missed pair anywhere (3,000 particles, all pairs checked)."""
    b = w.water_box(1000, None, seed=2300)
    rc, rl, nstprune = 1.0, 1.1, 5
    gb = gp.GpuBox(b, rl)
    frames = list(w.frame_walk(b.xyz, b.mass, 20, seed=2301))
    rp = float(np.float32(w.prune_radius(rc, rl, nstprune)))
    try:
        gb.grid(frames[0])
        g_or = oracle.grid(frames[0], b.q, b.types, b.box, 8)
        gb.build(float(np.float32(rl)))
        woff = (g_or.wrapped - frames[0]).astype(np.float32)
        which = 0
        for f, x in enumerate(frames):
            if f > 0 and f % nstprune == 0:
                gb.prune(rp, x)
                which = 1
            _, ient, cj, masks, sci = gb.list_arrays(which)
            a, bb, s, _ = __import__("gpu_path").expand_keys(ient, cj, masks, sci)
            g_f = oracle.Grid(**{**g_or.__dict__, "wrapped": (x + woff).astype(np.float32)})
            once, none, many = oracle.pair_cover(g_f, oracle.PairList(a, bb, s, np.zeros(a.size, np.uint64)), rc)
            assert none == 0 and many == 0 and once > 0, (f, once, none, many)
    finally:
        gb.close()


@pytest.mark.parametrize("cfg", ["cfg1", "cfg2"])
def test_pair_1x1_list_and_forces(gp, cfg, request):
    """The particle-pair comparison path: the full 1 x 1 list holds every pair
    within rlist twice (against the oracle's pair count; pairs within 1e-6 nm
    of rlist may differ), and its forces match the oracle."""
    import paper_1306_1737_gb300 as nb
    b, p = request.getfixturevalue(cfg)
    gb = gp.GpuBox(b, p["rlist"])
    torch = gb.torch
    try:
        gb.grid()
        rl = float(np.float32(p["rlist"]))
        gb.build(rl)
        max_nbr = 768
        nbr = torch.zeros((b.n, max_nbr), dtype=torch.int32, device=gb.dev)
        cnt = torch.zeros(b.n, dtype=torch.int32, device=gb.dev)
        nb.nb_pairlist_1x1(gb.ctx, rl, max_nbr, nbr, cnt)
        nb.nb_check(gb.ctx)
        counts = cnt.cpu().numpy()
        assert counts.max() <= max_nbr
        n_pairs = oracle.count_pairs_within(b.xyz, b.box, rl)
        n_edge = oracle.count_pairs_within(b.xyz, b.box, rl + 1e-6) - oracle.count_pairs_within(b.xyz, b.box, rl - 1e-6)
        assert abs(int(counts.sum()) - 2 * n_pairs) <= 2 * n_edge
        elec = p["elec"]
        prm = nb.make_params(elec, p["rc"], eps_rf=p.get("eps_rf", math.inf), beta=p.get("beta", 0.0),
                             want_energy=False)
        oprm = oracle.make_params(elec, float(np.float32(p["rc"])), beta=p.get("beta", 0.0))
        f = torch.zeros((b.n, 3), dtype=torch.float32, device=gb.dev)
        nb.nb_compute_1x1(gb.ctx, prm, None, nbr, cnt, max_nbr, f)
        nb.nb_check(gb.ctx)
        fo, _, _ = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        emax, erms, _ = gp.force_errors(f.cpu().numpy().astype(np.float64), fo)
        assert emax < FORCE_TOL, (emax, erms)
    finally:
        gb.close()


def test_tabulated_ewald_forces(gp, cfg2):
    """The tabulated force factor (linear interpolation in (beta r)^2) gives
    forces within 1e-4 of the RMS force of the oracle on the 24,000-atom box,
    before and after a prune."""
    import paper_1306_1737_gb300 as nb
    b, p = cfg2
    gb = gp.GpuBox(b, p["rlist"])
    try:
        gb.grid()
        gb.build(float(np.float32(p["rlist"])))
        prm = nb.make_params("ewald_tab", p["rc"], beta=p["beta"], want_energy=False)
        oprm = oracle.make_params("ewald", float(np.float32(p["rc"])), beta=p["beta"])
        f, _, _ = gb.compute(prm)
        fo, _, _ = oracle.forces_cells(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        emax, erms, _ = gp.force_errors(f, fo)
        assert emax < FORCE_TOL, (emax, erms)
        x5 = list(w.frame_walk(b.xyz, b.mass, 6, seed=2400))[5]
        gb.prune(float(np.float32(w.prune_radius(p["rc"], p["rlist"], 5))), x5)
        f5, _, _ = gb.compute(prm)
        fo5, _, _ = oracle.forces_cells(x5, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        emax, erms, _ = gp.force_errors(f5, fo5)
        assert emax < FORCE_TOL, (emax, erms)
    finally:
        gb.close()


def test_repeated_evaluations_agree(gp):
    """Twenty force evaluations in a row (energies on every other one) on the
    24,000-particle box: energies and virial equal to 1e-6 relative each
    time and forces equal up to the order of the FP32 additions (the work
    counters, slot accumulators and FP64 totals come back to zero after
    every evaluation)."""
    import paper_1306_1737_gb300 as nb
    b, p = w.config2()
    gb = gp.GpuBox(b, p["rlist"])
    try:
        gb.grid()
        gb.build(float(np.float32(p["rlist"])))
        pe = nb.make_params("ewald", p["rc"], beta=p["beta"], want_energy=True)
        pf = nb.make_params("ewald", p["rc"], beta=p["beta"], want_energy=False)
        f0, e0, v0 = gb.compute(pe)
        rms = np.sqrt((f0 ** 2).sum(1).mean())
        for k in range(20):
            f, e, v = gb.compute(pe if k % 2 else pf)
            assert np.abs(f - f0).max() < 1e-5 * rms
            if k % 2:
                assert np.abs(e - e0).max() <= 1e-6 * np.abs(e0).max()
                assert np.abs(v - v0).max() <= 1e-6 * np.abs(v0).max()
    finally:
        gb.close()
