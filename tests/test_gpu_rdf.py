"""Pair-distance histogram (pair correlation) on the GPU against the oracle.

Where every distance lies well inside a bin (a simple cubic lattice) the
histogram must be exact, and equal the lattice's shell counts.  On water
boxes the FP32 distances of the kernel may put a pair that sits within
delta of a bin edge on either side of it, so the cumulative counts are
compared: for every edge k the GPU's number of pairs below edge k differs
from the FP64 oracle's by at most the oracle's count of pairs within delta
of that edge.  Everything else is exact: the overflow bin plus the bins
equal the selected listed pairs (every counted pair of the list is binned,
no cut-off test), a second accumulated call doubles every count, and each
box of a batch gets its own histogram."""
import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

# nm: bound on |r_FP32 - r| for boxes below 8 nm (coordinate rounding of the
# difference ~1e-7, r^2 and the rsqrt-based r ~4e-7, the FP32 bin scale ~1.5e-7)
DELTA = 2e-6


@pytest.fixture(scope="module")
def env():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1306_1737_gb300 as nb
    nb.load()
    return torch, torch.device("cuda", 0), nb


def _gpu_hist(env, boxes_or_batch, r_max, nbins, rlist, C=8, sel=(-1, -1), excl=True, accumulate_twice=False):
    torch, dev, nb = env
    B = boxes_or_batch
    batch = hasattr(B, "counts")
    counts = B.counts if batch else B.n
    boxes = B.boxes if batch else B.box
    c6c12 = nb.nb_lj_combine(B.sigma, B.eps)
    cx = nb.Context(counts, boxes, rlist, B.q, B.types, c6c12, cluster_size=C)
    nbox = B.nbox if batch else 1
    try:
        ctx = cx.ctx
        nb.nb_grid_put(ctx, torch.as_tensor(B.xyz, device=dev), boxes)
        use_excl = excl and B.excl_idx.size > 0
        nb.nb_pairlist_build(ctx, float(np.float32(rlist)), 0.0,
                             torch.as_tensor(B.excl_off, device=dev) if use_excl else None,
                             torch.as_tensor(B.excl_idx, device=dev) if use_excl else None)
        nb.nb_check(ctx)
        h = torch.full((nbox, nbins + 1), 7, dtype=torch.int64, device=dev)   # zeroed by the call
        nb.nb_rdf(ctx, r_max, nbins, sel[0], sel[1], 0, h)
        if accumulate_twice:
            nb.nb_rdf(ctx, r_max, nbins, sel[0], sel[1], 1, h)
        nb.nb_check(ctx)
        out = h.cpu().numpy()
        listed = None
        if not batch:
            listed = _listed_selected(env, ctx, B, C, sel)
    finally:
        cx.close()
    return out, listed


def _listed_selected(env, ctx, b, C, sel):
    """Selected particle pairs whose mask bit is set in the outer list."""
    torch, dev, nb = env
    import gpu_path as gp
    info = nb.nb_check(ctx)
    ni, nj, S = int(info.n_ientries), int(info.n_jentries), int(info.super_size)
    ient = torch.zeros((max(ni, 1), 4), dtype=torch.int32, device=dev)
    cj = torch.zeros(max(nj, 1), dtype=torch.int32, device=dev)
    mask = torch.zeros((S, max(nj, 1)), dtype=torch.int64, device=dev)
    nb.nb_get_list(ctx, 0, ient, cj, mask)
    ns = info.n_clusters * C
    aos = torch.zeros(ns, dtype=torch.int32, device=dev)
    sci = torch.zeros((max(info.n_superclusters, 1), 2), dtype=torch.int32, device=dev)
    nb.nb_get_grid(ctx, atom_of_slot=aos, sc_info=sci)
    torch.cuda.synchronize()
    a, bb, s, m = gp.expand_keys(ient.cpu().numpy()[:ni], cj.cpu().numpy()[:nj],
                                 mask.cpu().numpy().view(np.uint64)[:, :nj],
                                 sci.cpu().numpy()[: info.n_superclusters])
    aos = aos.cpu().numpy()
    total = 0
    for p in range(C * C):
        i, j = divmod(p, C)
        on = ((m >> np.uint64(p)) & np.uint64(1)).astype(bool)
        ai, aj = aos[a[on] * C + i], aos[bb[on] * C + j]
        assert np.all(ai >= 0) and np.all(aj >= 0)
        if sel[0] < 0:
            total += int(on.sum())
        else:
            ti, tj = b.types[ai], b.types[aj]
            total += int((((ti == sel[0]) & (tj == sel[1])) | ((ti == sel[1]) & (tj == sel[0]))).sum())
    return total


def _lattice(ns, a, colour=True):
    g = np.stack(np.meshgrid(np.arange(ns), np.arange(ns), np.arange(ns), indexing="ij"), -1).reshape(-1, 3)
    xyz = (g * a + 0.05).astype(np.float32)
    n = xyz.shape[0]
    types = (g.sum(1) % 2).astype(np.int32) if colour else np.zeros(n, np.int32)
    return w.Box(xyz=xyz, q=np.zeros(n, np.float32), types=types, sigma=np.array([0.3, 0.3]),
                 eps=np.array([0.5, 0.5]), mass=np.ones(n), excl_off=np.zeros(n + 1, np.int32),
                 excl_idx=np.zeros(0, np.int32), box=np.full(3, ns * a))


def _shell_counts(n, a, r_max, nbins, parity=None):
    """Lattice pair counts per bin from the number of integer vectors of each
    squared length (the coordination shells), counted here by enumeration."""
    dr = r_max / nbins
    h = np.zeros(nbins, np.int64)
    m = int(r_max / a) + 1
    v = np.stack(np.meshgrid(*[np.arange(-m, m + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    s2 = (v ** 2).sum(1)
    for s in np.unique(s2[s2 > 0]):
        r = np.sqrt(s) * a
        if r >= r_max:
            continue
        if parity is not None and (s % 2) != parity:
            continue
        z = int((s2 == s).sum())
        h[int(r // dr)] += n * z // 2
    return h


@pytest.mark.parametrize("C", [8, 4])
def test_cubic_lattice_exact(env, C):
    ns, a = 10, 0.31
    b = _lattice(ns, a)
    r_max, nbins = 1.2, 113
    dr = r_max / nbins
    # every shell distance clears its bin edges by far more than FP32 error
    for s in range(1, 16):
        r = np.sqrt(s) * a
        if r < r_max:
            frac = (r / dr) % 1.0
            assert 0.02 < frac < 0.98
    h, listed = _gpu_hist(env, b, r_max, nbins, 1.2, C=C)
    want = _shell_counts(b.n, a, r_max, nbins)
    assert np.array_equal(h[0, :nbins], want)
    assert h[0, :nbins].sum() == oracle.rdf(b.xyz, b.types, b.box, r_max, nbins)[0].sum()
    assert h[0].sum() == listed
    # same-colour pairs are the even shells, opposite colours the odd ones
    h00, _ = _gpu_hist(env, b, r_max, nbins, 1.2, C=C, sel=(0, 0))
    h01, _ = _gpu_hist(env, b, r_max, nbins, 1.2, C=C, sel=(1, 0))
    assert np.array_equal(h00[0, :nbins], _shell_counts(b.n // 2, a, r_max, nbins, parity=0))
    assert np.array_equal(h01[0, :nbins], _shell_counts(b.n, a, r_max, nbins, parity=1))


def _check_bounds(g, hist, near):
    """Cumulative counts below every edge within the oracle's near-edge counts."""
    nbins = hist.shape[0]
    G = np.concatenate([[0], np.cumsum(g[:nbins])])
    H = np.concatenate([[0], np.cumsum(hist)])
    diff = np.abs(G - H)
    assert np.all(diff <= near), (np.nonzero(diff > near)[0][:10], diff[diff > near][:10])


@pytest.mark.parametrize("C,sel", [(8, (-1, -1)), (8, (0, 0)), (8, (0, 1)), (4, (-1, -1))])
def test_water_against_oracle(env, C, sel):
    b, p = w.config2()                      # 24,000-atom water box
    r_max, nbins = 1.0, 400
    g, listed = _gpu_hist(env, b, r_max, nbins, 1.0, C=C, sel=sel)
    hist, near = oracle.rdf(b.xyz, b.types, b.box, r_max, nbins, b.excl_off, b.excl_idx, *sel, delta=DELTA)
    _check_bounds(g[0], hist, near)
    assert g[0].sum() == listed                        # every selected listed pair binned once
    assert g[0, nbins] > 0                             # listed pairs beyond r_max: overflow bin
    assert near.sum() < 3e-3 * hist.sum()              # the bound leaves little room


def test_list_radius_above_r_max(env):
    """A list built for a larger radius: the extra pairs land in the overflow bin."""
    b = w.water_box(1000, None, seed=77)
    r_max, nbins = 0.9, 90
    g, listed = _gpu_hist(env, b, r_max, nbins, 1.2)
    hist, near = oracle.rdf(b.xyz, b.types, b.box, r_max, nbins, b.excl_off, b.excl_idx, delta=DELTA)
    _check_bounds(g[0], hist, near)
    assert g[0].sum() == listed
    assert g[0, nbins] > g[0, :nbins].sum() // 4


def test_accumulate_doubles(env):
    b = w.water_box(700, None, seed=78)
    g1, _ = _gpu_hist(env, b, 1.0, 50, 1.0)
    g2, _ = _gpu_hist(env, b, 1.0, 50, 1.0, accumulate_twice=True)
    assert np.array_equal(g2, 2 * g1)


def test_batch_per_box(env):
    sizes = [400, 1500, 300, 900]
    boxes = [w.water_box(m, None, seed=7100 + k) for k, m in enumerate(sizes)]
    one = _lattice(6, 0.31, colour=False)
    one.sigma, one.eps = boxes[0].sigma.copy(), boxes[0].eps.copy()
    boxes.insert(1, one)
    B = w.concat(boxes)
    r_max, nbins = 0.9, 120
    g, _ = _gpu_hist(env, B, r_max, nbins, 0.9)
    for k, b in enumerate(boxes):
        hist, near = oracle.rdf(b.xyz, b.types, b.box, r_max, nbins, b.excl_off, b.excl_idx, delta=DELTA)
        _check_bounds(g[k], hist, near)


def test_errors(env):
    torch, dev, nb = env
    b = w.water_box(300, None, seed=79)
    c6c12 = nb.nb_lj_combine(b.sigma, b.eps)
    cx = nb.Context(b.n, b.box, 1.0, b.q, b.types, c6c12)
    try:
        ctx = cx.ctx
        h = torch.zeros((1, 101), dtype=torch.int64, device=dev)
        x = torch.as_tensor(b.xyz, device=dev)
        nb.nb_grid_put(ctx, x, b.box)
        with pytest.raises(nb.NbError) as ei:
            nb.nb_rdf(ctx, 0.8, 100, -1, -1, 0, h)          # no list yet
        assert ei.value.status == nb.NB_ERR_STATE
        nb.nb_pairlist_build(ctx, 0.9, 0.0, None, None)
        for args, st in (((1.0, 100, -1, -1), nb.NB_ERR_BOX),       # r_max above rlist
                         ((0.8, 0, -1, -1), nb.NB_ERR_ARG),
                         ((0.8, nb.NB_RDF_MAX_BINS + 1, -1, -1), nb.NB_ERR_ARG),
                         ((0.8, 100, 0, -1), nb.NB_ERR_ARG),
                         ((0.8, 100, 0, b.ntypes), nb.NB_ERR_ARG),
                         ((0.0, 100, -1, -1), nb.NB_ERR_ARG)):
            with pytest.raises(nb.NbError) as ei:
                nb.nb_rdf(ctx, *args, 0, h)
            assert ei.value.status == st, args
        nb.nb_rdf(ctx, 0.8, 100, -1, -1, 0, h)
        nb.nb_set_coords(ctx, x)                              # new coordinates: list is stale
        with pytest.raises(nb.NbError) as ei:
            nb.nb_rdf(ctx, 0.8, 100, -1, -1, 0, h)
        assert ei.value.status == nb.NB_ERR_STATE
        nb.nb_check(ctx)
    finally:
        cx.close()
