"""Edge cases of the grid, list and forces against the oracle: fewer
particles than a cluster, particles on cell edges and on the periodic
boundaries (including coordinates in [-L, 0) and [L, 2L)), equal z values
(ties broken by particle index), empty grid columns, and a box that is a
single column; on each, the pair-distance histogram against the oracle and
the fused force + prune pass against the separate prune."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu


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


def _box(xyz, L, seed):
    rng = np.random.default_rng(seed)
    n = xyz.shape[0]
    q = rng.choice([-0.8, 0.4, 0.4], n).astype(np.float32)
    types = rng.integers(0, 2, n).astype(np.int32)
    return w.Box(xyz=np.asarray(xyz, np.float32), q=q, types=types, sigma=np.array([0.3166, 0.25]),
                 eps=np.array([0.65, 0.3]), mass=np.full(n, 16.0), excl_off=np.zeros(n + 1, np.int32),
                 excl_idx=np.zeros(0, np.int32), box=np.array(L, np.float64), seed=seed)


def _spread(rng, n, lo, hi, dmin=0.2, L=None):
    """n uniform points in the box [lo, hi) at least dmin apart (minimum
    image in a periodic box of edges L), by rejection."""
    pts = []
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    while len(pts) < n:
        p = rng.uniform(lo, hi)
        ok = True
        for q in pts:
            d = p - q
            if L is not None:
                d -= np.asarray(L) * np.round(d / np.asarray(L))
            if (d * d).sum() < dmin * dmin:
                ok = False
                break
        if ok:
            pts.append(p)
    return np.array(pts)


def _cases():
    rng = np.random.default_rng(5)
    L3 = [3.0, 3.0, 3.0]
    out = []
    # fewer particles than one cluster
    out.append(("five particles", _box(_spread(rng, 5, [0, 0, 0], L3, L=L3), L3, 1)))
    # equal z for many particles, on a lattice whose x/y sit on cell edges
    g = np.arange(6) * np.float32(0.5)
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), np.full(X.size, 1.25)], 1)
    pts = np.concatenate([pts, pts + [0.25, 0.25, 0.0]])
    out.append(("equal z, cell edges", _box(pts, L3, 2)))
    # all particles in one half: empty columns
    half = _spread(rng, 400, [0, 0, 0], [1.4, 3.0, 3.0], L=L3)
    out.append(("empty columns", _box(half, L3, 3)))
    # coordinates on and beyond the periodic boundaries
    edge = _spread(rng, 300, [0.01, 0.01, 0.01], [2.99, 2.99, 2.99], L=L3)
    edge[:20, 0] = 0.0
    edge[20:40, 0] = np.nextafter(np.float32(3.0), np.float32(0.0))
    edge[40:60, 1] -= 3.0          # in [-L, 0)
    edge[60:80, 2] += 3.0          # in [L, 2L)
    out.append(("periodic boundaries", _box(edge, L3, 4)))
    # a box that is one grid column (few particles in a tall box)
    out.append(("single column", _box(_spread(rng, 30, [0, 0, 0], [2.2, 2.2, 6.0], L=[2.2, 2.2, 6.0]),
                                       [2.2, 2.2, 6.0], 5)))
    return out


@pytest.mark.parametrize("C", [8, 4])
def test_edge_cases(gp, C):
    import paper_1306_1737_gb300 as nb
    from test_gpu_parity import check_grid, check_list
    rc, rl = 0.9, 1.0
    for name, b in _cases():
        gb = gp.GpuBox(b, rl, C=C)
        try:
            gb.grid()
            g_or = oracle.grid(b.xyz, b.q, b.types, b.box, C)
            check_grid(gb.grid_arrays(), g_or)
            rlf = float(np.float32(rl))
            gb.build(rlf)
            pl = oracle.pairlist(g_or, rlf, 0.0, b.excl_off, b.excl_idx)
            check_list(gb, g_or, pl, rlf)
            f, e, vir = gb.compute(nb.make_params("ewald", rc, beta=3.12))
            fo, eo, vo = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box,
                                             oracle.make_params("ewald", float(np.float32(rc)), beta=3.12))
            if np.abs(fo).max() > 0:
                emax, _, _ = gp.force_errors(f, fo)
                assert emax < 1e-4, (name, emax)
            else:
                assert np.abs(f).max() == 0.0, name
            assert np.allclose(e, eo, rtol=1e-5, atol=1e-6), (name, e, eo)
            # pair-distance histogram on the fresh list
            h = gb.torch.zeros((1, 51), dtype=gb.torch.int64, device=gb.dev)
            nb.nb_rdf(gb.ctx, rlf, 50, -1, -1, 0, h)
            hg = h.cpu().numpy()[0]
            ho, near = oracle.rdf(b.xyz, b.types, b.box, rlf, 50, b.excl_off, b.excl_idx, delta=2e-6)
            G = np.concatenate([[0], np.cumsum(hg[:50])])
            H = np.concatenate([[0], np.cumsum(ho)])
            assert np.all(np.abs(G - H) <= near), name
            # the separate prune and the fused force + prune pass: the same pruned list
            rp = 0.95
            nb.nb_prune(gb.ctx, None, rp)
            nb.nb_check(gb.ctx)
            _, ient_a, cj_a, m_a, _ = gb.list_arrays(1)
            nb.nb_prune_compute(gb.ctx, nb.make_params("ewald", rc, beta=3.12, want_energy=False), None, rp, gb.f)
            nb.nb_check(gb.ctx)
            _, ient_b, cj_b, m_b, _ = gb.list_arrays(1)
            assert np.array_equal(ient_a, ient_b) and np.array_equal(cj_a, cj_b) and np.array_equal(m_a, m_b), name
            f2 = gb.f.cpu().numpy().astype(np.float64)
            if np.abs(fo).max() > 0:
                emax, _, _ = gp.force_errors(f2, fo)
                assert emax < 1e-4, (name, emax)
            else:
                assert np.abs(f2).max() == 0.0, name
        finally:
            gb.close()
