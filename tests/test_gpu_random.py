"""Seeded random configurations against the FP64 oracle: anisotropic boxes,
random charges (neutral overall), 1 to 16 LJ types under either combination
rule, bonded-like force-field exclusions (triples of neighbouring
particles), random cut-offs, list radii and bounding-box shortcut radii,
reaction field (infinite or finite dielectric) or Ewald, clusters of 8 or 4.
Forces, energies and virial after the list build; then forces after small
random displacements, through the prune-and-compute call (the fused pass for
8-particle clusters, prune kernel then force kernel for 4)."""
import math

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-4     # of the RMS force, plus FP32 rounding of the particle's own force (R24)
F_ROUND = 4e-6
E_TOL = 1e-4         # energies and virial, relative to the largest component


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


def _config(seed):
    """A random box of particles on a jittered lattice (70 nm^-3, so no two
    particles closer than 0.17 nm) and its interaction parameters."""
    rng = np.random.default_rng(9100 + seed)
    aspect = rng.uniform(0.75, 1.35, 3)
    aspect /= aspect.prod() ** (1.0 / 3.0)
    rho = 70.0
    L = aspect * (float(rng.integers(800, 4000)) / rho) ** (1.0 / 3.0)
    rc = float(rng.uniform(0.6, 1.0))
    rlist = rc + float(rng.uniform(0.05, 0.15))
    lim = 0.49 * float(L.min())
    if rlist > lim:
        rc, rlist = rc * lim / rlist, lim
    a = rho ** (-1.0 / 3.0)
    nx = np.maximum(1, np.floor(L / a).astype(int))
    grid = np.stack(np.meshgrid(*[np.arange(k) for k in nx], indexing="ij"), -1).reshape(-1, 3)
    sp = L / nx
    xyz = ((grid + 0.5 + rng.uniform(-0.15, 0.15, grid.shape)) * sp).astype(np.float32)
    n = xyz.shape[0]
    q = (rng.uniform(0.1, 0.8, n) * rng.choice([-1.0, 1.0], n)).astype(np.float64)
    q = (q - q.mean()).astype(np.float32)
    nt = int(rng.integers(1, 17))
    sigma = rng.uniform(0.20, 0.28, nt)
    eps = rng.uniform(0.05, 1.0, nt)
    types = rng.integers(0, nt, n).astype(np.int32)
    # exclusions: triples of consecutive particles along a lattice row (z is
    # the fastest index, so they are spatial neighbours), for about half of
    # the triples
    part = [[] for _ in range(n)]
    nz = int(nx[2])
    for s in range(0, n - 2, 3):
        if (s % nz) + 2 < nz and rng.random() < 0.5:
            for i in range(s, s + 3):
                for j in range(s, s + 3):
                    if i != j:
                        part[i].append(j)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum([len(p_) for p_ in part])
    idx = np.array([j for p_ in part for j in p_], np.int32)
    b = w.Box(xyz=xyz, q=q, types=types, sigma=sigma, eps=eps, mass=np.full(n, 16.0), excl_off=off,
              excl_idx=idx, box=L.astype(np.float64), seed=seed)
    elec = ("rf", "ewald", "rf", "ewald")[seed % 4]
    eps_rf = math.inf if seed % 3 else 78.0
    prm = dict(rc=rc, rlist=rlist, elec=elec, eps_rf=eps_rf, beta=3.12 / rc,
               rbb=float(rng.choice([0.0, 0.5 * rlist, rlist])), C=(8, 4)[seed % 2],
               comb=("lb", "geom")[(seed // 2) % 2])
    return b, prm, rng


def _check_forces(f, fo):
    rms = np.sqrt((fo ** 2).sum(1).mean())
    err = np.sqrt(((f - fo) ** 2).sum(1))
    bound = FORCE_TOL * rms + F_ROUND * np.sqrt((fo ** 2).sum(1))
    assert (err <= bound).all(), (float((err / bound).max()), int((err > bound).sum()))


@pytest.mark.parametrize("seed", range(16))
def test_random_configuration(gp, seed):
    import paper_1306_1737_gb300 as nb
    b, p, rng = _config(seed)
    comb = nb.NB_COMB_LB if p["comb"] == "lb" else nb.NB_COMB_GEOM
    rcf = float(np.float32(p["rc"]))
    rlf = float(np.float32(p["rlist"]))
    oprm = oracle.make_params(p["elec"], rcf, eps_rf=p["eps_rf"], beta=p["beta"], comb=p["comb"])
    gb = gp.GpuBox(b, p["rlist"], C=p["C"], comb=comb)
    try:
        gb.grid()
        gb.build(rlf, p["rbb"])
        prm = nb.make_params(p["elec"], rcf, eps_rf=p["eps_rf"], beta=p["beta"])
        f, e, vir = gb.compute(prm)
        fo, eo, vo = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx,
                                         b.box, oprm)
        _check_forces(f, fo)
        scale = np.abs(eo).max()
        assert np.abs(e - eo).max() <= E_TOL * scale, (e, eo)
        assert np.abs(vir - vo).max() <= E_TOL * np.abs(vo).max(), (vir, vo)
        # a later frame: small displacements (well inside half the buffer),
        # pruned at the midpoint of rc and rlist in the same pass as the forces
        x1 = (b.xyz + rng.normal(0.0, 0.003, b.xyz.shape)).astype(np.float32)
        rp = float(np.float32(0.5 * (p["rc"] + p["rlist"])))
        prm_f = nb.make_params(p["elec"], rcf, eps_rf=p["eps_rf"], beta=p["beta"], want_energy=False)
        nb.nb_prune_compute(gb.ctx, prm_f, gb.torch.as_tensor(x1).to(gb.dev).contiguous(), rp, gb.f)
        nb.nb_check(gb.ctx)
        f1 = gb.f.cpu().numpy().astype(np.float64)
        fo1, _, _ = oracle.forces_brute(x1, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, oprm)
        _check_forces(f1, fo1)
        # and once more on the pruned list
        f2, _, _ = gb.compute(prm_f)
        _check_forces(f2, fo1)
    finally:
        gb.close()
