"""Pins of the brute-force oracle totals: Newton's third law, F = -dE/dx,
the virial against an affine-deformation derivative of the energy,
translation invariance, and the paper's pair count per particle."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1306_1737_gb300 import workloads as w

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def small():
    return w.water_box(256, None, seed=7)


def _params(elec):
    return oracle.make_params(elec, rc=0.9, beta=3.12)


def _energy(b, xyz, box, prm):
    _, e, _ = oracle.forces_brute(xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx,
                                  box, prm, exact=True)
    return e.sum()


@pytest.mark.parametrize("elec", ["rf", "ewald"])
def test_newton_third_law(small, elec):
    f, e, _ = oracle.forces_brute(small.xyz, small.q, small.types, small.sigma, small.eps,
                                  small.excl_off, small.excl_idx, small.box, _params(elec))
    rms = np.sqrt((f ** 2).sum(1).mean())
    assert rms > 100.0
    assert np.abs(f.sum(0)).max() < 1e-9 * rms * small.n


@pytest.mark.parametrize("elec", ["rf", "ewald"])
def test_force_is_minus_energy_gradient(small, elec):
    prm = _params(elec)
    xyz = small.xyz.astype(np.float64)
    box = small.box.astype(np.float32).astype(np.float64)
    f, _, _ = oracle.forces_brute(xyz, small.q, small.types, small.sigma, small.eps,
                                  small.excl_off, small.excl_idx, box, prm, exact=True)
    rng = np.random.default_rng(3)
    h = 1e-6
    for atom in rng.choice(small.n, 6, replace=False):
        for k in range(3):
            xp = xyz.copy()
            xp[atom, k] += h
            xm = xyz.copy()
            xm[atom, k] -= h
            fd = -(_energy(small, xp, box, prm) - _energy(small, xm, box, prm)) / (2 * h)
            assert fd == pytest.approx(f[atom, k], rel=2e-5, abs=2e-3)


@pytest.mark.parametrize("elec", ["rf", "ewald"])
def test_virial_diagonal_is_minus_strain_derivative(small, elec):
    # W = sum_{i<j} r_ij (x) F_ij.  Scaling the box and all coordinates along
    # axis a by (1 + e) changes every separation r_a by a factor (1 + e):
    # dE/de = -sum r_a F_a = -W[a][a].
    prm = _params(elec)
    xyz = small.xyz.astype(np.float64)
    box = small.box.astype(np.float32).astype(np.float64)
    _, _, vir = oracle.forces_brute(xyz, small.q, small.types, small.sigma, small.eps,
                                    small.excl_off, small.excl_idx, box, prm, exact=True)
    h = 1e-7
    for a in range(3):
        s = np.ones(3)
        s[a] = 1 + h
        ep = _energy(small, xyz * s, box * s, prm)
        s[a] = 1 - h
        em = _energy(small, xyz * s, box * s, prm)
        assert -(ep - em) / (2 * h) == pytest.approx(vir[a, a], rel=1e-5, abs=1e-2)


def test_virial_full_tensor_for_isolated_cluster():
    # A compact cluster of particles in a box much larger than the cut-off has
    # no periodic partners, so any affine deformation x -> (I + e) x applies:
    # dE/de_ab = -W[a][b] for all a, b (off-diagonal terms included).
    b = w.water_box(40, 1.05, seed=11)
    xyz = b.xyz.astype(np.float64) + 2.0
    box = np.array([9.0, 9.0, 9.0])
    prm = oracle.make_params("ewald", rc=2.5, beta=3.12)
    _, _, vir = oracle.forces_brute(xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, box,
                                    prm, exact=True)
    # make sure no pair is near the cut-off (energy would jump there)
    d = xyz[:, None, :] - xyz[None, :, :]
    assert np.sqrt((d ** 2).sum(-1)).max() < 2.5 - 1e-3
    h = 1e-7
    for a in range(3):
        for c in range(3):
            m = np.eye(3)
            m[a, c] += h
            ep = _energy(b, xyz @ m.T, box, prm)
            m[a, c] -= 2 * h
            em = _energy(b, xyz @ m.T, box, prm)
            assert -(ep - em) / (2 * h) == pytest.approx(vir[a, c], rel=1e-5, abs=1e-2)


@pytest.mark.parametrize("elec", ["rf", "ewald"])
def test_translation_invariance(small, elec):
    prm = _params(elec)
    box = small.box.astype(np.float32).astype(np.float64)
    xyz = small.xyz.astype(np.float64)
    f0, e0, v0 = oracle.forces_brute(xyz, small.q, small.types, small.sigma, small.eps,
                                     small.excl_off, small.excl_idx, box, prm, exact=True)
    t = np.array([0.37, -1.21, 5.3])
    f1, e1, v1 = oracle.forces_brute(xyz + t, small.q, small.types, small.sigma, small.eps,
                                     small.excl_off, small.excl_idx, box, prm, exact=True)
    rms = np.sqrt((f0 ** 2).sum(1).mean())
    assert np.abs(f1 - f0).max() < 1e-9 * rms
    assert e1 == pytest.approx(e0, rel=1e-10)
    assert np.abs(v1 - v0).max() < 1e-9 * np.abs(v0).max()


def test_two_particles_by_hand():
    # Two unit charges 0.5 nm apart in a 3 nm box, reaction field eps_rf = inf,
    # rc = 1: F on particle 0 = 3.5 f along x (repulsive, pointing away from 1).
    xyz = np.array([[0.2, 1.0, 1.0], [0.7, 1.0, 1.0]])
    q = np.array([1.0, 1.0], np.float32)
    t = np.zeros(2, np.int32)
    prm = oracle.make_params("rf", rc=1.0)
    f, e, vir = oracle.forces_brute(xyz, q, t, np.zeros(1), np.zeros(1), None, None,
                                    np.array([3.0, 3.0, 3.0]), prm, exact=True)
    assert f[0] == pytest.approx([-3.5 * oracle.FCOUL, 0, 0], abs=1e-9)
    assert f[1] == pytest.approx([3.5 * oracle.FCOUL, 0, 0], abs=1e-9)
    assert e[1] == pytest.approx(0.625 * oracle.FCOUL, rel=1e-14)
    # W_xx = r_x F_x = (-0.5)(-3.5 f)
    assert vir[0, 0] == pytest.approx(1.75 * oracle.FCOUL, rel=1e-14)
    # the same pair across the periodic boundary (minimum image)
    xyz2 = np.array([[0.2, 1.0, 1.0], [2.7, 1.0, 1.0]])
    f2, e2, _ = oracle.forces_brute(xyz2, q, t, np.zeros(1), np.zeros(1), None, None,
                                    np.array([3.0, 3.0, 3.0]), prm, exact=True)
    assert f2[0] == pytest.approx([3.5 * oracle.FCOUL, 0, 0], abs=1e-9)
    assert e2[1] == pytest.approx(e[1], rel=1e-14)


def test_excluded_pair_keeps_only_correction():
    # An excluded pair inside the cut-off contributes only the RF correction.
    xyz = np.array([[1.0, 1.0, 1.0], [1.1, 1.0, 1.0]])
    q = np.array([-0.82, 0.41], np.float32)
    t = np.zeros(2, np.int32)
    prm = oracle.make_params("rf", rc=1.0)
    eo = np.array([0, 1, 2], np.int32)
    ei = np.array([1, 0], np.int32)
    f, e, _ = oracle.forces_brute(xyz, q, t, np.array([0.3]), np.array([0.5]), eo, ei,
                                  np.array([3.0, 3.0, 3.0]), prm, exact=True)
    qq = float(q[0]) * float(q[1])
    # k = 1/2, c = 3/2: V = f qq (k r^2 - c), F_x on 0 = f qq (-2 k r) * (-1)
    assert e[0] == 0.0
    assert e[1] == pytest.approx(oracle.FCOUL * qq * (0.5 * 0.01 - 1.5), rel=1e-9)
    assert f[0, 0] == pytest.approx(oracle.FCOUL * qq * (-2 * 0.5 * 0.1) * -1.0, rel=1e-9)


def test_pairs_per_particle_matches_paper(cfg2):
    # Sec. 5: a 1 nm cut-off in water means about 210 non-zero pairs per
    # particle (half list).  The synthetic box has the paper's density.
    b, _ = cfg2
    rho = b.n / np.prod(b.box)
    assert rho == pytest.approx(GOLD["number_density_nm3"]["value"], rel=0.01)
    npairs = oracle.count_pairs_within(b.xyz, b.box, 1.0)
    per = npairs / b.n
    ideal = 2.0 / 3.0 * math.pi * rho
    assert per == pytest.approx(ideal, rel=0.02)
    assert per == pytest.approx(GOLD["nonzero_pairs_per_particle_1nm"]["value"], rel=0.03)


def test_cell_list_tier_matches_brute_force():
    """Tier B (cell list) equals Tier A (all pairs) to rounding: forces,
    energies and virial, including a box of two cells per axis and a
    selected-particle evaluation."""
    from paper_1306_1737_gb300 import workloads as wl
    cases = [(wl.water_box(512, 2.48, seed=1001), "rf", 0.9),
             (wl.water_box(100, 1.45, seed=100), "ewald", 0.65),
             (wl.water_box(2000, None, seed=5), "ewald", 1.0)]
    for b, elec, rc in cases:
        op = oracle.make_params(elec, float(np.float32(rc)), beta=3.12)
        fa, ea, va = oracle.forces_brute(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, op)
        fb, eb, vb = oracle.forces_cells(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, op)
        assert np.abs(fa - fb).max() <= 1e-12 * np.abs(fa).max()
        assert np.abs(ea - eb).max() <= 1e-12 * np.abs(ea).max()
        assert np.abs(va - vb).max() <= 1e-12 * np.abs(va).max()
        sel = np.arange(0, b.n, 7)
        fs, _, _ = oracle.forces_cells(b.xyz, b.q, b.types, b.sigma, b.eps, b.excl_off, b.excl_idx, b.box, op, sel=sel)
        assert np.abs(fs - fa[sel]).max() <= 1e-12 * np.abs(fa).max()
