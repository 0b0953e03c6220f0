"""The Verlet-buffer estimate of the library (Appendix; host code, no GPU)
against a composition of oracle parts: the drift integral by quadrature,
potential derivatives at rc by central differences of the oracle's pair
energies, Gaussian widths and class sums written out here."""
import math

import numpy as np
import pytest

import oracle

KB = 0.0083144626


def _v(p, r, qq, c6, c12):
    _, vl, vc = oracle.pair(p, r, qq, c6, c12)
    return vl + vc


def _drift_from_oracle(classes, sigma, eps, volume, elec, rc, beta, rb, t, T):
    op = oracle.make_params(elec, rc, beta=beta)
    h = 1e-5
    n = sum(c[0] for c in classes)
    total = 0.0
    for ci in classes:
        for cj in classes:
            c6, c12 = oracle.lj_pair_params("lb", sigma[ci[3]], eps[ci[3]], sigma[cj[3]], eps[cj[3]])
            qq = ci[2] * cj[2]
            # derivatives at rc from below (the potential is cut at rc)
            r0 = rc - 3 * h
            v = [_v(op, r0 + k * h, qq, c6, c12) for k in range(-2, 3)]
            d1 = (v[3] - v[1]) / (2 * h)
            d2 = (v[3] - 2 * v[2] + v[1]) / (h * h)
            # extrapolate the first derivative from r0 to rc with the second
            d1 += d2 * 3 * h
            s = t * math.sqrt(KB * T * (1 / ci[1] + 1 / cj[1]))
            i = oracle.buffer_drift_integral(d1, d2, rb, s)
            total += ci[0] * abs(4 * math.pi * (rc + rb + s) ** 2 * cj[0] / volume * i)
    return 0.5 * total / n / t


@pytest.fixture(scope="module")
def nb():
    import paper_1306_1737_gb300 as m
    from paper_1306_1737_gb300 import build
    build.build()
    m.load()
    return m


@pytest.mark.parametrize("elec", ["ewald", "rf"])
def test_buffer_drift_matches_oracle_composition(nb, elec):
    sigma, eps = np.array([0.3166, 0.0]), np.array([0.65, 0.0])
    classes = [(8000, 15.9994, -0.82, 0), (16000, 1.008, 0.41, 1)]
    volume = 6.21 ** 3
    table = nb.nb_lj_combine(sigma, eps)
    prm = nb.make_params(elec, 1.0, beta=3.12)
    for rb, t in ((0.05, 0.02), (0.1, 0.04), (0.0, 0.01)):
        got = nb.nb_buffer_drift(classes, table, volume, prm, rb, t, 300.0)
        want = _drift_from_oracle(classes, sigma, eps, volume, elec, 1.0, 3.12, rb, t, 300.0)
        assert abs(got - want) < 2e-3 * abs(want) + 1e-12, (rb, t, got, want)


def test_buffer_size_inverts_the_drift(nb):
    sigma, eps = np.array([0.3166, 0.0]), np.array([0.65, 0.0])
    classes = [(8000, 15.9994, -0.82, 0), (16000, 1.008, 0.41, 1)]
    table = nb.nb_lj_combine(sigma, eps)
    prm = nb.make_params("ewald", 1.0, beta=3.12)
    tol = 0.1 * KB * 298 / 1000          # 0.1 kB T per ns per particle (Table 3)
    rbs = [nb.nb_buffer_size(classes, table, 6.21 ** 3, prm, n * 0.002, 300.0, tol) for n in (5, 10, 20)]
    assert rbs[0] < rbs[1] < rbs[2]
    for n, rb in zip((5, 10, 20), rbs):
        d = nb.nb_buffer_drift(classes, table, 6.21 ** 3, prm, rb, n * 0.002, 300.0)
        assert d <= tol * (1 + 1e-9)
        d2 = nb.nb_buffer_drift(classes, table, 6.21 ** 3, prm, max(rb - 1e-3, 0.0), n * 0.002, 300.0)
        assert d2 > tol or rb < 1e-3
