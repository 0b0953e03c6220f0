"""Pins of the oracle's pair interaction (Sec. 3.2) against closed forms,
special cases and an independent high-precision erfc (mpmath)."""
import math

import mpmath
import pytest

import oracle

SIG_O, EPS_O = 0.3166, 0.650


def lj_params(comb="lb", si=SIG_O, ei=EPS_O, sj=SIG_O, ej=EPS_O):
    return oracle.lj_pair_params(comb, si, ei, sj, ej)


@pytest.mark.parametrize("comb", ["lb", "geom"])
def test_lj_minimum_at_two_to_the_sixth_sigma(comb):
    # LJ with C6 = 4 eps sigma^6, C12 = 4 eps sigma^12 has its minimum -eps at
    # r = 2^(1/6) sigma, where the force vanishes, and crosses zero at sigma.
    c6, c12 = lj_params(comb)
    prm = oracle.make_params("rf", rc=1.0)
    rmin = 2.0 ** (1.0 / 6.0) * SIG_O
    assert abs(rmin - 0.3553715) < 1e-6
    fs, vlj, _ = oracle.pair(prm, rmin, 0.0, c6, c12)
    assert abs(fs * rmin) < 1e-9
    assert vlj == pytest.approx(-EPS_O, rel=1e-12)
    _, v0, _ = oracle.pair(prm, SIG_O, 0.0, c6, c12)
    assert abs(v0) < 1e-12
    # repulsive inside, attractive outside (sign of F r_hat on i)
    assert oracle.pair(prm, 0.9 * rmin, 0.0, c6, c12)[0] > 0
    assert oracle.pair(prm, 1.1 * rmin, 0.0, c6, c12)[0] < 0


def test_lorentz_berthelot_mixed_pair():
    # LB: sigma_ij = (sigma_i + sigma_j)/2, eps_ij = sqrt(eps_i eps_j); the
    # mixed potential has its zero at sigma_ij and minimum -eps_ij.
    si, ei, sj, ej = 0.25, 0.1, 0.40, 1.0
    c6, c12 = oracle.lj_pair_params("lb", si, ei, sj, ej)
    prm = oracle.make_params("rf", rc=1.2)
    s = 0.5 * (si + sj)
    e = math.sqrt(ei * ej)
    assert abs(oracle.pair(prm, s, 0.0, c6, c12)[1]) < 1e-12
    rmin = 2 ** (1 / 6) * s
    assert oracle.pair(prm, rmin, 0.0, c6, c12)[1] == pytest.approx(-e, rel=1e-12)
    # geometric rule on C6/C12 differs from LB for unequal sigma
    g6, g12 = oracle.lj_pair_params("geom", si, ei, sj, ej)
    assert g6 != pytest.approx(c6, rel=1e-3)


def test_hydrogen_without_lj():
    c6, c12 = oracle.lj_pair_params("lb", SIG_O, EPS_O, 0.0, 0.0)
    assert c6 == 0.0 and c12 == 0.0


def test_coulomb_prefactor_from_codata():
    # 1/(4 pi eps0) in kJ mol^-1 nm e^-2 from SI constants
    e = 1.602176634e-19
    eps0 = 8.8541878128e-12
    na = 6.02214076e23
    f = e * e * na / (4 * math.pi * eps0) / 1e-9 / 1000.0
    assert oracle.FCOUL == pytest.approx(f, rel=1e-8)


@pytest.mark.parametrize("eps_rf", [math.inf, 78.0])
def test_reaction_field_properties(eps_rf):
    rc = 0.9
    prm = oracle.make_params("rf", rc=rc, eps_rf=eps_rf)
    qq = -0.82 * 0.41
    fs_in, _, vc_in = oracle.pair(prm, rc * (1 - 1e-9), qq, 0, 0)
    # energy shifted to zero at the cut-off
    assert abs(vc_in) < 1e-6
    if math.isinf(eps_rf):
        # conducting boundary: the force vanishes at rc too
        assert abs(fs_in * rc) < 1e-5
    # nothing at or beyond rc
    assert oracle.pair(prm, rc, qq, 0, 0) == (0.0, 0.0, 0.0)
    # force is minus the derivative of the energy (excluded and not)
    for excl in (False, True):
        for r in (0.1, 0.3, 0.6, 0.85):
            h = 1e-6
            vp = oracle.pair(prm, r + h, qq, 0, 0, excl)[2]
            vm = oracle.pair(prm, r - h, qq, 0, 0, excl)[2]
            f = oracle.pair(prm, r, qq, 0, 0, excl)[0] * r
            assert f == pytest.approx(-(vp - vm) / (2 * h), rel=1e-6, abs=1e-6)


def test_reaction_field_two_charges_by_hand():
    # eps_rf = inf, rc = 1: k = 1/2, c = 3/2; unit charges at r = 0.5:
    # V = f (2 + 0.125 - 1.5) = 0.625 f, F = f (4 - 0.5) = 3.5 f.
    prm = oracle.make_params("rf", rc=1.0)
    fs, _, vc = oracle.pair(prm, 0.5, 1.0, 0, 0)
    assert vc == pytest.approx(0.625 * oracle.FCOUL, rel=1e-14)
    assert fs * 0.5 == pytest.approx(3.5 * oracle.FCOUL, rel=1e-14)


def test_ewald_energy_against_mpmath_and_force_derivative():
    beta, rc = 3.12, 1.0
    prm = oracle.make_params("ewald", rc=rc, beta=beta)
    qq = 1.0
    mpmath.mp.dps = 30
    for r in (0.05, 0.1, 0.3, 0.7, 0.99):
        vc = oracle.pair(prm, r, qq, 0, 0)[2]
        ref = float(oracle.FCOUL * mpmath.erfc(beta * r) / r)
        assert vc == pytest.approx(ref, rel=1e-13)
        # excluded pair: only the correction, -f erf(beta r)/r
        vx = oracle.pair(prm, r, qq, 0, 0, True)[2]
        assert vx == pytest.approx(float(-oracle.FCOUL * mpmath.erf(beta * r) / r), rel=1e-13)
        for excl in (False, True):
            f = oracle.pair(prm, r, qq, 0, 0, excl)[0] * r
            dv = mpmath.diff(lambda x: oracle.FCOUL * ((0 if excl else 1) - mpmath.erf(beta * x)) / x, r)
            assert f == pytest.approx(float(-dv), rel=1e-10)


def test_ewald_force_factor_values():
    # c(r) = r^2 F / (f qq) = erfc(br) + 2br/sqrt(pi) exp(-b^2 r^2), from mpmath
    beta = 3.12
    prm = oracle.make_params("ewald", rc=1.5, beta=beta)
    mpmath.mp.dps = 30
    for r, expected in ((0.1, 0.9784422), (0.3, 0.6253933), (1.0, 2.1868e-4)):
        c = oracle.pair(prm, r, 1.0, 0, 0)[0] * r ** 3 / oracle.FCOUL
        x = mpmath.mpf(beta * r)
        ref = float(mpmath.erfc(x) + 2 * x / mpmath.sqrt(mpmath.pi) * mpmath.exp(-x * x))
        assert c == pytest.approx(ref, rel=1e-12)
        assert c == pytest.approx(expected, rel=2e-4)
    # the Ewald tolerance at the cut-off: erfc(beta rc) ~ 1e-5
    assert float(mpmath.erfc(3.12)) == pytest.approx(1.0226e-5, rel=1e-3)


def test_ewald_reduces_to_plain_coulomb_for_small_beta():
    prm = oracle.make_params("ewald", rc=1.0, beta=1e-9)
    for r in (0.2, 0.5):
        fs, _, vc = oracle.pair(prm, r, 1.0, 0, 0)
        assert vc == pytest.approx(oracle.FCOUL / r, rel=1e-8)
        assert fs * r == pytest.approx(oracle.FCOUL / r ** 2, rel=1e-8)
        # excluded pair: nothing left
        fx, _, vx = oracle.pair(prm, r, 1.0, 0, 0, True)
        assert abs(vx) < 1e-6 and abs(fx) < 1e-6


@pytest.mark.parametrize("elec", ["rf", "ewald"])
def test_exclusion_removes_exactly_plain_coulomb_and_lj(elec):
    # Sec. 2.4: an excluded pair loses the normal LJ and Coulomb terms but keeps
    # the long-range correction: the difference is the bare Coulomb pair.
    prm = oracle.make_params(elec, rc=1.0, beta=3.12)
    c6, c12 = lj_params()
    qq = 0.37
    for r in (0.1, 0.25, 0.8):
        fa, la, va = oracle.pair(prm, r, qq, c6, c12, False)
        fb, lb, vb = oracle.pair(prm, r, qq, c6, c12, True)
        flj = oracle.pair(prm, r, 0.0, c6, c12, False)[0]
        assert lb == 0.0
        assert (fa - flj - fb) * r == pytest.approx(oracle.FCOUL * qq / r ** 2, rel=1e-10)
        assert va - vb == pytest.approx(oracle.FCOUL * qq / r, rel=1e-10)
