"""Oracle pins for the Ewald force factor c(r) and the 1-32-32-1 SiLU network
that may stand in for it (CPU only).

c(r): values from the library erfc, the beta -> 0 limit, and the definition
as -r^2 d/dr[erfc(beta r)/r] (central differences of math.erfc).
Network: closed forms with chosen weights (SiLU(ln 3) = (3/4) ln 3, an
off-diagonal second-layer weight that a transposed index would miss),
linearity in the last layer, and the loss gradient against central finite
differences of the loss."""
import math

import numpy as np
import pytest

import oracle

H = oracle.MLP_HIDDEN
NP = oracle.MLP_NPARAMS
OFF_W1, OFF_B1, OFF_W2 = 0, H, 2 * H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H


def silu(z):
    return z / (1.0 + math.exp(-z))


def test_ewald_factor_values():
    beta = 3.12
    r = np.array([0.1, 0.3, 1.0, 0.05, 0.7])
    c = oracle.ewald_factor(r, beta)
    for ri, ci in zip(r, c):
        want = math.erfc(beta * ri) + 2 * beta * ri / math.sqrt(math.pi) * math.exp(-(beta * ri) ** 2)
        assert abs(ci - want) <= 1e-15 * max(1.0, abs(want))
    # printed values of the closed form at beta = 3.12
    assert abs(c[0] - 0.9784422) < 5e-8 and abs(c[1] - 0.6253933) < 5e-8 and abs(c[2] - 2.1868e-4) < 5e-8
    # no screening: the plain Coulomb force
    assert np.allclose(oracle.ewald_factor(r, 0.0), 1.0, rtol=0, atol=0)


def test_ewald_factor_is_minus_r2_dV_dr():
    beta, h = 3.12, 1e-6
    for r in (0.08, 0.2, 0.45, 0.9):
        v = lambda x: math.erfc(beta * x) / x
        dv = (v(r + h) - v(r - h)) / (2 * h)
        assert abs(oracle.ewald_factor([r], beta)[0] + r * r * dv) < 1e-8


def _zero():
    return np.zeros(NP)


def test_mlp_closed_form_single_path():
    # y = SiLU(w SiLU(a x)) + b3 with a x = ln 3 and w SiLU(ln 3) = ln 3
    p = _zero()
    rmin, rmax, r = 0.0, 2.0, 1.5          # x = r - 1 = 0.5
    a = 2.0 * math.log(3.0)
    p[OFF_W1 + 0] = a
    w = 4.0 / 3.0                          # (4/3) (3/4) ln 3 = ln 3
    p[OFF_W2 + 1 * H + 0] = w              # output unit 1 reads input unit 0
    p[OFF_W3 + 1] = 1.0
    p[OFF_B3] = 0.5
    y = oracle.mlp_forward(p, rmin, rmax, [r])[0]
    assert abs(silu(math.log(3.0)) - 0.75 * math.log(3.0)) < 1e-15
    assert abs(y - (0.75 * math.log(3.0) + 0.5)) < 1e-14
    # a transposed second layer (unit 0 reading unit 1) would give b3 only
    q = p.copy()
    q[OFF_W2 + 1 * H + 0] = 0.0
    q[OFF_W2 + 0 * H + 1] = w
    assert abs(oracle.mlp_forward(q, rmin, rmax, [r])[0] - 0.5) < 1e-15
    # negative branch: SiLU(-ln 3) = -(1/4) ln 3, bias path through b1 and b2
    p2 = _zero()
    p2[OFF_B1 + 5] = -math.log(3.0)
    p2[OFF_W2 + 7 * H + 5] = 1.0
    p2[OFF_B2 + 7] = 0.25 * math.log(3.0) + math.log(3.0)   # z2 = ln 3
    p2[OFF_W3 + 7] = 2.0
    y2 = oracle.mlp_forward(p2, rmin, rmax, [0.3])[0]
    assert abs(y2 - 2.0 * 0.75 * math.log(3.0)) < 1e-14


def test_mlp_last_layer_linear():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(NP) * 0.4
    r = rng.uniform(0.05, 1.0, 17)
    y = oracle.mlp_forward(p, 0.05, 1.0, r)
    q = p.copy()
    q[OFF_W3:] *= 2.0
    assert np.allclose(oracle.mlp_forward(q, 0.05, 1.0, r), 2.0 * y, rtol=1e-14, atol=1e-14)


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(4)
    p = rng.standard_normal(NP) * 0.4
    r = rng.uniform(0.05, 1.0, 64)
    t = np.cos(3 * r)
    w = rng.uniform(0.5, 2.0, 64)
    loss, g = oracle.mlp_loss_grad(p, 0.05, 1.0, r, t, w)
    y = oracle.mlp_forward(p, 0.05, 1.0, r)
    assert abs(loss - np.mean(w * (y - t) ** 2)) < 1e-13
    h = 1e-6
    idx = list(range(0, H, 5)) + list(range(H, 2 * H, 7)) + list(range(OFF_W2, OFF_B2, 97)) + \
        list(range(OFF_B2, OFF_W3, 6)) + list(range(OFF_W3, OFF_B3, 5)) + [OFF_B3]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, 0.05, 1.0, r, t, w)[0] - oracle.mlp_loss_grad(pm, 0.05, 1.0, r, t, w)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_buffer_drift_integral_pins():
    """The Appendix's drift integral by quadrature: at rb = 0 the first-order
    part is -sigma^2/4 and the second-order part sigma^3/(3 sqrt(2 pi))
    (elementary Gaussian moments); for rb > 0 it matches the integrals
    evaluated symbolically (sympy) -- a reference independent of the
    closed form the library uses."""
    s = 0.03
    assert abs(oracle.buffer_drift_integral(1.0, 0.0, 0.0, s) - (-0.25 * s * s)) < 1e-6 * s * s
    assert abs(oracle.buffer_drift_integral(0.0, 1.0, 0.0, s) - s ** 3 / (3 * math.sqrt(2 * math.pi))) < 1e-5 * s ** 3
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x", positive=True)
    for rb, sg in ((0.05, 0.03), (0.1, 0.05)):
        E = sp.erfc(x / sp.sqrt(2)) / 2
        # inner integral over r0 gives E((rb - u)/sigma); u = rb - sigma x
        i1 = float(sg * sp.Integral((rb - sg * x) * E, (x, rb / sg, sp.oo)).evalf(30))
        i2 = float(sg * sp.Integral(sp.Rational(1, 2) * (rb - sg * x) ** 2 * E, (x, rb / sg, sp.oo)).evalf(30))
        assert abs(oracle.buffer_drift_integral(1.0, 0.0, rb, sg) - i1) < 1e-6 * abs(i1)
        assert abs(oracle.buffer_drift_integral(0.0, 1.0, rb, sg) - i2) < 1e-4 * abs(i2)   # quadrature accuracy
