"""Fit the rational approximations of the Ewald real-space correction used by
the force kernel, and write them to nb_ewald_fit.h.

Sec. 3.2 of the paper evaluates the PME correction force analytically with a
quotient of two polynomials (about 24 multiply-adds and one division) instead
of erfc; the coefficients are not printed, so this project fits its own.

With x = beta r and w = x^2 the kernel needs, as smooth functions of w:
  G(w) = (erf(x) - 2x/sqrt(pi) exp(-x^2)) / x^3   (force:  F/r = qq (e r^-3 - beta^3 G))
  H(w) = erf(x) / x                              (energy: V   = qq (e r^-1 - beta H))
on w in [0, W] (W = 10, i.e. beta*rc <= 3.16, which covers the usual Ewald
splitting erfc(beta rc) ~ 1e-5; larger beta*rc falls back to erfcf).

Method: rational P(w)/Q(w), Q(0) = 1, fitted on Chebyshev-distributed points
by the Sanathanan-Koerner iteration (linear least squares on P - f Q,
re-weighted by 1/|Q| of the previous iterate) combined with Lawson's
re-weighting toward the minimax (equal-ripple) relative error.  Reference
values come from mpmath at 40 digits.  Run: python fit_ewald.py
"""
import os

import mpmath
import numpy as np

W_MAX = 10.0
# (numerator, denominator) degrees: the force factor G is evaluated for every
# pair, the energy factor H only in energy evaluations
DEGREES = {"G": (4, 4), "H": (5, 4)}
N_PTS = 4000
mpmath.mp.dps = 40


def g_exact(w):
    w = mpmath.mpf(w)
    if w < mpmath.mpf("1e-8"):
        c = 2 / mpmath.sqrt(mpmath.pi)
        return sum(c * (-1) ** (n + 1) * 2 * n / ((2 * n + 1) * mpmath.factorial(n)) * w ** (n - 1)
                   for n in range(1, 6))
    x = mpmath.sqrt(w)
    return (mpmath.erf(x) - 2 * x / mpmath.sqrt(mpmath.pi) * mpmath.exp(-w)) / x ** 3


def h_exact(w):
    w = mpmath.mpf(w)
    if w < mpmath.mpf("1e-8"):
        c = 2 / mpmath.sqrt(mpmath.pi)
        return sum(c * (-1) ** n * w ** n / (mpmath.factorial(n) * (2 * n + 1)) for n in range(0, 6))
    x = mpmath.sqrt(w)
    return mpmath.erf(x) / x


def fit(ws, f, p, q, iters=40):
    wt = np.full(ws.size, 1.0 / ws.size)
    qprev = np.ones_like(ws)
    best = None
    for _ in range(iters):
        A = np.zeros((ws.size, p + 1 + q))
        for k in range(p + 1):
            A[:, k] = ws ** k
        for k in range(1, q + 1):
            A[:, p + k] = -f * ws ** k
        sc = np.sqrt(wt) / (np.abs(f) * qprev)
        coef, *_ = np.linalg.lstsq(A * sc[:, None], f * sc, rcond=None)
        a = coef[: p + 1]
        b = np.concatenate([[1.0], coef[p + 1:]])
        P = np.polyval(a[::-1], ws)
        Q = np.polyval(b[::-1], ws)
        err = P / Q / f - 1.0
        m = np.abs(err).max()
        if best is None or m < best[0]:
            best = (m, a.copy(), b.copy())
        qprev = np.abs(Q)
        wt = wt * np.abs(err)
        wt = 0.5 * wt / wt.sum() + 0.5 / ws.size
    return best


def eval32(a, b, ws):
    a32 = a.astype(np.float32)
    b32 = b.astype(np.float32)
    w32 = ws.astype(np.float32)
    P = np.zeros_like(w32)
    for c in a32[::-1]:
        P = (P * w32 + c).astype(np.float32)
    Q = np.zeros_like(w32)
    for c in b32[::-1]:
        Q = (Q * w32 + c).astype(np.float32)
    return (P / Q).astype(np.float64), Q


def monic(a, b):
    """G's fit as lead * Pm(w) / Qm(w) with monic Pm, Qm (leading coefficient
    1): returns (Pm's lower coefficients, Qm's lower coefficients, lead)."""
    return a[:-1] / a[-1], b[:-1] / b[-1], a[-1] / b[-1]


def eval32_monic_scaled(pm, qm, lead, beta, ws):
    """FP32 evaluation as the force kernel does it: x = r^2 = w / beta^2, the
    monic polynomials in x with beta folded into their coefficients
    (c_k beta^(2(k - 4)), rounded to FP32), Horner with the first step x + c_3,
    the quotient as P times the reciprocal of Q; relative to lead (the leading
    ratio's beta^3 factor is the caller's)."""
    b2 = beta * beta
    pc = np.array([pm[k] * b2 ** (k - 4) for k in range(4)], np.float32)
    qc = np.array([qm[k] * b2 ** (k - 4) for k in range(4)], np.float32)
    x = (ws / b2).astype(np.float32)
    P = (x + pc[3]).astype(np.float32)
    Q = (x + qc[3]).astype(np.float32)
    for k in (2, 1, 0):
        P = (P * x + pc[k]).astype(np.float32)
        Q = (Q * x + qc[k]).astype(np.float32)
    return lead * (P * (np.float32(1.0) / Q).astype(np.float32)).astype(np.float64)


def main():
    t = np.cos(np.pi * (np.arange(N_PTS) + 0.5) / N_PTS)
    ws = np.sort((t + 1) / 2 * W_MAX)
    out = {}
    for name, fn in (("G", g_exact), ("H", h_exact)):
        f = np.array([float(fn(w)) for w in ws])
        m, a, b = fit(ws, f, *DEGREES[name])
        # check on a finer, different grid
        wchk = np.linspace(0.0, W_MAX, 20001)
        fchk = np.array([float(fn(w)) for w in wchk])
        v32, q32 = eval32(a, b, wchk)
        e32 = np.abs(v32 / fchk - 1).max()
        e64 = np.abs(np.polyval(a[::-1], wchk) / np.polyval(b[::-1], wchk) / fchk - 1).max()
        assert q32.min() > 0.0
        out[name] = (a, b, e64, e32)
    here = os.path.dirname(os.path.abspath(__file__))
    lines = [
        "// Generated by fit_ewald.py -- do not edit.",
        "// Rational approximations in w = (beta r)^2 on [0, %g] of" % W_MAX,
        "//   G(w) = (erf(x) - 2x/sqrt(pi) exp(-x^2)) / x^3  and  H(w) = erf(x) / x,  x = sqrt(w)",
        "// (Sanathanan-Koerner + Lawson fit of P/Q, Q(0) = 1; degrees G %s, H %s)." % (DEGREES["G"], DEGREES["H"]),
        "#pragma once",
        "",
        "namespace nbc {",
        "constexpr float kEwaldFitWMax = %.1ff;" % W_MAX,
        "// 1/x by the hardware's approximate reciprocal, denormals flushed (the",
        "// fits' denominators are at least 1 on their range; far outside it they",
        "// overflow to infinity and the quotient is selected away by the caller).",
        "__device__ __forceinline__ float fit_rcp(float x) {",
        "    float y;",
        "    asm(\"rcp.approx.ftz.f32 %0, %1;\" : \"=f\"(y) : \"f\"(x));",
        "    return y;",
        "}",
    ]
    for name in ("G", "H"):
        a, b, e64, e32 = out[name]
        lines.append("// %s(w): max relative error %.2e (double), %.2e (FP32 Horner)" % (name, e64, e32))
        lines.append("__device__ __forceinline__ float ewald_fit_%s(float w) {" % name.lower())

        def horner(c):
            expr = "%.9ef" % c[-1]
            for v in c[-2::-1]:
                expr = "fmaf(%s, w, %.9ef)" % (expr, v)
            return expr
        # scalar Horner: every coefficient is an immediate operand of its FMA
        lines.append("    const float p = %s;" % horner(a))
        lines.append("    const float q = %s;" % horner(b))
        lines.append("    return p * fit_rcp(q);")
        lines.append("}")
    # G in monic form over x = r^2 (beta folded into the coefficients by the host)
    a, b, _, _ = out["G"]
    pm, qm, lead = monic(a, b)
    fg = np.array([float(g_exact(w)) for w in ws])
    errs = []
    for beta in (2.0, 3.12, 4.0):
        v = eval32_monic_scaled(pm, qm, lead, beta, ws)
        errs.append(np.abs(v / fg - 1).max())
    lines += [
        "// G(w) = lead * Pm(w) / Qm(w) with monic Pm, Qm (below: their coefficients of",
        "// w^0..w^3; w^4 has 1).  With x = r^2 = w / beta^2 the kernel evaluates",
        "// Pm, Qm in x with coefficients c_k beta^(2(k-4)) (the common beta^8 cancels):",
        "// max relative error in FP32 %.2e, %.2e, %.2e at beta 2, 3.12, 4 nm^-1." % tuple(errs),
        "constexpr double kEwaldGMonicP[4] = {%s};" % ", ".join("%.17e" % v for v in pm),
        "constexpr double kEwaldGMonicQ[4] = {%s};" % ", ".join("%.17e" % v for v in qm),
        "constexpr double kEwaldGLead = %.17e;" % lead,
        "// Pm or Qm at x with the host-scaled coefficients c[0..3] (Horner, first step x + c[3]).",
        "__device__ __forceinline__ float ewald_monic4(float x, const float (&c)[4]) {",
        "    return fmaf(fmaf(fmaf(x + c[3], x, c[2]), x, c[1]), x, c[0]);",
        "}",
    ]
    lines += ["}  // namespace nbc", ""]
    path = os.path.join(here, "nb_ewald_fit.h")
    open(path, "w").write("\n".join(lines))
    for name in ("G", "H"):
        print(name, "max rel err double %.2e  fp32 %.2e" % (out[name][2], out[name][3]))
    print("wrote", path)


if __name__ == "__main__":
    main()
