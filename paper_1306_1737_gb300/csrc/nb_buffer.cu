// Verlet-buffer estimate (Appendix of the paper): an upper bound on the
// energy drift caused by pairs that move from outside the list radius
// rl = rc + rb to inside the cut-off during a list lifetime t, for particles
// moving freely at temperature T (which bounds the real, hindered motion).
//
// Per pair of particle classes (1, 2): the distance changes by a Gaussian
// of variance sigma^2 = t^2 kB T (1/m1 + 1/m2) (free flight for time t);
// with the pair potential expanded to second order at rc,
//   dV = 4 pi (rl + sigma)^2 rho2 { V'(rc)/2 [rb sigma G(rb/sigma)
//          - (rb^2 + sigma^2) E(rb/sigma)]
//        + V''(rc)/6 [sigma (rb^2 + 2 sigma^2) G(rb/sigma)
//          - rb (rb^2 + 3 sigma^2) E(rb/sigma)] },
// G the standard normal density and E(x) = erfc(x/sqrt 2)/2.  The drift per
// particle and time sums |dV| over ordered class pairs weighted by the
// first class's count, halves it (each pair is seen from both sides) and
// divides by the particle count and t.  Host code only.
#include <cmath>

#include "nb_ewald_fit.h"
#include "nb_internal.cuh"

namespace {

constexpr double kBoltzmann = 0.0083144626;   // kJ mol^-1 K^-1
constexpr double kCoulomb = 138.935458;       // kJ mol^-1 nm e^-2

double gauss_pdf(double x) { return std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI); }
double gauss_tail(double x) { return 0.5 * std::erfc(x / std::sqrt(2.0)); }

// V'(rc), V''(rc) of the Coulomb part for charge product qq.
void coulomb_derivs(const nb_params* p, double qq, double* d1, double* d2) {
    const double rc = p->rc, A = kCoulomb * qq;
    if (p->elec == NB_ELEC_RF) {
        double k;
        if (!(p->eps_rf > 0.f) || std::isinf(p->eps_rf)) k = 1.0 / (2.0 * rc * rc * rc);
        else k = ((double)p->eps_rf - 1.0) / ((2.0 * p->eps_rf + 1.0) * rc * rc * rc);
        *d1 = A * (-1.0 / (rc * rc) + 2.0 * k * rc);
        *d2 = A * (2.0 / (rc * rc * rc) + 2.0 * k);
    } else {
        const double b = p->beta, br = b * rc;
        const double g = 2.0 * b / std::sqrt(M_PI) * std::exp(-br * br);
        *d1 = A * (-g / rc - std::erfc(br) / (rc * rc));
        *d2 = A * (g * (2.0 * b * b + 2.0 / (rc * rc)) + 2.0 * std::erfc(br) / (rc * rc * rc));
    }
}

nb_status drift(int nclass, const nb_particle_class* cls, int ntypes, const float* c6c12, double volume,
                const nb_params* p, double rb, double t_ps, double temperature, double* out) {
    if (nclass <= 0 || !cls || ntypes <= 0 || !c6c12 || !p || !out || !(volume > 0.0) || !(rb >= 0.0) ||
        !(t_ps > 0.0) || !(temperature > 0.0) || !(p->rc > 0.f))
        return NB_ERR_ARG;
    if (p->elec != NB_ELEC_RF && p->elec != NB_ELEC_EWALD && p->elec != NB_ELEC_EWALD_MLP) return NB_ERR_ARG;
    const double rc = p->rc, kT = kBoltzmann * temperature;
    double total = 0.0, n = 0.0;
    for (int i = 0; i < nclass; ++i) {
        if (cls[i].type < 0 || cls[i].type >= ntypes || !(cls[i].mass > 0.0) || cls[i].count < 0.0) return NB_ERR_ARG;
        n += cls[i].count;
    }
    if (!(n > 0.0)) return NB_ERR_ARG;
    for (int i = 0; i < nclass; ++i) {
        for (int j = 0; j < nclass; ++j) {
            const int tt = cls[i].type * ntypes + cls[j].type;
            const double c6 = c6c12[2 * tt], c12 = c6c12[2 * tt + 1];
            // LJ C12/r^12 - C6/r^6
            double d1 = -12.0 * c12 / std::pow(rc, 13) + 6.0 * c6 / std::pow(rc, 7);
            double d2 = 156.0 * c12 / std::pow(rc, 14) - 42.0 * c6 / std::pow(rc, 8);
            double e1, e2;
            coulomb_derivs(p, cls[i].charge * cls[j].charge, &e1, &e2);
            d1 += e1;
            d2 += e2;
            const double s = t_ps * std::sqrt(kT * (1.0 / cls[i].mass + 1.0 / cls[j].mass));
            const double x = rb / s, G = gauss_pdf(x), E = gauss_tail(x);
            const double t1 = 0.5 * (rb * s * G - (rb * rb + s * s) * E);
            const double t2 = (s * (rb * rb + 2.0 * s * s) * G - rb * (rb * rb + 3.0 * s * s) * E) / 6.0;
            const double rl = rc + rb;
            const double dv = 4.0 * M_PI * (rl + s) * (rl + s) * (cls[j].count / volume) * (d1 * t1 + d2 * t2);
            total += cls[i].count * std::fabs(dv);
        }
    }
    *out = 0.5 * total / n / t_ps;
    return NB_OK;
}

}  // namespace

extern "C" {

nb_status nb_buffer_drift(int nclass, const nb_particle_class* classes, int ntypes, const float* c6c12,
                          double volume, const nb_params* p, double rb, double t_ps, double temperature,
                          double* drift_per_ps) {
    return drift(nclass, classes, ntypes, c6c12, volume, p, rb, t_ps, temperature, drift_per_ps);
}

nb_status nb_buffer_size(int nclass, const nb_particle_class* classes, int ntypes, const float* c6c12,
                         double volume, const nb_params* p, double t_ps, double temperature, double tolerance,
                         double* rb) {
    if (!rb || !(tolerance > 0.0)) return NB_ERR_ARG;
    double d = 0.0;
    nb_status st = drift(nclass, classes, ntypes, c6c12, volume, p, 0.0, t_ps, temperature, &d);
    if (st != NB_OK) return st;
    if (d <= tolerance) {
        *rb = 0.0;
        return NB_OK;
    }
    // the drift falls monotonically with the buffer: bisect on [0, hi]
    double lo = 0.0, hi = 0.05;
    for (int k = 0; k < 60; ++k) {
        st = drift(nclass, classes, ntypes, c6c12, volume, p, hi, t_ps, temperature, &d);
        if (st != NB_OK) return st;
        if (d <= tolerance) break;
        lo = hi;
        hi *= 2.0;
        if (hi > 100.0) return NB_ERR_ARG;
    }
    for (int k = 0; k < 60 && hi - lo > 1e-6; ++k) {
        const double mid = 0.5 * (lo + hi);
        st = drift(nclass, classes, ntypes, c6c12, volume, p, mid, t_ps, temperature, &d);
        if (st != NB_OK) return st;
        if (d <= tolerance) hi = mid;
        else lo = mid;
    }
    *rb = hi;
    return NB_OK;
}

}  // extern "C"
