// One particle pair of the force kernels (Sec. 3.2), shared by the 4 x 4
// cluster kernel and the particle-pair (1 x 1) comparison kernel.
#pragma once

#include "nb_ewald_fit.h"
#include "nb_internal.cuh"

namespace nbc {

// One particle pair.  FIT selects the fitted rational approximation of the
// Ewald correction (Sec. 3.2: quotient of two polynomials) over erfcf/expf.
template <int ELEC, bool ENERGY, bool FIT>
__device__ __forceinline__ void pair_fn(const ForceParams& P, bool inc, float bit, float r2, float qq,
                                        float2 lj, float& fs, float& vlj, float& vc) {
    const float r2s = inc ? r2 : 1.0f;
    const float rinv = rsqrtf(r2s);
    const float rinv2 = rinv * rinv;
    const float rinv6 = rinv2 * rinv2 * rinv2;
    // lj = {6 C6, 12 C12}
    const float flj = bit * (lj.y * rinv6 - lj.x) * rinv6 * rinv2;
    float fc;
    if (ELEC == NB_ELEC_RF) {
        fc = qq * (bit * rinv * rinv2 - P.two_k_rf);
        if (ENERGY) vc = inc ? qq * (bit * rinv + P.k_rf * r2s - P.c_rf) : 0.0f;
    } else if (FIT) {
        const float w = P.beta2 * r2s;
        const float g = ewald_fit_g(w);
        fc = qq * (bit * rinv * rinv2 - P.beta3 * g);
        if (ENERGY) {
            const float h = ewald_fit_h(w);
            vc = inc ? qq * (bit * rinv - P.beta * h) : 0.0f;
        }
    } else {
        const float r = r2s * rinv;
        const float br = P.beta * r;
        const float ec = erfcf(br) - (1.0f - bit);
        const float ex = __expf(-br * br);
        fc = qq * (ec + P.two_beta_sqrtpi * r * ex) * rinv * rinv2;
        if (ENERGY) vc = inc ? qq * ec * rinv : 0.0f;
    }
    fs = inc ? flj + fc : 0.0f;
    if (ENERGY)
        vlj = inc ? bit * (lj.y * (1.0f / 12.0f) * rinv6 - lj.x * (1.0f / 6.0f)) * rinv6 : 0.0f;
}

}  // namespace nbc
