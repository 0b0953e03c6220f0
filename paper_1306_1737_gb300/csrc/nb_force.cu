// Cluster-pair force/energy kernels (Sec. 3, Fig. 6); the FP64 totals and the
// return to the caller's order are in nb_finalize.cu.
//
// k_force8: one warp per i-entry {super-cluster, shift, j-range} of
// 8-particle clusters.  Lane (ih = lane / 8, j = lane % 8) owns particle pairs
// (ih, j) and (ih+4, j) of every i-cluster and j-cluster, so the 8 x 8
// cluster pair is two 8 x 4 halves spread over the warp, and the lane's two
// pairs are the two halves of packed FP32x2 operations.  The super-cluster's
// i-particles are staged in shared memory in that pairing, shifted by the
// entry's periodic image as an unevaluated FP32 sum hi + lo; each j-particle
// comes as two float4 of a duplicated layout ({-x, -x, -y, -y}, {-z, -z, q,
// q}) so that it enters packed operations without register copies.  The
// j-clusters' records (that layout and the LJ types, 288 bytes) reach a
// per-warp ring in shared memory by asynchronous copies, the next 8 entries'
// while the current 8 are computed, so that no entry waits for its j-data
// to come from L2.  A pair
// is computed when r^2 < rc^2 and either its mask bit is set (full LJ +
// Coulomb) or it is a counted pair without the bit (force-field exclusion:
// only the RF/Ewald correction, Sec. 2.4); the mask bit multiplies the plain
// terms (Sec. 3.1: masking by multiplication, conditional on the cut-off).
// j-entries whose interacting i-clusters all have full masks off the
// diagonal (most of them) take a path with the cut-off as the only
// condition.  Each lane adds its j-force (its two pairs' sum) with one
// vector atomic per j-cluster; i-forces are reduced at the end of the entry
// and added once per i-particle.
//
// Pair functions (Sec. 3.2), with qq = f q_i q_j and e = mask bit:
//   LJ      F/r = e (12 C12 r^-6 - 6 C6) r^-8,  V = e (C12 r^-6 - C6) r^-6
//   RF      F/r = qq (e r^-3 - 2k),             V = qq (e r^-1 + k r^2 - c_rf)
//   Ewald   F/r = qq (erfc(br) - (1-e) + 2br/sqrt(pi) exp(-b^2 r^2)) r^-3,
//           V = qq (erfc(br) - (1-e)) r^-1
#include <map>
#include <mutex>
#include <tuple>

#include "nb_internal.cuh"
#include "nb_ewald_fit.h"
#include "nb_mlp.cuh"
#include "nb_pair.cuh"

namespace nbc {

// The force kernels' arguments: only the arrays they touch, so that every
// field is a direct constant-bank operand.
struct ForceArgs {
    const int4* ient;                 // outer or pruned list
    const int* cj;
    const unsigned long long* mask;
    long long jstride;                // stride between the per-i-cluster mask arrays
    const float4* xyzq;
    const float4* xjd;                // j-cluster records: duplicated, negated j layout and LJ types
    const int* type_slot;
    float4* fslot;
    const float2* c6c12;
    const int2* sc_info;
    const long long* ient_off;        // box regions of the i-entries
    const DevState* st;
    const BoxGeom* geo;
    Accum* acc;
    const MlpTC* mlp;
    const float2* ewald_tab;          // tabulated Ewald force factor
    const int* ient_used;             // compact i-entry index per box
    int* work;                        // work counter (next i-entry to take)
    // pruned-list output of the fused force + prune kernel
    int4* ient_p;
    int* cj_p;
    unsigned long long* mask_p;
    DevState* stw;
    int nbox;
    ForceParams p;
};

constexpr int kForceWarps = 4;

// Packed FP32x2 helpers: component x is the lane's pair (ih, j), component y
// its pair (ih + 4, j).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sel2(bool p, bool q, float2 v) {
    return make_float2(p ? v.x : 0.0f, q ? v.y : 0.0f);
}

struct Lane8 {
    int j, ih;
    bool lower0, lower1;  // (ih, j) and (ih+4, j) on or below the diagonal
    unsigned sel;         // bit of this lane's pairs within each 32-bit half of a mask
};

constexpr int kSuper8 = super_size(8);
// Set in a staged j-word (sign bit, above the cluster index and the
// interaction bits) when every i-cluster of the super-cluster interacts with
// the j-cluster through an all-ones mask off the diagonal: the common case,
// computed with the cut-off as the only condition.
constexpr unsigned kFastBit = 1u << 31;
static_assert(kSuperShift + kSuper8 <= 31, "interaction bits overlap the fast bit");

// j-entries per group of the per-warp ring below.
constexpr int kJGroup = 8;
static_assert(kJGroup == 8, "the j-loop finds an entry's group as t >> 3");

// One j-cluster's record of the duplicated j layout, as the ring's copies
// bring it: the 8 slots' {-x, -x, -y, -y}, their {-z, -z, q, q}, their LJ
// types.
struct JTile {
    float4 a[8];
    float4 b[8];
    int t[8];
};
static_assert(sizeof(JTile) == kJRecord * sizeof(float4), "a record of the duplicated j layout");
static_assert(sizeof(JTile) % 16 == 0, "16-byte copies land on 16-byte boundaries");

// Per-warp shared staging of the force kernel.
struct WarpSmem {
    // i particles of the super-cluster, paired the way a lane uses them:
    // [k][ih] holds i-particles ih and ih + 4 of i-cluster k side by side
    float4 ixy[kSuper8][4];   // {x, x', y, y'} shifted coordinates, hi part
    float4 izq[kSuper8][4];   // {z, z', f q, f q'}
    float4 lxy[kSuper8][4];   // {x, x', y, y'} lo part of the shift
    float2 lz[kSuper8][4];    // {z, z'} lo part
    int2 row[kSuper8][4];     // LJ row byte offsets (type * ntypes * 8)
    int w[32];                // j-entry words of the current chunk (with the fast bit)
    unsigned long long m[kSuper8][32];  // their masks per i-cluster
    // a ring of two groups of j-clusters: the group being computed and the
    // next, copied in while the current one is computed
    JTile jt[2][kJGroup];
};

// Asynchronous 16-byte copies from global to shared memory (L2 only), in
// per-thread groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most the newest group of this thread's copies is in flight
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Request the j-clusters of group g of the staged chunk (entries g * kJGroup
// onwards, at most kJGroup of the chunk's nt) into ring buffer g & 1, whose
// previous group every lane has read (the warp synchronises here; the reads
// have completed, their values are in use): lane (k, q) = (lane / 4,
// lane % 4) copies the 16-byte pieces q, q + 4, ... of entry k's record; one
// commit group per lane.
static_assert(kJGroup * 4 == 32 && kJRecord <= 20, "four lanes per record, at most five pieces each");
__device__ __forceinline__ void jgroup_issue(const ForceArgs& A, WarpSmem& W, int g, int nt, int lane) {
    const int t0 = g * kJGroup, k = lane >> 2, q = lane & 3;
    __syncwarp();
    if (t0 + k < nt) {
        const long long cj = W.w[t0 + k] & kCjMask;
        const float4* src = A.xjd + kJRecord * cj + q;
        float4* dst = W.jt[g & 1][k].a + q;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (q + 4 * i < kJRecord) cp_async16(dst + 4 * i, src + 4 * i);
    }
    cp_async_commit();
}

// The j-particle of a lane with both halves of each packed pair holding it
// (the lane's two particle pairs share j): -x, -y, -z, so that a distance
// component is one packed add x_i + (-x_j), and the charge; from the
// j-cluster's record in the warp's ring.
struct JPart {
    float2 nx, ny, nz, q;
    int t;   // LJ type, as a byte offset into a row of the {-6 C6, 12 C12} table
};

__device__ __forceinline__ JPart load_jpart(const JTile& T, int j) {
    const float4 a = T.a[j], b = T.b[j];
    JPart J;
    J.nx = make_float2(a.x, a.y);
    J.ny = make_float2(a.z, a.w);
    J.nz = make_float2(b.x, b.y);
    J.q = make_float2(b.z, b.w);
    J.t = T.t[j] * (int)sizeof(float2);
    return J;
}

// LJ table entry at a byte offset (row of the i-type plus column of the j-type).
__device__ __forceinline__ float2 lj_entry(const float2* s_lj, int byte_off) {
    return *reinterpret_cast<const float2*>(reinterpret_cast<const char*>(s_lj) + byte_off);
}

// Distance vectors of the lane's two pairs with j-particle (xj) as packed
// pairs, from the paired i layout: d = (x_i + shift) - x_j with the shift
// as hi + lo, every operation rounded once (x_i^hi + (-x_j)) + x_i^lo.
template <bool SHIFTED>
__device__ __forceinline__ void pair_deltas(const WarpSmem& W, int k, int ih, float2 nx, float2 ny, float2 nz,
                                            float2& dx, float2& dy, float2& dz, float2& fq) {
    const float4 a = W.ixy[k][ih], b = W.izq[k][ih];
    dx = add2(make_float2(a.x, a.y), nx);
    dy = add2(make_float2(a.z, a.w), ny);
    dz = add2(make_float2(b.x, b.y), nz);
    fq = make_float2(b.z, b.w);
    if (SHIFTED) {
        const float4 l = W.lxy[k][ih];
        dx = add2(dx, make_float2(l.x, l.y));
        dy = add2(dy, make_float2(l.z, l.w));
        dz = add2(dz, W.lz[k][ih]);
    }
}

// The Ewald force factor G(w), w = (beta r)^2, from the table in shared
// memory: entry k = {G(k h), G((k+1) h) - G(k h)}, h = w_max / n, linear
// interpolation (Sec. 3.2: the tabulated kernels).  t = r^2 beta^2 / h.
__device__ __forceinline__ float ewald_tab_g(const float2* tab, int n, float t) {
    const int i = min((int)t, n - 1);
    const float2 v = tab[i];
    return fmaf(t - (float)i, v.y, v.x);
}

// 1/sqrt(x) by the hardware's approximate reciprocal square root, denormals
// flushed: squared distances of counted pairs are far above the denormal
// range, and any other pair's result is selected away.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Force/energy of the lane's two pairs (x and y components) given squared
// distances and the pair charge products qq = f q_i q_j.  Packed FP32x2 where
// both operands are pairs; scalar where one operand is a constant (an
// immediate or a kernel parameter is a direct operand of a scalar
// instruction, while a packed one would first need the constant copied into
// a register pair).  u0/u1: mask bits (full interaction); inc0/inc1: pair
// counted and inside rc.  Pairs that are not counted are computed on
// whatever r2 they have and selected away (no NaN escapes the selects).
// FULL: every pair inside rc is a full interaction (all-ones mask, no
// diagonal).
template <int ELEC, bool ENERGY, bool FIT, bool FULL>
__device__ __forceinline__ float2 pair_force2(const ForceParams& P, float2 r2, bool inc0, bool inc1, bool u0,
                                              bool u1, float2 qq, float2 lj0, float2 lj1, float& e_lj,
                                              float& e_c, const float2* s_tab) {
    const float2 rinv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 rinv2 = mul2(rinv, rinv);
    float2 rinv3 = mul2(rinv, rinv2);
    const float2 rinv6 = mul2(rinv3, rinv3);
    // LJ (12 C12 r^-6 - 6 C6) r^-8 with lj = {-6 C6, 12 C12}
    float2 flj = mul2(mul2(make_float2(fmaf(lj0.y, rinv6.x, lj0.x), fmaf(lj1.y, rinv6.y, lj1.x)), rinv6), rinv2);
    if (!FULL) {
        flj = sel2(u0, u1, flj);
        rinv3 = sel2(u0, u1, rinv3);
    }
    float2 fc;
    if (ELEC == NB_ELEC_RF) {
        fc = mul2(qq, make_float2(rinv3.x - P.two_k_rf, rinv3.y - P.two_k_rf));
    } else if (ELEC == NB_ELEC_EWALD_TAB) {
        fc = mul2(qq, make_float2(fmaf(-P.beta3, ewald_tab_g(s_tab, P.tab_n, r2.x * P.tab_scale), rinv3.x),
                                  fmaf(-P.beta3, ewald_tab_g(s_tab, P.tab_n, r2.y * P.tab_scale), rinv3.y)));
    } else if (FIT) {
        // the fitted factor as a quotient of monic polynomials in w whose
        // coefficients are immediate operands; -beta^3 times the leading
        // coefficients' ratio is fit_k
        const float g0 = ewald_fit_gm(P.beta2 * r2.x), g1 = ewald_fit_gm(P.beta2 * r2.y);
        fc = mul2(qq, make_float2(fmaf(P.fit_k, g0, rinv3.x), fmaf(P.fit_k, g1, rinv3.y)));
    } else {
        const float r0 = r2.x * rinv.x, r1 = r2.y * rinv.y;
        const float b0 = P.beta * r0, b1 = P.beta * r1;
        fc = mul2(qq, make_float2(
            rinv3.x + (erfcf(b0) - 1.0f + P.two_beta_sqrtpi * r0 * __expf(-b0 * b0)) * rinv2.x * rinv.x,
            rinv3.y + (erfcf(b1) - 1.0f + P.two_beta_sqrtpi * r1 * __expf(-b1 * b1)) * rinv2.y * rinv.y));
    }
    if (ENERGY) {
        // V_LJ = (C12 r^-6 - C6) r^-6;  V_C = qq (e/r - correction)
        float vl0 = fmaf(lj0.y * (1.0f / 12.0f), rinv6.x, lj0.x * (1.0f / 6.0f)) * rinv6.x;
        float vl1 = fmaf(lj1.y * (1.0f / 12.0f), rinv6.y, lj1.x * (1.0f / 6.0f)) * rinv6.y;
        const float re0 = FULL || u0 ? rinv.x : 0.0f, re1 = FULL || u1 ? rinv.y : 0.0f;
        float vc0, vc1;
        if (ELEC == NB_ELEC_RF) {
            vc0 = qq.x * (re0 + fmaf(P.k_rf, r2.x, -P.c_rf));
            vc1 = qq.y * (re1 + fmaf(P.k_rf, r2.y, -P.c_rf));
        } else if (FIT) {
            vc0 = qq.x * fmaf(-P.beta, ewald_fit_h(P.beta2 * r2.x), re0);
            vc1 = qq.y * fmaf(-P.beta, ewald_fit_h(P.beta2 * r2.y), re1);
        } else {
            vc0 = qq.x * ((erfcf(P.beta * r2.x * rinv.x) - 1.0f) * rinv.x + re0);
            vc1 = qq.y * ((erfcf(P.beta * r2.y * rinv.y) - 1.0f) * rinv.y + re1);
        }
        e_lj += (inc0 && (FULL || u0) ? vl0 : 0.0f) + (inc1 && (FULL || u1) ? vl1 : 0.0f);
        e_c += (inc0 ? vc0 : 0.0f) + (inc1 ? vc1 : 0.0f);
    }
    return sel2(inc0, inc1, add2(flj, fc));
}

// Add a warp's energy partial sums to box b's FP64 totals and clear them.
__device__ __forceinline__ void flush_energy(Accum* acc, int b, float& e_lj, float& e_c, unsigned& n_inc) {
    const unsigned full = 0xffffffffu;
    for (int o = 16; o > 0; o >>= 1) {
        e_lj += __shfl_xor_sync(full, e_lj, o);
        e_c += __shfl_xor_sync(full, e_c, o);
        n_inc += __shfl_xor_sync(full, n_inc, o);
    }
    if ((threadIdx.x & 31) == 0 && b >= 0) {
        atomicAdd(&acc[b].energy[0], (double)e_lj);
        atomicAdd(&acc[b].energy[1], (double)e_c);
        atomicAdd(&acc[b].n_inc, (unsigned long long)n_inc);
    }
    e_lj = e_c = 0.0f;
    n_inc = 0;
}

// Running force sums of a lane: i-forces per i-cluster, and the j-force of
// the current j-cluster, each over the lane's two pairs as packed pairs.
// The j-sum holds the force on i (the pair force times x_i - x_j); the
// j-particle receives its negative.
struct JSum {
    float2 x, y, z;
};

// The pairs of i-cluster k (of the super-cluster) with one j-cluster.
// Returns (warp-uniformly) whether any pair was inside rc.
// PRUNE: also sets bit k of keep when a counted pair (any pair but, on the
// unshifted diagonal, j <= i) is closer than the prune radius (Sec. 2.3),
// with the same FP32 distances as the separate prune kernel.
template <int ELEC, bool ENERGY, bool FIT, bool SHIFTED, bool FULL, bool PRUNE>
__device__ __forceinline__ bool icluster8(const ForceParams& P, const float2* s_lj, const WarpSmem& W,
                                          const Lane8& L, int2 row, int k, bool diag, unsigned long long m,
                                          const JPart& J, float2& fx, float2& fy, float2& fz, JSum& G,
                                          float& e_lj, float& e_c, unsigned& n_inc, unsigned& keep) {
    float2 dx, dy, dz, fq;
    pair_deltas<SHIFTED>(W, k, L.ih, J.nx, J.ny, J.nz, dx, dy, dz, fq);
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    if constexpr (PRUNE) {
        const bool c0 = FULL || !(diag && L.lower0), c1 = FULL || !(diag && L.lower1);
        if (__any_sync(0xffffffffu, (c0 && r2.x < P.rp2) || (c1 && r2.y < P.rp2))) keep |= 1u << k;
    }
    bool u0 = true, u1 = true;
    if (!FULL) {
        u0 = ((unsigned)m & L.sel) != 0u;
        u1 = ((unsigned)(m >> 32) & L.sel) != 0u;
    }
    bool inc0 = r2.x < P.rc2;
    bool inc1 = r2.y < P.rc2;
    if (!FULL && diag) {
        inc0 = inc0 && (u0 || !L.lower0);
        inc1 = inc1 && (u1 || !L.lower1);
    }
    if (!__any_sync(0xffffffffu, inc0 || inc1)) return false;
    const float2 lj0 = lj_entry(s_lj, row.x + J.t), lj1 = lj_entry(s_lj, row.y + J.t);
    const float2 fs = pair_force2<ELEC, ENERGY, FIT, FULL>(P, r2, inc0, inc1, u0, u1, mul2(fq, J.q), lj0, lj1,
                                                           e_lj, e_c, s_lj + P.ntypes * P.ntypes);
    if (ENERGY) n_inc += (unsigned)inc0 + (unsigned)inc1;
    fx = fma2(fs, dx, fx);
    fy = fma2(fs, dy, fy);
    fz = fma2(fs, dz, fz);
    G.x = fma2(fs, dx, G.x);
    G.y = fma2(fs, dy, G.y);
    G.z = fma2(fs, dz, G.z);
    return true;
}

// The common case of a j-entry, both i-clusters of the super-cluster with
// all-ones masks off the diagonal: one warp vote for the entry (does any of
// its 128 pairs lie inside rc?), then both 8 x 8 tiles as straight-line
// code.  Without a branch between them the two tiles' chains of dependent
// operations interleave, which hides their latencies (3M box: 2.6% less
// time per force launch than a vote and a branch per tile); a tile with no
// pair inside rc is computed as well and contributes zeros.
// PRUNE: as icluster8, per tile.
template <int ELEC, bool ENERGY, bool FIT, bool SHIFTED, bool PRUNE>
__device__ __forceinline__ bool icluster8_both(const ForceParams& P, const float2* s_lj, const WarpSmem& W,
                                               const Lane8& L, const int2 (&row)[kSuper8], const JPart& J,
                                               float2 (&fx)[kSuper8], float2 (&fy)[kSuper8],
                                               float2 (&fz)[kSuper8], JSum& G, float& e_lj, float& e_c,
                                               unsigned& n_inc, unsigned& keep) {
    static_assert(kSuper8 == 2, "a super-cluster of two 8-particle i-clusters");
    float2 dx[2], dy[2], dz[2], fq[2], r2[2];
    bool inc0[2], inc1[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        pair_deltas<SHIFTED>(W, k, L.ih, J.nx, J.ny, J.nz, dx[k], dy[k], dz[k], fq[k]);
        r2[k] = fma2(dx[k], dx[k], fma2(dy[k], dy[k], mul2(dz[k], dz[k])));
        if constexpr (PRUNE) {
            if (__any_sync(0xffffffffu, r2[k].x < P.rp2 || r2[k].y < P.rp2)) keep |= 1u << k;
        }
        inc0[k] = r2[k].x < P.rc2;
        inc1[k] = r2[k].y < P.rc2;
    }
    if (!__any_sync(0xffffffffu, inc0[0] || inc1[0] || inc0[1] || inc1[1])) return false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 lj0 = lj_entry(s_lj, row[k].x + J.t), lj1 = lj_entry(s_lj, row[k].y + J.t);
        const float2 fs = pair_force2<ELEC, ENERGY, FIT, true>(P, r2[k], inc0[k], inc1[k], true, true,
                                                               mul2(fq[k], J.q), lj0, lj1, e_lj, e_c,
                                                               s_lj + P.ntypes * P.ntypes);
        if (ENERGY) n_inc += (unsigned)inc0[k] + (unsigned)inc1[k];
        fx[k] = fma2(fs, dx[k], fx[k]);
        fy[k] = fma2(fs, dy[k], fy[k]);
        fz[k] = fma2(fs, dz[k], fz[k]);
        G.x = fma2(fs, dx[k], G.x);
        G.y = fma2(fs, dy[k], G.y);
        G.z = fma2(fs, dz[k], G.z);
    }
    return true;
}

// The surrogate form of icluster8 (forces only): unmasked pairs inside rc
// with r >= r_min take the Coulomb factor c(r) from the network, evaluated
// for the whole 8 x 8 tile at once on the tensor cores; force-field-excluded
// pairs (and any unmasked pair below r_min) keep the fitted analytic
// correction.
template <bool SHIFTED, bool FULL>
__device__ __forceinline__ bool icluster8_mlp(const ForceParams& P, const float2* s_lj, const WarpSmem& W,
                                              const Lane8& L, int2 row, int k, bool diag, unsigned long long m,
                                              const JPart& J, float2& fx, float2& fy, float2& fz, JSum& G,
                                              const MlpTC& M, float* mo) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float2 dx, dy, dz, fq;
    pair_deltas<SHIFTED>(W, k, L.ih, J.nx, J.ny, J.nz, dx, dy, dz, fq);
    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    bool u0 = true, u1 = true;
    if (!FULL) {
        u0 = ((unsigned)m & L.sel) != 0u;
        u1 = ((unsigned)(m >> 32) & L.sel) != 0u;
    }
    bool inc0 = r2.x < P.rc2;
    bool inc1 = r2.y < P.rc2;
    if (!FULL && diag) {
        inc0 = inc0 && (u0 || !L.lower0);
        inc1 = inc1 && (u1 || !L.lower1);
    }
    if (!__any_sync(full, inc0 || inc1)) return false;
    const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    const float2 rinv2 = mul2(rinv, rinv);
    const float2 rinv3 = mul2(rinv, rinv2);
    const float2 rinv6 = mul2(rinv3, rinv3);
    const float rr0 = r2.x * rinv.x, rr1 = r2.y * rinv.y;
    const bool n0 = inc0 && u0 && rr0 >= P.mlp_rmin, n1 = inc1 && u1 && rr1 >= P.mlp_rmin;
    float c0 = 0.0f, c1 = 0.0f;
    if (__any_sync(full, n0 || n1)) {
        // tile row p is the lane's first pair (p = lane) or its second
        // (p = lane + 32); m-tile t holds rows 16 t + g and 16 t + 8 + g
        const float ra = n0 ? rr0 : P.mlp_rmin, rb = n1 ? rr1 : P.mlp_rmin;
        const int g = lane >> 2;
#pragma unroll 1
        for (int t = 0; t < 4; ++t) {
            const float src = t < 2 ? ra : rb;
            const int base = g + 16 * (t & 1);
            const float x0 = (__shfl_sync(full, src, base) - M.c0) * M.c1;
            const float x1 = (__shfl_sync(full, src, base + 8) - M.c0) * M.c1;
            float o0, o1;
            mlp_mtile(M, lane, x0, x1, o0, o1);
            if ((lane & 3) == 0) {
                mo[16 * t + g] = o0;
                mo[16 * t + 8 + g] = o1;
            }
        }
        __syncwarp();
        c0 = mo[lane];
        c1 = mo[lane + 32];
        __syncwarp();
    }
    const bool a0f = inc0 && !n0, a1f = inc1 && !n1;   // analytic correction
    float g0 = 0.0f, g1 = 0.0f;
    if (__any_sync(full, a0f || a1f)) {
        g0 = a0f ? ewald_fit_g(P.beta2 * r2.x) : 0.0f;
        g1 = a1f ? ewald_fit_g(P.beta2 * r2.y) : 0.0f;
    }
    const float2 lj0 = lj_entry(s_lj, row.x + J.t), lj1 = lj_entry(s_lj, row.y + J.t);
    const float qq0 = fq.x * J.q.x, qq1 = fq.y * J.q.y;
    float flj0 = fmaf(lj0.y, rinv6.x, lj0.x) * rinv6.x * rinv2.x;
    float flj1 = fmaf(lj1.y, rinv6.y, lj1.x) * rinv6.y * rinv2.y;
    if (!FULL) {
        flj0 = u0 ? flj0 : 0.0f;
        flj1 = u1 ? flj1 : 0.0f;
    }
    const float fc0 = n0 ? qq0 * c0 * rinv3.x : qq0 * fmaf(-P.beta3, g0, u0 ? rinv3.x : 0.0f);
    const float fc1 = n1 ? qq1 * c1 * rinv3.y : qq1 * fmaf(-P.beta3, g1, u1 ? rinv3.y : 0.0f);
    const float2 fs = make_float2(inc0 ? flj0 + fc0 : 0.0f, inc1 ? flj1 + fc1 : 0.0f);
    fx = fma2(fs, dx, fx);
    fy = fma2(fs, dy, fy);
    fz = fma2(fs, dz, fz);
    G.x = fma2(fs, dx, G.x);
    G.y = fma2(fs, dy, G.y);
    G.z = fma2(fs, dz, G.z);
    return true;
}

// All j-entries [jb, je) (at most 32) of one super-cluster i-entry.  The
// j-clusters come through the warp's ring in groups of kJGroup entries, the
// next group copied in while the current one is computed.  PRUNE: the
// j-entries that keep an interacting i-cluster within the prune radius are
// appended in order to the pruned list at j_out + kept (the entry's offsets
// in the outer list), as the separate prune kernel does.
template <int ELEC, bool ENERGY, bool FIT, bool SHIFTED, bool PRUNE>
__device__ __forceinline__ void force_entry8(const ForceArgs& A, const float2* s_lj, WarpSmem& W,
                                             const Lane8& L, const int2 (&row)[kSuper8], int g0, bool center,
                                             int jb, int je, float2 (&fx)[kSuper8], float2 (&fy)[kSuper8],
                                             float2 (&fz)[kSuper8], float& e_lj, float& e_c,
                                             unsigned& n_inc, const MlpTC* M, float* mo, int j_out, int& kept,
                                             unsigned long long& keys) {
    constexpr bool MLP = ELEC == NB_ELEC_EWALD_MLP;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nt = je - jb;
    // the chunk's j-words and masks, one entry per lane; the fast bit marks
    // the words whose i-clusters all interact through full masks off the
    // diagonal
    if (lane < nt) {
        const int w = A.cj[jb + lane];
        const int cj = w & kCjMask;
        bool fast = ((unsigned)w >> kSuperShift) == (1u << kSuper8) - 1u;
#pragma unroll
        for (int k = 0; k < kSuper8; ++k) {
            const unsigned long long m = A.mask[k * A.jstride + jb + lane];
            W.m[k][lane] = m;
            fast = fast && m == ~0ull && !(center && cj == g0 + k);
        }
        W.w[lane] = fast ? (int)((unsigned)w | kFastBit) : w;
    }
    __syncwarp();
    jgroup_issue(A, W, 0, nt, lane);
    unsigned my_keep = 0;   // PRUNE: kept i-cluster bits of j-entry `lane`
    for (int t = 0; t < nt; ++t) {
        if ((t & (kJGroup - 1)) == 0) {
            // group t / kJGroup starts: request the one after it (into the
            // buffer of the group just finished; an empty commit group if
            // there is none), then wait for this one
            if (t + kJGroup < nt) jgroup_issue(A, W, (t >> 3) + 1, nt, lane);
            else cp_async_commit();
            cp_async_wait_prior();
            __syncwarp();
        }
        const int w = W.w[t];
        const int cjt = w & kCjMask;
        const JPart J = load_jpart(W.jt[0][t & (2 * kJGroup - 1)], L.j);
        JSum G;
        G.x = G.y = G.z = make_float2(0.f, 0.f);
        bool any = false;
        unsigned keep = 0;
        // (the network's form keeps one copy of each tile evaluator: its code
        // is large, and a third copy for the fast path costs more in
        // instruction fetch than the path saves)
        if (!MLP && w < 0) {
            any = icluster8_both<ELEC, ENERGY, FIT, SHIFTED, PRUNE>(A.p, s_lj, W, L, row, J, fx, fy, fz, G, e_lj,
                                                                    e_c, n_inc, keep);
        } else {
            const unsigned bits = ((unsigned)w >> kSuperShift) & ((1u << kSuper8) - 1u);
#pragma unroll
            for (int k = 0; k < kSuper8; ++k) {
                if (!((bits >> k) & 1u)) continue;
                const bool diag = center && (cjt == g0 + k);
                const unsigned long long m = W.m[k][t];
                if constexpr (MLP) {
                    if (!diag && m == ~0ull)
                        any |= icluster8_mlp<SHIFTED, true>(A.p, s_lj, W, L, row[k], k, false, m, J, fx[k], fy[k],
                                                            fz[k], G, *M, mo);
                    else
                        any |= icluster8_mlp<SHIFTED, false>(A.p, s_lj, W, L, row[k], k, diag, m, J, fx[k], fy[k],
                                                             fz[k], G, *M, mo);
                } else if (!diag && m == ~0ull) {
                    any |= icluster8<ELEC, ENERGY, FIT, SHIFTED, true, PRUNE>(A.p, s_lj, W, L, row[k], k, false, m,
                                                                              J, fx[k], fy[k], fz[k], G, e_lj, e_c,
                                                                              n_inc, keep);
                } else {
                    any |= icluster8<ELEC, ENERGY, FIT, SHIFTED, false, PRUNE>(A.p, s_lj, W, L, row[k], k, diag, m,
                                                                               J, fx[k], fy[k], fz[k], G, e_lj,
                                                                               e_c, n_inc, keep);
                }
            }
        }
        if constexpr (PRUNE) {
            if (lane == t) my_keep = keep;
        }
        if (!any) continue;
        // j-force: the lane's two pairs, added by every lane (the L2 adds
        // the 4 lanes' contributions to a j-particle faster than two rounds
        // of shuffles do)
        atomicAdd(&A.fslot[cjt * 8 + L.j],
                  make_float4(-(G.x.x + G.x.y), -(G.y.x + G.y.y), -(G.z.x + G.z.y), 0.0f));
    }
    if constexpr (PRUNE) {
        // compact the kept j-entries of this chunk, in order
        const unsigned kb = __ballot_sync(full, my_keep != 0);
        const int pos = __popc(kb & ((1u << lane) - 1u));
        if (my_keep) {
            const long long o = (long long)j_out + kept + pos;
            A.cj_p[o] = (W.w[lane] & kCjMask) | (int)(my_keep << kSuperShift);
#pragma unroll
            for (int k = 0; k < kSuper8; ++k)
                A.mask_p[k * A.jstride + o] = ((my_keep >> k) & 1u) ? W.m[k][lane] : 0ull;
        }
        kept += __popc(kb);
        unsigned nk = __popc(my_keep);
        for (int o = 16; o > 0; o >>= 1) nk += __shfl_xor_sync(full, nk, o);
        keys += nk;
    }
    __syncwarp();
}

// Blocks per SM the force kernels are compiled for (register budget, as
// measured fastest): the force kernel at 7 blocks of 4 warps (72
// registers), the energy and fused force + prune kernels at 6, the
// network's at 4.
template <int ELEC, bool ENERGY, bool PRUNE>
constexpr int force_min_blocks() {
    return ELEC == NB_ELEC_EWALD_MLP ? 4 : (ENERGY || PRUNE ? 6 : 7);
}

template <int ELEC, bool ENERGY, bool FIT, bool PRUNE = false>
__global__ void __launch_bounds__(32 * kForceWarps, force_min_blocks<ELEC, ENERGY, PRUNE>())
k_force8(ForceArgs A) {
    extern __shared__ float2 s_lj[];
    __shared__ WarpSmem s_w[kForceWarps];
    const unsigned full = 0xffffffffu;
    const int nt2 = A.p.ntypes * A.p.ntypes;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float2 v = A.c6c12[k];
        s_lj[k] = make_float2(-6.0f * v.x, 12.0f * v.y);
    }
    if constexpr (ELEC == NB_ELEC_EWALD_TAB) {
        // the force-factor table follows the LJ table
        for (int k = threadIdx.x; k < A.p.tab_n; k += blockDim.x) s_lj[nt2 + k] = A.ewald_tab[k];
    }
    const MlpTC* M = nullptr;
    float* mo = nullptr;
    if constexpr (ELEC == NB_ELEC_EWALD_MLP) {
        // the network in per-lane layout, and a 64-value exchange row per warp
        __shared__ MlpTC s_mlp;
        __shared__ float s_mo[kForceWarps][64];
        const uint4* src = reinterpret_cast<const uint4*>(A.mlp);
        uint4* dst = reinterpret_cast<uint4*>(&s_mlp);
        for (int k = threadIdx.x; k < (int)(sizeof(MlpTC) / 16); k += blockDim.x) dst[k] = src[k];
        M = &s_mlp;
        mo = s_mo[threadIdx.x >> 5];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    WarpSmem& W = s_w[threadIdx.x >> 5];
    Lane8 L;
    L.j = lane & 7;
    L.ih = lane >> 3;
    L.lower0 = L.j <= L.ih;
    L.lower1 = L.j <= L.ih + 4;
    L.sel = 1u << (L.ih * 8 + L.j);
    float e_lj = 0.0f, e_c = 0.0f;
    unsigned n_inc = 0;
    int b_acc = -1;
    int pb_acc = -1;                              // PRUNE: box of the pruned-list totals below
    unsigned long long kept_total = 0, keys_total = 0;
    const int n_used = A.ient_used[A.nbox];
    // warps take i-entries from a counter (entries differ in length); the
    // next index is requested while the current entry is processed
    // (the first entry of each warp is its warp index, so the launch does not
    // start with every warp contending for the counter; with only a few
    // entries per warp the static order wins and the counter is not used)
    const int n_warps = gridDim.x * kForceWarps;
    const bool dynamic = n_used > 8 * n_warps;
    int c_next = 0;
    for (int c = blockIdx.x * kForceWarps + (threadIdx.x >> 5); c < n_used; c = __shfl_sync(full, c_next, 0)) {
        if (lane == 0) c_next = dynamic ? n_warps + atomicAdd(A.work, 1) : c + n_warps;
        // the entry and its box by binary search (no state carried across entries)
        int b;
        const int e = ient_of(A.ient_used, A.ient_off, A.nbox, c, b);
        if (ENERGY && b != b_acc) {
            flush_energy(A.acc, b_acc, e_lj, e_c, n_inc);
            b_acc = b;
        }
        if (PRUNE && b != pb_acc) {
            if (lane == 0 && pb_acc >= 0 && kept_total) {
                atomicAdd(&A.stw[pb_acc].n_jent_pruned, kept_total);
                atomicAdd(&A.stw[pb_acc].n_keys_pruned, keys_total);
            }
            kept_total = keys_total = 0;
            pb_acc = b;
        }
        const int4 ie = A.ient[e];
        const int q = ie.x, s = ie.y, jb = ie.z, je = ie.w;
        if (jb >= je) {
            if (PRUNE && lane == 0) A.ient_p[e] = make_int4(q, s, jb, jb);
            continue;
        }
        const int2 info = A.sc_info[q];
        const int g0 = info.x, n = info.y;
        float sh[3];
        shift_vector(s, A.geo[b].L, sh);
        // stage the super-cluster's i particles: shifted coordinates as hi + lo
        if (lane < n * 8) {
            const float4 x = A.xyzq[g0 * 8 + lane];
            float4 h, l;
            two_sum(x.x, sh[0], h.x, l.x);
            two_sum(x.y, sh[1], h.y, l.y);
            two_sum(x.z, sh[2], h.z, l.z);
            h.w = x.w * A.p.fcoul;
            l.w = 0.0f;
            const int k = lane >> 3, ih = lane & 3, hh = (lane >> 2) & 1;
            float* pxy = reinterpret_cast<float*>(&W.ixy[k][ih]);
            float* pzq = reinterpret_cast<float*>(&W.izq[k][ih]);
            float* qxy = reinterpret_cast<float*>(&W.lxy[k][ih]);
            float* qz = reinterpret_cast<float*>(&W.lz[k][ih]);
            int* pr = reinterpret_cast<int*>(&W.row[k][ih]);
            pxy[hh] = h.x;
            pxy[2 + hh] = h.y;
            pzq[hh] = h.z;
            pzq[2 + hh] = h.w;
            qxy[hh] = l.x;
            qxy[2 + hh] = l.y;
            qz[hh] = l.z;
            pr[hh] = A.type_slot[g0 * 8 + lane] * A.p.ntypes * (int)sizeof(float2);
        }
        __syncwarp();
        int2 row[kSuper8];
#pragma unroll
        for (int k = 0; k < kSuper8; ++k) row[k] = W.row[k][L.ih];
        const bool center = (s == kShiftCenter);
        float2 fx[kSuper8], fy[kSuper8], fz[kSuper8];
#pragma unroll
        for (int k = 0; k < kSuper8; ++k) fx[k] = fy[k] = fz[k] = make_float2(0.f, 0.f);
        int kept = 0;
        for (int base = jb; base < je; base += 32) {
            const int bend = min(je, base + 32);
            // (the network's form runs the shifted code for every entry: its
            // tile evaluator is large, and a second copy for the unshifted
            // entries thrashes the instruction cache where both kinds are
            // frequent -- 24k box 0.75 -> 0.45 ms -- while the shift's lo
            // parts are exact zeros for an unshifted entry)
            if (center && ELEC != NB_ELEC_EWALD_MLP)
                force_entry8<ELEC, ENERGY, FIT, false, PRUNE>(A, s_lj, W, L, row, g0, true, base, bend, fx, fy, fz,
                                                              e_lj, e_c, n_inc, M, mo, jb, kept, keys_total);
            else
                force_entry8<ELEC, ENERGY, FIT, true, PRUNE>(A, s_lj, W, L, row, g0, center, base, bend, fx, fy,
                                                             fz, e_lj, e_c, n_inc, M, mo, jb, kept, keys_total);
        }
        if (PRUNE) {
            if (lane == 0) A.ient_p[e] = make_int4(q, s, jb, jb + kept);
            kept_total += kept;
        }
        // i-forces: per i-cluster, sum over the 8 lanes of each i row
        float tsum[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kSuper8; ++k) {
            if (k >= n) break;
            float f0[3] = {fx[k].x, fy[k].x, fz[k].x}, f1[3] = {fx[k].y, fy[k].y, fz[k].y};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    f0[d] += __shfl_xor_sync(full, f0[d], o);
                    f1[d] += __shfl_xor_sync(full, f1[d], o);
                }
                tsum[d] += f0[d] + f1[d];
            }
            if (L.j == 0) {
                atomicAdd(&A.fslot[(g0 + k) * 8 + L.ih], make_float4(f0[0], f0[1], f0[2], 0.0f));
                atomicAdd(&A.fslot[(g0 + k) * 8 + L.ih + 4], make_float4(f1[0], f1[1], f1[2], 0.0f));
            }
        }
        if (ENERGY && !center) {
            // i-side force of this shifted entry, for the virial
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                tsum[d] += __shfl_xor_sync(full, tsum[d], 8);
                tsum[d] += __shfl_xor_sync(full, tsum[d], 16);
            }
            if (lane == 0)
                for (int d = 0; d < 3; ++d) atomicAdd(&A.acc[b].fshift[s][d], (double)tsum[d]);
        }
        __syncwarp();
    }
    if (ENERGY) flush_energy(A.acc, b_acc, e_lj, e_c, n_inc);
    if (PRUNE && lane == 0 && pb_acc >= 0 && kept_total) {
        atomicAdd(&A.stw[pb_acc].n_jent_pruned, kept_total);
        atomicAdd(&A.stw[pb_acc].n_keys_pruned, keys_total);
    }
}

// Generic C = 4 kernel (super-clusters of one cluster): one warp per
// i-entry, lanes 0..15 hold the 4 x 4 pairs of one j-cluster and lanes
// 16..31 those of the next.
template <int ELEC, bool ENERGY, bool FIT>
__global__ void __launch_bounds__(32 * kForceWarps) k_force4(ForceArgs A) {
    extern __shared__ float2 s_lj[];
    const unsigned full = 0xffffffffu;
    const int nt2 = A.p.ntypes * A.p.ntypes;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float2 v = A.c6c12[k];
        s_lj[k] = make_float2(6.0f * v.x, 12.0f * v.y);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, i = (lane >> 2) & 3, j = lane & 3;
    float e_lj = 0.0f, e_c = 0.0f;
    unsigned n_inc = 0;
    int b_acc = -1;
    const int n_used = A.ient_used[A.nbox];
    for (int c = blockIdx.x * kForceWarps + (threadIdx.x >> 5); c < n_used; c += gridDim.x * kForceWarps) {
        // the entry and its box by binary search (no state carried across entries)
        int b;
        const int e = ient_of(A.ient_used, A.ient_off, A.nbox, c, b);
        if (ENERGY && b != b_acc) {
            flush_energy(A.acc, b_acc, e_lj, e_c, n_inc);
            b_acc = b;
        }
        const int4 ie = A.ient[e];
        const int ci = A.sc_info[ie.x].x, s = ie.y, jb = ie.z, je = ie.w;
        if (jb >= je) continue;
        float sh[3];
        shift_vector(s, A.geo[b].L, sh);
        const float4 x0 = A.xyzq[ci * 4 + i];
        float xh[3], xl[3];
        two_sum(x0.x, sh[0], xh[0], xl[0]);
        two_sum(x0.y, sh[1], xh[1], xl[1]);
        two_sum(x0.z, sh[2], xh[2], xl[2]);
        const float qi = x0.w * A.p.fcoul;
        const int ti = A.type_slot[ci * 4 + i] * A.p.ntypes;
        const bool center = (s == kShiftCenter);
        float fi[3] = {0.f, 0.f, 0.f};
        for (int k = jb; k < je; k += 2) {
            const int kk = k + half;
            const bool live = kk < je;
            const int cjt = live ? (A.cj[kk] & kCjMask) : ci;
            const unsigned long long m = live ? A.mask[kk] : 0ull;
            const float4 xj = A.xyzq[cjt * 4 + j];
            const int tj = A.type_slot[cjt * 4 + j];
            const bool diag = center && (cjt == ci);
            const float b = (float)((m >> (i * 4 + j)) & 1ull);
            const float dx = (xh[0] - xj.x) + xl[0];
            const float dy = (xh[1] - xj.y) + xl[1];
            const float dz = (xh[2] - xj.z) + xl[2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const bool inc = live && (r2 < A.p.rc2) && (b != 0.0f || !(diag && j <= i));
            if (!__any_sync(full, inc)) continue;
            float fs, vl = 0.f, vc = 0.f;
            pair_fn<ELEC, ENERGY, FIT>(A.p, inc, b, r2, qi * xj.w, s_lj[ti + tj], fs, vl, vc);
            if (ENERGY) {
                e_lj += vl;
                e_c += vc;
                n_inc += (unsigned)inc;
            }
            fi[0] = fmaf(fs, dx, fi[0]);
            fi[1] = fmaf(fs, dy, fi[1]);
            fi[2] = fmaf(fs, dz, fi[2]);
            float fjx = -fs * dx, fjy = -fs * dy, fjz = -fs * dz;
            for (int o = 4; o < 16; o <<= 1) {
                fjx += __shfl_xor_sync(full, fjx, o);
                fjy += __shfl_xor_sync(full, fjy, o);
                fjz += __shfl_xor_sync(full, fjz, o);
            }
            if (i == 0 && live) atomicAdd(&A.fslot[cjt * 4 + j], make_float4(fjx, fjy, fjz, 0.0f));
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            fi[d] += __shfl_xor_sync(full, fi[d], 1);
            fi[d] += __shfl_xor_sync(full, fi[d], 2);
            fi[d] += __shfl_xor_sync(full, fi[d], 16);
        }
        if (j == 0 && half == 0) atomicAdd(&A.fslot[ci * 4 + i], make_float4(fi[0], fi[1], fi[2], 0.0f));
        if (ENERGY && !center) {
            float t[3] = {fi[0], fi[1], fi[2]};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                t[d] += __shfl_xor_sync(full, t[d], 4);
                t[d] += __shfl_xor_sync(full, t[d], 8);
            }
            if (lane == 0)
                for (int d = 0; d < 3; ++d) atomicAdd(&A.acc[b].fshift[s][d], (double)t[d]);
        }
    }
    if (ENERGY) flush_energy(A.acc, b_acc, e_lj, e_c, n_inc);
}

// Resident blocks per SM of a force kernel at kForceWarps warps and smem
// bytes of dynamic shared memory, queried once per kernel, device and size
// (the query costs microseconds of host time, every frame otherwise).  All
// force kernels share one signature, so the kernel's address is in the key.
static cudaError_t force_blocks_per_sm(void (*kern)(ForceArgs), size_t smem, int* per_sm) {
    static std::mutex m;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_tuple(reinterpret_cast<const void*>(kern), dev, smem);
    std::lock_guard<std::mutex> lock(m);
    const auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, 32 * kForceWarps, smem);
    if (e != cudaSuccess) return e;
    if (*per_sm < 1) *per_sm = 1;
    cache[key] = *per_sm;
    return cudaSuccess;
}

template <int ELEC, bool ENERGY, bool FIT, bool PRUNE = false>
static cudaError_t launch_force_t(const ForceArgs& A, int C, int n_sm, cudaStream_t s) {
    const size_t smem = sizeof(float2) * A.p.ntypes * A.p.ntypes;
    auto kern = PRUNE ? k_force8<ELEC, ENERGY, FIT, PRUNE>
                      : ((C == 8) ? k_force8<ELEC, ENERGY, FIT> : k_force4<ELEC, ENERGY, FIT>);
    int per_sm = 0;
    const cudaError_t e = force_blocks_per_sm(kern, smem, &per_sm);
    if (e != cudaSuccess) return e;
    kern<<<n_sm * per_sm, 32 * kForceWarps, smem, s>>>(A);
    return cudaGetLastError();
}

template <int ELEC, bool ENERGY>
static cudaError_t launch_force_e(const ForceArgs& A, int C, int n_sm, cudaStream_t s) {
    if (ELEC == NB_ELEC_EWALD && A.p.use_fit) return launch_force_t<ELEC, ENERGY, true>(A, C, n_sm, s);
    return launch_force_t<ELEC, ENERGY, false>(A, C, n_sm, s);
}

// The tabulated kernel (forces only, 8-particle clusters): the table follows
// the LJ table in dynamic shared memory.
template <bool PRUNE>
static cudaError_t launch_force_tab(const ForceArgs& A, int n_sm, cudaStream_t s) {
    auto kern = k_force8<NB_ELEC_EWALD_TAB, false, true, PRUNE>;
    const size_t smem = sizeof(float2) * (A.p.ntypes * A.p.ntypes + A.p.tab_n);
    static std::atomic<unsigned long long> smem_set{0};
    cudaError_t e = smem_opt_in(kern, 64 * 1024, smem_set);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = force_blocks_per_sm(kern, smem, &per_sm);
    if (e != cudaSuccess) return e;
    kern<<<n_sm * per_sm, 32 * kForceWarps, smem, s>>>(A);
    return cudaGetLastError();
}

// The tabulated force factor G(w) = (erf(x) - 2x/sqrt(pi) exp(-x^2)) / x^3,
// x = sqrt(w), on w = k w_max / n (FP64, series near w = 0), stored as
// {G_k, G_{k+1} - G_k}.
__global__ void k_ewald_table(float2* tab, int n, double wmax) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double g[2];
        for (int d = 0; d < 2; ++d) {
            const double w = (k + d) * wmax / n;
            if (w < 1e-6) {
                g[d] = 4.0 / (3.0 * sqrt(M_PI)) * (1.0 - 0.6 * w + 3.0 / 14.0 * w * w);
            } else {
                const double x = sqrt(w);
                g[d] = (erf(x) - 2.0 * x / sqrt(M_PI) * exp(-w)) / (w * x);
            }
        }
        tab[k] = make_float2((float)g[0], (float)(g[1] - g[0]));
    }
}

cudaError_t launch_ewald_table(float2* tab, int n, double wmax, cudaStream_t s) {
    k_ewald_table<<<(n + 255) / 256, 256, 0, s>>>(tab, n, wmax);
    return cudaGetLastError();
}

cudaError_t launch_force(const Workspace& ws, const ForceParams& p, int C, int n_sm, cudaStream_t s) {
    ForceArgs A;
    A.ient = p.use_pruned ? ws.ient_p : ws.ient;
    A.cj = p.use_pruned ? ws.cj_p : ws.cj;
    A.mask = p.use_pruned ? ws.mask_p : ws.mask;
    A.jstride = ws.jstride;
    A.xyzq = ws.xyzq;
    A.xjd = ws.xjd;
    A.type_slot = ws.type_slot;
    A.fslot = ws.fslot;
    A.c6c12 = ws.c6c12;
    A.sc_info = ws.sc_info;
    A.ient_off = ws.lay.ient_off;
    A.st = ws.st;
    A.geo = ws.geo;
    A.acc = ws.acc;
    A.mlp = ws.mlp;
    A.nbox = ws.nbox;
    A.ient_used = ws.ient_used;
    A.ewald_tab = ws.ewald_tab;
    A.work = ws.work;
    A.ient_p = ws.ient_p;
    A.cj_p = ws.cj_p;
    A.mask_p = ws.mask_p;
    A.stw = ws.st;
    A.p = p;
    // the accumulators hold energies, pair counts and shift forces, which
    // only energy evaluations produce and read
    cudaError_t e = cudaSuccess;
    if (p.want_energy) {
        e = cudaMemsetAsync(ws.acc, 0, sizeof(Accum) * ws.nbox, s);
        if (e != cudaSuccess) return e;
    }
    if (p.prune) {
        // the fused force + prune kernel: forces only, 8-particle clusters,
        // not the surrogate (checked by the caller), on the outer list
        if (p.elec == NB_ELEC_EWALD_TAB) return launch_force_tab<true>(A, n_sm, s);
        if (p.elec == NB_ELEC_RF) return launch_force_t<NB_ELEC_RF, false, false, true>(A, C, n_sm, s);
        if (p.use_fit) return launch_force_t<NB_ELEC_EWALD, false, true, true>(A, C, n_sm, s);
        return launch_force_t<NB_ELEC_EWALD, false, false, true>(A, C, n_sm, s);
    }
    if (p.elec == NB_ELEC_EWALD_TAB) return launch_force_tab<false>(A, n_sm, s);
    if (p.elec == NB_ELEC_EWALD_MLP) {
        // forces only, 8-particle clusters (checked by the caller)
        auto kern = k_force8<NB_ELEC_EWALD_MLP, false, true>;
        const size_t smem = sizeof(float2) * A.p.ntypes * A.p.ntypes;
        int per_sm = 0;
        e = force_blocks_per_sm(kern, smem, &per_sm);
        if (e != cudaSuccess) return e;
        kern<<<n_sm * per_sm, 32 * kForceWarps, smem, s>>>(A);
        return cudaGetLastError();
    }
    if (p.elec == NB_ELEC_RF)
        return p.want_energy ? launch_force_e<NB_ELEC_RF, true>(A, C, n_sm, s)
                             : launch_force_e<NB_ELEC_RF, false>(A, C, n_sm, s);
    return p.want_energy ? launch_force_e<NB_ELEC_EWALD, true>(A, C, n_sm, s)
                         : launch_force_e<NB_ELEC_EWALD, false>(A, C, n_sm, s);
}

}  // namespace nbc
