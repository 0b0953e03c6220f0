// Pruning of the cluster-pair list with a particle-pair distance criterion
// (Sec. 2.3: done on the GPU, close to the cut-off).
//
// One warp per outer i-entry.  Each j-entry's C x C particle pairs are tested
// by the whole warp (C = 8: two pairs per lane); an entry is kept iff a pair
// the interaction counts (any pair except, on the unshifted diagonal, j <= i;
// dummies sit far away and never pass) is closer than r_prune.  Kept entries
// are compacted in order into the pruned arrays at the same offsets as the
// outer list, so the pruned i-entry e covers [j_begin, j_begin + kept).
#include "nb_internal.cuh"

namespace nbc {

struct PruneArgs {
    DevState* st;
    const float4* xyzq;
    const int4* ient;
    const int* cj;
    const unsigned long long* mask;
    int4* ient_p;
    int* cj_p;
    unsigned long long* mask_p;
    float L[3];
    float rp2;
    long long ient_cap;
};

constexpr int kPruneWarps = 4;

template <int C>
__global__ void __launch_bounds__(32 * kPruneWarps) k_prune(PruneArgs A) {
    constexpr int PPL = (C * C + 31) / 32;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long nient = min((long long)A.st->n_ient, A.ient_cap);
    unsigned long long kept_total = 0;
    for (long long e = (long long)blockIdx.x * kPruneWarps + (threadIdx.x >> 5); e < nient;
         e += (long long)gridDim.x * kPruneWarps) {
        const int4 ie = A.ient[e];
        const int ci = ie.x, s = ie.y, jb = ie.z, je = ie.w;
        const float sh[3] = {(float)(s / 9 - 1) * A.L[0], (float)((s / 3) % 3 - 1) * A.L[1],
                             (float)(s % 3 - 1) * A.L[2]};
        float xh[PPL][3], xl[PPL][3];
        int pi[PPL], pj[PPL];
        bool pv[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int p = lane + 32 * k;
            pv[k] = p < C * C;
            pi[k] = pv[k] ? p / C : 0;
            pj[k] = pv[k] ? p % C : 0;
            const float4 x = A.xyzq[ci * C + pi[k]];
            two_sum(x.x, sh[0], xh[k][0], xl[k][0]);
            two_sum(x.y, sh[1], xh[k][1], xl[k][1]);
            two_sum(x.z, sh[2], xh[k][2], xl[k][2]);
        }
        int kept = 0;
        for (int base = jb; base < je; base += 32) {
            const int nt = min(32, je - base);
            int my_cj = 0;
            unsigned long long my_m = 0;
            if (lane < nt) {
                my_cj = A.cj[base + lane];
                my_m = A.mask[base + lane];
            }
            bool my_keep = false;
            for (int t = 0; t < nt; ++t) {
                const int cjt = __shfl_sync(full, my_cj, t);
                const bool diag = (cjt == ci) && (s == kShiftCenter);
                bool hit = false;
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    if (!pv[k]) continue;
                    const float4 xj = A.xyzq[cjt * C + pj[k]];
                    const float dx = (xh[k][0] - xj.x) + xl[k][0];
                    const float dy = (xh[k][1] - xj.y) + xl[k][1];
                    const float dz = (xh[k][2] - xj.z) + xl[k][2];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const bool counted = !(diag && pj[k] <= pi[k]);
                    hit |= counted && (r2 < A.rp2);
                }
                const bool any = __any_sync(full, hit);
                if (lane == t) my_keep = any;
            }
            const unsigned kb = __ballot_sync(full, my_keep);
            const int pos = __popc(kb & ((1u << lane) - 1u));
            if (my_keep) {
                A.cj_p[jb + kept + pos] = my_cj;
                A.mask_p[jb + kept + pos] = my_m;
            }
            kept += __popc(kb);
        }
        if (lane == 0) A.ient_p[e] = make_int4(ci, s, jb, jb + kept);
        kept_total += kept;
    }
    if (lane == 0 && kept_total) atomicAdd(&A.st->n_jent_pruned, kept_total);
}

cudaError_t launch_prune(const Workspace& ws, const GridGeom& g, int C, float r_prune,
                         long long ient_cap, int n_sm, cudaStream_t s) {
    PruneArgs A;
    A.st = ws.st;
    A.xyzq = ws.xyzq;
    A.ient = ws.ient;
    A.cj = ws.cj;
    A.mask = ws.mask;
    A.ient_p = ws.ient_p;
    A.cj_p = ws.cj_p;
    A.mask_p = ws.mask_p;
    for (int k = 0; k < 3; ++k) A.L[k] = g.L[k];
    A.rp2 = r_prune * r_prune;
    A.ient_cap = ient_cap;
    cudaError_t e = cudaMemsetAsync(&ws.st->n_jent_pruned, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int blocks = n_sm * 16;
    if (C == 8)
        k_prune<8><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    else
        k_prune<4><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace nbc
