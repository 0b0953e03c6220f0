// Pruning of the cluster-pair list with a particle-pair distance criterion
// (Sec. 2.3: done on the GPU, close to the cut-off).
//
// One warp per outer i-entry (a super-cluster and a shift).  For every
// j-entry, each of its interacting i-clusters is re-tested: its C x C pairs
// are checked by the whole warp (C = 8: two pairs per lane) and its bit stays
// iff a pair the interaction counts (any pair except, on the unshifted
// diagonal, j <= i; dummies sit far away and never pass) is closer than
// r_prune.  Entries with a bit left are compacted in order into the pruned
// arrays at the outer list's offsets, so pruned i-entry e covers
// [j_begin, j_begin + kept).
#include "nb_internal.cuh"

namespace nbc {

struct PruneArgs {
    Workspace ws;
    float rp2;
};

constexpr int kPruneWarps = 4;

template <int C, int S>
__global__ void __launch_bounds__(32 * kPruneWarps) k_prune(PruneArgs A) {
    constexpr int PPL = (C * C + 31) / 32;
    constexpr int NA = S * C;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    // shifted i particles of the current super-cluster: hi and lo parts
    __shared__ float4 s_h[kPruneWarps][NA];
    __shared__ float4 s_l[kPruneWarps][NA];
    const Workspace& W = A.ws;
    int b = 0;
    unsigned long long kept_total = 0, keys_total = 0;
    int b_acc = -1;  // box whose totals are being accumulated
    int pi[PPL], pj[PPL];
    bool pv[PPL];
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int p = lane + 32 * k;
        pv[k] = p < C * C;
        pi[k] = pv[k] ? p / C : 0;
        pj[k] = pv[k] ? p % C : 0;
    }
    const int n_used = W.ient_used[W.nbox];
    // warps take i-entries from a counter (entries differ in length), the
    // next index requested while the current entry is processed
    // (the first entry of each warp is its warp index; with only a few
    // entries per warp the static order is kept)
    const int n_warps = gridDim.x * kPruneWarps;
    const bool dynamic = n_used > 8 * n_warps;
    int c_next = 0;
    for (int c = blockIdx.x * kPruneWarps + wib; c < n_used; c = __shfl_sync(full, c_next, 0)) {
        if (lane == 0) c_next = dynamic ? n_warps + atomicAdd(&W.work[1], 1) : c + n_warps;
        const int e = ient_of(W.ient_used, W.lay.ient_off, W.nbox, c, b);
        if (b != b_acc) {
            if (lane == 0 && b_acc >= 0 && kept_total) {
                atomicAdd(&W.st[b_acc].n_jent_pruned, kept_total);
                atomicAdd(&W.st[b_acc].n_keys_pruned, keys_total);
            }
            kept_total = keys_total = 0;
            b_acc = b;
        }
        const int4 ie = W.ient[e];
        const int q = ie.x, s = ie.y, jb = ie.z, je = ie.w;
        const int2 info = W.sc_info[q];
        const int g0 = info.x;
        float sh[3];
        shift_vector(s, W.geo[b].L, sh);
        if (lane < info.y * C) {
            const float4 x = W.xyzq[g0 * C + lane];
            float4 h, l;
            two_sum(x.x, sh[0], h.x, l.x);
            two_sum(x.y, sh[1], h.y, l.y);
            two_sum(x.z, sh[2], h.z, l.z);
            h.w = l.w = 0.0f;
            s_h[wib][lane] = h;
            s_l[wib][lane] = l;
        }
        __syncwarp();
        int kept = 0;
        for (int base = jb; base < je; base += 32) {
            const int nt = min(32, je - base);
            int my_w = 0;
            if (lane < nt) my_w = W.cj[base + lane];
            unsigned my_keep = 0;
            for (int t = 0; t < nt; ++t) {
                const int w = __shfl_sync(full, my_w, t);
                const int cjt = w & kCjMask;
                unsigned bits = (unsigned)w >> kSuperShift;
                float4 xj[PPL];
#pragma unroll
                for (int kk = 0; kk < PPL; ++kk) xj[kk] = W.xyzq[cjt * C + pj[kk]];
                unsigned keep = 0;
                while (bits) {
                    const int k = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const bool diag = (cjt == g0 + k) && (s == kShiftCenter);
                    bool hit = false;
#pragma unroll
                    for (int kk = 0; kk < PPL; ++kk) {
                        if (!pv[kk]) continue;
                        const float4 h = s_h[wib][k * C + pi[kk]], l = s_l[wib][k * C + pi[kk]];
                        const float dx = (h.x - xj[kk].x) + l.x;
                        const float dy = (h.y - xj[kk].y) + l.y;
                        const float dz = (h.z - xj[kk].z) + l.z;
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const bool counted = !(diag && pj[kk] <= pi[kk]);
                        hit |= counted && (r2 < A.rp2);
                    }
                    if (__any_sync(full, hit)) keep |= 1u << k;
                }
                if (lane == t) my_keep = keep;
            }
            const unsigned kb = __ballot_sync(full, my_keep != 0);
            const int pos = __popc(kb & ((1u << lane) - 1u));
            if (my_keep) {
                const long long o = jb + kept + pos;
                W.cj_p[o] = (my_w & kCjMask) | (int)(my_keep << kSuperShift);
#pragma unroll
                for (int k = 0; k < S; ++k)
                    W.mask_p[k * W.jstride + o] = ((my_keep >> k) & 1u) ? W.mask[k * W.jstride + base + lane] : 0ull;
            }
            kept += __popc(kb);
            unsigned nk = __popc(my_keep);
            for (int o = 16; o > 0; o >>= 1) nk += __shfl_xor_sync(full, nk, o);
            keys_total += nk;
        }
        if (lane == 0) W.ient_p[e] = make_int4(q, s, jb, jb + kept);
        kept_total += kept;
        __syncwarp();
    }
    if (lane == 0 && b_acc >= 0 && kept_total) {
        atomicAdd(&W.st[b_acc].n_jent_pruned, kept_total);
        atomicAdd(&W.st[b_acc].n_keys_pruned, keys_total);
    }
}

// Zero every box's pruned counters.
__global__ void k_prune_reset(Workspace ws) {
    if (threadIdx.x == 0) ws.work[1] = 0;
    for (int b = threadIdx.x; b < ws.nbox; b += blockDim.x) {
        ws.st[b].n_jent_pruned = 0;
        ws.st[b].n_keys_pruned = 0;
    }
}

cudaError_t launch_prune(const Workspace& ws, int C, float r_prune, int n_sm, cudaStream_t s) {
    PruneArgs A;
    A.ws = ws;
    A.rp2 = r_prune * r_prune;
    k_prune_reset<<<1, 256, 0, s>>>(ws);
    const int blocks = n_sm * 16;
    if (C == 8)
        k_prune<8, super_size(8)><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    else
        k_prune<4, super_size(4)><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace nbc
