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

// The 8-particle form: lane (ih, j) = (lane / 8, lane % 8) tests pairs
// (ih, j) and (ih + 4, j) of every i-cluster, as in the force kernel.  The
// lane's shifted i-particles stay in registers for the whole entry; the
// j-particles of a chunk of 32 j-entries (8 x 32 float4) are copied to shared
// memory with all copies in flight at once, so a chunk waits for one L2 round
// trip instead of one per j-entry.
template <int S>
__global__ void __launch_bounds__(32 * kPruneWarps) k_prune8(PruneArgs A) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int j = lane & 7, ih = lane >> 3;
    const bool lower0 = j <= ih, lower1 = j <= ih + 4;
    __shared__ float4 s_xj[kPruneWarps][32][8];
    const Workspace& W = A.ws;
    int b = 0;
    unsigned long long kept_total = 0, keys_total = 0;
    int b_acc = -1;
    const int n_used = W.ient_used[W.nbox];
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
        // shifted i-particles (ih) and (ih + 4) of each i-cluster: hi + lo
        float h0[S][3], l0[S][3], h1[S][3], l1[S][3];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int kk = k < info.y ? k : 0;
            const float4 a = W.xyzq[(g0 + kk) * 8 + ih], a1 = W.xyzq[(g0 + kk) * 8 + ih + 4];
            two_sum(a.x, sh[0], h0[k][0], l0[k][0]);
            two_sum(a.y, sh[1], h0[k][1], l0[k][1]);
            two_sum(a.z, sh[2], h0[k][2], l0[k][2]);
            two_sum(a1.x, sh[0], h1[k][0], l1[k][0]);
            two_sum(a1.y, sh[1], h1[k][1], l1[k][1]);
            two_sum(a1.z, sh[2], h1[k][2], l1[k][2]);
        }
        const bool center = s == kShiftCenter;
        int kept = 0;
        for (int base = jb; base < je; base += 32) {
            const int nt = min(32, je - base);
            int my_w = 0;
            if (lane < nt) my_w = W.cj[base + lane];
            // copy r covers j-entry t = 4 r + ih, particle j (8 lanes read
            // one cluster's 128 contiguous bytes)
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int t = 4 * r + ih;
                const int wt = __shfl_sync(full, my_w, t);
                if (t < nt) copy16_async(&s_xj[wib][t][j], W.xyzq + (wt & kCjMask) * 8 + j);
            }
            copy_async_wait_all();
            __syncwarp();
            unsigned my_keep = 0;
            for (int t = 0; t < nt; ++t) {
                const int w = __shfl_sync(full, my_w, t);
                const float4 xj = s_xj[wib][t][j];
                const int cjt = w & kCjMask;
                const unsigned bits = (unsigned)w >> kSuperShift;
                unsigned keep = 0;
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    if ((bits >> k) & 1u) {
                        const bool diag = center && (cjt == g0 + k);
                        const float dx0 = (h0[k][0] - xj.x) + l0[k][0], dx1 = (h1[k][0] - xj.x) + l1[k][0];
                        const float dy0 = (h0[k][1] - xj.y) + l0[k][1], dy1 = (h1[k][1] - xj.y) + l1[k][1];
                        const float dz0 = (h0[k][2] - xj.z) + l0[k][2], dz1 = (h1[k][2] - xj.z) + l1[k][2];
                        const float r20 = fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0));
                        const float r21 = fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1));
                        const bool hit = (r20 < A.rp2 && !(diag && lower0)) || (r21 < A.rp2 && !(diag && lower1));
                        if (__any_sync(full, hit)) keep |= 1u << k;
                    }
                }
                if (lane == t) my_keep = keep;
            }
            __syncwarp();   // s_xj is rewritten by the next chunk
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

cudaError_t launch_prune_reset(const Workspace& ws, cudaStream_t s) {
    k_prune_reset<<<1, 256, 0, s>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_prune(const Workspace& ws, int C, float r_prune, int n_sm, cudaStream_t s) {
    PruneArgs A;
    A.ws = ws;
    A.rp2 = r_prune * r_prune;
    k_prune_reset<<<1, 256, 0, s>>>(ws);
    const int blocks = n_sm * 16;
    if (C == 8)
        k_prune8<super_size(8)><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    else
        k_prune<4, super_size(4)><<<blocks, 32 * kPruneWarps, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace nbc
