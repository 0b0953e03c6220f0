// Pair-distance histogram over the cluster-pair list: the pair correlation
// function, limited-range pair work that the paper names beside force
// calculation (Sec. 1).  For such cheap pair work the paper rebuilds the
// list for every evaluation and drops both the particle-pair pruning and the
// cut-off conditional (Sec. 2.3): every listed pair is binned, and pairs at
// or beyond r_max fall into one overflow bin instead of being tested.
//
// One warp per outer i-entry.  The warp walks the (j-entry, particle pair)
// space of a chunk of up to 32 j-entries flat, 32 pairs per step (C = 8:
// half a cluster pair; C = 4: two cluster pairs), so every lane has a pair
// at every step.  A pair counts when its mask bit is set (distinct real
// particles, not force-field excluded; on the unshifted diagonal only
// j > i, so each pair once) and its types match the selection; its bin is
// min(int(r / dr), nbins) with r from the FP32 distance vector (shift as
// hi + lo, as in the other kernels).  Counts go to a per-warp histogram in
// shared memory (32-bit), which is added to the box's 64-bit histogram in
// global memory when the warp moves to another box and at the end.
#include "nb_internal.cuh"

namespace nbc {

struct RdfArgs {
    Workspace ws;
    float inv_dr;
    int nbins;
    int type_a, type_b;    // -1: every pair
    unsigned long long* hist;   // [nbox][nbins + 1]
};

constexpr int kRdfWarps = 4;

__device__ __forceinline__ void rdf_flush(unsigned* h, int nb1, unsigned long long* out, int lane) {
    __syncwarp();
    for (int k = lane; k < nb1; k += 32) {
        const unsigned v = h[k];
        if (v) atomicAdd(&out[k], (unsigned long long)v);
        h[k] = 0u;
    }
    __syncwarp();
}

template <int C, int S>
__global__ void __launch_bounds__(32 * kRdfWarps) k_rdf(RdfArgs A) {
    constexpr int NA = S * C;
    constexpr int PP = C * C;     // particle pairs per cluster pair
    extern __shared__ unsigned s_hist[];            // [kRdfWarps][nbins + 1]
    __shared__ float4 s_h[kRdfWarps][NA];           // shifted i particles: hi part
    __shared__ float4 s_l[kRdfWarps][NA];           // and lo part
    __shared__ int s_ti[kRdfWarps][NA];             // i types
    __shared__ int s_w[kRdfWarps][32];              // j-entry words of the chunk
    __shared__ unsigned long long s_m[kRdfWarps][S][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nb1 = A.nbins + 1;
    unsigned* hist = s_hist + wib * nb1;
    for (int k = lane; k < nb1; k += 32) hist[k] = 0u;
    __syncwarp();
    const Workspace& W = A.ws;
    const bool all_types = A.type_a < 0;
    const int n_used = W.ient_used[W.nbox];
    int b_acc = -1;
    for (int c = blockIdx.x * kRdfWarps + wib; c < n_used; c += gridDim.x * kRdfWarps) {
        int b;
        const int e = ient_of(W.ient_used, W.lay.ient_off, W.nbox, c, b);
        if (b != b_acc) {
            if (b_acc >= 0) rdf_flush(hist, nb1, A.hist + (long long)b_acc * nb1, lane);
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
            s_ti[wib][lane] = W.type_slot[g0 * C + lane];
        }
        for (int base = jb; base < je; base += 32) {
            const int nt = min(32, je - base);
            if (lane < nt) {
                s_w[wib][lane] = W.cj[base + lane];
#pragma unroll
                for (int k = 0; k < S; ++k) s_m[wib][k][lane] = W.mask[k * W.jstride + base + lane];
            }
            __syncwarp();
            for (int p = lane; p < nt * PP; p += 32) {
                const int t = p / PP, ij = p % PP, i = ij / C, j = ij % C;
                const unsigned w = (unsigned)s_w[wib][t];
                const int sj = (int)(w & kCjMask) * C + j;
                const unsigned bits = w >> kSuperShift;
                const float4 xj = W.xyzq[sj];
                const int tj = W.type_slot[sj];
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    const bool u = ((bits >> k) & 1u) && ((s_m[wib][k][t] >> ij) & 1ull);
                    const int ti = s_ti[wib][k * C + i];
                    const bool sel = all_types || (ti == A.type_a && tj == A.type_b) ||
                                     (ti == A.type_b && tj == A.type_a);
                    if (u && sel) {
                        const float4 h = s_h[wib][k * C + i], l = s_l[wib][k * C + i];
                        const float dx = (h.x - xj.x) + l.x;
                        const float dy = (h.y - xj.y) + l.y;
                        const float dz = (h.z - xj.z) + l.z;
                        const float r2 = fmaxf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)), 1e-30f);
                        // no cut-off test: a distance at or beyond r_max saturates
                        // into the overflow bin
                        const int bin = min((int)(r2 * rsqrtf(r2) * A.inv_dr), A.nbins);
                        atomicAdd(&hist[bin], 1u);
                    }
                }
            }
            __syncwarp();
        }
    }
    if (b_acc >= 0) rdf_flush(hist, nb1, A.hist + (long long)b_acc * nb1, lane);
}

cudaError_t launch_rdf(const Workspace& ws, int C, float r_max, int nbins, int type_a, int type_b,
                       unsigned long long* hist, int n_sm, cudaStream_t s) {
    RdfArgs A;
    A.ws = ws;
    A.inv_dr = (float)nbins / r_max;
    A.nbins = nbins;
    A.type_a = type_a;
    A.type_b = type_b;
    A.hist = hist;
    const size_t smem = sizeof(unsigned) * kRdfWarps * (size_t)(nbins + 1);
    const int blocks = n_sm * 4;
    if (C == 8)
        k_rdf<8, super_size(8)><<<blocks, 32 * kRdfWarps, smem, s>>>(A);
    else
        k_rdf<4, super_size(4)><<<blocks, 32 * kRdfWarps, smem, s>>>(A);
    return cudaGetLastError();
}

}  // namespace nbc
