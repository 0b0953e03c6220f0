// Pair-distance histogram over the cluster-pair list: the pair correlation
// function, limited-range pair work that the paper names beside force
// calculation (Sec. 1).  For such cheap pair work the paper rebuilds the
// list for every evaluation and drops both the particle-pair pruning and the
// cut-off conditional (Sec. 2.3): every listed pair is binned, and pairs at
// or beyond r_max fall into one overflow bin instead of being tested.
//
// One warp per outer i-entry.  k_rdf (any C, used for C = 4) walks the
// (j-entry, particle pair) space of a chunk of up to 32 j-entries flat, 32
// pairs per step (two 4 x 4 cluster pairs), so every lane has a pair at every
// step; k_rdf8 (C = 8) keeps the force kernel's lane layout.  A pair counts when its mask bit is set (distinct real
// particles, not force-field excluded; on the unshifted diagonal only
// j > i, so each pair once) and its types match the selection; its bin is
// min(int(r / dr), nbins) with r from the FP32 distance vector (shift as
// hi + lo, as in the other kernels).  Counts go to 32-bit histograms in
// shared memory (see RdfBins) that are added to the box's 64-bit histogram
// in global memory.
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

// Histogram bookkeeping of a block.  The block takes one contiguous range
// [c0, c1) of the compact i-entry index (so it meets few boxes) and keeps one
// shared histogram for its home box (the box of entry c0), fed by all of its
// warps and added to global memory once at the end; a warp that meets another
// box counts into its own histogram, flushed when its box changes.  One
// global flush per block instead of one per warp keeps the 64-bit atomics on
// each bin few.
struct RdfBins {
    unsigned* blk;      // [nbins + 1] home-box histogram
    unsigned* own;      // [nbins + 1] this warp's histogram for other boxes
    int nb1, c0, c1, home, b_own;
};

__device__ __forceinline__ RdfBins rdf_begin(const Workspace& W, int nbins, unsigned* s_hist) {
    RdfBins H;
    H.nb1 = nbins + 1;
    const int wib = threadIdx.x >> 5;
    H.blk = s_hist + kRdfWarps * H.nb1;
    H.own = s_hist + wib * H.nb1;
    for (int k = threadIdx.x; k < (kRdfWarps + 1) * H.nb1; k += blockDim.x) s_hist[k] = 0u;
    const int n_used = W.ient_used[W.nbox];
    const int per = (n_used + gridDim.x - 1) / gridDim.x;
    H.c0 = min(n_used, blockIdx.x * per);
    H.c1 = min(n_used, H.c0 + per);
    int home = -1;
    if (H.c0 < H.c1) ient_of(W.ient_used, W.lay.ient_off, W.nbox, H.c0, home);
    H.home = home;
    H.b_own = -1;
    __syncthreads();
    return H;
}

__device__ __forceinline__ unsigned* rdf_bins_for(RdfBins& H, int b, unsigned long long* out, int lane) {
    if (b == H.home) return H.blk;
    if (b != H.b_own) {
        if (H.b_own >= 0) rdf_flush(H.own, H.nb1, out + (long long)H.b_own * H.nb1, lane);
        H.b_own = b;
    }
    return H.own;
}

__device__ __forceinline__ void rdf_end(RdfBins& H, unsigned long long* out, int lane) {
    if (H.b_own >= 0) rdf_flush(H.own, H.nb1, out + (long long)H.b_own * H.nb1, lane);
    __syncthreads();
    if (H.home >= 0) {
        for (int k = threadIdx.x; k < H.nb1; k += blockDim.x) {
            const unsigned v = H.blk[k];
            if (v) atomicAdd(&out[(long long)H.home * H.nb1 + k], (unsigned long long)v);
        }
    }
}

template <int C, int S>
__global__ void __launch_bounds__(32 * kRdfWarps) k_rdf(RdfArgs A) {
    constexpr int NA = S * C;
    constexpr int PP = C * C;     // particle pairs per cluster pair
    extern __shared__ unsigned s_hist[];            // [kRdfWarps + 1][nbins + 1]
    __shared__ float4 s_h[kRdfWarps][NA];           // shifted i particles: hi part
    __shared__ float4 s_l[kRdfWarps][NA];           // and lo part
    __shared__ int s_ti[kRdfWarps][NA];             // i types
    __shared__ int s_w[kRdfWarps][32];              // j-entry words of the chunk
    __shared__ unsigned long long s_m[kRdfWarps][S][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const Workspace& W = A.ws;
    RdfBins H = rdf_begin(W, A.nbins, s_hist);
    const bool all_types = A.type_a < 0;
    for (int c = H.c0 + wib; c < H.c1; c += kRdfWarps) {
        int b;
        const int e = ient_of(W.ient_used, W.lay.ient_off, W.nbox, c, b);
        unsigned* hist = rdf_bins_for(H, b, A.hist, lane);
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
    rdf_end(H, A.hist, lane);
}

// The 8-particle form: lane (ih, j) = (lane / 8, lane % 8) bins pairs
// (ih, j) and (ih + 4, j) of every i-cluster, as in the force kernel; the
// lane's shifted i-particles and types stay in registers for the entry and
// the j-particles (and types) of a chunk of 32 j-entries are copied to
// shared memory with all copies in flight at once.
template <int S>
__global__ void __launch_bounds__(32 * kRdfWarps) k_rdf8(RdfArgs A) {
    extern __shared__ unsigned s_hist[];            // [kRdfWarps + 1][nbins + 1]
    __shared__ float4 s_xj[kRdfWarps][32][8];
    __shared__ int s_tj[kRdfWarps][32][8];
    __shared__ unsigned long long s_m[kRdfWarps][S][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int j = lane & 7, ih = lane >> 3;
    const int bit = ih * 8 + j;   // the lane's pairs: bit and bit + 32 of a mask
    const Workspace& W = A.ws;
    RdfBins H = rdf_begin(W, A.nbins, s_hist);
    const bool all_types = A.type_a < 0;
    for (int c = H.c0 + wib; c < H.c1; c += kRdfWarps) {
        int b;
        const int e = ient_of(W.ient_used, W.lay.ient_off, W.nbox, c, b);
        unsigned* hist = rdf_bins_for(H, b, A.hist, lane);
        const int4 ie = W.ient[e];
        const int q = ie.x, s = ie.y, jb = ie.z, je = ie.w;
        const int2 info = W.sc_info[q];
        const int g0 = info.x;
        float sh[3];
        shift_vector(s, W.geo[b].L, sh);
        float h0[S][3], l0[S][3], h1[S][3], l1[S][3];
        int ti0[S], ti1[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int kk = k < info.y ? k : 0;
            const int s0 = (g0 + kk) * 8 + ih;
            const float4 a = W.xyzq[s0], a1 = W.xyzq[s0 + 4];
            ti0[k] = W.type_slot[s0];
            ti1[k] = W.type_slot[s0 + 4];
            two_sum(a.x, sh[0], h0[k][0], l0[k][0]);
            two_sum(a.y, sh[1], h0[k][1], l0[k][1]);
            two_sum(a.z, sh[2], h0[k][2], l0[k][2]);
            two_sum(a1.x, sh[0], h1[k][0], l1[k][0]);
            two_sum(a1.y, sh[1], h1[k][1], l1[k][1]);
            two_sum(a1.z, sh[2], h1[k][2], l1[k][2]);
        }
        for (int base = jb; base < je; base += 32) {
            const int nt = min(32, je - base);
            int my_w = 0;
            if (lane < nt) {
                my_w = W.cj[base + lane];
#pragma unroll
                for (int k = 0; k < S; ++k) s_m[wib][k][lane] = W.mask[k * W.jstride + base + lane];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int t = 4 * r + ih;
                const int wt = __shfl_sync(full, my_w, t);
                if (t < nt) {
                    const int sj = (wt & kCjMask) * 8 + j;
                    copy16_async(&s_xj[wib][t][j], W.xyzq + sj);
                    copy4_async(&s_tj[wib][t][j], W.type_slot + sj);
                }
            }
            copy_async_wait_all();
            __syncwarp();
            for (int t = 0; t < nt; ++t) {
                const unsigned bits = (unsigned)__shfl_sync(full, my_w, t) >> kSuperShift;
                const float4 xj = s_xj[wib][t][j];
                const int tj = s_tj[wib][t][j];
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    if ((bits >> k) & 1u) {
                        const unsigned long long m = s_m[wib][k][t];
                        const bool u0 = ((unsigned)m >> bit) & 1u, u1 = ((unsigned)(m >> 32) >> bit) & 1u;
                        const bool sel0 = all_types || (ti0[k] == A.type_a && tj == A.type_b) ||
                                          (ti0[k] == A.type_b && tj == A.type_a);
                        const bool sel1 = all_types || (ti1[k] == A.type_a && tj == A.type_b) ||
                                          (ti1[k] == A.type_b && tj == A.type_a);
                        const float dx0 = (h0[k][0] - xj.x) + l0[k][0], dx1 = (h1[k][0] - xj.x) + l1[k][0];
                        const float dy0 = (h0[k][1] - xj.y) + l0[k][1], dy1 = (h1[k][1] - xj.y) + l1[k][1];
                        const float dz0 = (h0[k][2] - xj.z) + l0[k][2], dz1 = (h1[k][2] - xj.z) + l1[k][2];
                        const float r20 = fmaxf(fmaf(dx0, dx0, fmaf(dy0, dy0, dz0 * dz0)), 1e-30f);
                        const float r21 = fmaxf(fmaf(dx1, dx1, fmaf(dy1, dy1, dz1 * dz1)), 1e-30f);
                        // no cut-off test: distances at or beyond r_max saturate
                        // into the overflow bin
                        const int bin0 = min((int)(r20 * rsqrtf(r20) * A.inv_dr), A.nbins);
                        const int bin1 = min((int)(r21 * rsqrtf(r21) * A.inv_dr), A.nbins);
                        if (u0 && sel0) atomicAdd(&hist[bin0], 1u);
                        if (u1 && sel1) atomicAdd(&hist[bin1], 1u);
                    }
                }
            }
            __syncwarp();   // s_xj, s_tj and s_m are rewritten by the next chunk
        }
    }
    rdf_end(H, A.hist, lane);
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
    // histograms: one per warp and the block's; static staging up to ~21 KB
    const size_t smem = sizeof(unsigned) * (kRdfWarps + 1) * (size_t)(nbins + 1);
    const int blocks = n_sm * 6;   // 6 blocks of 4 warps fit an SM (registers)
    cudaError_t e;
    if (C == 8) {
        e = cudaFuncSetAttribute(k_rdf8<super_size(8)>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rdf8<super_size(8)><<<blocks, 32 * kRdfWarps, smem, s>>>(A);
    } else {
        e = cudaFuncSetAttribute(k_rdf<4, super_size(4)>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rdf<4, super_size(4)><<<blocks, 32 * kRdfWarps, smem, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace nbc
