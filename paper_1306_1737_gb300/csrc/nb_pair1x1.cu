// The particle-pair (1 x 1) comparison path: the classic Verlet list the
// paper measures its cluster pairs against (Sec. 4-5, Table 3: M x N versus
// 1 x 1 setups), run on the same GPU with the same interactions.
//
// k_pairlist_1x1: expands the outer cluster-pair list into a full particle
//   neighbour list (every pair within rlist stored for both particles),
//   one warp per i-entry; entries pack the neighbour's slot, the periodic
//   shift and whether the pair is force-field excluded.
// k_force_1x1: 4 to 16 lanes per particle walk its neighbours, compute each
//   pair with the cluster kernels' pair function (Sec. 3.2), sum the force
//   with shuffles and write it once (no atomics: the list is full, each pair
//   is computed twice).
#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace nbc {

constexpr int kNbrShiftBits = 5;            // shift index 0..26
constexpr int kNbrExclBit = 1 << kNbrShiftBits;
constexpr int kNbrSlotShift = kNbrShiftBits + 1;

struct Pair1x1Args {
    Workspace ws;
    float rl2;
    int max_nbr;
    int* nbr;      // [n_atoms][max_nbr]
    int* count;    // [n_atoms]
};

constexpr int kExpandWarps = 4;

template <int C, int S>
__global__ void __launch_bounds__(32 * kExpandWarps) k_pairlist_1x1(Pair1x1Args A) {
    constexpr int PPL = (C * C + 31) / 32;
    constexpr int NA = S * C;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    __shared__ float4 s_h[kExpandWarps][NA];
    __shared__ float4 s_l[kExpandWarps][NA];
    const Workspace& W = A.ws;
    const int n_used = W.ient_used[W.nbox];
    for (int c = blockIdx.x * kExpandWarps + wib; c < n_used; c += gridDim.x * kExpandWarps) {
        int b;
        const int e = ient_of(W.ient_used, W.lay.ient_off, W.nbox, c, b);
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
        for (int t = jb; t < je; ++t) {
            const unsigned w = (unsigned)W.cj[t];
            const int cjt = (int)(w & kCjMask);
            unsigned bits = w >> kSuperShift;
            while (bits) {
                const int k = __ffs(bits) - 1;
                bits &= bits - 1;
                const unsigned long long m = W.mask[k * W.jstride + t];
                const bool diag = (cjt == g0 + k) && (s == kShiftCenter);
#pragma unroll
                for (int kk = 0; kk < PPL; ++kk) {
                    const int p = lane + 32 * kk;
                    if (p >= C * C) continue;
                    const int i = p / C, j = p % C;
                    if (diag && j <= i) continue;
                    const int si = (g0 + k) * C + i, sj = cjt * C + j;
                    const int ai = W.atom_of_slot[si], aj = W.atom_of_slot[sj];
                    if (ai < 0 || aj < 0) continue;
                    const float4 h = s_h[wib][k * C + i], l = s_l[wib][k * C + i];
                    const float4 xj = W.xyzq[sj];
                    const float dx = (h.x - xj.x) + l.x;
                    const float dy = (h.y - xj.y) + l.y;
                    const float dz = (h.z - xj.z) + l.z;
                    if (!(fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < A.rl2)) continue;
                    const int excl = ((m >> p) & 1ull) ? 0 : kNbrExclBit;
                    const int pi = atomicAdd(&A.count[ai], 1);
                    const int pj = atomicAdd(&A.count[aj], 1);
                    if (pi < A.max_nbr)
                        A.nbr[(long long)ai * A.max_nbr + pi] = (sj << kNbrSlotShift) | excl | s;
                    if (pj < A.max_nbr)
                        A.nbr[(long long)aj * A.max_nbr + pj] = (si << kNbrSlotShift) | excl | (26 - s);
                    if (pi >= A.max_nbr || pj >= A.max_nbr) set_flag(&W.st[b], NB_ERR_CAPACITY);
                }
            }
        }
        __syncwarp();
    }
}

struct Force1x1Args {
    Workspace ws;
    ForceParams p;
    int C;
    int max_nbr;
    const int* nbr;
    const int* count;
};

// TPP consecutive lanes per slot (consecutive slot groups hold neighbouring
// particles): lane r of a group takes neighbours r, r + TPP, ... of the
// slot's list, and the group sums its partial forces with shuffles, so a box
// of a few ten thousand particles still fills the GPU (TPP = 16, 8 or 4 for
// small, medium and large boxes: the fastest measured per size).  Neighbour
// slots come from the list, which holds current slots only.
template <int ELEC, bool FIT, int TPP>
__global__ void __launch_bounds__(256) k_force_1x1(Force1x1Args A) {
    constexpr int kTpp = TPP;
    extern __shared__ float2 s_lj[];
    const int nt2 = A.p.ntypes * A.p.ntypes;
    for (int k = threadIdx.x; k < nt2; k += blockDim.x) {
        const float2 v = A.ws.c6c12[k];
        s_lj[k] = make_float2(6.0f * v.x, 12.0f * v.y);
    }
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const Workspace& W = A.ws;
    const int r = threadIdx.x % kTpp;
    const long long nslot = (long long)W.clu_total * A.C;
    const long long stride = (long long)gridDim.x * (blockDim.x / kTpp);
    // whole warps iterate together (the group reduction is a warp shuffle)
    const long long warp_first = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / kTpp;
    for (long long base = warp_first; base < nslot; base += stride) {
        const long long si = base + (threadIdx.x & 31) / kTpp;
        bool live = si < nslot;
        int a = -1, b = 0;
        if (live) {
            // only the slots of each box's current clusters hold particles; the
            // rest of the box's slot region is unused capacity
            const int g = (int)(si / A.C);
            b = find_box(W.lay.clu_off, W.nbox, g);
            if (g - W.lay.clu_off[b] >= W.st[b].nclu) live = false;
            else {
                a = W.atom_of_slot[si];
                if (a < 0 || a >= W.atom_total) live = false;
            }
        }
        float fx = 0.f, fy = 0.f, fz = 0.f;
        float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
            const float* L = W.geo[b].L;
            xi = W.xyzq[si];
            const float qi = xi.w * A.p.fcoul;
            const int ti = W.type_slot[si] * A.p.ntypes;
            const int cnt = min(A.count[a], A.max_nbr);
            const int* list = A.nbr + (long long)a * A.max_nbr;
            for (int k = r; k < cnt; k += kTpp) {
                const int v = list[k];
                const int sj = (int)((unsigned)v >> kNbrSlotShift), s = v & (kNbrExclBit - 1);
                const float bit = (v & kNbrExclBit) ? 0.0f : 1.0f;
                const float4 xj = W.xyzq[sj];
                float dx, dy, dz;
                if (s == kShiftCenter) {
                    dx = xi.x - xj.x;
                    dy = xi.y - xj.y;
                    dz = xi.z - xj.z;
                } else {
                    float sh[3], h, l;
                    shift_vector(s, L, sh);
                    two_sum(xi.x, sh[0], h, l);
                    dx = (h - xj.x) + l;
                    two_sum(xi.y, sh[1], h, l);
                    dy = (h - xj.y) + l;
                    two_sum(xi.z, sh[2], h, l);
                    dz = (h - xj.z) + l;
                }
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const bool inc = r2 < A.p.rc2;
                float fs, vl, vc;
                pair_fn<ELEC, false, FIT>(A.p, inc, bit, r2, qi * xj.w, s_lj[ti + W.type_slot[sj]], fs, vl, vc);
                fx = fmaf(fs, dx, fx);
                fy = fmaf(fs, dy, fy);
                fz = fmaf(fs, dz, fz);
            }
        }
#pragma unroll
        for (int o = kTpp / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(full, fx, o);
            fy += __shfl_xor_sync(full, fy, o);
            fz += __shfl_xor_sync(full, fz, o);
        }
        if (live && r == 0) W.fslot[si] = make_float4(fx, fy, fz, 0.0f);
    }
}

cudaError_t launch_pairlist_1x1(const Workspace& ws, int C, float rlist, int max_nbr, int* nbr, int* count,
                                int n_sm, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (ws.atom_total > 0 ? ws.atom_total : 1), s);
    if (e != cudaSuccess) return e;
    Pair1x1Args A;
    A.ws = ws;
    A.rl2 = rlist * rlist;
    A.max_nbr = max_nbr;
    A.nbr = nbr;
    A.count = count;
    const int blocks = n_sm * 16;
    if (C == 8)
        k_pairlist_1x1<8, super_size(8)><<<blocks, 32 * kExpandWarps, 0, s>>>(A);
    else
        k_pairlist_1x1<4, super_size(4)><<<blocks, 32 * kExpandWarps, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_force_1x1(const Workspace& ws, const ForceParams& p, int C, int max_nbr, const int* nbr,
                             const int* count, cudaStream_t s) {
    Force1x1Args A;
    A.ws = ws;
    A.p = p;
    A.C = C;
    A.max_nbr = max_nbr;
    A.nbr = nbr;
    A.count = count;
    const size_t smem = sizeof(float2) * p.ntypes * p.ntypes;
    const long long nslot = (long long)ws.clu_total * C;
    const int tpp = nslot < (1 << 17) ? 16 : (nslot < (1 << 20) ? 8 : 4);
    long long blocks = (nslot * tpp + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    const int nb = (int)blocks;
    if (p.elec == NB_ELEC_RF) {
        if (tpp == 16) k_force_1x1<NB_ELEC_RF, false, 16><<<nb, 256, smem, s>>>(A);
        else if (tpp == 8) k_force_1x1<NB_ELEC_RF, false, 8><<<nb, 256, smem, s>>>(A);
        else k_force_1x1<NB_ELEC_RF, false, 4><<<nb, 256, smem, s>>>(A);
    } else if (p.use_fit) {
        if (tpp == 16) k_force_1x1<NB_ELEC_EWALD, true, 16><<<nb, 256, smem, s>>>(A);
        else if (tpp == 8) k_force_1x1<NB_ELEC_EWALD, true, 8><<<nb, 256, smem, s>>>(A);
        else k_force_1x1<NB_ELEC_EWALD, true, 4><<<nb, 256, smem, s>>>(A);
    } else {
        if (tpp == 16) k_force_1x1<NB_ELEC_EWALD, false, 16><<<nb, 256, smem, s>>>(A);
        else if (tpp == 8) k_force_1x1<NB_ELEC_EWALD, false, 8><<<nb, 256, smem, s>>>(A);
        else k_force_1x1<NB_ELEC_EWALD, false, 4><<<nb, 256, smem, s>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace nbc
