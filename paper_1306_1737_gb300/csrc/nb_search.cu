// Cluster-pair search (Sec. 2.3, Fig. 3) and exclusion masks (Sec. 2.4).
//
// One warp per i-cluster a.  For each periodic shift s applied to a, the
// warp visits the grid columns whose x/y cells come within rlist of a's
// shifted bounding box; in each column (clusters sorted on z) a binary search
// bounds the j-clusters in z range.  Candidates b >= a (half list, Newton's
// third law; for b == a only s = 0 and the positive half of the shifts) are
// kept iff d_BB < rlist and (d_BB < rBB or some particle pair is closer than
// rlist).  Shifted coordinates are carried as an unevaluated FP32 sum hi + lo
// (TwoSum), so distances across the periodic boundary lose no precision.
// Accepted pairs get their 64-bit mask (bit i*C+j: full interaction) and are
// appended in chunks of at most kJChunk j-entries per i-entry.
#include "nb_internal.cuh"

namespace nbc {

struct SearchArgs {
    DevState* st;
    const float4* bb;
    const float4* xyzq;
    const int* atom_of_slot;
    const int* slot_of_atom;
    const int* col_clu_start;
    const int* excl_off;
    const int* excl_idx;
    float L[3];
    float inv_cx, inv_cy;
    int nx, ny;
    float rl, rl2, rbb2;
    int4* ient;
    int* cj;
    unsigned long long* mask;
    long long ient_cap, jent_cap;
    int n_atoms;
};

template <int C>
__host__ __device__ constexpr unsigned long long upper_mask() {
    unsigned long long m = 0;
    for (int i = 0; i < C; ++i)
        for (int j = i + 1; j < C; ++j) m |= 1ull << (i * C + j);
    return m;
}

template <int C>
__host__ __device__ constexpr unsigned long long diag_mask() {
    unsigned long long m = 0;
    for (int i = 0; i < C; ++i) m |= 1ull << (i * C + i);
    return m;
}

constexpr int kSearchWarps = 4;

template <int C>
__global__ void __launch_bounds__(32 * kSearchWarps) k_search(SearchArgs A) {
    constexpr int PPL = (C * C + 31) / 32;  // particle pairs per lane
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    __shared__ int s_ex_i[kSearchWarps][kMaxExclPerCluster];
    __shared__ int s_ex_s[kSearchWarps][kMaxExclPerCluster];
    __shared__ int s_buf_cj[kSearchWarps][kJChunk];
    __shared__ unsigned long long s_buf_m[kSearchWarps][kJChunk];

    const int nclu = A.st->nclu;
    const float eps = 1e-4f;
    for (int a = blockIdx.x * kSearchWarps + wib; a < nclu; a += gridDim.x * kSearchWarps) {
        const float4 blo = A.bb[2 * a], bhi = A.bb[2 * a + 1];
        const int aos = lane < C ? A.atom_of_slot[a * C + lane] : -1;
        const unsigned realA = __ballot_sync(full, aos >= 0);

        // force-field exclusions of a's particles as (row i, excluded slot)
        int nex = 0;
        if (A.excl_off) {
            int cnt = 0, off = 0;
            if (aos >= 0) {
                off = A.excl_off[aos];
                cnt = A.excl_off[aos + 1] - off;
            }
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(full, incl, 31);
            if (total > kMaxExclPerCluster && lane == 0) set_flag(A.st, NB_ERR_CAPACITY);
            for (int k = 0; k < cnt; ++k) {
                const int idx = incl - cnt + k;
                if (idx < kMaxExclPerCluster) {
                    const int q = A.excl_idx[off + k];
                    const bool ok = q >= 0 && q < A.n_atoms;
                    if (!ok) set_flag(A.st, NB_ERR_ARG);
                    s_ex_i[wib][idx] = lane;
                    s_ex_s[wib][idx] = ok ? A.slot_of_atom[q] : -1;
                }
            }
            nex = min(total, kMaxExclPerCluster);
        }
        __syncwarp();

        // i particles of this lane's pairs
        float xi[PPL][3];
        int pj[PPL];
        bool pv[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int p = lane + 32 * k;
            pv[k] = p < C * C;
            const int i = pv[k] ? p / C : 0;
            pj[k] = pv[k] ? p % C : 0;
            const float4 x = A.xyzq[a * C + i];
            xi[k][0] = x.x;
            xi[k][1] = x.y;
            xi[k][2] = x.z;
        }

        for (int s = 0; s < 27; ++s) {
            const float sh[3] = {(float)(s / 9 - 1) * A.L[0], (float)((s / 3) % 3 - 1) * A.L[1],
                                 (float)(s % 3 - 1) * A.L[2]};
            // candidate columns (plain FP32 with a margin; the exact test follows)
            const float lx = blo.x + sh[0], hx = bhi.x + sh[0];
            const float ly = blo.y + sh[1], hy = bhi.y + sh[1];
            const float lz = blo.z + sh[2], hz = bhi.z + sh[2];
            int ix0 = (int)floorf((lx - A.rl - eps) * A.inv_cx);
            int ix1 = (int)floorf((hx + A.rl + eps) * A.inv_cx);
            int iy0 = (int)floorf((ly - A.rl - eps) * A.inv_cy);
            int iy1 = (int)floorf((hy + A.rl + eps) * A.inv_cy);
            if (ix1 < 0 || ix0 > A.nx - 1 || iy1 < 0 || iy0 > A.ny - 1) continue;
            const float zlo = lz - A.rl - eps, zhi = hz + A.rl + eps;
            if (zhi < 0.0f || zlo >= A.L[2]) continue;
            ix0 = max(ix0, 0);
            ix1 = min(ix1, A.nx - 1);
            iy0 = max(iy0, 0);
            iy1 = min(iy1, A.ny - 1);
            const int ncy = iy1 - iy0 + 1;
            const int ncols = (ix1 - ix0 + 1) * ncy;

            // shifted bounding box and i particles as hi + lo
            float alo_h[3], alo_l[3], ahi_h[3], ahi_l[3];
            two_sum(blo.x, sh[0], alo_h[0], alo_l[0]);
            two_sum(blo.y, sh[1], alo_h[1], alo_l[1]);
            two_sum(blo.z, sh[2], alo_h[2], alo_l[2]);
            two_sum(bhi.x, sh[0], ahi_h[0], ahi_l[0]);
            two_sum(bhi.y, sh[1], ahi_h[1], ahi_l[1]);
            two_sum(bhi.z, sh[2], ahi_h[2], ahi_l[2]);
            float xh[PPL][3], xl[PPL][3];
#pragma unroll
            for (int k = 0; k < PPL; ++k)
#pragma unroll
                for (int d = 0; d < 3; ++d) two_sum(xi[k][d], sh[d], xh[k][d], xl[k][d]);

            int nbuf = 0;
            auto flush = [&]() {
                __syncwarp();
                unsigned long long jb = 0, ie = 0;
                if (lane == 0) {
                    jb = atomicAdd(&A.st->n_jent, (unsigned long long)nbuf);
                    ie = atomicAdd(&A.st->n_ient, 1ull);
                }
                jb = __shfl_sync(full, jb, 0);
                ie = __shfl_sync(full, ie, 0);
                if ((long long)(jb + nbuf) > A.jent_cap || (long long)ie >= A.ient_cap) {
                    // keep every stored i-entry valid: an empty range on overflow
                    if (lane == 0) {
                        set_flag(A.st, NB_ERR_CAPACITY);
                        if ((long long)ie < A.ient_cap) A.ient[ie] = make_int4(a, s, 0, 0);
                    }
                } else {
                    for (int t = lane; t < nbuf; t += 32) {
                        A.cj[jb + t] = s_buf_cj[wib][t];
                        A.mask[jb + t] = s_buf_m[wib][t];
                    }
                    if (lane == 0) A.ient[ie] = make_int4(a, s, (int)jb, (int)(jb + nbuf));
                }
                nbuf = 0;
                __syncwarp();
            };

            for (int cb = 0; cb < ncols; cb += 32) {
                const int cidx = cb + lane;
                int k0 = 0, cnt = 0;
                if (cidx < ncols) {
                    const int col = (ix0 + cidx / ncy) * A.ny + (iy0 + cidx % ncy);
                    const int g0 = A.col_clu_start[col], g1 = A.col_clu_start[col + 1];
                    int lo = g0, hi = g1;
                    while (lo < hi) {  // first cluster with zmax >= zlo
                        const int m = (lo + hi) >> 1;
                        if (A.bb[2 * m + 1].z < zlo) lo = m + 1; else hi = m;
                    }
                    const int f = lo;
                    hi = g1;
                    while (lo < hi) {  // first cluster with zmin > zhi
                        const int m = (lo + hi) >> 1;
                        if (A.bb[2 * m].z <= zhi) lo = m + 1; else hi = m;
                    }
                    const int f2 = max(f, a);
                    if (lo > f2) {
                        k0 = f2;
                        cnt = lo - f2;
                    }
                }
                int incl = cnt;
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(full, incl, o);
                    if (lane >= o) incl += v;
                }
                const int total = __shfl_sync(full, incl, 31);
                const int excl = incl - cnt;
                for (int base = 0; base < total; base += 32) {
                    const int idx = base + lane;
                    int owner = 0;
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int v = __shfl_sync(full, incl, owner + step - 1);
                        if (v <= idx) owner += step;
                    }
                    const int ok0 = __shfl_sync(full, k0, owner);
                    const int oex = __shfl_sync(full, excl, owner);
                    bool valid = idx < total;
                    const int b = ok0 + (idx - oex);
                    if (valid && b == a && s < kShiftCenter) valid = false;
                    bool pass = false, in_rbb = false;
                    if (valid) {
                        const float4 jlo = A.bb[2 * b], jhi = A.bb[2 * b + 1];
                        const float jl[3] = {jlo.x, jlo.y, jlo.z}, jh[3] = {jhi.x, jhi.y, jhi.z};
                        float d2 = 0.0f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float g1 = (jl[d] - ahi_h[d]) - ahi_l[d];
                            const float g2 = (alo_h[d] - jh[d]) + alo_l[d];
                            const float g = fmaxf(0.0f, fmaxf(g1, g2));
                            d2 = fmaf(g, g, d2);
                        }
                        pass = d2 < A.rl2;
                        in_rbb = d2 < A.rbb2;
                    }
                    unsigned need = __ballot_sync(full, pass && !in_rbb);
                    unsigned acc = __ballot_sync(full, pass && in_rbb);
                    while (need) {
                        const int t = __ffs(need) - 1;
                        need &= need - 1;
                        const int bt = __shfl_sync(full, b, t);
                        bool hit = false;
#pragma unroll
                        for (int k = 0; k < PPL; ++k) {
                            if (!pv[k]) continue;
                            const float4 xj = A.xyzq[bt * C + pj[k]];
                            const float dx = (xh[k][0] - xj.x) + xl[k][0];
                            const float dy = (xh[k][1] - xj.y) + xl[k][1];
                            const float dz = (xh[k][2] - xj.z) + xl[k][2];
                            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            hit |= r2 < A.rl2;
                        }
                        if (__any_sync(full, hit)) acc |= 1u << t;
                    }
                    while (acc) {
                        const int t = __ffs(acc) - 1;
                        acc &= acc - 1;
                        const int bt = __shfl_sync(full, b, t);
                        const int bos = lane < C ? A.atom_of_slot[bt * C + lane] : -1;
                        const unsigned realB = __ballot_sync(full, bos >= 0);
                        unsigned long long m = 0;
#pragma unroll
                        for (int i = 0; i < C; ++i)
                            if ((realA >> i) & 1u) m |= (unsigned long long)realB << (i * C);
                        if (bt == a) {
                            if (s == kShiftCenter) m &= upper_mask<C>();
                            else m &= ~diag_mask<C>();
                        }
                        unsigned lo32 = 0, hi32 = 0;
                        for (int e = lane; e < nex; e += 32) {
                            const int sl = s_ex_s[wib][e];
                            if (sl >= 0 && sl / C == bt) {
                                const int bit = s_ex_i[wib][e] * C + sl % C;
                                if (bit < 32) lo32 |= 1u << bit;
                                else hi32 |= 1u << (bit - 32);
                            }
                        }
                        lo32 = __reduce_or_sync(full, lo32);
                        hi32 = __reduce_or_sync(full, hi32);
                        m &= ~(((unsigned long long)hi32 << 32) | lo32);
                        if (lane == 0) {
                            s_buf_cj[wib][nbuf] = bt;
                            s_buf_m[wib][nbuf] = m;
                        }
                        ++nbuf;
                        if (nbuf == kJChunk) flush();
                    }
                }
            }
            if (nbuf > 0) flush();
        }
        __syncwarp();
    }
}

cudaError_t launch_search(const Workspace& ws, const GridGeom& g, int C, long long nclu_cap,
                          float rlist, float rbb, const int* excl_off, const int* excl_idx,
                          long long ient_cap, long long jent_cap, int n_atoms, int n_sm,
                          cudaStream_t s) {
    SearchArgs A;
    A.st = ws.st;
    A.bb = ws.bb;
    A.xyzq = ws.xyzq;
    A.atom_of_slot = ws.atom_of_slot;
    A.slot_of_atom = ws.slot_of_atom;
    A.col_clu_start = ws.col_clu_start;
    A.excl_off = excl_off;
    A.excl_idx = excl_idx;
    for (int k = 0; k < 3; ++k) A.L[k] = g.L[k];
    A.inv_cx = (float)g.nx / g.L[0];
    A.inv_cy = (float)g.ny / g.L[1];
    A.nx = g.nx;
    A.ny = g.ny;
    A.rl = rlist;
    A.rl2 = rlist * rlist;
    A.rbb2 = rbb * rbb;
    A.ient = ws.ient;
    A.cj = ws.cj;
    A.mask = ws.mask;
    A.ient_cap = ient_cap;
    A.jent_cap = jent_cap;
    A.n_atoms = n_atoms;
    long long want = (nclu_cap + kSearchWarps - 1) / kSearchWarps;
    long long blocks = (long long)n_sm * 16;
    if (blocks > want) blocks = want;
    if (blocks < 1) blocks = 1;
    if (C == 8)
        k_search<8><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
    else
        k_search<4><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace nbc
