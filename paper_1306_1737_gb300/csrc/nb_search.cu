// Cluster-pair search (Sec. 2.3, Fig. 3) and exclusion masks (Sec. 2.4),
// emitted as super-cluster lists (Sec. 3.1: the GPU kernel reads one j-list
// for several i-clusters, each j-entry carrying an interaction bit per
// i-cluster and that pair's exclusion mask).
//
// One warp per super-cluster (up to S consecutive clusters g0..g0+n-1 of one
// grid column).  For each periodic shift s applied to the i side, the warp
// visits the grid columns whose x/y cells come within rlist of the shifted
// union bounding box; in each column (clusters sorted on z) a binary search
// bounds the candidates in z.  For every candidate cj and every i-cluster ck
// with cj >= ck (half list, Newton's third law; cj == ck only for s = 0 and
// the positive half of the shifts) the pair is kept iff d_BB < rlist and
// (d_BB < rBB or some particle pair is closer than rlist).  Shifted
// coordinates are carried as an unevaluated FP32 sum hi + lo (TwoSum).
// Accepted j-clusters get their per-i-cluster 64-bit masks (bit i*C+j: full
// interaction) and are appended in chunks of at most kJChunk per i-entry.
#include "nb_internal.cuh"

namespace nbc {

struct SearchArgs {
    Workspace ws;
    const int* excl_off;
    const int* excl_idx;
    float rl, rl2, rbb2;
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
constexpr int kCoopSuperPerSm = 16;   // block-per-super-cluster mode up to this many per SM
constexpr int kMaxExclPerSuper = 512;

// COOP = false: one warp per super-cluster.  COOP = true (boxes with few
// super-clusters, where one warp each would leave the SMs mostly idle): the
// block's warps share one super-cluster and split its candidate columns
// (warp w takes columns w, w + kSearchWarps, ...); each warp writes full
// chunks of kJChunkCoop j-entries as it goes, and at the end of each shift
// the block merges the warps' remainders into full chunks, so the j-lists are
// not fragmented by the split.  The shorter chunks of this mode give a small
// box's force and prune kernels more i-entries than warps to balance.
template <int C, int S, bool COOP>
__global__ void __launch_bounds__(32 * kSearchWarps, 6) k_search(SearchArgs A) {
    constexpr int PPL = (C * C + 31) / 32;  // particle pairs per lane in an atom test
    constexpr int NA = S * C;               // i particles of a super-cluster (<= 32)
    static_assert(NA <= 32, "a super-cluster's particles must fit one warp");
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    __shared__ float4 s_xi[kSearchWarps][NA];
    __shared__ float4 s_h[kSearchWarps][NA];   // i particles shifted by the current shift: hi part
    __shared__ float4 s_l[kSearchWarps][NA];   // and lo part (TwoSum)
    __shared__ float s_bb[kSearchWarps][S][12];  // shifted BB: lo hi/lo, hi hi/lo per dimension
    // the super-cluster's exclusions: one copy per warp, or one per block
    // when the block's warps share the super-cluster
    __shared__ int s_ex_r[COOP ? 1 : kSearchWarps][kMaxExclPerSuper];
    __shared__ int s_ex_s[COOP ? 1 : kSearchWarps][kMaxExclPerSuper];
    __shared__ int s_buf_w[kSearchWarps][kJChunk];
    __shared__ unsigned long long s_buf_m[kSearchWarps][S][kJChunk];
    __shared__ float4 s_xc[kSearchWarps][COOP ? 32 * C : 1];  // particles of a batch's candidates
    __shared__ int s_nbuf[kSearchWarps];

    const Workspace& W = A.ws;
    const float eps = 1e-4f;
    int b = 0;
    const int part = COOP ? wib : 0;
    const int xw = COOP ? 0 : wib;   // the exclusion table this warp uses
    constexpr int P = COOP ? kSearchWarps : 1;
    constexpr int JC = COOP ? kJChunkCoop : kJChunk;   // j-entries per i-entry at most
    const int q0 = COOP ? blockIdx.x : blockIdx.x * kSearchWarps + wib;
    const int qstep = COOP ? gridDim.x : gridDim.x * kSearchWarps;
    for (int q = q0; q < W.sc_total; q += qstep) {
        b = advance_box(W.lay.sc_off, W.nbox, b, q);
        if (q - W.lay.sc_off[b] >= W.st[b].nsc) continue;
        DevState* st = &W.st[b];
        const BoxGeom G = W.geo[b];
        const int col_base = W.lay.col_off[b];
        const long long ient_base = W.lay.ient_off[b], ient_cap = W.lay.ient_off[b + 1] - ient_base;
        const long long jent_base = W.lay.jent_off[b], jent_cap = W.lay.jent_off[b + 1] - jent_base;
        const int2 info = W.sc_info[q];
        const int g0 = info.x, n = info.y;
        // i particles of the super-cluster, real-slot bits per i-cluster
        const int aos = lane < n * C ? W.atom_of_slot[g0 * C + lane] : -1;
        if (lane < NA) s_xi[wib][lane] = lane < n * C ? W.xyzq[g0 * C + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const unsigned realAll = __ballot_sync(full, aos >= 0);
        // union bounding box
        float ulo[3] = {INFINITY, INFINITY, INFINITY}, uhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = 0; k < n; ++k) {
            const float4 lo = W.bb[2 * (g0 + k)], hi = W.bb[2 * (g0 + k) + 1];
            ulo[0] = fminf(ulo[0], lo.x); ulo[1] = fminf(ulo[1], lo.y); ulo[2] = fminf(ulo[2], lo.z);
            uhi[0] = fmaxf(uhi[0], hi.x); uhi[1] = fmaxf(uhi[1], hi.y); uhi[2] = fmaxf(uhi[2], hi.z);
        }
        // force-field exclusions of the super-cluster's particles: (row, excluded slot)
        int nex = 0;
        int ex_lo = 0x7fffffff, ex_hi = -1;   // range of the excluded partners' clusters
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
            if (total > kMaxExclPerSuper && lane == 0) set_flag(st, NB_ERR_CAPACITY);
            for (int k = 0; k < cnt; ++k) {
                const int idx = incl - cnt + k;
                if (idx < kMaxExclPerSuper) {
                    const int qa = A.excl_idx[off + k];
                    const bool ok = qa >= 0 && qa < W.atom_total;
                    if (!ok) set_flag(st, NB_ERR_ARG);
                    const int sl = ok ? W.slot_of_atom[qa] : -1;
                    if (sl >= 0) {
                        ex_lo = min(ex_lo, sl / C);
                        ex_hi = max(ex_hi, sl / C);
                    }
                    if (!COOP || wib == 0) {
                        s_ex_r[xw][idx] = lane;
                        s_ex_s[xw][idx] = sl;
                    }
                }
            }
            nex = min(total, kMaxExclPerSuper);
            ex_lo = __reduce_min_sync(full, ex_lo);
            ex_hi = __reduce_max_sync(full, ex_hi);
        }
        if constexpr (COOP) __syncthreads();   // warp 0's exclusion table is complete
        __syncwarp();

        for (int s = 0; s < 27; ++s) {
            const float sh[3] = {(float)(s / 9 - 1) * G.L[0], (float)((s / 3) % 3 - 1) * G.L[1],
                                 (float)(s % 3 - 1) * G.L[2]};
            // candidate columns from the shifted union box (plain FP32 with a margin)
            int ix0 = (int)floorf((ulo[0] + sh[0] - A.rl - eps) * G.inv_cx);
            int ix1 = (int)floorf((uhi[0] + sh[0] + A.rl + eps) * G.inv_cx);
            int iy0 = (int)floorf((ulo[1] + sh[1] - A.rl - eps) * G.inv_cy);
            int iy1 = (int)floorf((uhi[1] + sh[1] + A.rl + eps) * G.inv_cy);
            if (ix1 < 0 || ix0 > G.nx - 1 || iy1 < 0 || iy0 > G.ny - 1) continue;
            const float zlo = ulo[2] + sh[2] - A.rl - eps, zhi = uhi[2] + sh[2] + A.rl + eps;
            if (zhi < 0.0f || zlo >= G.L[2]) continue;
            ix0 = max(ix0, 0);
            ix1 = min(ix1, G.nx - 1);
            iy0 = max(iy0, 0);
            iy1 = min(iy1, G.ny - 1);
            const int ncy = iy1 - iy0 + 1;
            const int ncols = (ix1 - ix0 + 1) * ncy;
            // exact shifted boxes of the i-clusters as hi + lo
            if (lane < n * 6) {
                const int k = lane / 6, c = lane % 6, d = c % 3;
                const float4 bx = c < 3 ? W.bb[2 * (g0 + k)] : W.bb[2 * (g0 + k) + 1];
                const float v = d == 0 ? bx.x : (d == 1 ? bx.y : bx.z);
                const float shd = d == 0 ? sh[0] : (d == 1 ? sh[1] : sh[2]);
                float h, l;
                two_sum(v, shd, h, l);
                s_bb[wib][k][2 * c] = h;
                s_bb[wib][k][2 * c + 1] = l;
            }
            if (lane < NA) {
                const float4 xi = s_xi[wib][lane];
                float4 h, l;
                two_sum(xi.x, sh[0], h.x, l.x);
                two_sum(xi.y, sh[1], h.y, l.y);
                two_sum(xi.z, sh[2], h.z, l.z);
                h.w = l.w = 0.0f;
                s_h[wib][lane] = h;
                s_l[wib][lane] = l;
            }
            __syncwarp();

            int nbuf = 0;
            auto flush = [&]() __attribute__((always_inline)) {
                __syncwarp();
                unsigned long long jb = 0, ie = 0;
                unsigned nk = 0;
                for (int t = lane; t < nbuf; t += 32) nk += __popc((unsigned)s_buf_w[wib][t] >> kSuperShift);
                for (int o = 16; o > 0; o >>= 1) nk += __shfl_xor_sync(full, nk, o);
                if (lane == 0) {
                    jb = atomicAdd(&st->n_jent, (unsigned long long)nbuf);
                    ie = atomicAdd(&st->n_ient, 1ull);
                    atomicAdd(&st->n_keys, (unsigned long long)nk);
                }
                jb = __shfl_sync(full, jb, 0);
                ie = __shfl_sync(full, ie, 0);
                if ((long long)(jb + nbuf) > jent_cap || (long long)ie >= ient_cap) {
                    // keep every stored i-entry valid: an empty range on overflow
                    if (lane == 0) {
                        set_flag(st, NB_ERR_CAPACITY);
                        if ((long long)ie < ient_cap) W.ient[ient_base + ie] = make_int4(q, s, 0, 0);
                    }
                } else {
                    const long long j0 = jent_base + (long long)jb;
                    for (int t = lane; t < nbuf; t += 32) {
                        W.cj[j0 + t] = s_buf_w[wib][t];
#pragma unroll
                        for (int k = 0; k < S; ++k) W.mask[k * W.jstride + j0 + t] = s_buf_m[wib][k][t];
                    }
                    if (lane == 0) W.ient[ient_base + ie] = make_int4(q, s, (int)j0, (int)(j0 + nbuf));
                }
                nbuf = 0;
                __syncwarp();
            };

            for (int cb = 0; cb * P + part < ncols; cb += 32) {
                const int cidx = (cb + lane) * P + part;
                int k0 = 0, cnt = 0;
                if (cidx < ncols) {
                    const int col = col_base + (ix0 + cidx / ncy) * G.ny + (iy0 + cidx % ncy);
                    const int c0 = W.col_clu_start[col], c1 = W.col_clu_start[col + 1];
                    int lo = c0, hi = c1;
                    while (lo < hi) {  // first cluster with zmax >= zlo
                        const int m = (lo + hi) >> 1;
                        if (W.bb[2 * m + 1].z < zlo) lo = m + 1; else hi = m;
                    }
                    const int f = lo;
                    hi = c1;
                    while (lo < hi) {  // first cluster with zmin > zhi
                        const int m = (lo + hi) >> 1;
                        if (W.bb[2 * m].z <= zhi) lo = m + 1; else hi = m;
                    }
                    const int f2 = max(f, g0);
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
                    const bool valid = idx < total;
                    const int cb_ = ok0 + (idx - oex);
                    unsigned need = 0, acc = 0;  // per candidate: i-clusters to test / accepted
                    unsigned realB_mine = 0;     // per candidate: its real (non-dummy) slots
                    if (valid) {
                        // the candidate's slot table, loaded beside its bounding box
                        const int4* ap = reinterpret_cast<const int4*>(W.atom_of_slot + (long long)cb_ * C);
#pragma unroll
                        for (int v = 0; v < C / 4; ++v) {
                            const int4 a = ap[v];
                            realB_mine |= ((a.x >= 0) ? 1u : 0u) << (4 * v) | ((a.y >= 0) ? 2u : 0u) << (4 * v) |
                                          ((a.z >= 0) ? 4u : 0u) << (4 * v) | ((a.w >= 0) ? 8u : 0u) << (4 * v);
                        }
                        const float4 jlo = W.bb[2 * cb_], jhi = W.bb[2 * cb_ + 1];
                        const float jl[3] = {jlo.x, jlo.y, jlo.z}, jh[3] = {jhi.x, jhi.y, jhi.z};
                        for (int k = 0; k < n; ++k) {
                            const int ck = g0 + k;
                            if (cb_ < ck || (cb_ == ck && s < kShiftCenter)) continue;
                            float d2 = 0.0f;
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                const float* sb = s_bb[wib][k];
                                const float g1 = (jl[d] - sb[6 + 2 * d]) - sb[6 + 2 * d + 1];
                                const float g2 = (sb[2 * d] - jh[d]) + sb[2 * d + 1];
                                const float g = fmaxf(0.0f, fmaxf(g1, g2));
                                d2 = fmaf(g, g, d2);
                            }
                            if (d2 < A.rl2) {
                                if (d2 < A.rbb2) acc |= 1u << k;
                                else need |= 1u << k;
                            }
                        }
                    }
                    // particle-distance tests, one warp-wide test per (candidate,
                    // i-cluster)
                    unsigned pending = __ballot_sync(full, need != 0);
                    if constexpr (COOP) {
                        // the particles of every candidate of the batch that needs a
                        // test are first copied to shared memory, all copies in
                        // flight at once (one L2 round trip per batch)
                        if (pending) {
#pragma unroll
                            for (int r = 0; r < C; ++r) {
                                const int t = r * (32 / C) + lane / C, jj = lane % C;
                                const int bt = __shfl_sync(full, cb_, t);
                                if ((pending >> t) & 1u)
                                    copy16_async(&s_xc[wib][t * C + jj], W.xyzq + (long long)bt * C + jj);
                            }
                            copy_async_wait_all();
                            __syncwarp();
                        }
                        while (pending) {
                            const int t = __ffs(pending) - 1;
                            pending &= pending - 1;
                            unsigned nk = __shfl_sync(full, need, t);
                            while (nk) {
                                const int k = __ffs(nk) - 1;
                                nk &= nk - 1;
                                bool hit = false;
#pragma unroll
                                for (int kk = 0; kk < PPL; ++kk) {
                                    const int p = lane + 32 * kk;
                                    if (p >= C * C) continue;
                                    const float4 h = s_h[wib][k * C + p / C], l = s_l[wib][k * C + p / C];
                                    const float4 xj = s_xc[wib][t * C + p % C];
                                    const float dx = (h.x - xj.x) + l.x;
                                    const float dy = (h.y - xj.y) + l.y;
                                    const float dz = (h.z - xj.z) + l.z;
                                    hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < A.rl2;
                                }
                                if (__any_sync(full, hit) && lane == t) acc |= 1u << k;
                            }
                        }
                        __syncwarp();   // s_xc is rewritten by the next batch
                    } else {
                        // two candidates per round so that their particle loads
                        // are in flight together
                        while (pending) {
                            const int t1 = __ffs(pending) - 1;
                            pending &= pending - 1;
                            const int t2 = pending ? __ffs(pending) - 1 : -1;
                            if (t2 >= 0) pending &= pending - 1;
                            const int bt1 = __shfl_sync(full, cb_, t1);
                            const int bt2 = __shfl_sync(full, cb_, t2 >= 0 ? t2 : t1);
                            unsigned nk1 = __shfl_sync(full, need, t1);
                            unsigned nk2 = __shfl_sync(full, need, t2 >= 0 ? t2 : t1);
                            if (t2 < 0) nk2 = 0u;
                            float4 xa[PPL], xb[PPL];
#pragma unroll
                            for (int kk = 0; kk < PPL; ++kk) {
                                const int jj = (lane + 32 * kk) % C;
                                xa[kk] = W.xyzq[bt1 * C + jj];
                                xb[kk] = W.xyzq[bt2 * C + jj];
                            }
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                unsigned nk = u == 0 ? nk1 : nk2;
                                while (nk) {
                                    const int k = __ffs(nk) - 1;
                                    nk &= nk - 1;
                                    bool hit = false;
#pragma unroll
                                    for (int kk = 0; kk < PPL; ++kk) {
                                        const int p = lane + 32 * kk;
                                        if (p >= C * C) continue;
                                        const float4 h = s_h[wib][k * C + p / C], l = s_l[wib][k * C + p / C];
                                        const float4 xj = u == 0 ? xa[kk] : xb[kk];
                                        const float dx = (h.x - xj.x) + l.x;
                                        const float dy = (h.y - xj.y) + l.y;
                                        const float dz = (h.z - xj.z) + l.z;
                                        hit |= fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < A.rl2;
                                    }
                                    if (__any_sync(full, hit) && lane == (u == 0 ? t1 : t2)) acc |= 1u << k;
                                }
                            }
                        }
                    }
                    // exclusion masks of the accepted candidates, one candidate per
                    // lane (bit i*C + j set: both particles real, distinct on the
                    // diagonal, not force-field excluded), appended to the buffer in
                    // lane order
                    const unsigned accepted = __ballot_sync(full, acc != 0);
                    unsigned long long my_m[S];
#pragma unroll
                    for (int k = 0; k < S; ++k) {
                        unsigned long long m = 0;
                        if ((acc >> k) & 1u) {
                            const unsigned realA = (realAll >> (k * C)) & ((1u << C) - 1u);
                            unsigned long long rows = 0;   // bit i*C for every real i-particle
#pragma unroll
                            for (int i = 0; i < C; ++i)
                                if ((realA >> i) & 1u) rows |= 1ull << (i * C);
                            // rows of C bits never overlap, so the product places the
                            // candidate's real j-bits in every real i-row
                            m = rows * (unsigned long long)realB_mine;
                            if (cb_ == g0 + k) {
                                if (s == kShiftCenter) m &= upper_mask<C>();
                                else m &= ~diag_mask<C>();
                            }
                            // only candidates in the range of excluded partners' clusters scan
                            if (cb_ >= ex_lo && cb_ <= ex_hi) {
                                for (int e = 0; e < nex; ++e) {
                                    const int sl = s_ex_s[xw][e];
                                    const int r = s_ex_r[xw][e];
                                    if (sl >= 0 && r / C == k && sl / C == cb_)
                                        m &= ~(1ull << ((r % C) * C + sl % C));
                                }
                            }
                        }
                        my_m[k] = m;
                    }
                    const int n_acc = __popc(accepted);
                    const int my_pos = __popc(accepted & ((1u << lane) - 1u));
                    for (int done = 0; done < n_acc;) {
                        const int take = min(JC - nbuf, n_acc - done);
                        if (acc && my_pos >= done && my_pos < done + take) {
                            const int slot = nbuf + my_pos - done;
                            s_buf_w[wib][slot] = cb_ | (int)(acc << kSuperShift);
#pragma unroll
                            for (int k = 0; k < S; ++k) s_buf_m[wib][k][slot] = my_m[k];
                        }
                        nbuf += take;
                        done += take;
                        if (nbuf == JC) flush();
                    }
                }
            }
            if constexpr (COOP) {
                // merge the warps' remainders (< JC each) into full chunks
                if (lane == 0) s_nbuf[wib] = nbuf;
                __syncthreads();
                if (wib == 0) {
                    const int cnt_w = lane < kSearchWarps ? s_nbuf[lane] : 0;
                    int incl = cnt_w;
                    for (int o = 1; o < 32; o <<= 1) {
                        const int v = __shfl_up_sync(full, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const int T = __shfl_sync(full, incl, 31);
                    const int e1 = __shfl_sync(full, incl, 0), e2 = __shfl_sync(full, incl, 1),
                              e3 = __shfl_sync(full, incl, 2);
                    static_assert(kSearchWarps == 4, "the merge below locates entries among 4 warps");
                    auto locate = [&](int idx, int& w, int& pos) {
                        w = (idx >= e1) + (idx >= e2) + (idx >= e3);
                        pos = idx - (w == 0 ? 0 : (w == 1 ? e1 : (w == 2 ? e2 : e3)));
                    };
                    if (T > 0) {
                        const int nch = (T + JC - 1) / JC;
                        unsigned nk = 0;
                        for (int idx = lane; idx < T; idx += 32) {
                            int w, pos;
                            locate(idx, w, pos);
                            nk += __popc((unsigned)s_buf_w[w][pos] >> kSuperShift);
                        }
                        for (int o = 16; o > 0; o >>= 1) nk += __shfl_xor_sync(full, nk, o);
                        unsigned long long jb = 0, ie = 0;
                        if (lane == 0) {
                            jb = atomicAdd(&st->n_jent, (unsigned long long)T);
                            ie = atomicAdd(&st->n_ient, (unsigned long long)nch);
                            atomicAdd(&st->n_keys, (unsigned long long)nk);
                        }
                        jb = __shfl_sync(full, jb, 0);
                        ie = __shfl_sync(full, ie, 0);
                        if ((long long)(jb + T) > jent_cap || (long long)(ie + nch) > ient_cap) {
                            if (lane == 0) set_flag(st, NB_ERR_CAPACITY);
                            for (int c = lane; c < nch; c += 32)
                                if ((long long)(ie + c) < ient_cap) W.ient[ient_base + ie + c] = make_int4(q, s, 0, 0);
                        } else {
                            const long long j0 = jent_base + (long long)jb;
                            for (int idx = lane; idx < T; idx += 32) {
                                int w, pos;
                                locate(idx, w, pos);
                                W.cj[j0 + idx] = s_buf_w[w][pos];
#pragma unroll
                                for (int k = 0; k < S; ++k) W.mask[k * W.jstride + j0 + idx] = s_buf_m[w][k][pos];
                            }
                            for (int c = lane; c < nch; c += 32)
                                W.ient[ient_base + ie + c] =
                                    make_int4(q, s, (int)(j0 + c * JC), (int)(j0 + min(T, (c + 1) * JC)));
                        }
                    }
                }
                __syncthreads();
                nbuf = 0;
            } else {
                if (nbuf > 0) flush();
            }
        }
        __syncwarp();
    }
}

// Compact i-entry index: per box the entries stored (clamped to the box's
// capacity), as an exclusive prefix over the boxes.
__global__ void k_ient_offsets(Workspace ws) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < ws.nbox; ++b) {
        ws.ient_used[b] = acc;
        const long long cap = ws.lay.ient_off[b + 1] - ws.lay.ient_off[b];
        acc += (int)min((long long)ws.st[b].n_ient, cap);
    }
    ws.ient_used[ws.nbox] = acc;
    ws.work[0] = 0;
    ws.work[1] = 0;
}

cudaError_t launch_search(const Workspace& ws, int C, float rlist, float rbb, const int* excl_off,
                          const int* excl_idx, int n_sm, cudaStream_t s) {
    SearchArgs A;
    A.ws = ws;
    A.excl_off = excl_off;
    A.excl_idx = excl_idx;
    A.rl = rlist;
    A.rl2 = rlist * rlist;
    A.rbb2 = rbb * rbb;
    // few super-clusters (fewer than about two per resident warp): a block per
    // super-cluster; else a warp per super-cluster
    const bool coop = (long long)ws.sc_total <= (long long)n_sm * kCoopSuperPerSm;
    long long want = coop ? (long long)ws.sc_total : ((long long)ws.sc_total + kSearchWarps - 1) / kSearchWarps;
    long long blocks = (long long)n_sm * 16;
    if (blocks > want) blocks = want;
    if (blocks < 1) blocks = 1;
    if (C == 8) {
        if (coop) k_search<8, super_size(8), true><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
        else k_search<8, super_size(8), false><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
    } else {
        if (coop) k_search<4, super_size(4), true><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
        else k_search<4, super_size(4), false><<<(int)blocks, 32 * kSearchWarps, 0, s>>>(A);
    }
    k_ient_offsets<<<1, 32, 0, s>>>(ws);
    return cudaGetLastError();
}

}  // namespace nbc
