// Spatial clustering on the GPU (Sec. 2.3, Fig. 2; pigeonhole sort Sec. 2.5),
// for every box of the context in the same launches:
//   k_wrap_col   wrap into the box, x/y column of each particle, count per column
//   k_scan_cols  per box (one block each): exclusive scans giving each
//                column's first particle, first cluster and first super-cluster
//   k_scatter    particles into column order as (z bits, index) keys
//   k_col_sort   per column: on-chip bitonic sort on (z, index), cut clusters
//                of C, pad with dummies, fill slot arrays, bounding boxes,
//                super-cluster table
//   k_set_coords new frame coordinates into the slots (wrap offset kept)
// Every float decision (wrap, cell index) is one FP32 operation rounded to
// nearest, so the grid is reproducible bit for bit.
#include "nb_internal.cuh"

namespace nbc {

__global__ void k_wrap_col(Workspace ws, const float* __restrict__ xyz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ws.atom_total) return;
    const int b = find_box(ws.lay.atom_off, ws.nbox, i);
    const BoxGeom G = ws.geo[b];
    float w[3];
    bool bad = false;
    for (int k = 0; k < 3; ++k) {
        const float x = xyz[3 * i + k];
        float v = x;
        if (v < 0.0f) v = __fadd_rn(v, G.L[k]);
        if (v >= G.L[k]) v = __fsub_rn(v, G.L[k]);
        if (!(v >= 0.0f && v < G.L[k])) {
            bad = true;
            v = 0.0f;
        }
        w[k] = v;
    }
    if (bad) set_flag(&ws.st[b], NB_ERR_COORD);
    ws.xw[i] = make_float4(w[0], w[1], w[2], ws.q[i]);
    ws.woff[i] = make_float4(__fsub_rn(w[0], xyz[3 * i]), __fsub_rn(w[1], xyz[3 * i + 1]),
                             __fsub_rn(w[2], xyz[3 * i + 2]), 0.0f);
    int ix = (int)__fmul_rn(w[0], G.inv_x);
    int iy = (int)__fmul_rn(w[1], G.inv_y);
    ix = min(ix, G.nx - 1);
    iy = min(iy, G.ny - 1);
    const int col = ws.lay.col_off[b] + ix * G.ny + iy;
    ws.col_of_atom[i] = col;
    ws.rank_in_col[i] = atomicAdd(&ws.col_count[col], 1);
}

// One block per box: exclusive scans over the box's columns of particles,
// clusters (ceil(count / C)) and super-clusters (ceil(clusters / S)), as batch
// indices; the column after the last holds the totals.
__global__ void k_scan_cols(Workspace ws, int C) {
    const int b = blockIdx.x;
    const int S = super_size(C);
    const BoxGeom G = ws.geo[b];
    const int ncol = G.nx * G.ny;
    const int c_base = ws.lay.col_off[b];
    const int* col_count = ws.col_count + c_base;
    __shared__ int s_a[1024];
    __shared__ int s_c[1024];
    __shared__ int s_g[1024];
    __shared__ int s_max;
    const int t = threadIdx.x;
    if (t == 0) s_max = 0;
    __syncthreads();
    const int per = (ncol + blockDim.x - 1) / blockDim.x;
    const int c0 = min(ncol, t * per), c1 = min(ncol, c0 + per);
    int sa = 0, sc = 0, sg = 0, mx = 0;
    for (int c = c0; c < c1; ++c) {
        const int k = col_count[c];
        const int nc = (k + C - 1) / C;
        sa += k;
        sc += nc;
        sg += (nc + S - 1) / S;
        mx = max(mx, k);
    }
    s_a[t] = sa;
    s_c[t] = sc;
    s_g[t] = sg;
    atomicMax(&s_max, mx);
    __syncthreads();
    // Hillis-Steele inclusive scan over the per-thread totals
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        int va = 0, vc = 0, vg = 0;
        if (t >= off) {
            va = s_a[t - off];
            vc = s_c[t - off];
            vg = s_g[t - off];
        }
        __syncthreads();
        s_a[t] += va;
        s_c[t] += vc;
        s_g[t] += vg;
        __syncthreads();
    }
    int ba = ws.lay.atom_off[b] + s_a[t] - sa;
    int bc = ws.lay.clu_off[b] + s_c[t] - sc;
    int bg = ws.lay.sc_off[b] + s_g[t] - sg;
    for (int c = c0; c < c1; ++c) {
        const int k = col_count[c];
        const int nc = (k + C - 1) / C;
        ws.col_atom_start[c_base + c] = ba;
        ws.col_clu_start[c_base + c] = bc;
        ws.col_sc_start[c_base + c] = bg;
        ba += k;
        bc += nc;
        bg += (nc + S - 1) / S;
    }
    if (t == blockDim.x - 1) {
        ws.col_clu_start[c_base + ncol] = ws.lay.clu_off[b] + s_c[t];
        ws.col_sc_start[c_base + ncol] = ws.lay.sc_off[b] + s_g[t];
        ws.st[b].nclu = s_c[t];
        ws.st[b].nsc = s_g[t];
    }
    if (t == 0) ws.st[b].max_col = s_max;
}

__global__ void k_scatter(Workspace ws) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ws.atom_total) return;
    const int pos = ws.col_atom_start[ws.col_of_atom[i]] + ws.rank_in_col[i];
    // z >= 0 after wrapping, so its IEEE bits order like the value
    ws.keys[pos] = ((unsigned long long)__float_as_uint(ws.xw[i].z) << 32) | (unsigned int)i;
}

// One block per batch column: sort the column's keys in shared memory
// (bitonic), then write its clusters' slots, bounding boxes and super-clusters.
__global__ void __launch_bounds__(512) k_col_sort(Workspace ws, int C, int ntypes) {
    extern __shared__ unsigned long long s_key[];
    const int cg = blockIdx.x;
    const int b = find_box(ws.lay.col_off, ws.nbox, cg);
    const BoxGeom G = ws.geo[b];
    const int c_local = cg - ws.lay.col_off[b];
    if (c_local >= G.nx * G.ny) return;  // capacity beyond this box's grid
    const int cnt = ws.col_count[cg];
    const int base = ws.col_atom_start[cg];
    const int g0 = ws.col_clu_start[cg], g1 = ws.col_clu_start[cg + 1];
    {
        // super-clusters: runs of up to S consecutive clusters of this column
        const int S = super_size(C);
        const int q0 = ws.col_sc_start[cg], q1 = ws.col_sc_start[cg + 1];
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const int first = g0 + (q - q0) * S;
            ws.sc_info[q] = make_int2(first, min(S, g1 - first));
        }
    }
    if (cnt > kMaxColumn) {
        // too long to sort on-chip: flag it, leave its particles without a
        // slot and fill its clusters with dummies, so later kernels only
        // ever see valid slots
        if (threadIdx.x == 0) set_flag(&ws.st[b], NB_ERR_CAPACITY);
        for (int k = threadIdx.x; k < cnt; k += blockDim.x)
            ws.slot_of_atom[(int)(ws.keys[base + k] & 0xffffffffull)] = -1;
    }
    const int cnt_s = cnt > kMaxColumn ? 0 : cnt;   // particles placed in slots
    int P = 1;
    while (P < cnt_s) P <<= 1;
    for (int k = threadIdx.x; k < P; k += blockDim.x) s_key[k] = k < cnt_s ? ws.keys[base + k] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                const int partner = k ^ stride;
                if (partner > k) {
                    const bool up = (k & size) == 0;
                    const unsigned long long x = s_key[k], y = s_key[partner];
                    if ((x > y) == up) {
                        s_key[k] = y;
                        s_key[partner] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    // slots of this column; a dummy's position uses its box-local slot index
    const long long slot0 = (long long)ws.lay.clu_off[b] * C;
    const int nsl = (g1 - g0) * C;
    for (int t = threadIdx.x; t < nsl; t += blockDim.x) {
        const long long s = (long long)g0 * C + t;
        ws.fslot[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < cnt_s) {
            const int a = (int)(s_key[t] & 0xffffffffull);
            const float4 x = ws.xw[a];
            ws.xyzq[s] = x;
            if (ws.xjd) store_xjd(ws.xjd, s, x);
            if (ws.woff_slot) ws.woff_slot[s] = ws.woff[a];
            ws.atom_of_slot[s] = a;
            ws.slot_of_atom[a] = (int)s;
            int ty = ws.type[a];
            if (ty < 0 || ty >= ntypes) {
                set_flag(&ws.st[b], NB_ERR_ARG);
                ty = 0;
            }
            ws.type_slot[s] = ty;
            if (ws.xjd) store_jtype(ws.xjd, s, ty);
        } else {
            const long long sl = s - slot0;
            const float4 x = make_float4(-G.dummy_g * (float)(1 + (int)(sl % 4096)),
                                         -G.dummy_g * (float)(1 + (int)(sl / 4096)), -G.dummy_g, 0.0f);
            ws.xyzq[s] = x;
            if (ws.xjd) store_xjd(ws.xjd, s, x);
            ws.atom_of_slot[s] = -1;
            ws.type_slot[s] = 0;
            if (ws.xjd) store_jtype(ws.xjd, s, 0);
        }
    }
    __syncthreads();
    // bounding boxes over the real particles (slots t < cnt of the column)
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        const int tb = (g - g0) * C;
        for (int t = tb; t < tb + C && t < cnt_s; ++t) {
            const float4 p = ws.xw[(int)(s_key[t] & 0xffffffffull)];
            lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
            lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
            lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
        }
        ws.bb[2 * g] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        ws.bb[2 * g + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    }
}

cudaError_t launch_grid(const Workspace& ws, int C, int ntypes, const float* xyz, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ws.col_count, 0, sizeof(int) * ws.col_total, s);
    if (e != cudaSuccess) return e;
    const int n = ws.atom_total;
    if (n > 0) k_wrap_col<<<(n + 255) / 256, 256, 0, s>>>(ws, xyz);
    k_scan_cols<<<ws.nbox, 1024, 0, s>>>(ws, C);
    if (n > 0) k_scatter<<<(n + 255) / 256, 256, 0, s>>>(ws);
    const size_t smem = sizeof(unsigned long long) * kMaxColumn;
    static std::atomic<unsigned long long> smem_set{0};
    e = smem_opt_in(k_col_sort, (int)smem, smem_set);
    if (e != cudaSuccess) return e;
    k_col_sort<<<ws.col_total, 512, smem, s>>>(ws, C, ntypes);
    return cudaGetLastError();
}

// One thread per slot of the current clusters (coalesced slot reads and
// writes; one gathered read of the particle's new coordinates): the slot's
// particle gets its new coordinates plus the wrap offset of the last
// gridding (kept per slot), its charge stays; dummy slots keep theirs.  The
// slot's force accumulator is cleared for the evaluation that follows.
// Particles without a slot (a column too long to grid, an error that is
// flagged) are not placed.
__global__ void k_set_coords(Workspace ws, int C, const float* __restrict__ xyz) {
    const long long nslot = (long long)ws.clu_total * C;
    const int n = ws.atom_total;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < nslot;
         s += (long long)gridDim.x * blockDim.x) {
        const int cl = (int)(s / C);
        const int b = find_box(ws.lay.clu_off, ws.nbox, cl);
        if (cl - ws.lay.clu_off[b] >= ws.st[b].nclu) continue;   // capacity beyond the box's grid
        ws.fslot[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int a = ws.atom_of_slot[s];
        if (a < 0 || a >= n) continue;
        const float4 o = ws.woff_slot[s];
        const float4 x = make_float4(__fadd_rn(xyz[3 * (long long)a], o.x), __fadd_rn(xyz[3 * (long long)a + 1], o.y),
                                     __fadd_rn(xyz[3 * (long long)a + 2], o.z), ws.xyzq[s].w);
        ws.xyzq[s] = x;
        store_xjd(ws.xjd, s, x);
    }
}

cudaError_t launch_set_coords(const Workspace& ws, int C, const float* xyz, cudaStream_t s) {
    long long blocks = ((long long)ws.clu_total * C + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (blocks < 1) blocks = 1;
    k_set_coords<<<(int)blocks, 256, 0, s>>>(ws, C, xyz);
    return cudaGetLastError();
}

}  // namespace nbc
