// Spatial clustering on the GPU (Sec. 2.3, Fig. 2; pigeonhole sort Sec. 2.5):
//   k_wrap_col   wrap into the box, x/y column of each particle, count per column
//   k_scan_cols  exclusive scans: first particle and first cluster per column
//   k_scatter    particles into column order as (z bits, index) keys
//   k_col_sort   per column: on-chip bitonic sort on (z, index), cut clusters
//                of C, pad with dummies, fill slot arrays, bounding boxes
//   k_set_coords new frame coordinates into the slots (wrap offset kept)
// Every float decision (wrap, cell index) is one FP32 operation rounded to
// nearest, so the grid is reproducible bit for bit.
#include "nb_internal.cuh"

namespace nbc {

__global__ void k_wrap_col(int n, const float* __restrict__ xyz, const float* __restrict__ q,
                           float Lx, float Ly, float Lz, float inv_x, float inv_y, int nx, int ny,
                           float4* __restrict__ xw, float4* __restrict__ woff,
                           int* __restrict__ col_of_atom, int* __restrict__ rank_in_col,
                           int* __restrict__ col_count, DevState* st) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float L[3] = {Lx, Ly, Lz};
    float w[3];
    bool bad = false;
    for (int k = 0; k < 3; ++k) {
        const float x = xyz[3 * i + k];
        float v = x;
        if (v < 0.0f) v = __fadd_rn(v, L[k]);
        if (v >= L[k]) v = __fsub_rn(v, L[k]);
        if (!(v >= 0.0f && v < L[k])) {
            bad = true;
            v = 0.0f;
        }
        w[k] = v;
    }
    if (bad) set_flag(st, NB_ERR_COORD);
    xw[i] = make_float4(w[0], w[1], w[2], q[i]);
    woff[i] = make_float4(__fsub_rn(w[0], xyz[3 * i]), __fsub_rn(w[1], xyz[3 * i + 1]),
                          __fsub_rn(w[2], xyz[3 * i + 2]), 0.0f);
    int ix = (int)__fmul_rn(w[0], inv_x);
    int iy = (int)__fmul_rn(w[1], inv_y);
    ix = min(ix, nx - 1);
    iy = min(iy, ny - 1);
    const int col = ix * ny + iy;
    col_of_atom[i] = col;
    rank_in_col[i] = atomicAdd(&col_count[col], 1);
}

// Single-block exclusive scans over the columns: particle offsets and cluster
// offsets (ceil(count / C) clusters per column).  Also records the longest
// column and the cluster count.
__global__ void k_scan_cols(int ncol, int C, const int* __restrict__ col_count,
                            int* __restrict__ col_atom_start, int* __restrict__ col_clu_start,
                            int* __restrict__ col_sc_start, DevState* st) {
    const int S = super_size(C);
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
    int ba = s_a[t] - sa, bc = s_c[t] - sc, bg = s_g[t] - sg;
    for (int c = c0; c < c1; ++c) {
        const int k = col_count[c];
        const int nc = (k + C - 1) / C;
        col_atom_start[c] = ba;
        col_clu_start[c] = bc;
        col_sc_start[c] = bg;
        ba += k;
        bc += nc;
        bg += (nc + S - 1) / S;
    }
    if (t == blockDim.x - 1) {
        col_clu_start[ncol] = s_c[t];
        col_sc_start[ncol] = s_g[t];
        st->nclu = s_c[t];
        st->nsc = s_g[t];
    }
    if (t == 0) st->max_col = s_max;
}

__global__ void k_scatter(int n, const int* __restrict__ col_of_atom,
                          const int* __restrict__ rank_in_col, const int* __restrict__ col_atom_start,
                          const float4* __restrict__ xw, unsigned long long* __restrict__ keys) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pos = col_atom_start[col_of_atom[i]] + rank_in_col[i];
    // z >= 0 after wrapping, so its IEEE bits order like the value
    keys[pos] = ((unsigned long long)__float_as_uint(xw[i].z) << 32) | (unsigned int)i;
}

// One block per column: sort the column's keys in shared memory (bitonic),
// then write its clusters' slots and bounding boxes.
__global__ void __launch_bounds__(512) k_col_sort(
    int ncol, int C, int ntypes, float dummy_g, const int* __restrict__ col_count,
    const int* __restrict__ col_atom_start, const int* __restrict__ col_clu_start,
    const int* __restrict__ col_sc_start, int2* __restrict__ sc_info,
    const unsigned long long* __restrict__ keys, const float4* __restrict__ xw,
    const int* __restrict__ type, float4* __restrict__ xyzq, int* __restrict__ atom_of_slot,
    int* __restrict__ slot_of_atom, int* __restrict__ type_slot, float4* __restrict__ bb,
    float4* __restrict__ fslot, DevState* st) {
    extern __shared__ unsigned long long s_key[];
    const int c = blockIdx.x;
    if (c >= ncol) return;
    const int cnt = col_count[c];
    const int base = col_atom_start[c];
    const int g0 = col_clu_start[c], g1 = col_clu_start[c + 1];
    {
        // super-clusters: runs of up to S consecutive clusters of this column
        const int S = super_size(C);
        const int q0 = col_sc_start[c], q1 = col_sc_start[c + 1];
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            const int first = g0 + (q - q0) * S;
            sc_info[q] = make_int2(first, min(S, g1 - first));
        }
    }
    if (cnt > kMaxColumn) {
        if (threadIdx.x == 0) set_flag(st, NB_ERR_CAPACITY);
        return;
    }
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int k = threadIdx.x; k < P; k += blockDim.x)
        s_key[k] = k < cnt ? keys[base + k] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = threadIdx.x; k < P; k += blockDim.x) {
                const int partner = k ^ stride;
                if (partner > k) {
                    const bool up = (k & size) == 0;
                    const unsigned long long a = s_key[k], b = s_key[partner];
                    if ((a > b) == up) {
                        s_key[k] = b;
                        s_key[partner] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // slots of this column
    const int nsl = (g1 - g0) * C;
    for (int t = threadIdx.x; t < nsl; t += blockDim.x) {
        const long long s = (long long)g0 * C + t;
        fslot[s] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < cnt) {
            const int a = (int)(s_key[t] & 0xffffffffull);
            const float4 p = xw[a];
            xyzq[s] = p;
            atom_of_slot[s] = a;
            slot_of_atom[a] = (int)s;
            int ty = type[a];
            if (ty < 0 || ty >= ntypes) {
                set_flag(st, NB_ERR_ARG);
                ty = 0;
            }
            type_slot[s] = ty;
        } else {
            xyzq[s] = make_float4(-dummy_g * (float)(1 + (int)(s % 4096)),
                                  -dummy_g * (float)(1 + (int)(s / 4096)), -dummy_g, 0.0f);
            atom_of_slot[s] = -1;
            type_slot[s] = 0;
        }
    }
    __syncthreads();
    // bounding boxes over the real particles (slots t < cnt of the column)
    for (int g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        const int tb = (g - g0) * C;
        for (int t = tb; t < tb + C && t < cnt; ++t) {
            const int a = (int)(s_key[t] & 0xffffffffull);
            const float4 p = xw[a];
            lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
            lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
            lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
        }
        bb[2 * g] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        bb[2 * g + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    }
}

cudaError_t launch_grid(const Workspace& ws, const GridGeom& g, int n, int C, int ntypes,
                        const float* xyz, int n_sm, cudaStream_t s) {
    (void)n_sm;
    const int ncol = g.nx * g.ny;
    cudaError_t e = cudaMemsetAsync(ws.col_count, 0, sizeof(int) * ncol, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        k_wrap_col<<<(n + 255) / 256, 256, 0, s>>>(n, xyz, ws.q, g.L[0], g.L[1], g.L[2], g.inv_x,
                                                   g.inv_y, g.nx, g.ny, ws.xw, ws.woff,
                                                   ws.col_of_atom, ws.rank_in_col, ws.col_count, ws.st);
    }
    k_scan_cols<<<1, 1024, 0, s>>>(ncol, C, ws.col_count, ws.col_atom_start, ws.col_clu_start,
                                   ws.col_sc_start, ws.st);
    if (n > 0) {
        k_scatter<<<(n + 255) / 256, 256, 0, s>>>(n, ws.col_of_atom, ws.rank_in_col,
                                                  ws.col_atom_start, ws.xw, ws.keys);
    }
    const size_t smem = sizeof(unsigned long long) * kMaxColumn;
    static bool attr_set = false;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_col_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_col_sort<<<ncol, 512, smem, s>>>(ncol, C, ntypes, g.dummy_g, ws.col_count, ws.col_atom_start,
                                       ws.col_clu_start, ws.col_sc_start, ws.sc_info, ws.keys, ws.xw,
                                       ws.type, ws.xyzq,
                                       ws.atom_of_slot, ws.slot_of_atom, ws.type_slot, ws.bb, ws.fslot,
                                       ws.st);
    return cudaGetLastError();
}

__global__ void k_set_coords(long long nslots_cap, const int* __restrict__ atom_of_slot,
                             const float* __restrict__ xyz, const float4* __restrict__ woff,
                             float4* __restrict__ xyzq, const DevState* st, int C) {
    const long long nslots = (long long)st->nclu * C;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nslots && s < nslots_cap;
         s += (long long)gridDim.x * blockDim.x) {
        const int a = atom_of_slot[s];
        if (a < 0) continue;
        const float4 o = woff[a];
        float4 p = xyzq[s];
        p.x = __fadd_rn(xyz[3 * a], o.x);
        p.y = __fadd_rn(xyz[3 * a + 1], o.y);
        p.z = __fadd_rn(xyz[3 * a + 2], o.z);
        xyzq[s] = p;
    }
}

cudaError_t launch_set_coords(const Workspace& ws, int n_slots_cap, int C, const float* xyz,
                              cudaStream_t s) {
    const int blocks = (int)((n_slots_cap + 255) / 256);
    k_set_coords<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(n_slots_cap, ws.atom_of_slot, xyz, ws.woff,
                                                         ws.xyzq, ws.st, C);
    return cudaGetLastError();
}

}  // namespace nbc
