// The force evaluation's epilogue: forces from the slot-ordered accumulator
// back to the caller's particle order, and with energies the FP64 per-box
// totals: energies, and the virial
// W = sum_i x_i (x) f_i + sum_s (s L) (x) f_shift(s) (the shift-force
// bookkeeping of the periodic images, Sec. 2.3).
#include "nb_internal.cuh"

namespace nbc {

// A warp's virial partial sums of box b added to the box's FP64 total, then cleared.
__device__ __forceinline__ void virial_flush(const Workspace& ws, double (&w)[9], int b, int lane) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        for (int o = 16; o > 0; o >>= 1) w[k] += __shfl_xor_sync(full, w[k], o);
        if (lane == 0 && b >= 0) atomicAdd(&ws.acc[b].vir_xf[k], w[k]);
        w[k] = 0.0;
    }
}

// Forces to the caller's order: one thread per particle reads its slot's
// accumulator (a gathered 16-byte read) and writes its force in place
// (coalesced).  The accumulators are left as they are: the next coordinate
// update, or a memset before the next force kernel, clears them.  Scattered
// writes, of forces to the caller's order or of cleared accumulators, cost
// several times more than these gathered reads on this GPU.  With want_vir
// also the FP64 sum per box of x (x) f (x the slot's wrapped coordinates):
// each warp takes a contiguous range of particles, 32 at a time, and the
// boxes' particles are contiguous, so its sums stay in registers until its
// box changes (one set of FP64 atomics per warp and box).  Particles
// without a slot (a column too long to grid, an error that is flagged) get
// zero force.  Block 0 also resets the force kernel's work counter.
__global__ void k_finalize(Workspace ws, int C, float* __restrict__ f_out, int want_vir) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) ws.work[0] = 0;
    const int n = ws.atom_total;
    const long long nslot = (long long)ws.clu_total * C;
    const long long n_warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wg = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long groups = ((long long)n + 31) / 32;
    const long long per = (groups + n_warps - 1) / n_warps;
    const long long g_end = min(groups, (wg + 1) * per);
    double w[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int b_cur = -1;
    for (long long g = wg * per; g < g_end; ++g) {
        const long long a = g * 32 + lane;
        int b = -1;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f), x = f;
        if (a < n) {
            const int sl = ws.slot_of_atom[a];
            if (sl >= 0 && sl < nslot) {
                f = ws.fslot[sl];
                if (want_vir) x = ws.xyzq[sl];
            }
            f_out[3 * a] = f.x;
            f_out[3 * a + 1] = f.y;
            f_out[3 * a + 2] = f.z;
            if (want_vir) b = find_box(ws.lay.atom_off, ws.nbox, (int)a);
        }
        if (!want_vir) continue;
        const int b0 = __shfl_sync(full, b, 0);   // lane 0 has a particle: g * 32 < n
        const bool uniform = __all_sync(full, b < 0 || b == b0);
        if (!uniform || b0 != b_cur) {
            virial_flush(ws, w, b_cur, lane);
            b_cur = uniform ? b0 : -1;
        }
        const double xa[3] = {x.x, x.y, x.z}, fb[3] = {f.x, f.y, f.z};
        if (uniform) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int c = 0; c < 3; ++c) w[3 * i + c] += xa[i] * fb[c];
        } else if (b >= 0) {
            // 32 particles straddling two boxes: add this group directly
            for (int i = 0; i < 3; ++i)
                for (int c = 0; c < 3; ++c) atomicAdd(&ws.acc[b].vir_xf[3 * i + c], xa[i] * fb[c]);
        }
    }
    if (want_vir) virial_flush(ws, w, b_cur, lane);
}

// Per box: the pair count of the evaluation, energies out, and
// W = sum x (x) f + sum_s (s L) (x) f_shift.
__global__ void k_finalize_small(Workspace ws, double* e_out, double* vir_out) {
    for (int b = threadIdx.x; b < ws.nbox; b += blockDim.x) {
        const Accum* acc = &ws.acc[b];
        ws.st[b].n_pairs_rc = acc->n_inc;
        if (e_out) {
            e_out[2 * b] = acc->energy[0];
            e_out[2 * b + 1] = acc->energy[1];
        }
        if (vir_out) {
            const float* L = ws.geo[b].L;
            double w[9];
            for (int k = 0; k < 9; ++k) w[k] = acc->vir_xf[k];
            for (int s = 0; s < 27; ++s) {
                const double sv[3] = {(double)(s / 9 - 1) * L[0], (double)((s / 3) % 3 - 1) * L[1],
                                      (double)(s % 3 - 1) * L[2]};
                for (int a = 0; a < 3; ++a)
                    for (int c = 0; c < 3; ++c) w[3 * a + c] += sv[a] * acc->fshift[s][c];
            }
            for (int k = 0; k < 9; ++k) vir_out[9 * b + k] = w[k];
        }
    }
}

cudaError_t launch_finalize(const Workspace& ws, const ForceParams& p, int C, float* f_out, double* e_out,
                            double* vir_out, cudaStream_t s) {
    const int want_vir = (p.want_energy && vir_out) ? 1 : 0;
    // one particle per thread without the virial; with it, fewer warps,
    // whose FP64 flushes meet on one box's nine addresses
    long long blocks = ((long long)ws.atom_total + 255) / 256;
    const long long cap = want_vir ? 1024 : 65535;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_finalize<<<(int)blocks, 256, 0, s>>>(ws, C, f_out, want_vir);
    if (p.want_energy) k_finalize_small<<<1, 256, 0, s>>>(ws, e_out, vir_out);
    return cudaGetLastError();
}

}  // namespace nbc
