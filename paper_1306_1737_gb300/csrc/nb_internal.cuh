// Internal declarations shared by the nbcluster CUDA sources (not part of the
// C ABI).
//
// A context holds one or more independent periodic boxes in one workspace.
// Every per-particle, per-column, per-cluster, per-super-cluster and list
// array is one batch array in which box b owns a region [off[b], off[b+1])
// fixed when the workspace is planned (capacity bounds); cluster, slot and
// list indices stored anywhere are batch-global.  Kernels find the box of a
// work item by binary search over the region offsets, so a single box is the
// batch of one and many small boxes share one launch per step.
// Layouts:
//   slots      : cluster g holds slots g*C .. g*C+C-1 (Sec. 2.3 clusters)
//   xyzq       : float4 per slot, wrapped coordinates + charge (dummies far away)
//   bb         : two float4 per cluster {xmin, ymin, zmin, 0}, {xmax, ymax, zmax, 0}
//   i-entry    : int4 {super-cluster, shift, j_begin, j_end}
//   j-entry    : word cj | (interaction bits << kSuperShift); masks [S][jstride]
//   fslot      : float4 per slot, force accumulators (w unused)
#pragma once

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nbcluster.h"

namespace nbc {

struct MlpTC;   // tensor-core form of the Ewald-factor network (nb_mlp.cuh)

constexpr int kMaxTypes = 64;          // LJ types (type table staged in shared memory)
constexpr int kMaxColumn = 8192;       // particles per grid column sorted on-chip
constexpr int kMaxBoxes = 4096;        // boxes per context
constexpr int kShiftCenter = 13;       // shift index of (0, 0, 0)
constexpr int kJChunk = 32;            // j-entries per i-entry at most (load balance)
constexpr int kJChunkCoop = 12;        // the same for boxes searched a block per super-cluster
// Super-clusters (Sec. 3.1, Fig. 6: several i-clusters share one j-list):
// up to super_size(C) consecutive clusters of one grid column.  A j-entry's
// word holds the j-cluster index in its low kSuperShift bits and one
// interaction bit per i-cluster of the super-cluster above them.
constexpr int kSuperShift = 27;
constexpr int kCjMask = (1 << kSuperShift) - 1;
__host__ __device__ constexpr int super_size(int C) { return C == 8 ? 2 : 1; }

// Device-resident state of one box: counters written by kernels, read back
// by nb_check.  Counts are box-local.
struct DevState {
    unsigned long long n_ient;          // outer list i-entries
    unsigned long long n_jent;          // outer list j-entries
    unsigned long long n_jent_pruned;   // j-entries kept by the last prune
    int nclu;                           // clusters of the current grid
    unsigned int flags;                 // 1 << nb_status_code
    int max_col;                        // largest column seen by the grid
    int nsc;                            // super-clusters of the current grid
    unsigned long long n_pairs_rc;      // pairs inside rc in the last energy evaluation
    unsigned long long n_keys;          // cluster pairs (i-cluster, j-cluster, shift) in the outer list
    unsigned long long n_keys_pruned;   // cluster pairs kept by the last prune
};

// FP64 accumulators of one force evaluation of one box.
struct Accum {
    double fshift[27][3];   // i-side force per periodic shift (virial bookkeeping)
    double energy[2];       // E_LJ, E_Coulomb
    double vir_xf[9];       // sum over slots x (x) f
    unsigned long long n_inc;  // pairs inside the cut-off (energy kernels only)
};

// Geometry of one box, rewritten by each nb_grid_put.
struct BoxGeom {
    float L[3];
    float inv_x, inv_y;     // FP32 n_x / L_x, n_y / L_y of the cell decision
    float inv_cx, inv_cy;   // the same, for the search's column ranges
    float dummy_g;          // dummy spacing (power of two >= 4 max L)
    int nx, ny;
};

// Region offsets of the boxes (device arrays of nbox + 1 entries, fixed by
// the workspace plan).  Column regions hold n_cols + 1 entries per box.
struct Layout {
    const int* atom_off;
    const int* col_off;
    const int* clu_off;
    const int* sc_off;
    const long long* ient_off;
    const long long* jent_off;
};

struct Workspace {
    int nbox;
    DevState* st;        // [nbox]
    Accum* acc;          // [nbox]
    BoxGeom* geo;        // [nbox]
    Layout lay;
    int atom_total, col_total, clu_total, sc_total;
    long long ient_total;
    // [nbox + 1]: exclusive prefix over boxes of the i-entries the last search
    // stored (clamped to capacity); entry nbox is their total.  Kernels that
    // walk the list index this compact range instead of the capacity.
    int* ient_used;
    // [2] work counters of the force and prune kernels (warps take the next
    // i-entry from them); zero between launches: the search's epilogue and
    // the kernel that follows each user reset them
    int* work;
    // per particle (caller order, all boxes concatenated)
    float4* xw;          // wrapped coordinates + charge
    float4* woff;        // wrap offset (wrapped - input), per particle
    int* col_of_atom;    // batch column index
    int* rank_in_col;
    int* slot_of_atom;   // batch slot index
    float* q;
    int* type;
    // per column (box regions of n_cols + 1)
    int* col_count;
    int* col_atom_start; // position of the column's first key in keys
    int* col_clu_start;  // first (batch) cluster of each column, end entry after the last
    int* col_sc_start;   // first (batch) super-cluster of each column
    int2* sc_info;       // per super-cluster {first batch cluster, number of clusters}
    unsigned long long* keys;  // sort keys in column order
    // per slot
    float4* xyzq;
    // per slot, two float4: {-x, -x, -y, -y}, {-z, -z, q, q} -- the
    // j-particle as the force kernel's packed pairs use it (both halves of a
    // lane's pair share j), written with xyzq -- and its LJ type; one record
    // of kJRecord float4 per group of 8 slots (an 8-particle cluster): the 8
    // first halves, the 8 second halves, the 8 types, 288 contiguous bytes
    float4* xjd;
    float4* woff_slot;   // the wrap offset of the slot's particle (written by the grid)
    int* atom_of_slot;   // batch particle index, -1 for dummies
    int* type_slot;
    float4* fslot;
    // per cluster
    float4* bb;          // [2 * clusters]
    // lists
    int4* ient;
    int* cj;
    unsigned long long* mask;
    int4* ient_p;
    int* cj_p;
    unsigned long long* mask_p;
    long long jstride;   // total j-entry capacity: stride between the S mask arrays
    // LJ table {C6, C12} [ntypes][ntypes]
    float2* c6c12;
    // the Ewald-factor network in tensor-core form (nb_set_surrogate)
    MlpTC* mlp;
    // the tabulated Ewald force factor [kEwaldTabN] (built with the workspace)
    float2* ewald_tab;
};

constexpr int kEwaldTabN = 2048;   // table intervals on w = (beta r)^2 in [0, kEwaldFitWMax]

// ---------------------------------------------------------------------------
// Host-side grid geometry (Sec. 2.3), shared by every gridding entry point so
// that they place particles identically.

// At most this many grid columns along x and along y, so that nx * ny fits
// an int; only slab-like boxes far thinner than the column spacing reach it.
constexpr int kMaxGridDim = 1 << 15;

inline int grid_extent(double L, double s) {
    const double g = std::floor(L / s);
    if (!(g >= 1.0)) return 1;
    return g > (double)kMaxGridDim ? kMaxGridDim : (int)g;
}

// Grid dimensions: spacing (C / rho)^(1/3) along x and y.
inline void grid_dims(int n, const float L[3], int C, int* nx, int* ny) {
    int gx = 1, gy = 1;
    if (n > 0) {
        const double Lx = L[0], Ly = L[1], Lz = L[2];
        const double rho = (double)n / (Lx * Ly * Lz);
        const double s = std::cbrt((double)C / rho);
        gx = grid_extent(Lx, s);
        gy = grid_extent(Ly, s);
    }
    *nx = gx;
    *ny = gy;
}

// Dummy spacing: the smallest power of two at least 4 times the longest edge.
inline float dummy_spacing(const float L[3]) {
    float m = L[0];
    if (L[1] > m) m = L[1];
    if (L[2] > m) m = L[2];
    float g = 1.0f;
    while (g < 4.0f * m) g *= 2.0f;
    return g;
}

// Geometry of a box of n particles with edges box[3] gridded with clusters of
// C: FP32 edges, grid dimensions, the FP32 inverse spacings of the cell
// decision and of the search's column ranges, and the dummy spacing.
inline BoxGeom box_geometry(int n, const double box[3], int C) {
    BoxGeom g{};
    for (int k = 0; k < 3; ++k) g.L[k] = (float)box[k];
    grid_dims(n, g.L, C, &g.nx, &g.ny);
    g.inv_x = (float)((double)g.nx / (double)g.L[0]);
    g.inv_y = (float)((double)g.ny / (double)g.L[1]);
    g.inv_cx = (float)g.nx / g.L[0];
    g.inv_cy = (float)g.ny / g.L[1];
    g.dummy_g = dummy_spacing(g.L);
    return g;
}

// Kernels whose dynamic shared memory exceeds the 48 KB default must opt in
// per device: the first launch on each device sets the attribute (host
// threads that race here set the same value).  done: one bit per device.
template <typename Kern>
inline cudaError_t smem_opt_in(Kern kern, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Kernel launchers (defined in the .cu files).
cudaError_t launch_grid(const Workspace& ws, int C, int ntypes, const float* xyz, cudaStream_t s);
cudaError_t launch_set_coords(const Workspace& ws, int C, const float* xyz, cudaStream_t s);
cudaError_t launch_search(const Workspace& ws, int C, float rlist, float rbb, const int* excl_off,
                          const int* excl_idx, int n_sm, cudaStream_t s);
cudaError_t launch_prune(const Workspace& ws, int C, float r_prune, int n_sm, cudaStream_t s);

struct ForceParams {
    int elec;
    int want_energy;
    float rc2;
    float fcoul;
    // reaction field
    float k_rf, two_k_rf, c_rf;
    // Ewald
    float beta, two_beta_sqrtpi;
    float beta2, beta3;   // beta^2, beta^3 for the fitted correction
    int use_fit;          // (beta rc)^2 within the fitted range
    // -beta^3 times the leading-coefficient ratio of the force factor's fit
    // in monic form: -beta^3 G(w) = fit_k Pm(w) / Qm(w)
    float fit_k;
    float mlp_rmin;       // network input range starts here (surrogate kernel)
    float tab_scale;      // beta^2 n / w_max: r^2 to table coordinate (tabulated kernel)
    int tab_n;            // table intervals
    int ntypes;
    int use_pruned;
    int prune;            // also prune the (outer) list being computed, at rp2
    float rp2;
};

cudaError_t launch_force(const Workspace& ws, const ForceParams& p, int C, int n_sm, cudaStream_t s);
cudaError_t launch_prune_reset(const Workspace& ws, cudaStream_t s);
cudaError_t launch_ewald_table(float2* tab, int n, double wmax, cudaStream_t s);
cudaError_t launch_finalize(const Workspace& ws, const ForceParams& p, int C, float* f_out, double* e_out,
                            double* vir_out, cudaStream_t s);

cudaError_t launch_pairlist_1x1(const Workspace& ws, int C, float rlist, int max_nbr, int* nbr, int* count,
                                int n_sm, cudaStream_t s);
cudaError_t launch_rdf(const Workspace& ws, int C, float r_max, int nbins, int type_a, int type_b,
                       unsigned long long* hist, int n_sm, cudaStream_t s);
cudaError_t launch_force_1x1(const Workspace& ws, const ForceParams& p, int C, int max_nbr, const int* nbr,
                             const int* count, cudaStream_t s);

// Kernels each launcher issues (for launch accounting).
constexpr int kLaunchesGrid = 4, kLaunchesSearch = 2, kLaunchesPrune = 2, kLaunchesSetCoords = 1;

// ---------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ void set_flag(DevState* st, int code) {
    atomicOr(&st->flags, 1u << code);
}

// Box b with off[b] <= x < off[b+1] (off ascending, nbox + 1 entries).
template <typename T>
__device__ __forceinline__ int find_box(const T* off, int nbox, T x) {
    int lo = 0, hi = nbox;
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (off[m] <= x) lo = m; else hi = m;
    }
    return lo;
}

// i-entry of compact index c (0 <= c < ient_used[nbox]) and its box.
__device__ __forceinline__ int ient_of(const int* ient_used, const long long* ient_off, int nbox, int c,
                                       int& b) {
    b = find_box(ient_used, nbox, c);
    return (int)ient_off[b] + (c - ient_used[b]);
}

// Advance box b (ascending walk) until off[b] <= x < off[b+1].
template <typename T>
__device__ __forceinline__ int advance_box(const T* off, int nbox, int b, T x) {
    while (b + 1 < nbox && off[b + 1] <= x) ++b;
    return b;
}

// Error-free sum a + b = s + e (Knuth TwoSum), every operation rounded once.
// Asynchronous global -> shared copies (cp.async, bypassing registers) of
// 16 or 4 bytes, and the wait for all of the thread's outstanding copies.
__device__ __forceinline__ void copy16_async(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void copy4_async(void* smem, const void* gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The two float4 of a slot's duplicated j layout and its LJ type (see
// Workspace::xjd).
constexpr int kJRecord = 18;
__device__ __forceinline__ void store_xjd(float4* xjd, long long s, float4 x) {
    float4* g = xjd + kJRecord * (s >> 3) + (s & 7);
    g[0] = make_float4(-x.x, -x.x, -x.y, -x.y);
    g[8] = make_float4(-x.z, -x.z, x.w, x.w);
}
__device__ __forceinline__ void store_jtype(float4* xjd, long long s, int type) {
    reinterpret_cast<int*>(xjd + kJRecord * (s >> 3) + 16)[s & 7] = type;
}

__device__ __forceinline__ void shift_vector(int s, const float L[3], float sh[3]) {
    sh[0] = (float)(s / 9 - 1) * L[0];
    sh[1] = (float)((s / 3) % 3 - 1) * L[1];
    sh[2] = (float)(s % 3 - 1) * L[2];
}

}  // namespace nbc
