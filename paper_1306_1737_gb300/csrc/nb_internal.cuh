// Internal declarations shared by the nbcluster CUDA sources (not part of the
// C ABI).  Layouts of the workspace-resident data:
//   slots      : cluster g holds slots g*C .. g*C+C-1 (Sec. 2.3 clusters)
//   xyzq       : float4 per slot, wrapped coordinates + charge (dummies far away)
//   bb         : two float4 per cluster {xmin, ymin, zmin, 0}, {xmax, ymax, zmax, 0}
//   i-entry    : int4 {ci, shift, j_begin, j_end}; j-entry: cj (int) + mask (u64)
//   fslot      : float4 per slot, force accumulators (w unused)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/nbcluster.h"

namespace nbc {

constexpr int kMaxTypes = 64;          // LJ types (type table staged in shared memory)
constexpr int kMaxColumn = 8192;       // particles per grid column sorted on-chip
constexpr int kShiftCenter = 13;       // shift index of (0, 0, 0)
constexpr int kJChunk = 32;            // j-entries per i-entry at most (load balance)
constexpr int kMaxExclPerCluster = 256;
// Super-clusters (Sec. 3.1, Fig. 6: several i-clusters share one j-list):
// up to kSuper consecutive clusters of one grid column.  A j-entry's word
// holds the j-cluster index in its low kSuperShift bits and one interaction
// bit per i-cluster of the super-cluster above them.
constexpr int kSuperShift = 27;
constexpr int kCjMask = (1 << kSuperShift) - 1;
__host__ __device__ constexpr int super_size(int C) { return C == 8 ? 2 : 1; }

// Device-resident state: counters written by kernels, read back by nb_check.
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

// FP64 accumulators of one force evaluation.
struct Accum {
    double fshift[27][3];   // i-side force per periodic shift (virial bookkeeping)
    double energy[2];       // E_LJ, E_Coulomb
    double vir_xf[9];       // sum over slots x (x) f
    unsigned long long n_inc;  // pairs inside the cut-off (energy kernels only)
};

struct Workspace {
    DevState* st;
    Accum* acc;
    // per particle (caller order)
    float4* xw;          // wrapped coordinates + charge
    float4* woff;        // wrap offset (wrapped - input), per particle
    int* col_of_atom;
    int* rank_in_col;
    int* slot_of_atom;
    float* q;
    int* type;
    // per column
    int* col_count;
    int* col_atom_start;
    int* col_clu_start;  // [ncol + 1]
    int* col_sc_start;   // [ncol + 1] first super-cluster of each column
    int2* sc_info;       // per super-cluster {first cluster, number of clusters}
    // sort keys (column order)
    unsigned long long* keys;
    // per slot
    float4* xyzq;
    int* atom_of_slot;
    int* type_slot;
    float4* fslot;
    // per cluster
    float4* bb;          // [2 * nclu]
    // lists: i-entry {super-cluster, shift, j_begin, j_end}; j-entry word
    // = cj | (interaction bits << kSuperShift); masks [S][jent capacity]
    int4* ient;
    int* cj;
    unsigned long long* mask;
    int4* ient_p;
    int* cj_p;
    unsigned long long* mask_p;
    long long jstride;   // j-entry capacity: stride between the S mask arrays
    // LJ table {C6, C12} [ntypes][ntypes]
    float2* c6c12;
};

struct GridGeom {
    float L[3];
    float inv_x, inv_y;
    int nx, ny;
    float dummy_g;
};

// Kernel launchers (defined in the .cu files).
cudaError_t launch_grid(const Workspace& ws, const GridGeom& g, int n, int C, int ntypes,
                        const float* xyz, int n_sm, cudaStream_t s);
cudaError_t launch_set_coords(const Workspace& ws, int n_slots_cap, int C, const float* xyz,
                              cudaStream_t s);
cudaError_t launch_search(const Workspace& ws, const GridGeom& g, int C, long long nclu_cap,
                          float rlist, float rbb, const int* excl_off, const int* excl_idx,
                          long long ient_cap, long long jent_cap, int n_atoms, int n_sm,
                          cudaStream_t s);
cudaError_t launch_prune(const Workspace& ws, const GridGeom& g, int C, float r_prune,
                         long long ient_cap, int n_sm, cudaStream_t s);

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
    int ntypes;
    float L[3];
    int use_pruned;
    long long ient_cap;
};

cudaError_t launch_force(const Workspace& ws, const ForceParams& p, int C, int n_sm,
                         long long n_slots_cap, cudaStream_t s);
cudaError_t launch_finalize(const Workspace& ws, const ForceParams& p, int n, float* f_out,
                            double* e_out, double* vir_out, cudaStream_t s);

// Kernels each launcher issues (for launch accounting).
constexpr int kLaunchesGrid = 4, kLaunchesSearch = 1, kLaunchesPrune = 1, kLaunchesSetCoords = 1;

// ---------------------------------------------------------------------------
// Device helpers

__device__ __forceinline__ void set_flag(DevState* st, int code) {
    atomicOr(&st->flags, 1u << code);
}

// Error-free sum a + b = s + e (Knuth TwoSum), every operation rounded once.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ int shift_comp(int s, int k) {
    return k == 0 ? s / 9 - 1 : (k == 1 ? (s / 3) % 3 - 1 : s % 3 - 1);
}

}  // namespace nbc
