/*
 * nbcluster -- cluster-pair non-bonded interactions on one GB300 (sm_103a).
 *
 * C ABI of the method of Pall & Hess, "A flexible algorithm for calculating
 * pair interactions on SIMD architectures": particles are gridded into
 * fixed-size spatial clusters (Sec. 2.3), a buffered cluster-pair list with
 * exclusion bitmasks is built (Sec. 2.3, Fig. 3, Sec. 2.4), pruned with a
 * particle-pair distance criterion (Sec. 2.3), and Lennard-Jones plus Coulomb
 * (reaction-field or Ewald real-space) forces and energies are computed per
 * cluster pair (Sec. 3, Fig. 6).
 *
 * Conventions
 *  - Units: nm, kJ/mol, elementary charge; forces in kJ mol^-1 nm^-1.
 *  - Rectangular periodic box; every cut-off and list radius must be below
 *    half of every box edge (minimum image).
 *  - Particle arrays are in the caller's order.  xyz is float [n][3].
 *  - Every pointer argument named *_dev is a device pointer owned by the
 *    caller; host arrays are named explicitly.  The library never allocates
 *    device memory: it works inside the workspace the caller provides.
 *  - Every call that takes a stream is asynchronous on that stream (a
 *    cudaStream_t; NULL = the legacy default stream) and performs no host
 *    synchronisation, so a sequence of calls can be captured in a CUDA graph.
 *    Errors that only the device can detect (list capacity overflow, a
 *    particle outside [-L, 2L), a column too long to sort on-chip, an LJ type
 *    or exclusion index out of range) raise a device flag that nb_check()
 *    reads.
 *  - Return value: NB_OK or an nb_status_code; nb_last_error() gives text.
 *  - A context keeps host-side state (plan, list state, events, the last
 *    error): one host thread at a time may call with it.  Calls on different
 *    contexts may run concurrently, as may the context-free entry points
 *    except nb_grid_put_noalloc (one fixed scratch array per device: see its
 *    own rule below).
 */
#ifndef NBCLUSTER_H
#define NBCLUSTER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx;
typedef void* nb_stream; /* cudaStream_t */
typedef int nb_status;

enum nb_status_code {
    NB_OK = 0,
    NB_ERR_ARG = 1,      /* null pointer, size or option out of range */
    NB_ERR_BOX = 2,      /* box edge <= 0 or >= 1e30, or a radius >= half a box edge */
    NB_ERR_CAPACITY = 3, /* workspace or list capacity exceeded */
    NB_ERR_CUDA = 4,     /* a CUDA runtime call failed */
    NB_ERR_STATE = 5,    /* call out of order (no workspace, no grid, no list) */
    NB_ERR_TIMEOUT = 6,  /* a bounded device wait expired (reserved: no kernel waits) */
    NB_ERR_COORD = 7     /* a coordinate outside [-L, 2L) at gridding */
};

enum nb_elec {
    NB_ELEC_RF = 0,    /* reaction field, g(r) = -2 k r (Sec. 3.2) */
    NB_ELEC_EWALD = 1, /* Ewald real space, g(r) = d/dr[erf(beta r)/r] (Sec. 3.2) */
    NB_ELEC_EWALD_MLP = 2, /* Ewald real space with the force factor c(r) of unmasked pairs
                              taken from a trained network (nb_set_surrogate); forces only */
    NB_ELEC_EWALD_TAB = 3  /* Ewald real space with the correction factor from a table in
                              (beta r)^2 with linear interpolation (Sec. 3.2, tabulated
                              kernels; 2,048 intervals on [0, 10], relative error 1.3e-6);
                              forces only, 8-particle clusters, (beta rc)^2 <= 10 */
};

enum nb_comb {
    NB_COMB_LB = 0,   /* Lorentz-Berthelot: sigma_ij = (s_i+s_j)/2, eps_ij = sqrt(e_i e_j) */
    NB_COMB_GEOM = 1  /* geometric: C6_ij = sqrt(C6_i C6_j), C12_ij = sqrt(C12_i C12_j) */
};

/* Creation options. */
typedef struct {
    int cluster_size; /* particles per cluster C (M = N = C); 4 or 8.  Sec. 2.2-2.3 */
    int device;       /* CUDA device ordinal the context is bound to */
} nb_options;

/* Interaction parameters (Sec. 3.2). */
typedef struct {
    int elec;          /* enum nb_elec */
    int want_energy;   /* 0: forces only; 1: also energies and virial */
    float rc;          /* interaction cut-off for LJ and Coulomb (nm) */
    float eps_rf;      /* reaction-field dielectric; <= 0 or inf means infinity */
    float beta;        /* Ewald splitting parameter (nm^-1) */
} nb_params;

/* Sizes of the current grid and lists (read back by nb_check), summed over
 * the boxes it covers (all boxes for nb_check, one for nb_box_info). */
typedef struct {
    int n_atoms;          /* particles gridded */
    int nx, ny;           /* grid columns along x and y (one box only; else 0) */
    int n_clusters;       /* clusters, including padded ones */
    int64_t n_ientries;   /* i-entries of the outer (rlist) list */
    int64_t n_jentries;   /* j-entries of the outer list */
    int64_t n_jentries_pruned; /* j-entries kept by the last prune (nb_prune or nb_prune_compute; -1: none) */
    int64_t ient_capacity, jent_capacity;
    int64_t n_pairs_rc;   /* particle pairs inside rc in the last energy evaluation */
    int64_t n_cluster_pairs;        /* cluster pairs (i-cluster, j-cluster, shift) in the outer list */
    int64_t n_cluster_pairs_pruned; /* cluster pairs kept by the last prune (-1: none) */
    int n_superclusters;  /* super-clusters (runs of up to super_size clusters of a column) */
    int super_size;       /* i-clusters per super-cluster: 2 for C = 8, 1 for C = 4 */
    int64_t n_launches;   /* kernels this context has launched */
    uint32_t flags;       /* device error flags (bit mask of 1 << nb_status_code) */
    int n_boxes;          /* boxes covered */
    int atom_offset;      /* index of the first box's first particle in the particle arrays */
} nb_info;

/* Kernel kinds reported by nb_profile_read. */
enum nb_kernel_kind {
    NB_KERNEL_GRID = 0,    /* the gridding kernels of nb_grid_put, as one span */
    NB_KERNEL_SEARCH = 1,  /* nb_pairlist_build's search kernel */
    NB_KERNEL_PRUNE = 2,   /* nb_prune's prune kernel */
    NB_KERNEL_FORCE = 3,   /* nb_compute's force/energy kernel */
    NB_KERNEL_FORCE_1X1 = 4, /* nb_compute_1x1's particle-pair force kernel */
    NB_KERNEL_RDF = 5,      /* nb_rdf's pair-distance histogram kernel */
    NB_KERNEL_FORCE_PRUNE = 6, /* nb_prune_compute's fused force + prune kernel */
    NB_KERNEL_FINALIZE = 7,  /* forces back to caller order, energies and virial out */
    NB_KERNEL_COORDS = 8     /* nb_set_coords (also inside the calls that take coordinates) */
};

/* --- context ------------------------------------------------------------ */

/* Create a context bound to opt->device (opt may be NULL: C = 8, device 0).
 * Errors: NB_ERR_ARG (C not 4 or 8), NB_ERR_CUDA. */
nb_status nb_create(nb_ctx** ctx, const nb_options* opt);

/* Destroy a context.  Does not free the caller's workspace. */
nb_status nb_destroy(nb_ctx* ctx);

/* Text of the last error on this context (never NULL). */
const char* nb_last_error(const nb_ctx* ctx);

/* Name of a status code. */
const char* nb_status_string(nb_status s);

/* --- host helpers -------------------------------------------------------- */

/* LJ pair table from per-type sigma (nm) and epsilon (kJ/mol) with a
 * combination rule (Sec. 3.2: geometric or Lorentz-Berthelot; C6 = 4 eps
 * sigma^6, C12 = 4 eps sigma^12).  Host arrays; c6c12_host is written as
 * float [ntypes][ntypes][2] = {C6, C12}.  Errors: NB_ERR_ARG. */
nb_status nb_lj_combine(int ntypes, const double* sigma_host, const double* eps_host, int comb,
                        float* c6c12_host);

/* --- workspace ------------------------------------------------------------ */

/* Bytes of device workspace needed for n_atoms particles in a box of edges
 * box_host[3] (nm), lists up to radius rlist_max (nm) and ntypes <= 64 LJ
 * types.  list_factor (>= 1; 0 = default 1.5) scales the density-based
 * estimate of the cluster-pair list capacity.  Fixes the context's plan (one
 * box); nb_set_workspace must follow.  The grid has at most 2^15 columns along
 * x and along y (reached only by boxes far thinner than the column spacing).
 * Errors: NB_ERR_ARG (more than 2^31 - 1 particles), NB_ERR_BOX,
 * NB_ERR_CAPACITY (more than 2^31 - 1 slots, i-entries or j-entries, or more
 * than 2^27 - 1 clusters: a j-entry word holds a 27-bit cluster index). */
nb_status nb_workspace_query(nb_ctx* ctx, int n_atoms, const double* box_host, double rlist_max,
                             int ntypes, double list_factor, size_t* bytes);

/* The same for a batch of nbox <= 4096 independent periodic boxes handled by
 * every call of the context together (one launch per kernel for all boxes).
 * Box b holds n_atoms_host[b] particles, which are the b-th consecutive range
 * of every particle array (q, type, xyz, f, exclusion CSR indices are
 * batch-global), in a box of edges boxes_host[3b..3b+2] (nm) used to size its
 * grid and list capacity.  The plan (particles per box) is fixed until the
 * next query; box edges may change at every nb_grid_put within the capacity.
 * Errors: as nb_workspace_query, with the limits on the sums over the boxes. */
nb_status nb_workspace_query_boxes(nb_ctx* ctx, int nbox, const int* n_atoms_host,
                                   const double* boxes_host, double rlist_max, int ntypes,
                                   double list_factor, size_t* bytes);

/* The bytes nb_workspace_query_boxes would return for a context of the given
 * cluster size (4 or 8), computed without a context or a device (host
 * arithmetic only), e.g. to size allocations ahead of time.
 * Errors: as nb_workspace_query_boxes; NB_ERR_ARG for another cluster size. */
nb_status nb_workspace_bytes(int cluster_size, int nbox, const int* n_atoms_host, const double* boxes_host,
                             double rlist_max, int ntypes, double list_factor, size_t* bytes);

/* Hand the context a device buffer of at least the queried size (256-byte
 * aligned).  The caller owns it and keeps it alive while the context uses
 * it.  Resets all state.  Errors: NB_ERR_ARG, NB_ERR_CAPACITY (too small). */
nb_status nb_set_workspace(nb_ctx* ctx, void* ws_dev, size_t bytes);

/* --- the hot path ---------------------------------------------------------- */

/* Particle charges (float [n]), LJ types (int [n], 0 <= type < ntypes) and the
 * LJ pair table c6c12_dev (float [ntypes][ntypes][2], e.g. nb_lj_combine;
 * shared by all boxes) are copied into the workspace on the stream.  Sec. 3.2.
 * n must equal the planned number of particles (summed over the boxes).  A
 * type outside 0 .. ntypes - 1 is not read here: the next nb_grid_put uses
 * type 0 for it and raises its box's NB_ERR_ARG device flag.
 * Errors: NB_ERR_ARG, NB_ERR_STATE (no workspace), NB_ERR_CAPACITY (n not the
 * planned number, or ntypes above 64), NB_ERR_CUDA. */
nb_status nb_set_atoms(nb_ctx* ctx, int n, const float* q_dev, const int* type_dev, int ntypes,
                       const float* c6c12_dev, nb_stream stream);

/* Spatial clustering (Sec. 2.3, Fig. 2): wrap xyz_dev (float [n][3], each
 * coordinate in [-L, 2L) of its own box) into its box, grid x/y into columns
 * of spacing (C/rho)^(1/3), sort each column on z, cut clusters of C with
 * dummy padding, compute bounding boxes.  boxes_host: double [nbox][3] edge
 * lengths (nm) of every box, used as FP32.  Invalidates the lists.  Inside
 * a stream capture the edges must equal those of the previous call (new
 * edges are staged through host memory, which a captured graph would re-read
 * at every replay): NB_ERR_STATE otherwise.
 * Errors: NB_ERR_ARG, NB_ERR_BOX, NB_ERR_STATE (no atoms set),
 * NB_ERR_CAPACITY (more columns/slots than the workspace holds), NB_ERR_CUDA;
 * device flags NB_ERR_COORD, NB_ERR_CAPACITY (column > 8192 particles),
 * NB_ERR_ARG (an LJ type outside 0 .. ntypes - 1, used as type 0). */
nb_status nb_grid_put(nb_ctx* ctx, const float* xyz_dev, const double* boxes_host, nb_stream stream);

/* Cluster-pair search (Sec. 2.3, Fig. 3) with exclusion bitmasks (Sec. 2.4):
 * every cluster pair (a <= b, periodic shift s applied to a; for a == b only
 * s = 0 and the positive half of the shifts) whose bounding boxes are closer
 * than rlist and either closer than rbb or holding a particle pair closer
 * than rlist.  Bit i*C+j of a pair's mask is 1 iff particles i of a and j of b
 * get the full interaction.  excl_off_dev (int [n+1]) and excl_idx_dev (int
 * [excl_off[n]]) give each particle's force-field exclusions (CSR, caller
 * order, both directions; an exclusion never links two boxes); both may be
 * NULL for none.  They are read on the stream and must stay valid until it
 * reaches this call.
 * Errors: NB_ERR_ARG, NB_ERR_BOX (rlist >= L/2 of a box), NB_ERR_STATE (no grid),
 * NB_ERR_CUDA; device flags NB_ERR_CAPACITY (list or exclusion overflow),
 * NB_ERR_ARG (an exclusion index outside 0 .. n - 1, ignored). */
nb_status nb_pairlist_build(nb_ctx* ctx, float rlist, float rbb, const int* excl_off_dev,
                            const int* excl_idx_dev, nb_stream stream);

/* New coordinates for the current grid and lists (float [n][3], caller order,
 * same periodic image as at nb_grid_put: the wrap offset applied then is
 * added again, so particles do not jump between images while a list lives).
 * Errors: NB_ERR_ARG, NB_ERR_STATE (no grid), NB_ERR_CUDA. */
nb_status nb_set_coords(nb_ctx* ctx, const float* xyz_dev, nb_stream stream);

/* Prune the outer list (Sec. 2.3): keep a cluster pair iff one of its counted
 * particle pairs (full or force-field-excluded; on the unshifted diagonal only
 * j > i) is closer than r_prune under the current coordinates.  Writes the
 * pruned list beside the outer list (which is kept for later prunes);
 * nb_compute uses the pruned list from then on.  xyz_dev may be NULL (keep
 * the current coordinates), else it is applied as by nb_set_coords.
 * Errors: NB_ERR_ARG, NB_ERR_STATE (no list), NB_ERR_BOX, NB_ERR_CUDA. */
nb_status nb_prune(nb_ctx* ctx, const float* xyz_dev, float r_prune, nb_stream stream);

/* Forces (and with p->want_energy, energies and virial) over the current list
 * (the pruned one after nb_prune, else the outer one) -- Sec. 3, Fig. 6:
 * per cluster pair, LJ (type table) plus Coulomb (RF or Ewald real space),
 * normal pairs by mask bit, force-field-excluded pairs within rc with the
 * correction only.  xyz_dev may be NULL (current coordinates).
 * f_dev: float [n][3], caller order, overwritten.
 * e_dev: double [nbox][2] {E_LJ, E_Coulomb} per box (kJ/mol), overwritten;
 * may be NULL.
 * vir_dev: double [nbox][9], per box W = sum over pairs r_ij (x) F_ij
 * (row-major), with r_ij = x_i - x_j and F_ij the force on i; overwritten;
 * may be NULL.
 * With p->elec == NB_ELEC_EWALD_MLP (C = 8 contexts with a network set by
 * nb_set_surrogate), the Coulomb force of every unmasked pair inside rc with
 * r >= r_min is f qq c_net(r) / r^2, c_net evaluated per 8 x 8 tile on the
 * tensor cores; excluded pairs keep the analytic correction.  That mode, and
 * NB_ELEC_EWALD_TAB (the correction factor from a table), compute forces
 * only: with want_energy set, the analytic Ewald kernel runs instead (forces,
 * energies and virial all analytic).
 * Errors: NB_ERR_ARG, NB_ERR_BOX (rc >= L/2, or rc above the list's radius:
 * rlist, or after nb_prune the smaller of rlist and r_prune), NB_ERR_STATE (no
 * list; no network for NB_ELEC_EWALD_MLP), NB_ERR_CUDA. */
nb_status nb_compute(nb_ctx* ctx, const nb_params* p, const float* xyz_dev, float* f_dev,
                     double* e_dev, double* vir_dev, nb_stream stream);

/* Synchronise the stream, read the device flags and sizes of every box into
 * *info (totals; may be NULL) and turn a raised flag into its status (the
 * message names the first box that raised it).  Clears the flags.  Not
 * callable during stream capture. */
nb_status nb_check(nb_ctx* ctx, nb_stream stream, nb_info* info);

/* Sizes and flags of one box as read by the last nb_check (host only).
 * Errors: NB_ERR_ARG (box out of range), NB_ERR_STATE (no nb_check yet). */
nb_status nb_box_info(nb_ctx* ctx, int box, nb_info* info);

/* --- timing --------------------------------------------------------------- */

/* enable != 0: from now on record a pair of CUDA events on the launching
 * stream around each hot-path kernel (kinds above; at most 256 spans are kept
 * until read).  Inside a stream capture the events become event-record nodes
 * of the graph, recorded at every replay.  enable == 2 does the same and also
 * keeps the spans across nb_profile_read calls, so that each replay of a
 * captured graph can be read; enable == 0 stops recording.
 * Errors: NB_ERR_CUDA. */
nb_status nb_profile(nb_ctx* ctx, int enable);

/* Wait for the recorded spans and return them in launch order: kinds[k] and
 * ms[k] for k < *count (at most max), then forget them (unless recording was
 * enabled with 2).  Host arrays.
 * Errors: NB_ERR_ARG, NB_ERR_CUDA. */
nb_status nb_profile_read(nb_ctx* ctx, int* kinds_host, float* ms_host, int max, int* count);

/* --- introspection (tests) -------------------------------------------------- */

/* Copy the grid (device to device, on the stream).  Any pointer may be NULL.
 * atom_of_slot_dev: int [nslots] (-1 for dummies), slot_of_atom_dev: int [n],
 * col_clu_start_dev: int [nx*ny+1], xyzq_dev: float [nslots][4] (wrapped
 * coordinates and charge; dummies far outside the box), type_slot_dev: int
 * [nslots], bb_dev: float [nclusters][6] (min xyz, max xyz), col_of_atom_dev:
 * int [n], sc_info_dev: int [n_superclusters][2] = {first cluster, number of
 * clusters} of each super-cluster.  nslots = n_clusters * C from nb_check.
 * One-box contexts only.
 * Errors: NB_ERR_STATE, NB_ERR_CUDA. */
nb_status nb_get_grid(nb_ctx* ctx, int* atom_of_slot_dev, int* slot_of_atom_dev,
                      int* col_clu_start_dev, float* xyzq_dev, int* type_slot_dev, float* bb_dev,
                      int* col_of_atom_dev, int* sc_info_dev, nb_stream stream);

/* Copy a list (which = 0: outer, 1: pruned) in its storage form, device to
 * device.  The list is kept per super-cluster (Sec. 3.1: several i-clusters
 * share one j-list): ient_dev int [n_ientries][4] = {super-cluster, shift,
 * j_begin, j_end}; cj_dev int [n_jentries], each the j-cluster index in bits
 * 0..26 and, in bits 27.., one interaction bit per i-cluster k of the
 * super-cluster (cluster first + k); mask_dev uint64 [super_size][n_jentries],
 * the exclusion mask of i-cluster k with that j-cluster (bit i*C+j: full
 * interaction).  Shift index s encodes (sx, sy, sz) in {-1,0,1}^3 as
 * (sx+1)*9 + (sy+1)*3 + (sz+1), applied to the i side.  Sizes from nb_check
 * (j-entries are indexed by the i-entries' ranges; for the pruned list use
 * the outer list's n_jentries as the array size).  One-box contexts only.
 * Errors: NB_ERR_STATE, NB_ERR_CUDA. */
nb_status nb_get_list(nb_ctx* ctx, int which, int* ient_dev, int* cj_dev, uint64_t* mask_dev,
                      nb_stream stream);

/* --- Verlet-buffer estimate (Appendix) ------------------------------------- */

/* Particles sharing mass, charge and LJ type, for the buffer estimate. */
typedef struct {
    double count;   /* particles of the class in the volume */
    double mass;    /* atomic mass units */
    double charge;  /* e */
    int type;       /* LJ type: row of the c6c12 table */
} nb_particle_class;

/* Upper bound on the energy drift (kJ mol^-1 ps^-1 per particle) caused by a
 * Verlet buffer rb (nm) over a list lifetime t_ps at temperature T (K), for
 * the classes in volume (nm^3) with interactions p (rc, electrostatics) and
 * the LJ table c6c12_host (float [ntypes][ntypes][2] = {C6, C12}): the
 * Appendix's estimate with free-flight displacements, sigma^2 = t^2 kB T
 * (1/m1 + 1/m2), and the pair potential expanded to second order at rc
 * (the second-order term integrated exactly: sigma (rb^2 + 2 sigma^2)).
 * Host-only arithmetic.  Errors: NB_ERR_ARG. */
nb_status nb_buffer_drift(int nclass, const nb_particle_class* classes_host, int ntypes,
                          const float* c6c12_host, double volume, const nb_params* p, double rb, double t_ps,
                          double temperature, double* drift_per_ps);

/* The smallest buffer rb (nm, to 1e-6) whose drift bound is at most
 * tolerance (kJ mol^-1 ps^-1 per particle).  Errors: NB_ERR_ARG. */
nb_status nb_buffer_size(int nclass, const nb_particle_class* classes_host, int ntypes, const float* c6c12_host,
                         double volume, const nb_params* p, double t_ps, double temperature, double tolerance,
                         double* rb);

/* Prune and compute in one pass (Sec. 2.3: pruning on the GPU).  With xyz_dev
 * (may be NULL: current coordinates) the forces (and energies, virial as in
 * nb_compute) are computed on the outer list of the last nb_pairlist_build,
 * and the same pass writes the pruned list at r_prune that later nb_compute
 * calls use; the pruned list equals the one nb_prune would write for these
 * coordinates.  One fused kernel for 8-particle clusters computing forces
 * with the analytic or tabulated factor; otherwise (4-particle clusters,
 * energies, the surrogate factor) nb_prune's kernel followed by the force
 * kernel on the pruned list.  rc must not exceed r_prune nor the list
 * radius.  Errors: as nb_compute and nb_prune. */
nb_status nb_prune_compute(nb_ctx* ctx, const nb_params* p, const float* xyz_dev, float r_prune, float* f_dev,
                           double* e_dev, double* vir_dev, nb_stream stream);

/* --- frames from host memory ---------------------------------------------------- */

/* A run of frames whose coordinates are in host memory, for a caller that
 * holds them there (a trajectory, or an integrator on the host).  The list
 * is built on the first frame and reused, pruned every nstprune frames
 * (Sec. 2.3: the Verlet buffer and pruning).  Frame f's coordinates are
 * copied in on copy_stream while frame f - 1 computes on stream, and frame
 * f's forces are copied out while frame f + 1 computes (two device buffers
 * each, ordered by events the context owns), so with page-locked host
 * memory the transfers overlap the kernels.  All host pointers must stay
 * valid, and unmodified or unread, until the streams have finished. */
typedef struct {
    int n_frames;                 /* >= 1 */
    int n_atoms, n_boxes;         /* the context's particle and box counts (the sizes below) */
    const float* x_host;          /* float [n_frames][n][3], caller order (page-locked for overlap) */
    float* f_host;                /* float [n_frames][n][3], overwritten */
    const unsigned char* energy_frames_host; /* [n_frames]: nonzero = energies (and virial) on that
                                     frame; NULL: forces only on every frame */
    double* e_host;               /* double [n_frames][nbox][2], written on energy frames; may be NULL */
    double* vir_host;             /* double [n_frames][nbox][9], written on energy frames; may be NULL */
    float* x_dev[2];              /* device staging, float [n][3] each */
    float* f_dev[2];              /* device staging, float [n][3] each */
    double* e_dev[2];             /* device staging, double [nbox][2] each (when e_host) */
    double* vir_dev[2];           /* device staging, double [nbox][9] each (when vir_host) */
    int build;                    /* nonzero: grid and list on frame 0 (boxes_host, rlist, rbb,
                                     exclusions as nb_grid_put and nb_pairlist_build); zero:
                                     every frame updates the coordinates of the current list */
    const double* boxes_host;     /* as nb_grid_put (build only) */
    float rlist, rbb;             /* as nb_pairlist_build (build only) */
    const int* excl_off_dev;      /* as nb_pairlist_build (build only) */
    const int* excl_idx_dev;
    int first_frame;              /* index of frame 0 within the list's lifetime (0 with build) */
    int nstprune;                 /* frames f with first_frame + f > 0 and a multiple of nstprune
                                     prune at r_prune in their force pass (nb_prune_compute);
                                     0: no pruning */
    float r_prune;
} nb_frames;

/* Forces (and, on the chosen frames, energies and virial) of every frame of
 * fr with the interactions p (p->want_energy is ignored: energy_frames_host
 * decides), as nb_compute and nb_prune_compute would give them frame by
 * frame.  stream computes; copy_stream copies (must differ from stream; both
 * on the context's device).  Returns after queuing the work: stream waits for
 * copy_stream's last copy, so synchronising stream makes every output
 * readable.  Errors: NB_ERR_ARG (null pointers, n_frames < 1, n_atoms or
 * n_boxes not the context's, equal streams, nstprune < 0), and those of the calls it makes (nb_grid_put,
 * nb_pairlist_build, nb_compute, nb_prune_compute), returned at the first
 * failing frame with the frames before it queued.
 * Runs with build set are the same work whenever their arguments are the
 * same: every field of fr and *p, the box edges and energy flags (by value)
 * and the context's state (workspace, atoms, network, geometry, profiling).
 * The first such run is made call by call, the second is captured in a CUDA
 * graph and later ones replay it on stream (its copies are graph nodes,
 * copy_stream is not used); a replay reads the host frames anew, so new
 * coordinates in the same buffers give their own forces.  Not while stream
 * is being captured by the caller, nor with nb_profile on (those runs are
 * made call by call). */
nb_status nb_run_frames(nb_ctx* ctx, const nb_params* p, const nb_frames* fr, nb_stream stream,
                        nb_stream copy_stream);

/* --- the particle-pair (1 x 1) comparison path -------------------------------- */

/* A full particle-pair Verlet list (every pair within rlist stored for both
 * particles) expanded from the current outer cluster-pair list, for the
 * comparison the paper makes between cluster-pair (M x N) and particle-pair
 * (1 x 1) setups (Sec. 4-5, Table 3).  rlist must not exceed the radius of
 * the last nb_pairlist_build, and the coordinates must be the ones that list
 * was built from (no nb_set_coords, nb_prune or nb_compute with new
 * coordinates since).  nbr_dev: int [n][max_nbr] entries, each
 * (neighbour slot << 6) | (force-field excluded << 5) | shift index (the
 * shift applied to the particle owning the row); count_dev: int [n] entries
 * per particle (a row holds min(count, max_nbr); a count above max_nbr
 * raises the NB_ERR_CAPACITY device flag).  Caller order, device memory.
 * Errors: NB_ERR_ARG, NB_ERR_STATE (no list, or new coordinates since it was
 * built), NB_ERR_BOX, NB_ERR_CUDA. */
nb_status nb_pairlist_1x1(nb_ctx* ctx, float rlist, int max_nbr, int* nbr_dev, int* count_dev,
                          nb_stream stream);

/* Forces over a 1 x 1 list from nb_pairlist_1x1: 16, 8 or 4 lanes per
 * particle (fewer for more particles) summing its row, each pair computed for
 * both of its particles (no atomics), with the same pair interactions as
 * nb_compute (RF or Ewald; forces only, p->want_energy must be 0).  rc must
 * not exceed the radius the list was built with (the list is the caller's:
 * not checked).  xyz_dev may be NULL (current coordinates);
 * f_dev: float [n][3], caller order, overwritten.
 * Errors: NB_ERR_ARG, NB_ERR_STATE, NB_ERR_BOX, NB_ERR_CUDA. */
nb_status nb_compute_1x1(nb_ctx* ctx, const nb_params* p, const float* xyz_dev, const int* nbr_dev,
                         const int* count_dev, int max_nbr, float* f_dev, nb_stream stream);

/* --- pair-distance histogram (pair correlation) ------------------------------ */

#define NB_RDF_MAX_BINS 2048

/* Histogram of particle-pair distances over the current outer cluster-pair
 * list: the pair correlation analysis that the paper names as limited-range
 * pair work (Sec. 1) and for which it rebuilds the list for every evaluation
 * and uses neither pruning nor a cut-off conditional in the kernel (Sec. 2.3).
 * Every listed pair whose mask bit is set (distinct real particles, not
 * force-field excluded; each pair once) and whose types match the selection
 * (type_a = type_b = -1: every pair; else {type_i, type_j} = {type_a, type_b})
 * adds one to bin min(int(r / dr), nbins) of its box, dr = r_max / nbins, r
 * from the FP32 distance vector (periodic shift as hi + lo): bins
 * 0 .. nbins - 1 cover [0, r_max), bin nbins counts the listed pairs at
 * r >= r_max.  hist_dev: uint64 [nbox][nbins + 1], device memory, zeroed
 * first unless accumulate != 0 (to sum several frames).  The list must come
 * from nb_pairlist_build on the current coordinates (no nb_set_coords,
 * nb_prune or nb_compute with new coordinates since) with rlist >= r_max, so
 * that it holds every pair closer than r_max.  For N_a and N_b particles of
 * the selected types in volume V, g(r) in bin k is h_k V / (P dV_k) with
 * dV_k = 4 pi / 3 ((k + 1)^3 - k^3) dr^3 and P = N_a N_b pairs (P =
 * N_a (N_a - 1) / 2 for one type or every pair) less the force-field-excluded
 * pairs among them.
 * Errors: NB_ERR_ARG (nbins outside 1 .. NB_RDF_MAX_BINS, r_max <= 0, a type
 * outside -1 .. ntypes - 1 or only one of them -1, null hist_dev),
 * NB_ERR_STATE (no list, or coordinates changed since it was built),
 * NB_ERR_BOX (r_max above the list radius), NB_ERR_CUDA. */
nb_status nb_rdf(nb_ctx* ctx, float r_max, int nbins, int type_a, int type_b, int accumulate,
                 uint64_t* hist_dev, nb_stream stream);

/* --- learned Ewald force factor --------------------------------------------- */

/* The network: a multilayer perceptron 1 -> 32 -> 32 -> 1 with SiLU hidden
 * layers that stands in for the Ewald real-space force factor
 * c(r) = erfc(beta r) + 2 beta r / sqrt(pi) exp(-beta^2 r^2) (Sec. 3.2: the
 * non-excluded real-space Coulomb force is f qq c(r) / r^2).  Input
 * x = (r - (r_min + r_max)/2) * 2 / (r_max - r_min).  Parameters: float
 * [NB_MLP_NPARAMS] = W1[32], b1[32], W2[32][32] (row = output unit), b2[32],
 * W3[32], b3.  All pointers are device pointers; all calls are asynchronous
 * on the stream.  The paper has no network; it is an alternative to the
 * paper's analytic approximation of the same factor. */
#define NB_MLP_NPARAMS 1153

/* FP64 c(r) for n distances (the training targets).  Errors: NB_ERR_ARG,
 * NB_ERR_CUDA. */
nb_status nb_ewald_factor(const double* r_dev, int64_t n, double beta, double* out_dev, nb_stream stream);

/* y = network(r) for n distances on the CUDA cores in FP32.
 * Errors: NB_ERR_ARG (r_max <= r_min, null pointers), NB_ERR_CUDA. */
nb_status nb_mlp_forward(const float* params_dev, float r_min, float r_max, const float* r_dev, int64_t n,
                         float* y_dev, nb_stream stream);

/* Bytes of the tensor-core form of a network (per-lane fragments of W2 as
 * BF16 hi + lo parts and the lane's FP32 layer-1/3 parameters). */
size_t nb_mlp_packed_bytes(void);

/* Write the tensor-core form of params into packed_dev (16-byte aligned, at
 * least nb_mlp_packed_bytes()).  Errors: NB_ERR_ARG, NB_ERR_CUDA. */
nb_status nb_mlp_pack(const float* params_dev, float r_min, float r_max, void* packed_dev, nb_stream stream);

/* y = network(r) through the tensor-core tile evaluator of the force kernel
 * (64 distances per warp; layer 2 as BF16 mma.sync with hi/lo splitting and
 * FP32 accumulation).  Errors: NB_ERR_ARG, NB_ERR_CUDA. */
nb_status nb_mlp_forward_tc(const void* packed_dev, const float* r_dev, int64_t n, float* y_dev,
                            nb_stream stream);

/* Loss L = (1/n) sum_i w_i (y(r_i) - t_i)^2 (w_dev may be NULL: weights 1)
 * into *loss_dev (may be NULL) and dL/dparams into grad_dev
 * [NB_MLP_NPARAMS], FP32.  Errors: NB_ERR_ARG, NB_ERR_CUDA. */
nb_status nb_mlp_loss_grad(const float* params_dev, float r_min, float r_max, const float* r_dev,
                           const float* t_dev, const float* w_dev, int64_t n, float* grad_dev,
                           float* loss_dev, nb_stream stream);

/* steps Adam updates (beta1 0.9, beta2 0.999, eps 1e-8) of params_dev on
 * minibatches of `batch` consecutive samples of (r, t, w) (wrapping around
 * the n samples; step k of the schedule starts at sample k * batch mod n),
 * learning rate lr_min + (lr_max - lr_min) (1 + cos(pi k / total_steps)) / 2
 * for schedule steps k = step0 .. step0 + steps - 1.  state_dev: float
 * [3 * NB_MLP_NPARAMS] = Adam first and second moments and a gradient
 * buffer; zero it before step 0.  loss_dev: float [steps] minibatch losses,
 * or NULL.  Errors: NB_ERR_ARG, NB_ERR_CUDA. */
nb_status nb_mlp_train(float* params_dev, float* state_dev, float r_min, float r_max, const float* r_dev,
                       const float* t_dev, const float* w_dev, int64_t n, int batch, int steps, int step0,
                       int total_steps, float lr_max, float lr_min, float* loss_dev, nb_stream stream);

/* Give the context a network for NB_ELEC_EWALD_MLP (copied into the
 * workspace in tensor-core form on the stream; params_dev may be freed once
 * the stream reaches this call).  The network is used for unmasked pairs
 * with r_min <= r < rc, so r_max must be >= the rc of later nb_compute calls.
 * Errors: NB_ERR_ARG (C != 8, bad range), NB_ERR_STATE (no workspace),
 * NB_ERR_CUDA. */
nb_status nb_set_surrogate(nb_ctx* ctx, const float* params_dev, float r_min, float r_max, nb_stream stream);

/* --- gridding without device allocation ------------------------------------ */

/* nb_grid_put's gridding (wrap, columns, z sort, clusters with dummies,
 * bounding boxes) for callers that cannot allocate device memory at all:
 * code that must not call cudaMalloc (for example inside a host callback or
 * a graph node, a plug-in whose device memory is owned and capped by its
 * host application, or a process whose allocations go through another
 * runtime's allocator).  It needs no context and no workspace: its scratch
 * lives in a fixed-size array that the library's module carries on every GPU
 * that loads it (about 2.8 MB, held until the process exits).  The paper has
 * no counterpart to this entry point; the results are bit-identical to
 * nb_grid_put followed by nb_get_grid.
 *
 * Limits: n <= 32768 particles, at most 4096 grid columns, and
 * n + columns * (C - 1) <= 61440 slots; beyond them the call returns
 * NB_ERR_CAPACITY and does nothing.
 * Inputs (device): xyz float [n][3] (each coordinate in [-L, 2L)), q float
 * [n], type int [n] (0 <= type < ntypes <= 64); box_host double[3].
 * Outputs (device, written on the stream): atom_of_slot int [max_slots]
 * (-1 for a dummy), xyzq float [max_slots][4] (wrapped coordinates and
 * charge), type_slot int [max_slots], bb float [max_slots / C][8]
 * ({xmin, ymin, zmin, 0, xmax, ymax, zmax, 0} per cluster), col_clu_start
 * int [max_columns + 1], info int [2] = {number of clusters, device flags
 * (1 << NB_ERR_COORD for a coordinate outside [-L, 2L), 1 << NB_ERR_ARG for
 * a type out of range, 1 << NB_ERR_CAPACITY for a grid column holding more
 * than 8192 particles: that column's particles get no slot, its clusters
 * are dummies, and the call still returns NB_OK)}.  Only the first
 * clusters * C slots and nx * ny + 1 column entries are written.  xyzq and
 * bb must be 16-byte aligned.
 * The first call on a device (with that device current) looks up the
 * scratch array's device address; make that first call before any stream
 * capture.  All calls share the one array and each call clears the parts
 * that must start at zero, so calls whose work overlaps on the GPU race:
 * serialise them (one stream, or events between streams).
 * Errors: NB_ERR_ARG, NB_ERR_BOX, NB_ERR_CAPACITY, NB_ERR_CUDA. */
nb_status nb_grid_put_noalloc(int n, const float* xyz_dev, const float* q_dev, const int* type_dev,
                              int ntypes, const double* box_host, int cluster_size,
                              int* atom_of_slot_dev, float* xyzq_dev, int* type_slot_dev,
                              float* bb_dev, int* col_clu_start_dev, int* info_dev, int max_slots,
                              int max_columns, nb_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* NBCLUSTER_H */
