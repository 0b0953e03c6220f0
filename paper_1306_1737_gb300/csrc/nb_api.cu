// C ABI of nbcluster (declared in include/nbcluster.h): context, workspace
// carving, argument checks, and the stream-ordered launch sequence of the
// hot path.  No device allocation happens here; all device data lives in the
// caller's workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "nb_internal.cuh"
#include "nb_ewald_fit.h"

using namespace nbc;

struct nb_ctx {
    int C = 8;
    int device = 0;
    int n_sm = 0;
    // workspace sizes
    char* ws_base = nullptr;
    size_t ws_bytes = 0;
    int n_cap = 0;
    int ncol_cap = 0;
    long long nslot_cap = 0, nclu_cap = 0, nsc_cap = 0, ient_cap = 0, jent_cap = 0;
    int ntypes_cap = 0;
    Workspace ws{};
    DevState* st_host = nullptr;  // pinned read-back buffer
    // state
    int n = 0, ntypes = 0;
    bool have_atoms = false, have_grid = false, have_list = false, have_pruned = false;
    GridGeom geom{};
    float rlist = 0.f, r_prune = 0.f;
    DevState last{};
    bool last_valid = false;
    long long n_launches = 0;
    // timing spans (nb_profile)
    static constexpr int kMaxSpans = 256;
    bool prof = false;
    cudaEvent_t ev[2 * kMaxSpans] = {};
    int ev_kind[kMaxSpans] = {};
    int ev_n = 0;
    char err[512] = {0};
};

// Record the start of a timed span (returns its slot or -1).
static int span_begin(nb_ctx* c, int kind, cudaStream_t s) {
    if (!c->prof || c->ev_n >= nb_ctx::kMaxSpans) return -1;
    const int k = c->ev_n++;
    c->ev_kind[k] = kind;
    cudaEventRecord(c->ev[2 * k], s);
    return k;
}

static void span_end(nb_ctx* c, int k, cudaStream_t s) {
    if (k >= 0) cudaEventRecord(c->ev[2 * k + 1], s);
}

static nb_status fail(nb_ctx* c, nb_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

static nb_status cuda_fail(nb_ctx* c, cudaError_t e, const char* where) {
    return fail(c, NB_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NB_CUDA(ctx, call)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

static bool box_ok(const double* box) {
    if (!box) return false;
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 0.0) || !std::isfinite(box[k])) return false;
    return true;
}

// Grid dimensions (Sec. 2.3): spacing (C / rho)^(1/3) along x and y.
static void grid_dims(int n, const float L[3], int C, int* nx, int* ny) {
    int gx = 1, gy = 1;
    if (n > 0) {
        const double Lx = L[0], Ly = L[1], Lz = L[2];
        const double rho = (double)n / (Lx * Ly * Lz);
        const double s = std::cbrt((double)C / rho);
        gx = (int)std::floor(Lx / s);
        gy = (int)std::floor(Ly / s);
        if (gx < 1) gx = 1;
        if (gy < 1) gy = 1;
    }
    *nx = gx;
    *ny = gy;
}

static float dummy_spacing(const float L[3]) {
    float m = L[0];
    if (L[1] > m) m = L[1];
    if (L[2] > m) m = L[2];
    float g = 1.0f;
    while (g < 4.0f * m) g *= 2.0f;
    return g;
}

struct Sizes {
    int n, ncol, ntypes, S;
    long long nslot, nclu, nsc, ient, jent;
};

// Lay the workspace out from base (nullptr: only count bytes).
static size_t carve(const Sizes& z, char* base, Workspace* ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    Workspace w{};
    w.st = (DevState*)take(sizeof(DevState));
    w.acc = (Accum*)take(sizeof(Accum));
    w.xw = (float4*)take(sizeof(float4) * z.n);
    w.woff = (float4*)take(sizeof(float4) * z.n);
    w.col_of_atom = (int*)take(sizeof(int) * z.n);
    w.rank_in_col = (int*)take(sizeof(int) * z.n);
    w.slot_of_atom = (int*)take(sizeof(int) * z.n);
    w.q = (float*)take(sizeof(float) * z.n);
    w.type = (int*)take(sizeof(int) * z.n);
    w.col_count = (int*)take(sizeof(int) * z.ncol);
    w.col_atom_start = (int*)take(sizeof(int) * z.ncol);
    w.col_clu_start = (int*)take(sizeof(int) * (z.ncol + 1));
    w.col_sc_start = (int*)take(sizeof(int) * (z.ncol + 1));
    w.sc_info = (int2*)take(sizeof(int2) * z.nsc);
    w.keys = (unsigned long long*)take(sizeof(unsigned long long) * z.n);
    w.xyzq = (float4*)take(sizeof(float4) * z.nslot);
    w.atom_of_slot = (int*)take(sizeof(int) * z.nslot);
    w.type_slot = (int*)take(sizeof(int) * z.nslot);
    w.fslot = (float4*)take(sizeof(float4) * z.nslot);
    w.bb = (float4*)take(sizeof(float4) * 2 * z.nclu);
    w.ient = (int4*)take(sizeof(int4) * z.ient);
    w.cj = (int*)take(sizeof(int) * z.jent);
    w.mask = (unsigned long long*)take(sizeof(unsigned long long) * z.jent * z.S);
    w.ient_p = (int4*)take(sizeof(int4) * z.ient);
    w.cj_p = (int*)take(sizeof(int) * z.jent);
    w.mask_p = (unsigned long long*)take(sizeof(unsigned long long) * z.jent * z.S);
    w.jstride = z.jent;
    w.c6c12 = (float2*)take(sizeof(float2) * z.ntypes * z.ntypes);
    if (ws) *ws = w;
    return (off + 255) & ~(size_t)255;
}

// Sizes for n particles in box L with lists up to rlist.  The number of
// j-entries is estimated from the density: j-clusters whose bounding box is
// within rlist of a super-cluster's box (half of them, Newton's third law),
// i.e. the cluster density times the volume of the rounded box of side
// (super-cluster extent + cluster extent) dilated by rlist, scaled by factor.
static Sizes plan(int n, const float L[3], int C, double rlist, int ntypes, double factor) {
    Sizes z{};
    int nx, ny;
    grid_dims(n, L, C, &nx, &ny);
    z.n = n > 0 ? n : 1;
    z.ncol = nx * ny;
    z.ntypes = ntypes;
    z.S = super_size(C);
    z.nslot = (long long)n + (long long)z.ncol * (C - 1);
    z.nclu = z.nslot / C + 1;
    z.nsc = z.nclu / z.S + z.ncol + 1;
    const double V = (double)L[0] * L[1] * L[2];
    const double wx = (double)L[0] / nx, wy = (double)L[1] / ny;
    const double rho = n > 0 ? n / V : 1.0;
    const double hz = C / (rho * wx * wy);
    const double a = 2 * wx, b = 2 * wy, c = (z.S + 1) * hz, r = rlist;
    const double vm = a * b * c + 2 * r * (a * b + b * c + c * a) + M_PI * r * r * (a + b + c) +
                      4.0 / 3.0 * M_PI * r * r * r;
    const double rho_c = (double)z.nclu / V;
    double per = 0.5 * rho_c * vm + z.S;
    const double maxper = 0.5 * 27.0 * (double)z.nclu + 1.0;
    if (per > maxper) per = maxper;
    z.jent = (long long)std::ceil(factor * per * (double)z.nsc) + 1024;
    z.ient = z.nsc * 27 + z.jent / kJChunk + 1024;
    return z;
}

extern "C" {

const char* nb_status_string(nb_status s) {
    switch (s) {
        case NB_OK: return "NB_OK";
        case NB_ERR_ARG: return "NB_ERR_ARG";
        case NB_ERR_BOX: return "NB_ERR_BOX";
        case NB_ERR_CAPACITY: return "NB_ERR_CAPACITY";
        case NB_ERR_CUDA: return "NB_ERR_CUDA";
        case NB_ERR_STATE: return "NB_ERR_STATE";
        case NB_ERR_TIMEOUT: return "NB_ERR_TIMEOUT";
        case NB_ERR_COORD: return "NB_ERR_COORD";
        default: return "NB_UNKNOWN";
    }
}

nb_status nb_create(nb_ctx** out, const nb_options* opt) {
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    const int C = opt ? opt->cluster_size : 8;
    const int dev = opt ? opt->device : 0;
    if (C != 4 && C != 8) return NB_ERR_ARG;
    nb_ctx* c = new (std::nothrow) nb_ctx();
    if (!c) return NB_ERR_ARG;
    c->C = C;
    c->device = dev;
    cudaError_t e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->st_host, sizeof(DevState));
    if (e != cudaSuccess) {
        delete c;
        return NB_ERR_CUDA;
    }
    *out = c;
    return NB_OK;
}

nb_status nb_destroy(nb_ctx* c) {
    if (!c) return NB_ERR_ARG;
    if (c->st_host) cudaFreeHost(c->st_host);
    for (int k = 0; k < 2 * nb_ctx::kMaxSpans; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    delete c;
    return NB_OK;
}

const char* nb_last_error(const nb_ctx* c) { return c ? c->err : "null context"; }

nb_status nb_lj_combine(int ntypes, const double* sigma, const double* eps, int comb, float* out) {
    if (ntypes <= 0 || !sigma || !eps || !out) return NB_ERR_ARG;
    if (comb != NB_COMB_LB && comb != NB_COMB_GEOM) return NB_ERR_ARG;
    for (int a = 0; a < ntypes; ++a) {
        for (int b = 0; b < ntypes; ++b) {
            double c6, c12;
            if (comb == NB_COMB_LB) {
                const double s = 0.5 * (sigma[a] + sigma[b]);
                const double e = std::sqrt(eps[a] * eps[b]);
                const double s6 = s * s * s * s * s * s;
                c6 = 4.0 * e * s6;
                c12 = c6 * s6;
            } else {
                const double sa6 = std::pow(sigma[a], 6.0), sb6 = std::pow(sigma[b], 6.0);
                c6 = std::sqrt(4.0 * eps[a] * sa6 * 4.0 * eps[b] * sb6);
                c12 = std::sqrt(4.0 * eps[a] * sa6 * sa6 * 4.0 * eps[b] * sb6 * sb6);
            }
            out[2 * (a * ntypes + b)] = (float)c6;
            out[2 * (a * ntypes + b) + 1] = (float)c12;
        }
    }
    return NB_OK;
}

nb_status nb_workspace_query(nb_ctx* c, int n, const double* box, double rlist_max, int ntypes,
                             double list_factor, size_t* bytes) {
    if (!c || !bytes || n < 0 || ntypes <= 0) return fail(c, NB_ERR_ARG, "workspace_query: bad argument");
    if (ntypes > kMaxTypes) return fail(c, NB_ERR_ARG, "at most %d LJ types", kMaxTypes);
    if (!box_ok(box)) return fail(c, NB_ERR_BOX, "box edges must be positive");
    if (!(rlist_max > 0.0)) return fail(c, NB_ERR_ARG, "rlist_max must be positive");
    if (list_factor == 0.0) list_factor = 1.5;
    if (list_factor < 1.0) return fail(c, NB_ERR_ARG, "list_factor must be >= 1");
    const float L[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const Sizes z = plan(n, L, c->C, rlist_max, kMaxTypes, list_factor);
    *bytes = carve(z, nullptr, nullptr);
    // remember the plan for nb_set_workspace
    c->n_cap = z.n;
    c->ncol_cap = z.ncol;
    c->nslot_cap = z.nslot;
    c->nclu_cap = z.nclu;
    c->nsc_cap = z.nsc;
    c->ient_cap = z.ient;
    c->jent_cap = z.jent;
    c->ntypes_cap = kMaxTypes;
    (void)ntypes;
    return NB_OK;
}

nb_status nb_set_workspace(nb_ctx* c, void* ws, size_t bytes) {
    if (!c || !ws) return fail(c, NB_ERR_ARG, "set_workspace: null");
    if (((uintptr_t)ws & 255) != 0) return fail(c, NB_ERR_ARG, "workspace must be 256-byte aligned");
    if (c->n_cap == 0) return fail(c, NB_ERR_STATE, "call nb_workspace_query first");
    Sizes z{};
    z.n = c->n_cap;
    z.ncol = c->ncol_cap;
    z.ntypes = c->ntypes_cap;
    z.nslot = c->nslot_cap;
    z.nclu = c->nclu_cap;
    z.nsc = c->nsc_cap;
    z.S = super_size(c->C);
    z.ient = c->ient_cap;
    z.jent = c->jent_cap;
    const size_t need = carve(z, nullptr, nullptr);
    if (bytes < need) return fail(c, NB_ERR_CAPACITY, "workspace has %zu bytes, needs %zu", bytes, need);
    NB_CUDA(c, cudaSetDevice(c->device));
    carve(z, (char*)ws, &c->ws);
    c->ws_base = (char*)ws;
    c->ws_bytes = bytes;
    c->have_atoms = c->have_grid = c->have_list = c->have_pruned = false;
    c->last_valid = false;
    NB_CUDA(c, cudaMemset(c->ws.st, 0, sizeof(DevState)));
    return NB_OK;
}

nb_status nb_set_atoms(nb_ctx* c, int n, const float* q, const int* type, int ntypes,
                       const float* c6c12, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->ws_base) return fail(c, NB_ERR_STATE, "no workspace");
    if (n < 0 || (n > 0 && (!q || !type)) || ntypes <= 0 || !c6c12)
        return fail(c, NB_ERR_ARG, "set_atoms: bad argument");
    if (n > c->n_cap) return fail(c, NB_ERR_CAPACITY, "%d particles, workspace holds %d", n, c->n_cap);
    if (ntypes > c->ntypes_cap) return fail(c, NB_ERR_CAPACITY, "too many LJ types");
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        NB_CUDA(c, cudaMemcpyAsync(c->ws.q, q, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        NB_CUDA(c, cudaMemcpyAsync(c->ws.type, type, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    NB_CUDA(c, cudaMemcpyAsync(c->ws.c6c12, c6c12, sizeof(float2) * ntypes * ntypes,
                               cudaMemcpyDeviceToDevice, s));
    c->n = n;
    c->ntypes = ntypes;
    c->have_atoms = true;
    c->have_grid = c->have_list = c->have_pruned = false;
    return NB_OK;
}

nb_status nb_grid_put(nb_ctx* c, const float* xyz, const double* box, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_atoms) return fail(c, NB_ERR_STATE, "nb_set_atoms first");
    if (c->n > 0 && !xyz) return fail(c, NB_ERR_ARG, "xyz is null");
    if (!box_ok(box)) return fail(c, NB_ERR_BOX, "box edges must be positive");
    GridGeom g{};
    for (int k = 0; k < 3; ++k) g.L[k] = (float)box[k];
    grid_dims(c->n, g.L, c->C, &g.nx, &g.ny);
    if (g.nx * g.ny > c->ncol_cap) return fail(c, NB_ERR_CAPACITY, "grid has more columns than the workspace");
    if ((long long)c->n + (long long)g.nx * g.ny * (c->C - 1) > c->nslot_cap)
        return fail(c, NB_ERR_CAPACITY, "grid may need more slots than the workspace");
    g.inv_x = (float)((double)g.nx / (double)g.L[0]);
    g.inv_y = (float)((double)g.ny / (double)g.L[1]);
    g.dummy_g = dummy_spacing(g.L);
    NB_CUDA(c, cudaSetDevice(c->device));
    const int sp = span_begin(c, NB_KERNEL_GRID, (cudaStream_t)stream);
    cudaError_t e = launch_grid(c->ws, g, c->n, c->C, c->ntypes, xyz, c->n_sm, (cudaStream_t)stream);
    span_end(c, sp, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "grid kernels");
    c->n_launches += kLaunchesGrid;
    c->geom = g;
    c->have_grid = true;
    c->have_list = c->have_pruned = false;
    c->last_valid = false;
    return NB_OK;
}

nb_status nb_pairlist_build(nb_ctx* c, float rlist, float rbb, const int* excl_off,
                            const int* excl_idx, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_grid) return fail(c, NB_ERR_STATE, "nb_grid_put first");
    if (!(rlist > 0.f) || !(rbb >= 0.f) || ((excl_off == nullptr) != (excl_idx == nullptr)))
        return fail(c, NB_ERR_ARG, "pairlist_build: bad argument");
    for (int k = 0; k < 3; ++k)
        if (!(rlist < 0.5f * c->geom.L[k])) return fail(c, NB_ERR_BOX, "rlist must be below half the box");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    NB_CUDA(c, cudaMemsetAsync(c->ws.st, 0, 2 * sizeof(unsigned long long), s));
    NB_CUDA(c, cudaMemsetAsync(&c->ws.st->n_keys, 0, sizeof(unsigned long long), s));
    const int sp = span_begin(c, NB_KERNEL_SEARCH, s);
    cudaError_t e = launch_search(c->ws, c->geom, c->C, c->nclu_cap, rlist, rbb, excl_off, excl_idx,
                                  c->ient_cap, c->jent_cap, c->n, c->n_sm, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "search kernel");
    c->n_launches += kLaunchesSearch;
    c->rlist = rlist;
    c->have_list = true;
    c->have_pruned = false;
    c->last_valid = false;
    return NB_OK;
}

nb_status nb_set_coords(nb_ctx* c, const float* xyz, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_grid) return fail(c, NB_ERR_STATE, "nb_grid_put first");
    if (!xyz && c->n > 0) return fail(c, NB_ERR_ARG, "xyz is null");
    NB_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_set_coords(c->ws, (int)c->nslot_cap, c->C, xyz, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_coords kernel");
    c->n_launches += kLaunchesSetCoords;
    return NB_OK;
}

nb_status nb_prune(nb_ctx* c, const float* xyz, float r_prune, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (!(r_prune > 0.f)) return fail(c, NB_ERR_ARG, "r_prune must be positive");
    for (int k = 0; k < 3; ++k)
        if (!(r_prune < 0.5f * c->geom.L[k])) return fail(c, NB_ERR_BOX, "r_prune must be below half the box");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    const int sp = span_begin(c, NB_KERNEL_PRUNE, (cudaStream_t)stream);
    cudaError_t e = launch_prune(c->ws, c->geom, c->C, r_prune, c->ient_cap, c->n_sm, (cudaStream_t)stream);
    span_end(c, sp, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "prune kernel");
    c->n_launches += kLaunchesPrune;
    c->r_prune = r_prune;
    c->have_pruned = true;
    c->last_valid = false;
    return NB_OK;
}

nb_status nb_compute(nb_ctx* c, const nb_params* p, const float* xyz, float* f, double* e_out,
                     double* vir_out, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!p || (!f && c->n > 0)) return fail(c, NB_ERR_ARG, "compute: null argument");
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (p->elec != NB_ELEC_RF && p->elec != NB_ELEC_EWALD) return fail(c, NB_ERR_ARG, "unknown electrostatics");
    if (!(p->rc > 0.f)) return fail(c, NB_ERR_ARG, "rc must be positive");
    for (int k = 0; k < 3; ++k)
        if (!(p->rc < 0.5f * c->geom.L[k])) return fail(c, NB_ERR_BOX, "rc must be below half the box");
    const float rlive = c->have_pruned ? c->r_prune : c->rlist;
    if (p->rc > rlive) return fail(c, NB_ERR_BOX, "rc above the list radius");
    if (p->elec == NB_ELEC_EWALD && !(p->beta >= 0.f)) return fail(c, NB_ERR_ARG, "beta must be >= 0");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    ForceParams fp{};
    fp.elec = p->elec;
    fp.want_energy = p->want_energy ? 1 : 0;
    fp.rc2 = p->rc * p->rc;
    fp.fcoul = 138.935458f;
    const double rc = p->rc;
    double k = 0.0;
    if (!(p->eps_rf > 0.f) || std::isinf(p->eps_rf)) k = 1.0 / (2.0 * rc * rc * rc);
    else k = ((double)p->eps_rf - 1.0) / ((2.0 * p->eps_rf + 1.0) * rc * rc * rc);
    fp.k_rf = (float)k;
    fp.two_k_rf = (float)(2.0 * k);
    fp.c_rf = (float)(1.0 / rc + k * rc * rc);
    fp.beta = p->beta;
    fp.two_beta_sqrtpi = (float)(2.0 * (double)p->beta / std::sqrt(M_PI));
    fp.beta2 = (float)((double)p->beta * p->beta);
    fp.beta3 = (float)((double)p->beta * p->beta * p->beta);
    fp.use_fit = ((double)p->beta * p->beta * rc * rc <= (double)kEwaldFitWMax) ? 1 : 0;
    fp.ntypes = c->ntypes;
    for (int d = 0; d < 3; ++d) fp.L[d] = c->geom.L[d];
    fp.use_pruned = c->have_pruned ? 1 : 0;
    fp.ient_cap = c->ient_cap;
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    const int sp = span_begin(c, NB_KERNEL_FORCE, s);
    cudaError_t e = launch_force(c->ws, fp, c->C, c->n_sm, c->nslot_cap, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "force kernel");
    e = launch_finalize(c->ws, fp, c->n, f, e_out, vir_out, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernels");
    c->n_launches += 2 + (fp.want_energy ? 1 : 0);
    return NB_OK;
}

nb_status nb_check(nb_ctx* c, nb_stream stream, nb_info* info) {
    if (!c) return NB_ERR_ARG;
    if (!c->ws_base) return fail(c, NB_ERR_STATE, "no workspace");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    NB_CUDA(c, cudaMemcpyAsync(c->st_host, c->ws.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    c->last = *c->st_host;
    c->last_valid = true;
    const unsigned flags = c->last.flags;
    if (flags) {
        NB_CUDA(c, cudaMemsetAsync(&c->ws.st->flags, 0, sizeof(unsigned), s));
        NB_CUDA(c, cudaStreamSynchronize(s));
    }
    if (info) {
        info->n_atoms = c->n;
        info->nx = c->geom.nx;
        info->ny = c->geom.ny;
        info->n_clusters = c->have_grid ? c->last.nclu : 0;
        info->n_ientries = c->have_list ? (int64_t)c->last.n_ient : 0;
        info->n_jentries = c->have_list ? (int64_t)c->last.n_jent : 0;
        info->n_jentries_pruned = c->have_pruned ? (int64_t)c->last.n_jent_pruned : -1;
        info->ient_capacity = c->ient_cap;
        info->jent_capacity = c->jent_cap;
        info->n_pairs_rc = (int64_t)c->last.n_pairs_rc;
        info->n_superclusters = c->have_grid ? c->last.nsc : 0;
        info->n_cluster_pairs = c->have_list ? (int64_t)c->last.n_keys : 0;
        info->n_cluster_pairs_pruned = c->have_pruned ? (int64_t)c->last.n_keys_pruned : -1;
        info->super_size = super_size(c->C);
        info->n_launches = c->n_launches;
        info->flags = flags;
    }
    if (flags & (1u << NB_ERR_COORD)) return fail(c, NB_ERR_COORD, "a coordinate was outside [-L, 2L)");
    if (flags & (1u << NB_ERR_CAPACITY))
        return fail(c, NB_ERR_CAPACITY, "device capacity exceeded (list %llu/%lld j-entries, longest column %d)",
                    (unsigned long long)c->last.n_jent, c->jent_cap, c->last.max_col);
    if (flags & (1u << NB_ERR_TIMEOUT)) return fail(c, NB_ERR_TIMEOUT, "a bounded device wait expired");
    if (flags) return fail(c, NB_ERR_CUDA, "device flags 0x%x", flags);
    return NB_OK;
}

nb_status nb_profile(nb_ctx* c, int enable) {
    if (!c) return NB_ERR_ARG;
    if (enable && !c->ev[0]) {
        NB_CUDA(c, cudaSetDevice(c->device));
        for (int k = 0; k < 2 * nb_ctx::kMaxSpans; ++k) NB_CUDA(c, cudaEventCreate(&c->ev[k]));
    }
    c->prof = enable != 0;
    return NB_OK;
}

nb_status nb_profile_read(nb_ctx* c, int* kinds, float* ms, int max, int* count) {
    if (!c || !count || max < 0 || (max > 0 && (!kinds || !ms))) return fail(c, NB_ERR_ARG, "profile_read: bad argument");
    const int n = c->ev_n < max ? c->ev_n : max;
    for (int k = 0; k < n; ++k) {
        NB_CUDA(c, cudaEventSynchronize(c->ev[2 * k + 1]));
        NB_CUDA(c, cudaEventElapsedTime(&ms[k], c->ev[2 * k], c->ev[2 * k + 1]));
        kinds[k] = c->ev_kind[k];
    }
    *count = n;
    c->ev_n = 0;
    return NB_OK;
}

nb_status nb_get_grid(nb_ctx* c, int* atom_of_slot, int* slot_of_atom, int* col_clu_start, float* xyzq,
                      int* type_slot, float* bb, int* col_of_atom, int* sc_info, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_grid || !c->last_valid) return fail(c, NB_ERR_STATE, "need a grid and nb_check");
    cudaStream_t s = (cudaStream_t)stream;
    const long long nclu = c->last.nclu;
    const long long ns = nclu * c->C;
    const int ncol = c->geom.nx * c->geom.ny;
    auto cp = [&](void* dst, const void* src, size_t bytes) -> cudaError_t {
        if (!dst || bytes == 0) return cudaSuccess;
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s);
    };
    NB_CUDA(c, cp(atom_of_slot, c->ws.atom_of_slot, sizeof(int) * ns));
    NB_CUDA(c, cp(slot_of_atom, c->ws.slot_of_atom, sizeof(int) * c->n));
    NB_CUDA(c, cp(col_clu_start, c->ws.col_clu_start, sizeof(int) * (ncol + 1)));
    NB_CUDA(c, cp(xyzq, c->ws.xyzq, sizeof(float4) * ns));
    NB_CUDA(c, cp(type_slot, c->ws.type_slot, sizeof(int) * ns));
    NB_CUDA(c, cp(col_of_atom, c->ws.col_of_atom, sizeof(int) * c->n));
    NB_CUDA(c, cp(sc_info, c->ws.sc_info, sizeof(int2) * (size_t)c->last.nsc));
    if (bb && nclu > 0) {
        // float4 pairs -> float [nclu][6]
        NB_CUDA(c, cudaMemcpy2DAsync(bb, 6 * sizeof(float), c->ws.bb, 8 * sizeof(float), 3 * sizeof(float),
                                     nclu, cudaMemcpyDeviceToDevice, s));
        NB_CUDA(c, cudaMemcpy2DAsync(bb + 3, 6 * sizeof(float), (const char*)c->ws.bb + 4 * sizeof(float),
                                     8 * sizeof(float), 3 * sizeof(float), nclu, cudaMemcpyDeviceToDevice, s));
    }
    return NB_OK;
}

nb_status nb_get_list(nb_ctx* c, int which, int* ient, int* cj, uint64_t* mask, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (which != 0 && which != 1) return fail(c, NB_ERR_ARG, "which must be 0 or 1");
    if (!c->have_list || !c->last_valid || (which == 1 && !c->have_pruned))
        return fail(c, NB_ERR_STATE, "need a list and nb_check");
    cudaStream_t s = (cudaStream_t)stream;
    const long long ni = (long long)c->last.n_ient, nj = (long long)c->last.n_jent;
    if (ni > c->ient_cap || nj > c->jent_cap) return fail(c, NB_ERR_CAPACITY, "list overflowed");
    const int4* si = which ? c->ws.ient_p : c->ws.ient;
    const int* sc = which ? c->ws.cj_p : c->ws.cj;
    const unsigned long long* sm = which ? c->ws.mask_p : c->ws.mask;
    if (ient && ni) NB_CUDA(c, cudaMemcpyAsync(ient, si, sizeof(int4) * ni, cudaMemcpyDeviceToDevice, s));
    if (cj && nj) NB_CUDA(c, cudaMemcpyAsync(cj, sc, sizeof(int) * nj, cudaMemcpyDeviceToDevice, s));
    if (mask && nj)
        for (int k = 0; k < super_size(c->C); ++k)
            NB_CUDA(c, cudaMemcpyAsync(mask + (size_t)k * nj, sm + (size_t)k * c->ws.jstride, sizeof(uint64_t) * nj,
                                       cudaMemcpyDeviceToDevice, s));
    return NB_OK;
}

}  // extern "C"
