// C ABI of nbcluster (declared in include/nbcluster.h): context, workspace
// planning and carving for one or many boxes, argument checks, and the
// stream-ordered launch sequence of the hot path.  No device allocation
// happens here; all device data lives in the caller's workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "nb_ewald_fit.h"
#include "nb_internal.cuh"
#include "nb_mlp.cuh"

using namespace nbc;

namespace {

struct BoxPlan {
    int n, ncol_cap;
    long long nclu_cap, nsc_cap, ient_cap, jent_cap;
};

constexpr int kGeoRing = 8;  // pinned staging buffers for box geometry uploads

}  // namespace

struct nb_ctx {
    int C = 8;
    int device = 0;
    int n_sm = 0;
    // plan (fixed by nb_workspace_query*)
    int nbox = 0;
    std::vector<BoxPlan> plan;
    std::vector<int> atom_off, col_off, clu_off, sc_off;
    std::vector<long long> ient_off, jent_off;
    int ntypes_cap = 0;
    // workspace
    char* ws_base = nullptr;
    size_t ws_bytes = 0;
    Workspace ws{};
    // geometry mirror and upload ring
    std::vector<BoxGeom> geo_host;
    bool geo_uploaded = false;
    BoxGeom* geo_pinned[kGeoRing] = {};
    cudaEvent_t geo_ev[kGeoRing] = {};
    bool geo_ev_used[kGeoRing] = {};
    int geo_slot = 0;
    // read-back
    DevState* st_host = nullptr;  // pinned [nbox]
    std::vector<DevState> last;
    bool last_valid = false;
    // state
    int n = 0, ntypes = 0;
    bool have_atoms = false, have_grid = false, have_list = false, have_pruned = false;
    bool list_fresh = false;   // no new coordinates since the last list build
    bool fslot_zero = false;   // the slot force accumulators hold zeros (cleared by the grid and
                               // the coordinate update)
    bool have_mlp = false;
    float mlp_rmin = 0.f, mlp_rmax = 0.f;
    float rlist = 0.f, r_prune = 0.f;
    long long n_launches = 0;
    // timing spans (nb_profile)
    static constexpr int kMaxSpans = 256;
    bool prof = false;
    bool prof_keep = false;   // spans survive reads (graph replays re-record them)
    cudaEvent_t ev[2 * kMaxSpans] = {};
    int ev_kind[kMaxSpans] = {};
    // nb_run_frames: x_ready[2], x_free[2], f_done[2], f_free[2], fork
    cudaEvent_t run_ev[9] = {};
    // nb_run_frames: the graph of the last run's work, replayed when the
    // next run has the same arguments; gen counts the changes (workspace,
    // atoms, network, geometry, profiling) a captured run depends on
    unsigned long long gen = 0;
    std::vector<unsigned char> run_key;
    int run_seen = 0;
    cudaGraphExec_t run_exec = nullptr;
    long long run_launches = 0;
    cudaStream_t run_cap = nullptr;   // captures are made on this stream (the caller's may be the legacy one)
    int ev_n = 0;
    char err[512] = {0};
};

// Timing spans: a pair of events around a kernel.  Inside a stream capture
// the events become event-record nodes of the graph (recorded at every
// replay), so a replayed graph can be timed span by span.
static cudaError_t span_record(cudaEvent_t ev, cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal);
    return cudaEventRecord(ev, s);
}

static int span_begin(nb_ctx* c, int kind, cudaStream_t s) {
    if (!c->prof || c->ev_n >= nb_ctx::kMaxSpans) return -1;
    const int k = c->ev_n;
    if (span_record(c->ev[2 * k], s) != cudaSuccess) return -1;
    c->ev_n = k + 1;
    c->ev_kind[k] = kind;
    return k;
}

static void span_end(nb_ctx* c, int k, cudaStream_t s) {
    if (k >= 0) span_record(c->ev[2 * k + 1], s);
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

#define NB_CUDA(ctx, call)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

static bool box_ok(const double* box) {
    if (!box) return false;
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 0.0) || !(box[k] < 1e30)) return false;
    return true;
}

// Capacities of one box holding n particles in box L with lists up to rlist.
// The number of j-entries is estimated from the density: j-clusters whose
// bounding box is within rlist of a super-cluster's box (half of them,
// Newton's third law) -- the cluster density times the volume of the rounded
// box of side (super-cluster extent + cluster extent) dilated by rlist --
// scaled by factor.
static BoxPlan plan_box(int n, const float L[3], int C, double rlist, double factor) {
    BoxPlan z{};
    int nx, ny;
    grid_dims(n, L, C, &nx, &ny);
    const int S = super_size(C);
    z.n = n;
    z.ncol_cap = nx * ny;
    const long long nslot = (long long)n + (long long)z.ncol_cap * (C - 1);
    z.nclu_cap = nslot / C + 1;
    z.nsc_cap = z.nclu_cap / S + z.ncol_cap + 1;
    const double V = (double)L[0] * L[1] * L[2];
    const double wx = (double)L[0] / nx, wy = (double)L[1] / ny;
    const double rho = n > 0 ? n / V : 1.0;
    const double hz = C / (rho * wx * wy);
    const double a = 2 * wx, b = 2 * wy, c = (S + 1) * hz, r = rlist;
    const double vm = a * b * c + 2 * r * (a * b + b * c + c * a) + M_PI * r * r * (a + b + c) +
                      4.0 / 3.0 * M_PI * r * r * r;
    const double rho_c = (double)z.nclu_cap / V;
    double per = 0.5 * rho_c * vm + S;
    const double maxper = 0.5 * 27.0 * (double)z.nclu_cap + 1.0;
    if (per > maxper) per = maxper;
    // saturated far above the 2^31-entry limit the query enforces
    const double jent = std::ceil(factor * per * (double)z.nsc_cap) + 64.0;
    z.jent_cap = jent < 1e15 ? (long long)jent : (long long)1e15;
    z.ient_cap = z.nsc_cap * 27 + z.jent_cap / kJChunkCoop + 64;
    return z;
}

// Lay the workspace out from base (nullptr: only count bytes).
static size_t carve(const nb_ctx* c, char* base, Workspace* ws) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        off = (off + 255) & ~(size_t)255;
        char* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    const int nb = c->nbox, C = c->C, S = super_size(C);
    Workspace w{};
    w.nbox = nb;
    w.atom_total = c->atom_off[nb];
    w.col_total = c->col_off[nb];
    w.clu_total = c->clu_off[nb];
    w.sc_total = c->sc_off[nb];
    w.ient_total = c->ient_off[nb];
    w.jstride = c->jent_off[nb];
    const size_t na = w.atom_total > 0 ? w.atom_total : 1;
    w.st = (DevState*)take(sizeof(DevState) * nb);
    w.acc = (Accum*)take(sizeof(Accum) * nb);
    w.geo = (BoxGeom*)take(sizeof(BoxGeom) * nb);
    w.lay.atom_off = (int*)take(sizeof(int) * (nb + 1));
    w.lay.col_off = (int*)take(sizeof(int) * (nb + 1));
    w.lay.clu_off = (int*)take(sizeof(int) * (nb + 1));
    w.lay.sc_off = (int*)take(sizeof(int) * (nb + 1));
    w.lay.ient_off = (long long*)take(sizeof(long long) * (nb + 1));
    w.lay.jent_off = (long long*)take(sizeof(long long) * (nb + 1));
    w.xw = (float4*)take(sizeof(float4) * na);
    w.woff = (float4*)take(sizeof(float4) * na);
    w.col_of_atom = (int*)take(sizeof(int) * na);
    w.rank_in_col = (int*)take(sizeof(int) * na);
    w.slot_of_atom = (int*)take(sizeof(int) * na);
    w.q = (float*)take(sizeof(float) * na);
    w.type = (int*)take(sizeof(int) * na);
    w.col_count = (int*)take(sizeof(int) * w.col_total);
    w.col_atom_start = (int*)take(sizeof(int) * w.col_total);
    w.col_clu_start = (int*)take(sizeof(int) * w.col_total);
    w.col_sc_start = (int*)take(sizeof(int) * w.col_total);
    w.sc_info = (int2*)take(sizeof(int2) * w.sc_total);
    w.keys = (unsigned long long*)take(sizeof(unsigned long long) * na);
    const size_t ns = (size_t)w.clu_total * C;
    w.xyzq = (float4*)take(sizeof(float4) * ns);
    w.xjd = (float4*)take(sizeof(float4) * kJRecord * ((ns + 7) / 8));   // a record per group of 8 slots
    w.woff_slot = (float4*)take(sizeof(float4) * ns);
    w.atom_of_slot = (int*)take(sizeof(int) * ns);
    w.type_slot = (int*)take(sizeof(int) * ns);
    w.fslot = (float4*)take(sizeof(float4) * ns);
    w.bb = (float4*)take(sizeof(float4) * 2 * (size_t)w.clu_total);
    w.ient = (int4*)take(sizeof(int4) * w.ient_total);
    w.cj = (int*)take(sizeof(int) * w.jstride);
    w.mask = (unsigned long long*)take(sizeof(unsigned long long) * w.jstride * S);
    w.ient_p = (int4*)take(sizeof(int4) * w.ient_total);
    w.cj_p = (int*)take(sizeof(int) * w.jstride);
    w.mask_p = (unsigned long long*)take(sizeof(unsigned long long) * w.jstride * S);
    w.ient_used = (int*)take(sizeof(int) * (nb + 1));
    w.work = (int*)take(sizeof(int) * 2);
    w.c6c12 = (float2*)take(sizeof(float2) * kMaxTypes * kMaxTypes);
    w.mlp = (MlpTC*)take(sizeof(MlpTC));
    w.ewald_tab = (float2*)take(sizeof(float2) * kEwaldTabN);
    if (ws) *ws = w;
    return (off + 255) & ~(size_t)255;
}

static void set_plan(nb_ctx* c, const std::vector<BoxPlan>& plans) {
    const int nb = (int)plans.size();
    c->nbox = nb;
    c->plan = plans;
    c->atom_off.assign(nb + 1, 0);
    c->col_off.assign(nb + 1, 0);
    c->clu_off.assign(nb + 1, 0);
    c->sc_off.assign(nb + 1, 0);
    c->ient_off.assign(nb + 1, 0);
    c->jent_off.assign(nb + 1, 0);
    for (int b = 0; b < nb; ++b) {
        c->atom_off[b + 1] = c->atom_off[b] + plans[b].n;
        c->col_off[b + 1] = c->col_off[b] + plans[b].ncol_cap + 1;
        c->clu_off[b + 1] = c->clu_off[b] + (int)plans[b].nclu_cap;
        c->sc_off[b + 1] = c->sc_off[b] + (int)plans[b].nsc_cap;
        c->ient_off[b + 1] = c->ient_off[b] + plans[b].ient_cap;
        c->jent_off[b + 1] = c->jent_off[b] + plans[b].jent_cap;
    }
    c->ntypes_cap = kMaxTypes;
    c->ws_base = nullptr;
    c->have_atoms = c->have_grid = c->have_list = c->have_pruned = false;
    c->geo_uploaded = false;
    c->last_valid = false;
}

// Upload the boxes' geometry if it changed (pinned ring, each slot reused
// only after its previous copy has completed).
static nb_status upload_geometry(nb_ctx* c, const std::vector<BoxGeom>& geo, cudaStream_t s) {
    if (c->geo_uploaded && memcmp(geo.data(), c->geo_host.data(), sizeof(BoxGeom) * c->nbox) == 0)
        return NB_OK;
    // a captured copy would read the staging buffer at every replay, after
    // later calls may have reused it: new geometry needs an uncaptured call
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NB_CUDA(c, cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone)
        return fail(c, NB_ERR_STATE, "box edges changed during stream capture: call nb_grid_put with them once before capturing");
    const int k = c->geo_slot;
    c->geo_slot = (k + 1) % kGeoRing;
    if (c->geo_ev_used[k]) NB_CUDA(c, cudaEventSynchronize(c->geo_ev[k]));
    memcpy(c->geo_pinned[k], geo.data(), sizeof(BoxGeom) * c->nbox);
    NB_CUDA(c, cudaMemcpyAsync(c->ws.geo, c->geo_pinned[k], sizeof(BoxGeom) * c->nbox,
                               cudaMemcpyHostToDevice, s));
    NB_CUDA(c, cudaEventRecord(c->geo_ev[k], s));
    c->geo_ev_used[k] = true;
    c->geo_host = geo;
    c->geo_uploaded = true;
    ++c->gen;
    return NB_OK;
}

static void release_host(nb_ctx* c) {
    for (int k = 0; k < kGeoRing; ++k) {
        if (c->geo_pinned[k]) cudaFreeHost(c->geo_pinned[k]);
        if (c->geo_ev[k]) cudaEventDestroy(c->geo_ev[k]);
        c->geo_pinned[k] = nullptr;
        c->geo_ev[k] = nullptr;
        c->geo_ev_used[k] = false;
    }
    if (c->st_host) cudaFreeHost(c->st_host);
    c->st_host = nullptr;
}

// Reset every box's list counters.
static __global__ void k_list_reset(Workspace ws) {
    for (int b = threadIdx.x; b < ws.nbox; b += blockDim.x) {
        ws.st[b].n_ient = 0;
        ws.st[b].n_jent = 0;
        ws.st[b].n_keys = 0;
    }
}

static float min_edge(const nb_ctx* c) {
    float m = INFINITY;
    for (int b = 0; b < c->nbox; ++b)
        for (int k = 0; k < 3; ++k) m = fminf(m, c->geo_host[b].L[k]);
    return m;
}

static void fill_info(const nb_ctx* c, int b0, int b1, nb_info* info, unsigned flags) {
    memset(info, 0, sizeof(*info));
    info->n_jentries_pruned = c->have_pruned ? 0 : -1;
    info->n_cluster_pairs_pruned = c->have_pruned ? 0 : -1;
    for (int b = b0; b < b1; ++b) {
        const DevState& d = c->last[b];
        info->n_atoms += c->plan[b].n;
        if (c->have_grid) {
            info->n_clusters += d.nclu;
            info->n_superclusters += d.nsc;
        }
        if (c->have_list) {
            info->n_ientries += (int64_t)d.n_ient;
            info->n_jentries += (int64_t)d.n_jent;
            info->n_cluster_pairs += (int64_t)d.n_keys;
        }
        if (c->have_pruned) {
            info->n_jentries_pruned += (int64_t)d.n_jent_pruned;
            info->n_cluster_pairs_pruned += (int64_t)d.n_keys_pruned;
        }
        info->n_pairs_rc += (int64_t)d.n_pairs_rc;
        info->ient_capacity += c->plan[b].ient_cap;
        info->jent_capacity += c->plan[b].jent_cap;
    }
    if (b1 - b0 == 1 && c->geo_uploaded) {
        info->nx = c->geo_host[b0].nx;
        info->ny = c->geo_host[b0].ny;
    }
    info->super_size = super_size(c->C);
    info->n_launches = c->n_launches;
    info->n_boxes = b1 - b0;
    info->atom_offset = c->atom_off[b0];
    info->flags = flags;
}

// Kernel constants of an interaction setup (Sec. 3.2).
static nb_status force_params(nb_ctx* c, const nb_params* p, ForceParams* fp) {
    *fp = ForceParams{};
    // the surrogate and tabulated kernels compute forces only; energy
    // evaluations are analytic
    const bool forces_only = p->elec == NB_ELEC_EWALD_MLP || p->elec == NB_ELEC_EWALD_TAB;
    fp->elec = (forces_only && p->want_energy) ? NB_ELEC_EWALD : p->elec;
    fp->tab_n = kEwaldTabN;
    fp->tab_scale = (float)((double)p->beta * p->beta * kEwaldTabN / (double)kEwaldFitWMax);
    fp->mlp_rmin = c->mlp_rmin;
    fp->want_energy = p->want_energy ? 1 : 0;
    fp->rc2 = p->rc * p->rc;
    fp->fcoul = 138.935458f;
    const double rc = p->rc;
    double k = 0.0;
    if (!(p->eps_rf > 0.f) || std::isinf(p->eps_rf)) k = 1.0 / (2.0 * rc * rc * rc);
    else k = ((double)p->eps_rf - 1.0) / ((2.0 * p->eps_rf + 1.0) * rc * rc * rc);
    fp->k_rf = (float)k;
    fp->two_k_rf = (float)(2.0 * k);
    fp->c_rf = (float)(1.0 / rc + k * rc * rc);
    fp->beta = p->beta;
    fp->two_beta_sqrtpi = (float)(2.0 * (double)p->beta / std::sqrt(M_PI));
    fp->beta2 = (float)((double)p->beta * p->beta);
    fp->beta3 = (float)((double)p->beta * p->beta * p->beta);
    fp->use_fit = ((double)p->beta * p->beta * rc * rc <= (double)kEwaldFitWMax) ? 1 : 0;
    fp->fit_k = (float)(-(double)p->beta * p->beta * p->beta * kEwaldGLead);
    if ((fp->elec == NB_ELEC_EWALD_MLP || fp->elec == NB_ELEC_EWALD_TAB) && !fp->use_fit)
        return fail(c, NB_ERR_ARG, "the surrogate and tabulated kernels need (beta rc)^2 <= %g",
                    (double)kEwaldFitWMax);
    if (fp->elec == NB_ELEC_EWALD_TAB && c->C != 8)
        return fail(c, NB_ERR_ARG, "the tabulated kernel needs 8-particle clusters");
    fp->ntypes = c->ntypes;
    fp->use_pruned = c->have_pruned ? 1 : 0;
    return NB_OK;
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
    if (e != cudaSuccess) {
        delete c;
        return NB_ERR_CUDA;
    }
    *out = c;
    return NB_OK;
}

nb_status nb_destroy(nb_ctx* c) {
    if (!c) return NB_ERR_ARG;
    release_host(c);
    for (int k = 0; k < 2 * nb_ctx::kMaxSpans; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    for (int k = 0; k < 9; ++k)
        if (c->run_ev[k]) cudaEventDestroy(c->run_ev[k]);
    if (c->run_exec) cudaGraphExecDestroy(c->run_exec);
    if (c->run_cap) cudaStreamDestroy(c->run_cap);
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

nb_status nb_workspace_query_boxes(nb_ctx* c, int nbox, const int* n_atoms, const double* boxes,
                                   double rlist_max, int ntypes, double list_factor, size_t* bytes) {
    if (!c || !bytes || nbox <= 0 || !n_atoms || !boxes || ntypes <= 0)
        return fail(c, NB_ERR_ARG, "workspace_query: bad argument");
    if (nbox > kMaxBoxes) return fail(c, NB_ERR_ARG, "at most %d boxes", kMaxBoxes);
    if (ntypes > kMaxTypes) return fail(c, NB_ERR_ARG, "at most %d LJ types", kMaxTypes);
    if (!(rlist_max > 0.0)) return fail(c, NB_ERR_ARG, "rlist_max must be positive");
    if (list_factor == 0.0) list_factor = 1.5;
    if (list_factor < 1.0) return fail(c, NB_ERR_ARG, "list_factor must be >= 1");
    std::vector<BoxPlan> plans(nbox);
    long long total = 0;
    for (int b = 0; b < nbox; ++b) {
        if (n_atoms[b] < 0) return fail(c, NB_ERR_ARG, "negative particle count");
        if (!box_ok(boxes + 3 * b)) return fail(c, NB_ERR_BOX, "box %d: edges must be positive and below 1e30 nm", b);
        const float L[3] = {(float)boxes[3 * b], (float)boxes[3 * b + 1], (float)boxes[3 * b + 2]};
        plans[b] = plan_box(n_atoms[b], L, c->C, rlist_max, list_factor);
        total += n_atoms[b];
    }
    if (total > 0x7fffffffLL) return fail(c, NB_ERR_ARG, "too many particles");
    long long ient_sum = 0, jent_sum = 0, slot_sum = 0;
    for (const BoxPlan& z : plans) {
        ient_sum += z.ient_cap;
        jent_sum += z.jent_cap;
        slot_sum += z.nclu_cap * c->C;
    }
    // list and slot indices are stored as 32-bit integers
    if (ient_sum > 0x7fffffffLL || jent_sum > 0x7fffffffLL || slot_sum > 0x7fffffffLL)
        return fail(c, NB_ERR_CAPACITY, "list or slot capacity above 2^31 entries");
    // a j-entry word keeps the j-cluster index in its low kSuperShift bits
    if (slot_sum / c->C > (long long)kCjMask)
        return fail(c, NB_ERR_CAPACITY, "more than 2^%d clusters", kSuperShift);
    set_plan(c, plans);
    *bytes = carve(c, nullptr, nullptr);
    return NB_OK;
}

nb_status nb_workspace_query(nb_ctx* c, int n, const double* box, double rlist_max, int ntypes,
                             double list_factor, size_t* bytes) {
    if (!c) return NB_ERR_ARG;
    if (!box_ok(box)) return fail(c, NB_ERR_BOX, "box edges must be positive and below 1e30 nm");
    return nb_workspace_query_boxes(c, 1, &n, box, rlist_max, ntypes, list_factor, bytes);
}

nb_status nb_workspace_bytes(int cluster_size, int nbox, const int* n_atoms, const double* boxes,
                             double rlist_max, int ntypes, double list_factor, size_t* bytes) {
    if (cluster_size != 4 && cluster_size != 8) return NB_ERR_ARG;
    nb_ctx plan;   // planning is host arithmetic: no device state is touched
    plan.C = cluster_size;
    return nb_workspace_query_boxes(&plan, nbox, n_atoms, boxes, rlist_max, ntypes, list_factor, bytes);
}

nb_status nb_set_workspace(nb_ctx* c, void* ws, size_t bytes) {
    if (!c || !ws) return fail(c, NB_ERR_ARG, "set_workspace: null");
    if (((uintptr_t)ws & 255) != 0) return fail(c, NB_ERR_ARG, "workspace must be 256-byte aligned");
    if (c->nbox == 0) return fail(c, NB_ERR_STATE, "call nb_workspace_query first");
    const size_t need = carve(c, nullptr, nullptr);
    if (bytes < need) return fail(c, NB_ERR_CAPACITY, "workspace has %zu bytes, needs %zu", bytes, need);
    NB_CUDA(c, cudaSetDevice(c->device));
    ++c->gen;
    carve(c, (char*)ws, &c->ws);
    c->ws_base = (char*)ws;
    c->ws_bytes = bytes;
    c->have_atoms = c->have_grid = c->have_list = c->have_pruned = false;
    c->have_mlp = false;
    c->last_valid = false;
    c->geo_uploaded = false;
    release_host(c);
    for (int k = 0; k < kGeoRing; ++k) {
        NB_CUDA(c, cudaMallocHost((void**)&c->geo_pinned[k], sizeof(BoxGeom) * c->nbox));
        NB_CUDA(c, cudaEventCreateWithFlags(&c->geo_ev[k], cudaEventDisableTiming));
    }
    NB_CUDA(c, cudaMallocHost((void**)&c->st_host, sizeof(DevState) * c->nbox));
    c->last.assign(c->nbox, DevState{});
    const int nb = c->nbox;
    NB_CUDA(c, cudaMemset(c->ws.st, 0, sizeof(DevState) * nb));
    NB_CUDA(c, cudaMemset(c->ws.work, 0, sizeof(int) * 2));
    NB_CUDA(c, launch_ewald_table(c->ws.ewald_tab, kEwaldTabN, (double)kEwaldFitWMax, 0));
    NB_CUDA(c, cudaDeviceSynchronize());
    NB_CUDA(c, cudaMemset(c->ws.geo, 0, sizeof(BoxGeom) * nb));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.atom_off, c->atom_off.data(), sizeof(int) * (nb + 1),
                          cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.col_off, c->col_off.data(), sizeof(int) * (nb + 1),
                          cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.clu_off, c->clu_off.data(), sizeof(int) * (nb + 1),
                          cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.sc_off, c->sc_off.data(), sizeof(int) * (nb + 1),
                          cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.ient_off, c->ient_off.data(), sizeof(long long) * (nb + 1),
                          cudaMemcpyHostToDevice));
    NB_CUDA(c, cudaMemcpy((void*)c->ws.lay.jent_off, c->jent_off.data(), sizeof(long long) * (nb + 1),
                          cudaMemcpyHostToDevice));
    return NB_OK;
}

nb_status nb_set_atoms(nb_ctx* c, int n, const float* q, const int* type, int ntypes,
                       const float* c6c12, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->ws_base) return fail(c, NB_ERR_STATE, "no workspace");
    if (n < 0 || (n > 0 && (!q || !type)) || ntypes <= 0 || !c6c12)
        return fail(c, NB_ERR_ARG, "set_atoms: bad argument");
    ++c->gen;
    if (n != c->atom_off[c->nbox])
        return fail(c, NB_ERR_CAPACITY, "%d particles, the workspace is planned for %d", n, c->atom_off[c->nbox]);
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

nb_status nb_grid_put(nb_ctx* c, const float* xyz, const double* boxes, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_atoms) return fail(c, NB_ERR_STATE, "nb_set_atoms first");
    if (c->n > 0 && !xyz) return fail(c, NB_ERR_ARG, "xyz is null");
    if (!boxes) return fail(c, NB_ERR_BOX, "box is null");
    std::vector<BoxGeom> geo(c->nbox);
    for (int b = 0; b < c->nbox; ++b) {
        if (!box_ok(boxes + 3 * b)) return fail(c, NB_ERR_BOX, "box %d: edges must be positive and below 1e30 nm", b);
        BoxGeom& g = geo[b];
        const int nb_atoms = c->plan[b].n;
        g = box_geometry(nb_atoms, boxes + 3 * b, c->C);
        if (g.nx * g.ny > c->plan[b].ncol_cap)
            return fail(c, NB_ERR_CAPACITY, "box %d: grid has more columns than the workspace", b);
        if ((long long)nb_atoms + (long long)g.nx * g.ny * (c->C - 1) > c->plan[b].nclu_cap * c->C)
            return fail(c, NB_ERR_CAPACITY, "box %d: grid may need more slots than the workspace", b);
    }
    NB_CUDA(c, cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    nb_status st = upload_geometry(c, geo, s);
    if (st != NB_OK) return st;
    const int sp = span_begin(c, NB_KERNEL_GRID, s);
    cudaError_t e = launch_grid(c->ws, c->C, c->ntypes, xyz, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "grid kernels");
    c->n_launches += kLaunchesGrid;
    c->have_grid = true;
    c->fslot_zero = true;
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
    if (!(rlist < 0.5f * min_edge(c))) return fail(c, NB_ERR_BOX, "rlist must be below half the box");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    k_list_reset<<<1, 256, 0, s>>>(c->ws);
    const int sp = span_begin(c, NB_KERNEL_SEARCH, s);
    cudaError_t e = launch_search(c->ws, c->C, rlist, rbb, excl_off, excl_idx, c->n_sm, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "search kernel");
    c->n_launches += kLaunchesSearch + 1;
    c->rlist = rlist;
    c->have_list = true;
    c->list_fresh = true;
    c->have_pruned = false;
    c->last_valid = false;
    return NB_OK;
}

// The force kernels add into the slot accumulators: clear them first unless
// the grid or a coordinate update left them cleared.
static nb_status clear_slot_forces(nb_ctx* c, cudaStream_t s) {
    if (!c->fslot_zero)
        NB_CUDA(c, cudaMemsetAsync(c->ws.fslot, 0, sizeof(float4) * (size_t)c->ws.clu_total * c->C, s));
    c->fslot_zero = false;
    return NB_OK;
}

nb_status nb_set_coords(nb_ctx* c, const float* xyz, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_grid) return fail(c, NB_ERR_STATE, "nb_grid_put first");
    if (!xyz && c->n > 0) return fail(c, NB_ERR_ARG, "xyz is null");
    NB_CUDA(c, cudaSetDevice(c->device));
    const int sp = span_begin(c, NB_KERNEL_COORDS, (cudaStream_t)stream);
    cudaError_t e = launch_set_coords(c->ws, c->C, xyz, (cudaStream_t)stream);
    c->fslot_zero = true;
    span_end(c, sp, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_coords kernel");
    c->n_launches += kLaunchesSetCoords;
    c->list_fresh = false;
    return NB_OK;
}

nb_status nb_prune(nb_ctx* c, const float* xyz, float r_prune, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (!(r_prune > 0.f)) return fail(c, NB_ERR_ARG, "r_prune must be positive");
    if (!(r_prune < 0.5f * min_edge(c))) return fail(c, NB_ERR_BOX, "r_prune must be below half the box");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    const int sp = span_begin(c, NB_KERNEL_PRUNE, (cudaStream_t)stream);
    cudaError_t e = launch_prune(c->ws, c->C, r_prune, c->n_sm, (cudaStream_t)stream);
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
    if (p->elec != NB_ELEC_RF && p->elec != NB_ELEC_EWALD && p->elec != NB_ELEC_EWALD_MLP &&
        p->elec != NB_ELEC_EWALD_TAB)
        return fail(c, NB_ERR_ARG, "unknown electrostatics");
    if (p->elec == NB_ELEC_EWALD_MLP) {
        if (!c->have_mlp) return fail(c, NB_ERR_STATE, "no network: call nb_set_surrogate first");
        if (p->rc > c->mlp_rmax) return fail(c, NB_ERR_ARG, "rc above the network's input range");
    }
    if (!(p->rc > 0.f)) return fail(c, NB_ERR_ARG, "rc must be positive");
    if (!(p->rc < 0.5f * min_edge(c))) return fail(c, NB_ERR_BOX, "rc must be below half the box");
    // a prune at a radius above the list's keeps the list's radius
    const float rlive = c->have_pruned && c->r_prune < c->rlist ? c->r_prune : c->rlist;
    if (p->rc > rlive) return fail(c, NB_ERR_BOX, "rc above the list radius");
    if (p->elec != NB_ELEC_RF && !(p->beta >= 0.f)) return fail(c, NB_ERR_ARG, "beta must be >= 0");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    ForceParams fp{};
    const nb_status pst = force_params(c, p, &fp);
    if (pst != NB_OK) return pst;
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    const int sp = span_begin(c, NB_KERNEL_FORCE, s);
    nb_status zs = clear_slot_forces(c, s);
    if (zs != NB_OK) return zs;
    cudaError_t e = launch_force(c->ws, fp, c->C, c->n_sm, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "force kernel");
    const int sz = span_begin(c, NB_KERNEL_FINALIZE, s);
    e = launch_finalize(c->ws, fp, c->C, f, e_out, vir_out, s);
    c->fslot_zero = false;
    span_end(c, sz, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernels");
    c->n_launches += 2 + (fp.want_energy ? 1 : 0);
    return NB_OK;
}

nb_status nb_prune_compute(nb_ctx* c, const nb_params* p, const float* xyz, float r_prune, float* f,
                           double* e_out, double* vir_out, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!p || (!f && c->n > 0)) return fail(c, NB_ERR_ARG, "prune_compute: null argument");
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (p->elec != NB_ELEC_RF && p->elec != NB_ELEC_EWALD && p->elec != NB_ELEC_EWALD_MLP &&
        p->elec != NB_ELEC_EWALD_TAB)
        return fail(c, NB_ERR_ARG, "unknown electrostatics");
    if (p->elec == NB_ELEC_EWALD_MLP) {
        if (!c->have_mlp) return fail(c, NB_ERR_STATE, "no network: call nb_set_surrogate first");
        if (p->rc > c->mlp_rmax) return fail(c, NB_ERR_ARG, "rc above the network's input range");
    }
    if (!(p->rc > 0.f) || !(r_prune > 0.f)) return fail(c, NB_ERR_ARG, "rc and r_prune must be positive");
    if (!(r_prune < 0.5f * min_edge(c))) return fail(c, NB_ERR_BOX, "r_prune must be below half the box");
    if (p->rc > r_prune || p->rc > c->rlist) return fail(c, NB_ERR_BOX, "rc above the prune or list radius");
    if (p->elec != NB_ELEC_RF && !(p->beta >= 0.f)) return fail(c, NB_ERR_ARG, "beta must be >= 0");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    ForceParams fp{};
    const nb_status pst = force_params(c, p, &fp);
    if (pst != NB_OK) return pst;
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    // one pass where the fused kernel exists (8-particle clusters, forces
    // only, analytic or tabulated factor); else the prune kernel, then the
    // force kernel on the pruned list
    const bool fused = c->C == 8 && !fp.want_energy && fp.elec != NB_ELEC_EWALD_MLP;
    cudaError_t e;
    if (fused) {
        e = launch_prune_reset(c->ws, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "prune reset");
        fp.prune = 1;
        fp.rp2 = r_prune * r_prune;
        fp.use_pruned = 0;
        const int sp = span_begin(c, NB_KERNEL_FORCE_PRUNE, s);
        const nb_status zs = clear_slot_forces(c, s);
        if (zs != NB_OK) return zs;
        e = launch_force(c->ws, fp, c->C, c->n_sm, s);
        span_end(c, sp, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "force + prune kernel");
        c->n_launches += 2;
    } else {
        const int sp = span_begin(c, NB_KERNEL_PRUNE, s);
        e = launch_prune(c->ws, c->C, r_prune, c->n_sm, s);
        span_end(c, sp, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "prune kernel");
        c->n_launches += kLaunchesPrune;
        fp.use_pruned = 1;
        const int sf = span_begin(c, NB_KERNEL_FORCE, s);
        const nb_status zs = clear_slot_forces(c, s);
        if (zs != NB_OK) return zs;
        e = launch_force(c->ws, fp, c->C, c->n_sm, s);
        span_end(c, sf, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "force kernel");
        c->n_launches += 1;
    }
    c->r_prune = r_prune;
    c->have_pruned = true;
    c->last_valid = false;
    const int sz = span_begin(c, NB_KERNEL_FINALIZE, s);
    e = launch_finalize(c->ws, fp, c->C, f, e_out, vir_out, s);
    c->fslot_zero = false;
    span_end(c, sz, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernels");
    c->n_launches += 1 + (fp.want_energy ? 1 : 0);
    return NB_OK;
}

// Frames from host memory: the per-frame calls of a list lifetime with the
// transfers on a second stream.  Events (created on first use, owned by the
// context): x_ready[k] (coordinates in buffer k), x_free[k] (buffer k read
// by its frame's kernels), f_done[k] (forces of buffer k written), f_free[k]
// (buffer k's outputs copied out), and a fork event that orders the copy
// stream after all work queued on the compute stream before the run
// (earlier runs, replayed graphs included).  Only the events recorded in
// this run are waited on.
static nb_status run_frames_enqueue(nb_ctx* c, const nb_params* p, const nb_frames* fr, cudaStream_t s,
                                    cudaStream_t cs, bool captured) {
    cudaEvent_t* x_ready = c->run_ev;
    cudaEvent_t* x_free = c->run_ev + 2;
    cudaEvent_t* f_done = c->run_ev + 4;
    cudaEvent_t* f_free = c->run_ev + 6;
    unsigned recorded = 0;   // the events recorded in this run (bit = index in run_ev)
    auto record = [&](cudaEvent_t* ev, int k, cudaStream_t st) -> cudaError_t {
        recorded |= 1u << (int)(ev - c->run_ev + k);
        return cudaEventRecord(ev[k], st);
    };
    auto wait = [&](cudaStream_t st, cudaEvent_t* ev, int k) -> cudaError_t {
        if (!((recorded >> (int)(ev - c->run_ev + k)) & 1u)) return cudaSuccess;
        return cudaStreamWaitEvent(st, ev[k], 0);
    };
    const size_t xb = (size_t)c->n * 3 * sizeof(float);
    const size_t eb = (size_t)c->nbox * 2 * sizeof(double), vb = (size_t)c->nbox * 9 * sizeof(double);
    (void)captured;
    NB_CUDA(c, cudaEventRecord(c->run_ev[8], s));
    NB_CUDA(c, cudaStreamWaitEvent(cs, c->run_ev[8], 0));
    // frame 0's coordinates
    if (xb) NB_CUDA(c, cudaMemcpyAsync(fr->x_dev[0], fr->x_host, xb, cudaMemcpyHostToDevice, cs));
    NB_CUDA(c, record(x_ready, 0, cs));
    for (int f = 0; f < fr->n_frames; ++f) {
        const int k = f & 1;
        if (f + 1 < fr->n_frames) {
            const int kn = k ^ 1;
            NB_CUDA(c, wait(cs, x_free, kn));   // frame f - 1 has read it
            if (xb)
                NB_CUDA(c, cudaMemcpyAsync(fr->x_dev[kn], fr->x_host + (size_t)(f + 1) * c->n * 3, xb,
                                           cudaMemcpyHostToDevice, cs));
            NB_CUDA(c, record(x_ready, kn, cs));
        }
        NB_CUDA(c, wait(s, x_ready, k));
        NB_CUDA(c, wait(s, f_free, k));   // frame f - 2's outputs are copied out
        const bool energy = fr->energy_frames_host && fr->energy_frames_host[f];
        nb_params q = *p;
        q.want_energy = energy ? 1 : 0;
        double* e_dev = energy && fr->e_host ? fr->e_dev[k] : nullptr;
        double* v_dev = energy && fr->vir_host ? fr->vir_dev[k] : nullptr;
        const float* x = fr->x_dev[k];
        nb_status st;
        if (f == 0 && fr->build) {
            st = nb_grid_put(c, x, fr->boxes_host, s);
            if (st != NB_OK) return st;
            st = nb_pairlist_build(c, fr->rlist, fr->rbb, fr->excl_off_dev, fr->excl_idx_dev, s);
            if (st != NB_OK) return st;
            x = nullptr;   // the list's own coordinates
        }
        const int g = fr->first_frame + f;
        if (fr->nstprune > 0 && g > 0 && g % fr->nstprune == 0)
            st = nb_prune_compute(c, &q, x, fr->r_prune, fr->f_dev[k], e_dev, v_dev, s);
        else
            st = nb_compute(c, &q, x, fr->f_dev[k], e_dev, v_dev, s);
        if (st != NB_OK) return st;
        NB_CUDA(c, record(x_free, k, s));
        NB_CUDA(c, record(f_done, k, s));
        NB_CUDA(c, wait(cs, f_done, k));
        if (xb)
            NB_CUDA(c, cudaMemcpyAsync(fr->f_host + (size_t)f * c->n * 3, fr->f_dev[k], xb,
                                       cudaMemcpyDeviceToHost, cs));
        if (e_dev)
            NB_CUDA(c, cudaMemcpyAsync(fr->e_host + (size_t)f * c->nbox * 2, e_dev, eb, cudaMemcpyDeviceToHost,
                                       cs));
        if (v_dev)
            NB_CUDA(c, cudaMemcpyAsync(fr->vir_host + (size_t)f * c->nbox * 9, v_dev, vb,
                                       cudaMemcpyDeviceToHost, cs));
        NB_CUDA(c, record(f_free, k, cs));
    }
    // the compute stream waits for the last copy out
    NB_CUDA(c, wait(s, f_free, (fr->n_frames - 1) & 1));
    return NB_OK;
}

// The arguments a captured run depends on, as bytes: every field of the
// frames description and the parameters, the box edges and energy flags the
// call reads, and the context's generation.
static std::vector<unsigned char> run_key(const nb_ctx* c, const nb_params* p, const nb_frames* fr) {
    std::vector<unsigned char> k;
    auto put = [&](const void* v, size_t n) {
        const unsigned char* b = (const unsigned char*)v;
        k.insert(k.end(), b, b + n);
    };
    put(&c->gen, sizeof(c->gen));
    put(&p->elec, sizeof(p->elec));
    put(&p->rc, sizeof(p->rc));
    put(&p->eps_rf, sizeof(p->eps_rf));
    put(&p->beta, sizeof(p->beta));
    put(&fr->n_frames, sizeof(fr->n_frames));
    const void* ptrs[] = {fr->x_host, fr->f_host, fr->energy_frames_host, fr->e_host, fr->vir_host,
                          fr->x_dev[0], fr->x_dev[1], fr->f_dev[0], fr->f_dev[1], fr->e_dev[0],
                          fr->e_dev[1], fr->vir_dev[0], fr->vir_dev[1], fr->excl_off_dev, fr->excl_idx_dev};
    put(ptrs, sizeof(ptrs));
    put(&fr->build, sizeof(fr->build));
    put(&fr->rlist, sizeof(fr->rlist));
    put(&fr->rbb, sizeof(fr->rbb));
    put(&fr->first_frame, sizeof(fr->first_frame));
    put(&fr->nstprune, sizeof(fr->nstprune));
    put(&fr->r_prune, sizeof(fr->r_prune));
    if (fr->boxes_host) put(fr->boxes_host, sizeof(double) * 3 * c->nbox);
    if (fr->energy_frames_host) put(fr->energy_frames_host, (size_t)fr->n_frames);
    return k;
}

// A run that builds its own list is the same work every time its arguments
// are the same: the first such run is made eagerly, the second is captured
// in a CUDA graph, and later ones replay the graph on the compute stream
// (its copies are graph nodes; copy_stream is not used), which spares the
// host a few microseconds per launch and the device the gaps between them.
nb_status nb_run_frames(nb_ctx* c, const nb_params* p, const nb_frames* fr, nb_stream stream,
                        nb_stream copy_stream) {
    if (!c) return NB_ERR_ARG;
    if (!p || !fr) return fail(c, NB_ERR_ARG, "run_frames: null argument");
    if (fr->n_frames < 1) return fail(c, NB_ERR_ARG, "run_frames: n_frames must be >= 1");
    if (fr->n_atoms != c->n || fr->n_boxes != c->nbox)
        return fail(c, NB_ERR_ARG, "run_frames: %d particles in %d boxes given, the context has %d in %d",
                    fr->n_atoms, fr->n_boxes, c->n, c->nbox);
    if (stream == copy_stream) return fail(c, NB_ERR_ARG, "run_frames: the copy stream must differ");
    if (fr->nstprune < 0 || fr->first_frame < 0) return fail(c, NB_ERR_ARG, "run_frames: negative schedule");
    if (c->n > 0 && (!fr->x_host || !fr->f_host)) return fail(c, NB_ERR_ARG, "run_frames: null host buffer");
    for (int k = 0; k < 2; ++k) {
        if (c->n > 0 && (!fr->x_dev[k] || !fr->f_dev[k]))
            return fail(c, NB_ERR_ARG, "run_frames: null device buffer");
        if ((fr->e_host && !fr->e_dev[k]) || (fr->vir_host && !fr->vir_dev[k]))
            return fail(c, NB_ERR_ARG, "run_frames: null energy or virial staging");
    }
    if (fr->build && !fr->boxes_host) return fail(c, NB_ERR_ARG, "run_frames: build needs the boxes");
    NB_CUDA(c, cudaSetDevice(c->device));
    for (int k = 0; k < 9; ++k)
        if (!c->run_ev[k]) NB_CUDA(c, cudaEventCreateWithFlags(&c->run_ev[k], cudaEventDisableTiming));
    cudaStream_t s = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NB_CUDA(c, cudaStreamIsCapturing(s, &cap));
    const bool graphable = fr->build && !c->prof && cap == cudaStreamCaptureStatusNone;
    std::vector<unsigned char> key = run_key(c, p, fr);
    const bool same = graphable && key == c->run_key;
    if (same && c->run_exec) {
        NB_CUDA(c, cudaGraphLaunch(c->run_exec, s));
        c->n_launches += c->run_launches;
        return NB_OK;
    }
    if (c->run_exec && !same) {
        cudaGraphExecDestroy(c->run_exec);
        c->run_exec = nullptr;
    }
    if (same && c->run_seen >= 1 && !c->run_cap)
        NB_CUDA(c, cudaStreamCreateWithFlags(&c->run_cap, cudaStreamNonBlocking));
    bool capturing = false;
    if (same && c->run_seen >= 1) {
        capturing = cudaStreamBeginCapture(c->run_cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (!capturing) cudaGetLastError();   // no graph this time: made call by call below
    }
    if (capturing) {
        // the second run with these arguments: captured on the context's
        // stream, then launched on the caller's
        const long long n0 = c->n_launches;
        const nb_status st = run_frames_enqueue(c, p, fr, c->run_cap, cs, true);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->run_cap, &g);
        cudaError_t ei = cudaErrorUnknown;
        if (st == NB_OK && e == cudaSuccess) ei = cudaGraphInstantiate(&c->run_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st == NB_OK && e == cudaSuccess && ei == cudaSuccess) {
            c->run_launches = c->n_launches - n0;
            NB_CUDA(c, cudaGraphLaunch(c->run_exec, s));
            return NB_OK;
        }
        // no graph for these arguments: this run and the next ones eagerly
        c->run_exec = nullptr;
        cudaGetLastError();
        c->n_launches = n0;
        if (st != NB_OK) {
            c->run_key.clear();
            c->run_seen = 0;
            return st;
        }
        const nb_status st2 = run_frames_enqueue(c, p, fr, s, cs, false);
        c->run_seen = -1000000;
        return st2;
    }
    const nb_status st = run_frames_enqueue(c, p, fr, s, cs, false);
    if (st != NB_OK || !graphable) {
        c->run_key.clear();
        c->run_seen = 0;
        return st;
    }
    // remembered with the generation after the run (it may have uploaded geometry)
    c->run_key = run_key(c, p, fr);
    c->run_seen = same ? c->run_seen + 1 : 1;
    return NB_OK;
}

nb_status nb_pairlist_1x1(nb_ctx* c, float rlist, int max_nbr, int* nbr, int* count, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (!(rlist > 0.f) || max_nbr <= 0 || (c->n > 0 && (!nbr || !count)))
        return fail(c, NB_ERR_ARG, "pairlist_1x1: bad argument");
    if (!c->list_fresh) return fail(c, NB_ERR_STATE, "pairlist_1x1: coordinates changed since the list was built");
    if (rlist > c->rlist) return fail(c, NB_ERR_BOX, "rlist above the cluster list's radius");
    NB_CUDA(c, cudaSetDevice(c->device));
    cudaError_t e = launch_pairlist_1x1(c->ws, c->C, rlist, max_nbr, nbr, count, c->n_sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "1x1 list kernel");
    c->n_launches += 1;
    return NB_OK;
}

nb_status nb_compute_1x1(nb_ctx* c, const nb_params* p, const float* xyz, const int* nbr, const int* count,
                         int max_nbr, float* f, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!p || (c->n > 0 && (!f || !nbr || !count)) || max_nbr <= 0)
        return fail(c, NB_ERR_ARG, "compute_1x1: null argument");
    if (!c->have_grid) return fail(c, NB_ERR_STATE, "nb_grid_put first");
    if (p->elec != NB_ELEC_RF && p->elec != NB_ELEC_EWALD)
        return fail(c, NB_ERR_ARG, "the 1x1 kernel supports reaction field and Ewald");
    if (p->want_energy) return fail(c, NB_ERR_ARG, "the 1x1 kernel computes forces only");
    if (!(p->rc > 0.f) || !(p->rc < 0.5f * min_edge(c))) return fail(c, NB_ERR_BOX, "rc out of range");
    if (xyz) {
        nb_status st = nb_set_coords(c, xyz, stream);
        if (st != NB_OK) return st;
    }
    ForceParams fp{};
    const nb_status pst = force_params(c, p, &fp);
    if (pst != NB_OK) return pst;
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    const int sp = span_begin(c, NB_KERNEL_FORCE_1X1, s);
    c->fslot_zero = false;   // the 1 x 1 kernel overwrites the real slots' accumulators
    cudaError_t e = launch_force_1x1(c->ws, fp, c->C, max_nbr, nbr, count, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "1x1 force kernel");
    const int sz = span_begin(c, NB_KERNEL_FINALIZE, s);
    e = launch_finalize(c->ws, fp, c->C, f, nullptr, nullptr, s);
    c->fslot_zero = false;
    span_end(c, sz, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "finalize kernel");
    c->n_launches += 2;
    return NB_OK;
}

nb_status nb_rdf(nb_ctx* c, float r_max, int nbins, int type_a, int type_b, int accumulate, uint64_t* hist,
                 nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!hist || nbins < 1 || nbins > NB_RDF_MAX_BINS || !(r_max > 0.f))
        return fail(c, NB_ERR_ARG, "rdf: bad argument");
    if ((type_a < 0) != (type_b < 0) || type_a < -1 || type_b < -1 || type_a >= c->ntypes || type_b >= c->ntypes)
        return fail(c, NB_ERR_ARG, "rdf: type selection must be two types in range or both -1");
    if (!c->have_list) return fail(c, NB_ERR_STATE, "nb_pairlist_build first");
    if (!c->list_fresh) return fail(c, NB_ERR_STATE, "rdf: coordinates changed since the list was built");
    if (r_max > c->rlist) return fail(c, NB_ERR_BOX, "rdf: r_max above the list radius");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint64_t) * (size_t)c->nbox * (size_t)(nbins + 1), s);
        if (e != cudaSuccess) return cuda_fail(c, e, "rdf: clearing the histogram");
    }
    const int sp = span_begin(c, NB_KERNEL_RDF, s);
    cudaError_t e = launch_rdf(c->ws, c->C, r_max, nbins, type_a, type_b,
                               reinterpret_cast<unsigned long long*>(hist), c->n_sm, s);
    span_end(c, sp, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "rdf kernel");
    c->n_launches += 1;
    return NB_OK;
}

nb_status nb_set_surrogate(nb_ctx* c, const float* params, float r_min, float r_max, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->ws_base) return fail(c, NB_ERR_STATE, "no workspace");
    if (c->C != 8) return fail(c, NB_ERR_ARG, "the surrogate kernel needs 8-particle clusters");
    ++c->gen;
    if (!params || !(r_min >= 0.f) || !(r_max > r_min) || !std::isfinite(r_max))
        return fail(c, NB_ERR_ARG, "set_surrogate: bad argument");
    NB_CUDA(c, cudaSetDevice(c->device));
    const nb_status st = nb_mlp_pack(params, r_min, r_max, c->ws.mlp, stream);
    if (st != NB_OK) return fail(c, st, "packing the network failed");
    c->n_launches += 1;
    c->have_mlp = true;
    c->mlp_rmin = r_min;
    c->mlp_rmax = r_max;
    return NB_OK;
}

nb_status nb_check(nb_ctx* c, nb_stream stream, nb_info* info) {
    if (!c) return NB_ERR_ARG;
    if (!c->ws_base) return fail(c, NB_ERR_STATE, "no workspace");
    cudaStream_t s = (cudaStream_t)stream;
    NB_CUDA(c, cudaSetDevice(c->device));
    NB_CUDA(c, cudaMemcpyAsync(c->st_host, c->ws.st, sizeof(DevState) * c->nbox, cudaMemcpyDeviceToHost, s));
    NB_CUDA(c, cudaStreamSynchronize(s));
    unsigned flags = 0;
    int worst = -1;
    for (int b = 0; b < c->nbox; ++b) {
        c->last[b] = c->st_host[b];
        if (c->last[b].flags && worst < 0) worst = b;
        flags |= c->last[b].flags;
    }
    c->last_valid = true;
    if (flags) {
        for (int b = 0; b < c->nbox; ++b)
            if (c->last[b].flags) NB_CUDA(c, cudaMemsetAsync(&c->ws.st[b].flags, 0, sizeof(unsigned), s));
        NB_CUDA(c, cudaStreamSynchronize(s));
    }
    if (info) fill_info(c, 0, c->nbox, info, flags);
    if (flags & (1u << NB_ERR_COORD))
        return fail(c, NB_ERR_COORD, "box %d: a coordinate was outside [-L, 2L)", worst);
    if (flags & (1u << NB_ERR_CAPACITY))
        return fail(c, NB_ERR_CAPACITY, "box %d: device capacity exceeded (list %llu/%lld j-entries, longest column %d)",
                    worst, (unsigned long long)c->last[worst].n_jent, c->plan[worst].jent_cap,
                    c->last[worst].max_col);
    if (flags & (1u << NB_ERR_ARG)) return fail(c, NB_ERR_ARG, "box %d: a type or exclusion index out of range", worst);
    if (flags & (1u << NB_ERR_TIMEOUT)) return fail(c, NB_ERR_TIMEOUT, "a bounded device wait expired");
    if (flags) return fail(c, NB_ERR_CUDA, "device flags 0x%x", flags);
    return NB_OK;
}

nb_status nb_box_info(nb_ctx* c, int box, nb_info* info) {
    if (!c || !info) return NB_ERR_ARG;
    if (box < 0 || box >= c->nbox) return fail(c, NB_ERR_ARG, "box index out of range");
    if (!c->last_valid) return fail(c, NB_ERR_STATE, "call nb_check first");
    fill_info(c, box, box + 1, info, c->last[box].flags);
    return NB_OK;
}

nb_status nb_profile(nb_ctx* c, int enable) {
    if (!c) return NB_ERR_ARG;
    ++c->gen;
    if (enable && !c->ev[0]) {
        NB_CUDA(c, cudaSetDevice(c->device));
        for (int k = 0; k < 2 * nb_ctx::kMaxSpans; ++k) NB_CUDA(c, cudaEventCreate(&c->ev[k]));
    }
    c->prof = enable != 0;
    c->prof_keep = enable == 2;
    return NB_OK;
}

nb_status nb_profile_read(nb_ctx* c, int* kinds, float* ms, int max, int* count) {
    if (!c || !count || max < 0 || (max > 0 && (!kinds || !ms)))
        return fail(c, NB_ERR_ARG, "profile_read: bad argument");
    const int n = c->ev_n < max ? c->ev_n : max;
    for (int k = 0; k < n; ++k) {
        NB_CUDA(c, cudaEventSynchronize(c->ev[2 * k + 1]));
        NB_CUDA(c, cudaEventElapsedTime(&ms[k], c->ev[2 * k], c->ev[2 * k + 1]));
        kinds[k] = c->ev_kind[k];
    }
    *count = n;
    if (!c->prof_keep) c->ev_n = 0;
    return NB_OK;
}

nb_status nb_get_grid(nb_ctx* c, int* atom_of_slot, int* slot_of_atom, int* col_clu_start, float* xyzq,
                      int* type_slot, float* bb, int* col_of_atom, int* sc_info, nb_stream stream) {
    if (!c) return NB_ERR_ARG;
    if (!c->have_grid || !c->last_valid) return fail(c, NB_ERR_STATE, "need a grid and nb_check");
    if (c->nbox != 1) return fail(c, NB_ERR_STATE, "grid copies are for single-box contexts");
    cudaStream_t s = (cudaStream_t)stream;
    const long long nclu = c->last[0].nclu;
    const long long ns = nclu * c->C;
    const int ncol = c->geo_host[0].nx * c->geo_host[0].ny;
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
    NB_CUDA(c, cp(sc_info, c->ws.sc_info, sizeof(int2) * (size_t)c->last[0].nsc));
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
    if (c->nbox != 1) return fail(c, NB_ERR_STATE, "list copies are for single-box contexts");
    cudaStream_t s = (cudaStream_t)stream;
    const long long ni = (long long)c->last[0].n_ient, nj = (long long)c->last[0].n_jent;
    if (ni > c->plan[0].ient_cap || nj > c->plan[0].jent_cap) return fail(c, NB_ERR_CAPACITY, "list overflowed");
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
