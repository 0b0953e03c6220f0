// nb_grid_put_noalloc: the gridding kernels of nb_grid_put run on scratch
// memory that is a file-scope __device__ array instead of a caller-provided
// workspace, for callers that cannot allocate device memory at all (code that
// runs where cudaMalloc is forbidden or unavailable, e.g. inside a host
// callback, a memory-capped plug-in, or a process whose allocator belongs to
// another runtime).  The paper has no counterpart to this entry point.
//
// The array is loaded with the module on every GPU that uses the library and
// stays allocated until the process exits.  Host code cannot use the array's
// name as a device address, so the first call on each device (with that
// device current) asks the runtime for the address with cudaGetSymbolAddress
// and keeps it; that first call should therefore happen before any stream
// capture.  Every call shares the one array: calls whose work overlaps on the
// GPU (different streams, or different host threads on one device) race.
#include <mutex>

#include "nb_internal.cuh"

namespace nbc {

constexpr int kNoallocMaxAtoms = 32768;
constexpr int kNoallocMaxColumns = 4096;
constexpr long long kNoallocMaxSlots = kNoallocMaxAtoms + (long long)kNoallocMaxColumns * 7;
// Clusters and super-clusters of a grid with at most slots slots and
// columns columns, as the entry point plans them (the super-cluster bound is
// largest for clusters of 4, one cluster each).
constexpr long long noalloc_clusters(long long slots, int C) { return slots / C + 1; }
constexpr long long noalloc_superclusters(long long slots, long long columns, int C) {
    return noalloc_clusters(slots, C) / super_size(C) + columns + 1;
}
constexpr long long kNoallocMaxSuperclusters = noalloc_superclusters(kNoallocMaxSlots, kNoallocMaxColumns, 4);
static_assert(kNoallocMaxSuperclusters >= noalloc_superclusters(kNoallocMaxSlots, kNoallocMaxColumns, 8),
              "super-cluster capacity");
constexpr int kNoallocMaxDevices = 64;

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout (byte offsets).
constexpr size_t kOffState = 0;
constexpr size_t kOffGeo = align256(kOffState + sizeof(DevState));
constexpr size_t kOffLayout = align256(kOffGeo + sizeof(BoxGeom));
constexpr size_t kOffXw = align256(kOffLayout + 4 * 2 * sizeof(int) + 2 * 2 * sizeof(long long));
constexpr size_t kOffWoff = align256(kOffXw + sizeof(float4) * kNoallocMaxAtoms);
constexpr size_t kOffColOfAtom = align256(kOffWoff + sizeof(float4) * kNoallocMaxAtoms);
constexpr size_t kOffRank = align256(kOffColOfAtom + sizeof(int) * kNoallocMaxAtoms);
constexpr size_t kOffSlotOfAtom = align256(kOffRank + sizeof(int) * kNoallocMaxAtoms);
constexpr size_t kOffKeys = align256(kOffSlotOfAtom + sizeof(int) * kNoallocMaxAtoms);
constexpr size_t kOffColCount = align256(kOffKeys + sizeof(unsigned long long) * kNoallocMaxAtoms);
constexpr size_t kOffColAtomStart = align256(kOffColCount + sizeof(int) * (kNoallocMaxColumns + 1));
constexpr size_t kOffColScStart = align256(kOffColAtomStart + sizeof(int) * (kNoallocMaxColumns + 1));
constexpr size_t kOffScInfo = align256(kOffColScStart + sizeof(int) * (kNoallocMaxColumns + 1));
constexpr size_t kOffFslot = align256(kOffScInfo + sizeof(int2) * kNoallocMaxSuperclusters);
constexpr size_t kNoallocScratchBytes = align256(kOffFslot + sizeof(float4) * kNoallocMaxSlots);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mutex;
static unsigned char* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
static cudaError_t noalloc_scratch(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (unsigned char*)p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Box geometry, the one-box region offsets and a cleared state, written into
// the scratch on the stream (the values travel as kernel arguments, so no host
// staging buffer is involved).
__global__ void k_noalloc_setup(Workspace ws, BoxGeom g, int n, int ncol, int nclu_cap, int nsc_cap) {
    if (threadIdx.x != 0) return;
    *ws.geo = g;
    int* a = const_cast<int*>(ws.lay.atom_off);
    int* c = const_cast<int*>(ws.lay.col_off);
    int* u = const_cast<int*>(ws.lay.clu_off);
    int* q = const_cast<int*>(ws.lay.sc_off);
    long long* ie = const_cast<long long*>(ws.lay.ient_off);
    long long* je = const_cast<long long*>(ws.lay.jent_off);
    a[0] = c[0] = u[0] = q[0] = 0;
    a[1] = n;
    c[1] = ncol + 1;
    u[1] = nclu_cap;
    q[1] = nsc_cap;
    ie[0] = ie[1] = je[0] = je[1] = 0;
    DevState z{};
    *ws.st = z;
}

}  // namespace nbc

using namespace nbc;

extern "C" nb_status nb_grid_put_noalloc(int n, const float* xyz, const float* q, const int* type,
                                         int ntypes, const double* box, int cluster_size,
                                         int* atom_of_slot, float* xyzq, int* type_slot, float* bb,
                                         int* col_clu_start, int* info, int max_slots, int max_columns,
                                         nb_stream stream) {
    const int C = cluster_size;
    if (C != 4 && C != 8) return NB_ERR_ARG;
    if (n <= 0 || !xyz || !q || !type || !atom_of_slot || !xyzq || !type_slot || !bb || !col_clu_start ||
        !info || ntypes <= 0 || ntypes > kMaxTypes || max_slots <= 0 || max_columns <= 0)
        return NB_ERR_ARG;
    if (((uintptr_t)xyzq & 15) || ((uintptr_t)bb & 15)) return NB_ERR_ARG;
    if (!box) return NB_ERR_BOX;
    for (int k = 0; k < 3; ++k)
        if (!(box[k] > 0.0) || !(box[k] < 1e30)) return NB_ERR_BOX;
    // the same geometry as nb_grid_put (dimensions, inverse spacings, dummies)
    const BoxGeom g = box_geometry(n, box, C);
    const long long ncol = (long long)g.nx * g.ny;
    const long long nslot_bound = (long long)n + ncol * (C - 1);
    if (n > kNoallocMaxAtoms || ncol > kNoallocMaxColumns || nslot_bound > kNoallocMaxSlots)
        return NB_ERR_CAPACITY;
    if (nslot_bound > max_slots || ncol > max_columns) return NB_ERR_CAPACITY;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocMaxDevices) return NB_ERR_CUDA;
    unsigned char* base = nullptr;
    if (noalloc_scratch(dev, &base) != cudaSuccess) return NB_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int nclu_cap = (int)noalloc_clusters(nslot_bound, C);
    const int nsc_cap = (int)noalloc_superclusters(nslot_bound, ncol, C);
    Workspace ws{};
    ws.nbox = 1;
    ws.st = (DevState*)(base + kOffState);
    ws.geo = (BoxGeom*)(base + kOffGeo);
    {
        int* li = (int*)(base + kOffLayout);
        ws.lay.atom_off = li;
        ws.lay.col_off = li + 2;
        ws.lay.clu_off = li + 4;
        ws.lay.sc_off = li + 6;
        long long* ll = (long long*)(li + 8);
        ws.lay.ient_off = ll;
        ws.lay.jent_off = ll + 2;
    }
    ws.atom_total = n;
    ws.col_total = (int)ncol + 1;
    ws.clu_total = nclu_cap;
    ws.sc_total = nsc_cap;
    ws.xw = (float4*)(base + kOffXw);
    ws.woff = (float4*)(base + kOffWoff);
    ws.col_of_atom = (int*)(base + kOffColOfAtom);
    ws.rank_in_col = (int*)(base + kOffRank);
    ws.slot_of_atom = (int*)(base + kOffSlotOfAtom);
    ws.keys = (unsigned long long*)(base + kOffKeys);
    ws.col_count = (int*)(base + kOffColCount);
    ws.col_atom_start = (int*)(base + kOffColAtomStart);
    ws.fslot = (float4*)(base + kOffFslot);
    ws.col_sc_start = (int*)(base + kOffColScStart);
    ws.sc_info = (int2*)(base + kOffScInfo);
    ws.q = const_cast<float*>(q);
    ws.type = const_cast<int*>(type);
    ws.col_clu_start = col_clu_start;
    ws.xyzq = (float4*)xyzq;
    ws.atom_of_slot = atom_of_slot;
    ws.type_slot = type_slot;
    ws.bb = (float4*)bb;
    // geometry, offsets and a cleared state (the previous call's flags and counts)
    k_noalloc_setup<<<1, 32, 0, s>>>(ws, g, n, (int)ncol, nclu_cap, nsc_cap);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;
    if (launch_grid(ws, C, ntypes, xyz, s) != cudaSuccess) return NB_ERR_CUDA;
    if (cudaMemcpyAsync(&info[0], &ws.st->nclu, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(&info[1], &ws.st->flags, sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return NB_ERR_CUDA;
    return NB_OK;
}
