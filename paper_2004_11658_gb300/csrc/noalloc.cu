// noalloc.cu -- dp_format_nlist_noalloc: the formatted neighbour list
// (candidates + Algorithm 1) computed without allocating any memory.
//
// Some callers cannot allocate device memory when they need the list: a host
// MD engine that owns a fixed device memory budget and forbids allocations
// after start-up, or code that runs where cudaMalloc is not allowed.  This
// entry point takes only the caller's inputs and outputs and keeps all of its
// scratch (candidate lists, sort keys, status word) in one file-scope
// __device__ array of fixed size, which every GPU that loads the library holds
// until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "dp_internal.cuh"

namespace {

constexpr int kMaxAtoms = DP_NOALLOC_MAX_ATOMS;
constexpr int kCap = DP_NOALLOC_CAND_CAP;
constexpr int kMaxDevices = 64;

// Scratch layout (byte offsets, each 256-aligned).
constexpr size_t kOffStatus = 0;
constexpr size_t kOffNcand = 256;
constexpr size_t kOffTypeStart = kOffNcand + sizeof(int32_t) * kMaxAtoms;
constexpr size_t kOffTypePerm = kOffTypeStart + 256;
constexpr size_t kOffXref = kOffTypePerm + sizeof(int32_t) * kMaxAtoms;
constexpr size_t kOffCand = kOffXref + sizeof(double) * 3 * kMaxAtoms;
constexpr size_t kOffKeys = kOffCand + sizeof(int32_t) * (size_t)kMaxAtoms * kCap;
constexpr size_t kOffRetry = kOffKeys + sizeof(uint64_t) * (size_t)kMaxAtoms * DP_MAX_NM;
constexpr size_t kScratchBytes = kOffRetry + sizeof(int32_t) * (kMaxAtoms + 64);
static_assert(kOffNcand % 256 == 0 && kOffTypeStart % 256 == 0 && kOffTypePerm % 256 == 0 &&
                  kOffXref % 256 == 0 && kOffCand % 256 == 0 && kOffKeys % 256 == 0 && kOffRetry % 256 == 0,
              "scratch regions must stay 256-byte aligned");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol, not a device address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char dp_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

}  // namespace

// Defined in dp_api.cu: keeps dp_last_error() in sync for this entry point.
void dp_set_last_error(const char *msg);

extern "C" dp_status dp_format_nlist_noalloc(const dp_model_desc *desc, const double *coords,
                                             const int32_t *types, const double box[9], int64_t N,
                                             double skin, int32_t *nlist, int32_t *nreal, void *stream)
{
    auto fail = [](dp_status s, const std::string &m) {
        dp_set_last_error(m.c_str());
        return s;
    };
    if (!desc || !coords || !types || !box || !nlist || !nreal)
        return fail(DP_ERR_ARG, "dp_format_nlist_noalloc: a pointer argument is NULL");
    if (desc->ntypes < 1 || desc->ntypes > DP_MAX_TYPES)
        return fail(DP_ERR_UNSUPPORTED, "dp_format_nlist_noalloc: ntypes must be in [1, 8]");
    int nm = 0;
    for (int a = 0; a < desc->ntypes; ++a) {
        if (desc->sel[a] < 0) return fail(DP_ERR_ARG, "dp_format_nlist_noalloc: sel must be >= 0");
        nm += desc->sel[a];
    }
    if (nm < 1 || nm > DP_MAX_NM) return fail(DP_ERR_UNSUPPORTED, "dp_format_nlist_noalloc: sum(sel) must be in [1, 1024]");
    if (N < 1 || N > kMaxAtoms)
        return fail(DP_ERR_CAPACITY, "dp_format_nlist_noalloc: N must be in [1, " + std::to_string(kMaxAtoms) +
                                         "] (the fixed scratch holds at most that many atoms)");
    if (!(desc->rcut > 0.0) || !(skin >= 0.0)) return fail(DP_ERR_ARG, "dp_format_nlist_noalloc: need rcut > 0, skin >= 0");
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            if (r != c && box[3 * r + c] != 0.0)
                return fail(DP_ERR_BOX, "dp_format_nlist_noalloc: only orthorhombic (diagonal) cells are supported");
    Box3 b;
    const double rlist = desc->rcut + skin;
    for (int a = 0; a < 3; ++a) {
        b.L[a] = box[4 * a];
        if (!(b.L[a] >= 2.0 * rlist)) return fail(DP_ERR_BOX, "dp_format_nlist_noalloc: every cell edge must be >= 2 (rcut + skin)");
    }

    // One-time set-up per device, with that device current: the device
    // address of the scratch array.
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(DP_ERR_UNSUPPORTED, "dp_format_nlist_noalloc: device index too large");
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, dp_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return fail(DP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = (unsigned char *)p;
        }
        base = g_addr[dev];
    }

    DevModel m;
    std::memset(&m, 0, sizeof(m));
    m.ntypes = desc->ntypes;
    for (int a = 0, off = 0; a < desc->ntypes; ++a) {
        m.sel[a] = desc->sel[a];
        m.sel_off[a] = off;
        off += desc->sel[a];
    }
    m.nm = nm;
    m.rcut = desc->rcut;

    NlistBuffers nb;
    std::memset(&nb, 0, sizeof(nb));
    nb.ncand = (int32_t *)(base + kOffNcand);
    nb.type_start = (int32_t *)(base + kOffTypeStart);
    nb.type_perm = (int32_t *)(base + kOffTypePerm);
    nb.xref = (double *)(base + kOffXref);
    nb.cand = (int32_t *)(base + kOffCand);
    FormatBuffers fb;
    fb.nlist = nlist;
    fb.nreal = nreal;
    fb.keys = (uint64_t *)(base + kOffKeys);
    int32_t *status = (int32_t *)(base + kOffStatus);

    cudaStream_t st = (cudaStream_t)stream;
    int64_t launches = 0;
    int nc[3] = {1, 1, 1};  // brute-force candidates: no cell arrays needed
    e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = dp_launch_build(st, m, coords, types, b, (int)N, rlist, kCap, nc, nb, status, nullptr, &launches);
    if (e == cudaSuccess)
        e = dp_launch_format(st, m, coords, types, b, (int)N, kCap, kCap, 0.0, nb, fb, status,
                             (int32_t *)(base + kOffRetry), &launches);
    int32_t flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("dp_format_nlist_noalloc: ") + cudaGetErrorString(e));
    if (flags & DPF_BAD_TYPE) return fail(DP_ERR_TYPE, "dp_format_nlist_noalloc: an atom type is outside [0, ntypes)");
    if (flags & DPF_CAND_OVERFLOW)
        return fail(DP_ERR_CAPACITY, "dp_format_nlist_noalloc: an atom has more than " + std::to_string(kCap) +
                                         " candidates within rcut + skin");
    if (flags & DPF_SEL_OVERFLOW) return fail(DP_ERR_SEL_OVERFLOW, "dp_format_nlist_noalloc: a neighbour within rcut did not fit sel");
    return DP_OK;
}
