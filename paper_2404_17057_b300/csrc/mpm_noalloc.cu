// mpm_noalloc.cu -- mpm_sort_keys_static: the stable key re-order for callers
// that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: components that live inside another
// framework's memory pool and must not grow the device footprint behind its
// back, and latency-critical loops where an allocation can synchronise the
// device.  For them this entry point keeps all of its scratch space in fixed
// arrays that are part of the library image itself.  Every GPU that loads
// the library holds these arrays (3.1 MiB) until the process exits.
//
// This file is compiled into the same translation unit as mpm_api.cu (it is
// included at its end) and reuses the radix-sort kernels of mpm_sort.cuh.
#include <mutex>

namespace mpm {

constexpr int64_t kStaticSortMaxKeys = MPM_SORT_STATIC_MAX_KEYS;
constexpr int64_t kStaticSortMaxBlocks = (kStaticSortMaxKeys + kSortTile - 1) / kSortTile;
constexpr int64_t kStaticSortHist = 256 * kStaticSortMaxBlocks;

// The scratch: two (key, index) ping-pong buffers, the digit histograms and
// the partial sums of their scan.  Shared by every call on a device.
static __device__ __align__(256) uint32_t g_sort_keys[2][kStaticSortMaxKeys];
static __device__ __align__(256) uint32_t g_sort_idx[kStaticSortMaxKeys];
static __device__ __align__(256) uint32_t g_sort_hist[kStaticSortHist];
static __device__ __align__(256) uint32_t g_sort_part[kScanTile];
// set by a call that meets a key >= nkeys, cleared by the same call
static __device__ __align__(256) uint32_t g_sort_bad[4];

struct StaticSortScratch {
    uint32_t* keys[2];
    uint32_t* idx;
    uint32_t* hist;
    uint32_t* part;
    uint32_t* bad;
    bool ready;
};

constexpr int kStaticSortMaxDevices = 64;
static StaticSortScratch g_scratch[kStaticSortMaxDevices];
static std::mutex g_scratch_mutex;

// Device addresses of the scratch arrays on the current device, looked up
// once per device.  In host code the array names are host-side stand-ins,
// not device addresses, so only these looked-up pointers go to kernels.
static cudaError_t static_sort_scratch(int dev, StaticSortScratch* out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    StaticSortScratch& s = g_scratch[dev];
    if (!s.ready) {
        cudaError_t e;
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_sort_keys)) != cudaSuccess) return e;
        s.keys[0] = static_cast<uint32_t*>(p);
        s.keys[1] = s.keys[0] + kStaticSortMaxKeys;
        if ((e = cudaGetSymbolAddress(&p, g_sort_idx)) != cudaSuccess) return e;
        s.idx = static_cast<uint32_t*>(p);
        if ((e = cudaGetSymbolAddress(&p, g_sort_hist)) != cudaSuccess) return e;
        s.hist = static_cast<uint32_t*>(p);
        if ((e = cudaGetSymbolAddress(&p, g_sort_part)) != cudaSuccess) return e;
        s.part = static_cast<uint32_t*>(p);
        if ((e = cudaGetSymbolAddress(&p, g_sort_bad)) != cudaSuccess) return e;
        s.bad = static_cast<uint32_t*>(p);
        s.ready = true;
    }
    *out = s;
    return cudaSuccess;
}

// Any key >= nkeys marks the call as invalid.
__global__ void k_static_sort_verify(const uint32_t* __restrict__ keys, int64_t n, int64_t nkeys, uint32_t* bad)
{
    bool b = false;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        b = b || (int64_t)keys[j] >= nkeys;
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// After the cell starts are written: an invalid call replaces
// cell_start[nkeys] (n otherwise) by 0xffffffff; the flag is cleared for the
// next call.
__global__ void k_static_sort_finish(uint32_t* bad, uint32_t* cell_start, int64_t nkeys)
{
    if (*bad) cell_start[nkeys] = 0xffffffffu;
    *bad = 0u;
}

}  // namespace mpm

extern "C" mpm_status mpm_sort_keys_static(const uint32_t* keys, int64_t n, int64_t nkeys, uint32_t* perm,
                                           uint32_t* cell_start, void* stream)
{
    using namespace mpm;
    if (n < 0 || n > kStaticSortMaxKeys)
        return fail(nullptr, MPM_EINVAL, "mpm_sort_keys_static: n must be in [0, MPM_SORT_STATIC_MAX_KEYS]");
    if (nkeys < 1 || nkeys > MPM_SORT_STATIC_MAX_SPANS)
        return fail(nullptr, MPM_EINVAL, "mpm_sort_keys_static: nkeys must be in [1, MPM_SORT_STATIC_MAX_SPANS]");
    if ((n > 0 && (!keys || !perm)) || !cell_start)
        return fail(nullptr, MPM_EINVAL, "mpm_sort_keys_static: NULL device pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kStaticSortMaxDevices) {
        cudaGetLastError();
        return fail(nullptr, MPM_ECUDA, "mpm_sort_keys_static: no usable CUDA device");
    }
    StaticSortScratch sc;
    e = static_sort_scratch(dev, &sc);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, MPM_ECUDA, std::string("mpm_sort_keys_static: scratch lookup: ") + cudaGetErrorString(e));
    }
    cudaStream_t st = (cudaStream_t)stream;
    int bits = 1;
    while (((int64_t)1 << bits) < nkeys) ++bits;
    const int passes = (bits + 7) / 8;
    const int dbits = (bits + passes - 1) / passes;
    const unsigned nb = (unsigned)std::max<int64_t>(1, (n + kSortTile - 1) / kSortTile);
    const int64_t nhist = (int64_t)(1 << dbits) * nb;
    if (n > 0) {
        // the digit histograms are fully rewritten by every pass; only the
        // invalid-key flag must start at zero (every call clears it at its end)
        k_static_sort_verify<<<(unsigned)std::min<int64_t>(256, (n + 255) / 256), 256, 0, st>>>(keys, n, nkeys,
                                                                                              sc.bad);
        const uint32_t* kin = keys;
        const uint32_t* iin = nullptr;
        for (int pass = 0; pass < passes; ++pass) {
            const int shift = pass * dbits;
            uint32_t* kout = sc.keys[pass & 1];
            // indices ping-pong between the scratch and the caller's perm so
            // that the last pass writes perm and never reads its own output
            uint32_t* iout = ((passes - 1 - pass) % 2 == 0) ? perm : sc.idx;
            k_radix_hist<<<nb, kSortThreads, 0, st>>>(kin, n, shift, dbits, sc.hist, nullptr);
            scan_exclusive(sc.hist, sc.hist, nhist, sc.part, 0, st, nullptr);
            k_radix_scatter<<<nb, kSortThreads, 0, st>>>(kin, iin, kout, iout, n, shift, dbits, sc.hist, nullptr,
                                                          pass == 0);
            kin = kout;
            iin = iout;
        }
        k_cell_start<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(kin, n, nkeys, cell_start, nullptr);
    } else {
        k_cell_start<<<1, 256, 0, st>>>(keys, 0, nkeys, cell_start, nullptr);
    }
    k_static_sort_finish<<<1, 1, 0, st>>>(sc.bad, cell_start, nkeys);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, MPM_ECUDA, std::string("mpm_sort_keys_static: ") + cudaGetErrorString(e));
    return MPM_OK;
}
