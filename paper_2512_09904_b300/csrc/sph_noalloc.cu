// sph_noalloc.cu -- allocation-free cell sort (sph_cell_sort_noalloc).
//
// Some callers cannot let a library allocate device memory: a process whose
// HBM is already reserved by its own caching allocator (a new driver
// allocation fails there), a latency-critical loop that cannot afford the
// implicit device synchronisation of cudaMalloc/cudaFree, or a host that
// forbids allocations outside its own memory manager.  For them this file
// keeps the sort's scratch in a fixed device array, placed on a device when
// this library's module is loaded there (at the first call on that device
// under lazy module loading, the default; at library load with
// CUDA_MODULE_LOADING=EAGER) and held until the process exits.
#include <mutex>

#include "sph.h"
#include "sph_kernels.cuh"

namespace sph {
void set_stateless_error(const char* msg);
}

namespace {

constexpr size_t kMaxN = (size_t)SPH_NOALLOC_MAX_N;
constexpr size_t kMaxCells = (size_t)SPH_NOALLOC_MAX_CELLS;
constexpr size_t kScanWords = kMaxCells / sph::SCAN_TILE + 2;
// keys, ranks, scattered slots (n each), per-cell counts, scan tile totals
constexpr size_t kWords = 3 * kMaxN + kMaxCells + kScanWords;

static __device__ __align__(256) uint32_t g_scratch[kWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per
// device.  In host code the name g_scratch is only a host-side stand-in, so
// the address must come from cudaGetSymbolAddress with the device current.
// The cached address is not refreshed: a device reset (cudaDeviceReset, or a
// primary-context reset) after the first call is not supported.
cudaError_t scratch_address(uint32_t** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sph_status sph_cell_sort_noalloc(const double* pos, int64_t n, const double origin[3],
                                            const double cellw[3], const int ncell[3], int32_t* perm,
                                            int32_t* cell_start, void* stream) {
    if (!origin || !cellw || !ncell) {
        sph::set_stateless_error("sph_cell_sort_noalloc: null grid argument");
        return SPH_EINVAL;
    }
    static const char* too_big =
        "sph_cell_sort_noalloc: n or the cell count exceeds the fixed scratch "
        "(SPH_NOALLOC_MAX_N / SPH_NOALLOC_MAX_CELLS); use sph_cell_sort";
    // the running product is checked after every factor, so it stays below
    // kMaxCells * INT_MAX and never overflows
    int64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (ncell[a] < 1 || !(cellw[a] > 0)) {
            sph::set_stateless_error("sph_cell_sort_noalloc: ncell must be >= 1 and cellw > 0");
            return SPH_EINVAL;
        }
        nc *= ncell[a];
        if (nc > (int64_t)kMaxCells) {
            sph::set_stateless_error(too_big);
            return SPH_EINVAL;
        }
    }
    if (n > (int64_t)kMaxN) {
        sph::set_stateless_error(too_big);
        return SPH_EINVAL;
    }
    if (n < 0 || (n > 0 && (!pos || !perm)) || !cell_start) {
        sph::set_stateless_error("sph_cell_sort_noalloc: null pointer or negative n");
        return SPH_EINVAL;
    }
    uint32_t* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        sph::set_stateless_error("sph_cell_sort_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return SPH_ECUDA;
    }
    uint32_t* keys = base;
    uint32_t* rank = keys + kMaxN;
    uint32_t* tmp = rank + kMaxN;
    uint32_t* cnt = tmp + kMaxN;   // cleared by launch_cell_sort before use
    uint32_t* blk = cnt + kMaxCells;
    e = sph::launch_cell_sort(pos, (int)n, origin, cellw, ncell, keys, rank, cnt, tmp, blk, perm, cell_start,
                              (cudaStream_t)stream);
    if (e != cudaSuccess) {
        sph::set_stateless_error("sph_cell_sort_noalloc: kernel launch failed");
        return SPH_ECUDA;
    }
    return SPH_OK;
}
