// otm_noalloc.cu -- the linked-cell support search for callers that cannot allocate device
// memory: the same kernels as otm_support_search, with their scratch in a fixed static device
// array instead of a caller-provided buffer.
//
// Who needs it: code that runs where device allocation is not an option at call time -- a
// host process whose device memory is already fully reserved by another allocator, a latency-
// sensitive loop that must not pay cudaMalloc's implicit device synchronisation, or an embedding
// that must not fail on an out-of-memory at run time. Such callers still own their inputs and
// outputs; only the scratch is provided here.
//
// The static array below lives in every GPU that loads this library, from module load until
// process exit (16 MiB). In host code its name is only a host-side stand-in, so the device
// address is looked up once per device with cudaGetSymbolAddress while that device is current,
// and that address is what the kernels receive.
#include <mutex>

#include "otm_dev.cuh"

namespace otm {

constexpr size_t kNoallocScratchBytes = (size_t)16 << 20;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[kNoallocMaxDevices];

// Device address of the static scratch on the current device (set up on first use).
static cudaError_t noalloc_scratch(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        if (!p) return cudaErrorInvalidSymbol;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace otm

using namespace otm;

extern "C" int otm_support_search_noalloc(const double *node_x, int64_t n_nodes, const double *mp_x, int64_t n_mps,
                                          double rs2, double cell_size, int32_t max_support, int32_t *ids,
                                          int32_t *counts, double *grid_out, int32_t *status, void *stream)
{
    if (!node_x || !mp_x || !ids || !counts || !status || n_nodes <= 0 || n_mps < 0) return OTM_ERR_ARG;
    if (max_support < 1 || max_support > kMaxS) return OTM_ERR_ARG;
    if (!(rs2 > 0) || !(cell_size * 2.0 >= sqrt(rs2))) return OTM_ERR_ARG;
    if (n_nodes > OTM_NOALLOC_MAX_NODES) return OTM_ERR_CAPACITY;
    if (search_scratch_bytes(n_nodes) > kNoallocScratchBytes) return OTM_ERR_CAPACITY;
    void *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return OTM_ERR_CUDA;
    if (launch_search_only(node_x, n_nodes, mp_x, n_mps, rs2, cell_size, max_support, ids, counts, scratch,
                           kNoallocScratchBytes, grid_out, status, (cudaStream_t)stream) != cudaSuccess)
        return OTM_ERR_CUDA;
    return OTM_OK;
}
