// otm_replay.cu -- the supports of a state as a compact CSR in caller device memory, and such a
// CSR replayed as the supports of a step. A finite-difference check of the adjoint differences
// perturbed runs whose topology must be that of the differentiated trajectory; recording the
// supports of every step on the device keeps a long trajectory's record (hundreds of steps of
// ~10^8 pairs) off the host, and the replay of rows in the library's own order reproduces the
// unperturbed run bit for bit.
#include "otm_dev.cuh"

namespace otm {

static int replay_blocks(int64_t warps)
{
    int64_t b = (warps * kWarp + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

// ids[off[p] + k] = slot k of MP p's padded row, k < cnt[p]; one warp per MP (grid-stride)
__global__ void k_csr_gather(const Dev D, const int32_t *__restrict__ off, int32_t *__restrict__ ids)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w0; p < D.nm; p += nw) {
        const int n = D.cnt[p];
        const int64_t o = off[p], base = p * (int64_t)D.S;
        for (int k = lane; k < n; k += kWarp) ids[o + k] = D.ids[base + k];
    }
}

// Checks a caller CSR before anything reads through it: for every MP, 0 <= off[p],
// off[p + 1] <= len, and 1 <= off[p + 1] - off[p] <= S; only then are the row's IDs read, each
// in [0, nn). Any violation sets *bad (zeroed by the caller).
__global__ void k_csr_check(const int32_t *__restrict__ off, const int32_t *__restrict__ ids, int64_t nm, int S,
                            int64_t len, int64_t nn, int32_t *bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w0; p < nm; p += nw) {
        const int64_t o0 = off[p], o1 = off[p + 1];
        const int64_t n = o1 - o0;
        if (o0 < 0 || o1 > len || n < 1 || n > S) {
            if (lane == 0) atomicExch(bad, 1);
            continue;
        }
        bool ok = true;
        for (int64_t k = lane; k < n; k += kWarp) {
            const int32_t id = ids[o0 + k];
            ok = ok && id >= 0 && (int64_t)id < nn;
        }
        if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicExch(bad, 1);
    }
}

// the checked CSR as the padded rows of the state: cnt[p] and ids[p * S + k]
__global__ void k_csr_scatter(const Dev D, const int32_t *__restrict__ off, const int32_t *__restrict__ ids)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w0; p < D.nm; p += nw) {
        const int64_t o = off[p];
        const int n = (int)(off[p + 1] - o);
        const int64_t base = p * (int64_t)D.S;
        for (int k = lane; k < n; k += kWarp) D.ids[base + k] = ids[o + k];
        if (lane == 0) D.cnt[p] = n;
    }
}

cudaError_t launch_csr_gather(const Dev &D, const int32_t *off, int32_t *ids, cudaStream_t s, long long *launches)
{
    if (D.nm <= 0) return cudaSuccess;
    k_csr_gather<<<replay_blocks(D.nm), 256, 0, s>>>(D, off, ids);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_csr_check(const int32_t *off, const int32_t *ids, int64_t nm, int S, int64_t len, int64_t nn,
                             int32_t *bad, cudaStream_t s, long long *launches)
{
    if (nm <= 0) return cudaSuccess;
    k_csr_check<<<replay_blocks(nm), 256, 0, s>>>(off, ids, nm, S, len, nn, bad);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_csr_scatter(const Dev &D, const int32_t *off, const int32_t *ids, cudaStream_t s,
                               long long *launches)
{
    if (D.nm <= 0) return cudaSuccess;
    k_csr_scatter<<<replay_blocks(D.nm), 256, 0, s>>>(D, off, ids);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace otm
