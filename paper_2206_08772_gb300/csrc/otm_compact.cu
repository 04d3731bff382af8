// otm_compact.cu -- changes of the node and MP sets as device stream compactions (the paper adds
// and removes nodes and MPs during the run, Sec. 1 and Sec. 3.2; erosion by the Johnson-Cook
// fracture criterion, Sec. 4.2):
//  - material points flagged by the fracture criterion leave the body after the constitutive
//    update of their step, and nodes that belong to no support once the new supports are built
//    are removed. Both compactions are stable (survivors keep ascending ID order): keep flags, an
//    exclusive scan, and a gather of every per-entry array; the support IDs are renumbered
//    through the monotone old->new node map, so rows stay consistent.
//  - node insertion: for each MP whose LME solve failed, a node is appended one spacing beyond
//    the MP, away from the centroid of its support (slots by an exclusive scan of the failure
//    flags, so new IDs follow ascending MP ID).
// Scratch comes from regions of the workspace that are dead at that point of the step (see the
// comments at each call).
#include "otm_dev.cuh"

namespace otm {

static int cblocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

__global__ void k_keep_from_u8(const uint8_t *failed, int64_t n, int32_t *keep, int32_t *n_drop)
{
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = failed[i] ? 0 : 1;
        keep[i] = k;
        local += 1 - k;
    }
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(n_drop, local);
}

__global__ void k_keep_from_count(const int32_t *count, int64_t n, int32_t *keep, int32_t *n_drop)
{
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = count[i] > 0 ? 1 : 0;
        keep[i] = k;
        local += 1 - k;
    }
    local = __reduce_add_sync(0xffffffffu, local);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(n_drop, local);
}

// dst[newidx[i]] = src[i] for kept rows; rows of `words` 32-bit words
__global__ void k_gather_rows(const uint32_t *src, uint32_t *dst, int64_t n, int words, const int32_t *keep,
                              const int32_t *newidx)
{
    const int64_t total = n * words;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / words;
        if (!keep[i]) continue;
        const int w = (int)(t - i * words);
        dst[(int64_t)newidx[i] * words + w] = src[t];
    }
}

__global__ void k_gather_bytes(const uint8_t *src, uint8_t *dst, int64_t n, const int32_t *keep,
                               const int32_t *newidx)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (keep[i]) dst[newidx[i]] = src[i];
}

__global__ void k_remap_ids(int32_t *ids, const int32_t *cnt, int64_t nm, int S, const int32_t *newid)
{
    const int64_t total = nm * (int64_t)S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / S;
        const int k = (int)(t - p * S);
        if (k < cnt[p]) ids[t] = newid[ids[t]];
    }
}

// compact the rows of one array in place through `tmp` (tmp holds n * row_bytes bytes)
static cudaError_t compact_array(void *base, int64_t n, size_t row_bytes, const int32_t *keep, const int32_t *newidx,
                                 int64_t n_new, void *tmp, cudaStream_t s, long long *launches)
{
    const int words = (int)(row_bytes / 4);
    k_gather_rows<<<cblocks(n * words, 256), 256, 0, s>>>((const uint32_t *)base, (uint32_t *)tmp, n, words, keep,
                                                          newidx);
    if (launches) *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(base, tmp, (size_t)n_new * row_bytes, cudaMemcpyDeviceToDevice, s);
}

// Erode the MPs flagged in D.failed. Scratch: the node-major contribution region (consumed by the
// node update of this step, rewritten by the LME kernel later in the step). Returns the number
// of eroded MPs through *n_drop_host (synchronises the stream).
cudaError_t erode_mps(Dev &D, int32_t *scan_tmp, int64_t *n_drop_host, cudaStream_t s, long long *launches)
{
    const int64_t nm = D.nm;
    char *scratch = D.precision == OTM_PRECISION_MIXED ? (char *)D.contrib32 : (char *)D.contrib64;
    int32_t *n_drop = (int32_t *)scratch;
    int32_t *keep = n_drop + 64;
    int32_t *newidx = keep + ((nm + 63) / 64) * 64;
    void *tmp = (void *)(newidx + ((nm + 1 + 63) / 64) * 64 + 64);
    cudaError_t e = cudaMemsetAsync(n_drop, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_keep_from_u8<<<cblocks(nm, 256), 256, 0, s>>>(D.failed, nm, keep, n_drop);
    if (launches) *launches += 1;
    int32_t nd = 0;
    if ((e = cudaMemcpyAsync(&nd, n_drop, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *n_drop_host = nd;
    if (nd == 0) return cudaSuccess;
    if ((e = launch_exclusive_scan_tmp(keep, newidx, nm, scan_tmp, s, launches)) != cudaSuccess) return e;
    const int64_t nn_new = nm - nd;
    struct F {
        void *p;
        size_t row;
    } fields[] = {{D.xp, 32}, {D.xp_prev, 32}, {D.F, 72}, {D.dF, 72}, {D.be, 48}, {D.sig, 48}, {D.vol, 8}, {D.mass, 8},
                  {D.ebar, 8}, {D.T, 8}, {D.rate, 8}, {D.lam, 24}, {D.lam_prev, 24}, {D.lam_prev2, 24}, {D.lam_prev3, 24}, {D.Qe, 72}, {D.logz, 8}, {D.logz_in, 8}, {D.mat_id, 4},
                  {D.newton_it, 4}, {D.mgid, 8}};
    for (auto &f : fields)
        if ((e = compact_array(f.p, nm, f.row, keep, newidx, nn_new, tmp, s, launches)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(D.failed, 0, (size_t)nm, s)) != cudaSuccess) return e;
    D.nm = nn_new;
    return cudaSuccess;
}

// Remove nodes that belong to no support (influence count 0). Runs after the LME kernel, so the
// node-major contribution offsets of the survivors do not move (removed nodes own no pairs).
// Scratch: the linked-cell arrays and node positions in cell order (rebuilt next step).
cudaError_t remove_orphan_nodes(Dev &D, int32_t *scan_tmp, int64_t *n_drop_host, cudaStream_t s, long long *launches)
{
    const int64_t nn = D.nn;
    int32_t *n_drop = D.node_cell;                    // nn ints
    int32_t *keep = D.node_rank;                      // nn ints
    int32_t *newid = D.cell_start;                    // >= nn + 1 ints
    void *tmp = (void *)D.spos;                       // 32 nn bytes
    cudaError_t e = cudaMemsetAsync(n_drop, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    // keep flags are written to node_rank; the drop counter lives in node_cell[0]
    k_keep_from_count<<<cblocks(nn, 256), 256, 0, s>>>(D.ncount, nn, keep, n_drop);
    if (launches) *launches += 1;
    int32_t nd = 0;
    if ((e = cudaMemcpyAsync(&nd, n_drop, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *n_drop_host = nd;
    if (nd == 0) return cudaSuccess;
    if ((e = launch_exclusive_scan_tmp(keep, newid, nn, scan_tmp, s, launches)) != cudaSuccess) return e;
    const int64_t nn_new = nn - nd;
    k_remap_ids<<<cblocks(D.nm * (int64_t)D.S, 256), 256, 0, s>>>(D.ids, D.cnt, D.nm, D.S, newid);
    if (launches) *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    struct F {
        void *p;
        size_t row;
    } fields[] = {{D.x, 32}, {D.x_prev, 32}, {D.du, 32}, {D.mr, 32}, {D.du32, 16}, {D.ngid, 8},
                  {D.ncount, 4}, {D.noff, 4}};
    for (auto &f : fields)
        if ((e = compact_array(f.p, nn, f.row, keep, newid, nn_new, tmp, s, launches)) != cudaSuccess) return e;
    k_gather_bytes<<<cblocks(nn, 256), 256, 0, s>>>(D.nflags, (uint8_t *)tmp, nn, keep, newid);
    if (launches) *launches += 1;
    if ((e = cudaMemcpyAsync(D.nflags, tmp, (size_t)nn_new, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
    // the total pair count (offset past the last node) moves to the new end
    if ((e = cudaMemcpyAsync(D.noff + nn_new, D.noff + nn, sizeof(int32_t), cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
        return e;
    D.nn = nn_new;
    return cudaSuccess;
}

// one warp per MP flagged in lme_fail: the new node at slot nn + slot[p] (see insert_nodes)
__global__ void k_insert_nodes(const Dev D, const int32_t *slot, int64_t next_gid)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = w0; p < D.nm; p += nw) {
        if (!D.lme_fail[p]) continue;             // warp-uniform
        const int n = D.cnt[p];
        const int32_t *row = D.ids + p * (int64_t)D.S;
        double c0 = 0.0, c1 = 0.0, c2 = 0.0;
        for (int k = lane; k < n; k += kWarp) {
            const double4_32a a = D.x[row[k]];
            c0 += a.x; c1 += a.y; c2 += a.z;
        }
        c0 = warp_sum(c0); c1 = warp_sum(c1); c2 = warp_sum(c2);
        if (lane != 0) continue;
        const double4_32a xp = D.xp[p], xq = D.xp_prev[p];
        const double u0 = xp.x - c0 / (double)n, u1 = xp.y - c1 / (double)n, u2 = xp.z - c2 / (double)n;
        const double len = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        const int64_t i = D.nn + slot[p];
        if (!(len > 1e-12 * D.h) || n <= 0) {
            raise_error(D.err, OTM_ERR_LME_NOCONV, D.mgid[p]);
            continue;
        }
        const double x0 = xp.x + D.h * (u0 / len), x1 = xp.y + D.h * (u1 / len), x2 = xp.z + D.h * (u2 / len);
        const double d0 = xp.x - xq.x, d1 = xp.y - xq.y, d2 = xp.z - xq.z;
        D.x[i] = make_double4_32a(x0, x1, x2, 0.0);
        D.x_prev[i] = make_double4_32a(x0 - d0, x1 - d1, x2 - d2, 0.0);
        D.du[i] = make_double4_32a(d0, d1, d2, 0.0);
        D.du32[i] = make_float4((float)d0, (float)d1, (float)d2, 0.f);
        D.mr[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        D.nflags[i] = 0;
        D.ngid[i] = next_gid + slot[p];
        D.ncount[i] = 0;
    }
}

__global__ void k_keep_flag(const uint8_t *flag, int64_t n, int32_t *keep)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        keep[i] = flag[i] ? 1 : 0;
}

// Append one node per MP flagged in D.lme_fail (n_fail of them; the caller checked the slots).
// Scratch: the node-major contribution region, which the LME kernel rewrites after the repeated
// search. D.nn grows by n_fail.
cudaError_t insert_nodes(Dev &D, int32_t *scan_tmp, int64_t n_fail, int64_t next_gid, cudaStream_t s,
                         long long *launches)
{
    const int64_t nm = D.nm;
    int32_t *keep = D.precision == OTM_PRECISION_MIXED ? (int32_t *)D.contrib32 : (int32_t *)D.contrib64;
    int32_t *slot = keep + ((nm + 63) / 64) * 64;
    k_keep_flag<<<cblocks(nm, 256), 256, 0, s>>>(D.lme_fail, nm, keep);
    if (launches) *launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_exclusive_scan_tmp(keep, slot, nm, scan_tmp, s, launches)) != cudaSuccess) return e;
    k_insert_nodes<<<cblocks(nm * 32, 256), 256, 0, s>>>(D, slot, next_gid);
    if (launches) *launches += 1;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    D.nn += n_fail;
    return cudaSuccess;
}

__global__ void k_raise_flagged(const Dev D, int code)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < D.nm; p += (int64_t)gridDim.x * blockDim.x)
        if (D.lme_fail[p]) raise_error(D.err, code, D.mgid[p]);
}

// the error `code` for every flagged MP (the smallest ID wins)
cudaError_t raise_flagged(const Dev &D, int code, cudaStream_t s, long long *launches)
{
    k_raise_flagged<<<cblocks(D.nm, 256), 256, 0, s>>>(D, code);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace otm
