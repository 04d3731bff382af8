// otm_grid.cu -- linked-cell grid as a device counting sort (Algorithm 3, step 1), the
// node-major (influence-domain) permutation of the support pairs, and integer scans.
//
// Grid: origin = componentwise minimum of the node positions (exact, ordered-integer atomics),
// dims = floor((max - min) / cell) + 1 per axis, cell id = (iz * ny + iy) * nx + ix.
// Nodes are counted into cells with integer atomics, the counts are scanned, the nodes are
// scattered, and each cell's short list is sorted by node ID, so the final (cell, ID) order is
// unique whatever order the atomics ran in.
#include "otm_dev.cuh"

namespace otm {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------------------ bounding box
__global__ void k_bbox_init(GridDev *g)
{
    if (threadIdx.x < 3) {
        g->key_lo[threadIdx.x] = ~0ULL;
        g->key_hi[threadIdx.x] = 0ULL;
    }
}

__global__ void k_bbox(const double4_32a *__restrict__ x, int64_t n, GridDev *g)
{
    unsigned long long lo[3] = {~0ULL, ~0ULL, ~0ULL}, hi[3] = {0ULL, 0ULL, 0ULL};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double4_32a p = x[i];
        unsigned long long k0 = dkey(p.x), k1 = dkey(p.y), k2 = dkey(p.z);
        lo[0] = min(lo[0], k0); hi[0] = max(hi[0], k0);
        lo[1] = min(lo[1], k1); hi[1] = max(hi[1], k1);
        lo[2] = min(lo[2], k2); hi[2] = max(hi[2], k2);
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = min(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = max(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; d++) {
            atomicMin(&g->key_lo[d], lo[d]);
            atomicMax(&g->key_hi[d], hi[d]);
        }
    }
}

__global__ void k_grid_setup(GridDev *g, double cell, int max_cells, unsigned long long *err)
{
    if (threadIdx.x != 0) return;
    // the cell count is formed in FP64: each axis is at most max_cells (< 2^31), so the product
    // is below 2^93 and cannot wrap, and any product above max_cells is reported as capacity
    double total = 1.0;
    bool ok = true;
    for (int d = 0; d < 3; d++) {
        double lo = dkey_inv(g->key_lo[d]), hi = dkey_inv(g->key_hi[d]);
        g->origin[d] = lo;
        if (!isfinite(lo) || !isfinite(hi)) {
            ok = false;
            raise_error(err, OTM_ERR_NONFINITE, 0);
            g->dims[d] = 0;
            continue;
        }
        double nd = floor(__ddiv_rn(__dsub_rn(hi, lo), cell)) + 1.0;
        if (!(nd <= (double)max_cells)) {
            ok = false;
            nd = 0;
        }
        g->dims[d] = (int)nd;
        total *= nd;
    }
    if (ok && !(total <= (double)max_cells)) ok = false;
    if (!ok) raise_error(err, OTM_ERR_CAPACITY, 0);
    g->n_cells = ok ? (int)total : 0;
}

// ------------------------------------------------------------------------ counting sort
__global__ void k_cell_zero(int32_t *cell_count, const GridDev *g)
{
    int n = g->n_cells;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cell_count[i] = 0;
}

__global__ void k_cell_count(const double4_32a *__restrict__ x, int64_t n, const GridDev *g, double cell,
                             int32_t *cell_count, int32_t *node_cell, int32_t *node_rank)
{
    if (g->n_cells == 0) return;
    const double o0 = g->origin[0], o1 = g->origin[1], o2 = g->origin[2];
    const int n0 = g->dims[0], n1 = g->dims[1], n2 = g->dims[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double4_32a p = x[i];
        int ix = cell_coord(p.x, o0, cell, n0, true);
        int iy = cell_coord(p.y, o1, cell, n1, true);
        int iz = cell_coord(p.z, o2, cell, n2, true);
        int c = (iz * n1 + iy) * n0 + ix;
        node_cell[i] = c;
        node_rank[i] = atomicAdd(&cell_count[c], 1);
    }
}

// single-block exclusive scan of cell_count[0..n_cells) into cell_start[0..n_cells]
__global__ void __launch_bounds__(kScanThreads) k_scan_cells(const int32_t *count, int32_t *start,
                                                             const GridDev *g)
{
    __shared__ int32_t wsum[kWarp];
    __shared__ int32_t carry_s;
    const int n = g->n_cells;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < n; base += kScanTile) {
        int v[kScanItems];
        int tsum = 0;
        int i0 = base + threadIdx.x * kScanItems;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            v[k] = (i0 + k < n) ? count[i0 + k] : 0;
            tsum += v[k];
        }
        int incl = tsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int ws = wsum[lane];
            int wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;   // exclusive warp offsets
        }
        __syncthreads();
        int run = carry_s + wsum[warp] + incl - tsum;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (i0 + k < n) start[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry_s = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry_s;
}

__global__ void k_cell_fill(int64_t n, const int32_t *node_cell, const int32_t *node_rank,
                            const int32_t *cell_start, int32_t *sorted, const GridDev *g)
{
    if (g->n_cells == 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        sorted[cell_start[node_cell[i]] + node_rank[i]] = (int32_t)i;
}

// each cell's (short) node list sorted by ID: insertion sort, one thread per cell
__global__ void k_cell_sort(int32_t *sorted, const int32_t *cell_start, const GridDev *g)
{
    const int n = g->n_cells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        int b = cell_start[c], e = cell_start[c + 1];
        for (int i = b + 1; i < e; i++) {
            int v = sorted[i];
            int j = i - 1;
            while (j >= b && sorted[j] > v) {
                sorted[j + 1] = sorted[j];
                j--;
            }
            sorted[j + 1] = v;
        }
    }
}

__global__ void k_spos(int64_t n, const int32_t *sorted, const double4_32a *__restrict__ x, double4_32a *spos,
                       float4 *spos32, const GridDev *g)
{
    if (g->n_cells == 0) return;
    const double o0 = g->origin[0], o1 = g->origin[1], o2 = g->origin[2];
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int id = sorted[s];
        double4_32a p = x[id];
        p.w = __longlong_as_double((long long)id);
        spos[s] = p;
        spos32[s] = make_float4((float)(p.x - o0), (float)(p.y - o1), (float)(p.z - o2), __int_as_float(id));
    }
}

static int grid_blocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

static cudaError_t grid_build_impl(const double4_32a *x, int64_t nn, double cell, int max_cells, GridDev *g,
                                   int32_t *cell_count, int32_t *cell_start, int32_t *node_cell,
                                   int32_t *node_rank, int32_t *sorted, double4_32a *spos, float4 *spos32,
                                   unsigned long long *err, cudaStream_t s, long long *launches)
{
    k_bbox_init<<<1, 32, 0, s>>>(g);
    k_bbox<<<grid_blocks(nn, 256), 256, 0, s>>>(x, nn, g);
    k_grid_setup<<<1, 32, 0, s>>>(g, cell, max_cells, err);
    k_cell_zero<<<grid_blocks(max_cells, 256), 256, 0, s>>>(cell_count, g);
    k_cell_count<<<grid_blocks(nn, 256), 256, 0, s>>>(x, nn, g, cell, cell_count, node_cell, node_rank);
    k_scan_cells<<<1, kScanThreads, 0, s>>>(cell_count, cell_start, g);
    k_cell_fill<<<grid_blocks(nn, 256), 256, 0, s>>>(nn, node_cell, node_rank, cell_start, sorted, g);
    k_cell_sort<<<grid_blocks(max_cells, 128), 128, 0, s>>>(sorted, cell_start, g);
    k_spos<<<grid_blocks(nn, 256), 256, 0, s>>>(nn, sorted, x, spos, spos32, g);
    if (launches) *launches += 9;
    return cudaGetLastError();
}

cudaError_t launch_grid_build(const Dev &D, cudaStream_t s, long long *launches)
{
    return grid_build_impl(D.x, D.nn, D.cell, D.max_cells, D.grid, D.cell_count, D.cell_start,
                           D.node_cell, D.node_rank, D.sorted, D.spos, D.spos32, D.err, s, launches);
}

// ------------------------------------------------------------------------ generic scan
// Exclusive scan of n int32 values into out[0..n] (out[n] = total). Three phases: tile sums,
// a single-block scan of the tile sums, and a rescan of every tile with its offset.
__global__ void __launch_bounds__(kScanThreads) k_tile_sums(const int32_t *in, int64_t n, int32_t *tile_sum)
{
    __shared__ int32_t wsum[kWarp];
    int64_t i0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int t = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) t += (i0 + k < n) ? in[i0 + k] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = wsum[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) tile_sum[blockIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(int32_t *tile_sum, int64_t ntiles)
{
    __shared__ int32_t wsum[kWarp];
    __shared__ int32_t carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += kScanThreads) {
        int64_t i = base + threadIdx.x;
        int v = (i < ntiles) ? tile_sum[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int ws = wsum[lane], wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - ws;
        }
        __syncthreads();
        int excl = carry_s + wsum[warp] + incl - v;
        if (i < ntiles) tile_sum[i] = excl;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry_s = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) tile_sum[ntiles] = carry_s;
}

__global__ void __launch_bounds__(kScanThreads) k_tile_rescan(const int32_t *in, int64_t n,
                                                              const int32_t *tile_off, int32_t *out,
                                                              int64_t ntiles)
{
    __shared__ int32_t wsum[kWarp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t i0 = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = (i0 + k < n) ? in[i0 + k] : 0;
        tsum += v[k];
    }
    int incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int ws = wsum[lane], wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - ws;
    }
    __syncthreads();
    int run = tile_off[blockIdx.x] + wsum[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (i0 + k < n) out[i0 + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_off[ntiles];
}

// tile scratch: ntiles + 1 ints directly after out[n] is not available, so it lives in
// a static-size region of the caller's buffer `tmp`
cudaError_t launch_exclusive_scan_tmp(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp,
                                      cudaStream_t s, long long *launches)
{
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles < 1) ntiles = 1;
    k_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_tile_sums<<<1, kScanThreads, 0, s>>>(tmp, ntiles);
    k_tile_rescan<<<(unsigned)ntiles, kScanThreads, 0, s>>>(in, n, tmp, out, ntiles);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

size_t scan_tmp_ints(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile + 2); }

// ------------------------------------------------------------------------ node-major offsets
// noff = exclusive scan of the influence counts; the LME kernel then writes each pair's
// contribution at noff[node] + rank, so every node's influence list is contiguous.
cudaError_t launch_node_offsets(const Dev &D, int32_t *tmp, cudaStream_t s, long long *launches)
{
    return launch_exclusive_scan_tmp(D.ncount, D.noff, D.nn, tmp, s, launches);
}

// ------------------------------------------------------------------------ stand-alone search scratch
static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

static int search_max_cells(int64_t nn) { return (int)(16 * nn + 65536); }

size_t search_scratch_bytes(int64_t nn)
{
    int mc = search_max_cells(nn);
    size_t b = 0;
    b += align256(sizeof(GridDev));
    b += 2 * align256((size_t)nn * sizeof(double4_32a));
    b += align256((size_t)nn * sizeof(float4));
    b += 2 * align256(((size_t)mc + 1) * sizeof(int32_t));
    b += 3 * align256((size_t)nn * sizeof(int32_t));
    b += align256(sizeof(unsigned long long));
    return b;
}

bool carve_search_scratch(void *base, size_t bytes, int64_t nn, SearchScratch *S)
{
    if (search_scratch_bytes(nn) > bytes) return false;
    char *p = (char *)base;
    int mc = search_max_cells(nn);
    S->g = (GridDev *)p; p += align256(sizeof(GridDev));
    S->x4 = (double4_32a *)p; p += align256((size_t)nn * sizeof(double4_32a));
    S->spos = (double4_32a *)p; p += align256((size_t)nn * sizeof(double4_32a));
    S->spos32 = (float4 *)p; p += align256((size_t)nn * sizeof(float4));
    S->cell_count = (int32_t *)p; p += align256(((size_t)mc + 1) * sizeof(int32_t));
    S->cell_start = (int32_t *)p; p += align256(((size_t)mc + 1) * sizeof(int32_t));
    S->node_cell = (int32_t *)p; p += align256((size_t)nn * sizeof(int32_t));
    S->node_rank = (int32_t *)p; p += align256((size_t)nn * sizeof(int32_t));
    S->sorted = (int32_t *)p; p += align256((size_t)nn * sizeof(int32_t));
    S->err = (unsigned long long *)p;
    S->max_cells = mc;
    return true;
}

__global__ void k_pack3to4(const double *__restrict__ x3, int64_t n, double4_32a *x4)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x4[i] = make_double4_32a(x3[3 * i], x3[3 * i + 1], x3[3 * i + 2], 0.0);
}

// rows of `width` bytes (a multiple of 8) between a pitched layout and a dense one, 8 bytes per
// thread: a state transfer then moves one contiguous block instead of many short rows
__global__ void k_rows_to_dense(const char *__restrict__ src, size_t pitch, size_t width, int64_t rows,
                                double *__restrict__ dst)
{
    const int64_t words = (int64_t)(width / 8), total = rows * words;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / words, w = t - r * words;
        dst[t] = *(const double *)(src + (size_t)r * pitch + (size_t)w * 8);
    }
}

__global__ void k_rows_from_dense(const double *__restrict__ src, size_t pitch, size_t width, int64_t rows,
                                  char *__restrict__ dst)
{
    const int64_t words = (int64_t)(width / 8), total = rows * words;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / words, w = t - r * words;
        *(double *)(dst + (size_t)r * pitch + (size_t)w * 8) = src[t];
    }
}

cudaError_t launch_rows_to_dense(const void *src, size_t pitch, size_t width, int64_t rows, void *dst, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_rows_to_dense<<<grid_blocks(rows * (int64_t)(width / 8), 256), 256, 0, s>>>((const char *)src, pitch, width,
                                                                                  rows, (double *)dst);
    return cudaGetLastError();
}

cudaError_t launch_rows_from_dense(const void *src, size_t pitch, size_t width, int64_t rows, void *dst,
                                   cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    k_rows_from_dense<<<grid_blocks(rows * (int64_t)(width / 8), 256), 256, 0, s>>>((const double *)src, pitch,
                                                                                    width, rows, (char *)dst);
    return cudaGetLastError();
}

cudaError_t launch_pack3to4(const double *x3, int64_t n, double4_32a *x4, cudaStream_t s, long long *launches)
{
    if (n <= 0) return cudaSuccess;
    k_pack3to4<<<grid_blocks(n, 256), 256, 0, s>>>(x3, n, x4);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// initial state (Algorithm 1, REQUIRE): F = dF = b^e = 1, sigma = 0, ebar = 0, T = T0,
// lambda = 0, original IDs, x_prev = x, du32 = du
__global__ void k_init_state(const Dev D, double T0)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < D.nm;
         p += (int64_t)gridDim.x * blockDim.x) {
        for (int i = 0; i < 9; i++) D.F[9 * p + i] = D.dF[9 * p + i] = (i % 4 == 0) ? 1.0 : 0.0;
        for (int i = 0; i < 6; i++) {
            D.be[6 * p + i] = (i < 3) ? 1.0 : 0.0;
            D.sig[6 * p + i] = 0.0;
        }
        D.ebar[p] = 0.0;
        D.T[p] = T0;
        D.xp_prev[p] = D.xp[p];
        D.rate[p] = 0.0;
        D.lam[3 * p] = D.lam[3 * p + 1] = D.lam[3 * p + 2] = 0.0;
        D.lam_prev[3 * p] = D.lam_prev[3 * p + 1] = D.lam_prev[3 * p + 2] = 0.0;
        D.lam_prev2[3 * p] = D.lam_prev2[3 * p + 1] = D.lam_prev2[3 * p + 2] = 0.0;
        D.lam_prev3[3 * p] = D.lam_prev3[3 * p + 1] = D.lam_prev3[3 * p + 2] = 0.0;
        for (int i = 0; i < 9; i++) D.Qe[9 * p + i] = (i % 4 == 0) ? 1.0 : 0.0;
        D.logz[p] = 0.0;
        D.logz_in[p] = 0.0;
        D.failed[p] = 0;
        D.cnt[p] = 0;
        D.newton_it[p] = 0;
        D.mgid[p] = p;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        D.ngid[i] = i;
        D.x_prev[i] = D.x[i];
        const double4_32a u = D.du[i];
        D.du32[i] = make_float4((float)u.x, (float)u.y, (float)u.z, 0.f);
        D.mr[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
}

__global__ void k_du_to_f32(const Dev D)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D.nn;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double4_32a u = D.du[i];
        D.du32[i] = make_float4((float)u.x, (float)u.y, (float)u.z, 0.f);
    }
}

cudaError_t launch_du_to_f32(const Dev &D, cudaStream_t s, long long *launches)
{
    k_du_to_f32<<<grid_blocks(D.nn, 256), 256, 0, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_init_state(const Dev &D, double T0, cudaStream_t s, long long *launches)
{
    int64_t n = D.nm > D.nn ? D.nm : D.nn;
    k_init_state<<<grid_blocks(n, 256), 256, 0, s>>>(D, T0);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

__global__ void k_grid_out(const GridDev *g, double *out)
{
    if (threadIdx.x < 3) {
        out[threadIdx.x] = g->origin[threadIdx.x];
        out[3 + threadIdx.x] = (double)g->dims[threadIdx.x];
    }
}

cudaError_t build_search_grid(const double *node_x, int64_t nn, double cell, SearchScratch *S,
                              double *grid_out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(S->err, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_pack3to4<<<grid_blocks(nn, 256), 256, 0, s>>>(node_x, nn, S->x4);
    e = grid_build_impl(S->x4, nn, cell, S->max_cells, S->g, S->cell_count, S->cell_start, S->node_cell,
                        S->node_rank, S->sorted, S->spos, S->spos32, S->err, s, nullptr);
    if (e != cudaSuccess) return e;
    if (grid_out) k_grid_out<<<1, 32, 0, s>>>(S->g, grid_out);
    return cudaGetLastError();
}

}  // namespace otm
