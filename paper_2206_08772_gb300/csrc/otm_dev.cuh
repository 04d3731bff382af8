// otm_dev.cuh -- device-side state and helpers shared by the OTM kernels (sm_103a).
//
// Layout in HBM (all carved from the caller's workspace, see otm_api.cu):
//   nodes  : x, x_prev, du (double4_32a, w unused), du32 (float4, mixed path), mass/force (double4_32a),
//            flags, influence counts, node-major offsets, linked-cell arrays
//   MPs    : x_p (double4_32a), F, dF (9), b^e, sigma (6), vol, mass, ebar, T, rate, J, lambda (3),
//            material, support count, Newton iterations, failure flag, original ID
//   pairs  : padded MP-major rows of S slots: node ID (int32), shape (double4_32a: N, e = N d),
//            rank in the node's influence list (uint16); node-major contributions
//            (double4_32a or float4: m_p N, -v sigma grad N) at noff[node] + rank
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/otm.h"

namespace otm {

constexpr int kWarp = 32;
constexpr int kMaxS = 1024;          // largest per-MP support capacity
constexpr int kNodeSegMax = 4096;    // largest influence list reduced in shared memory
constexpr int kSearchWarps = 4;      // warps per block in the search + LME kernel
constexpr int kNodeWarps = 4;        // warps per block in the node kernel

struct GridDev {
    unsigned long long key_lo[3];    // ordered-integer keys of the node bounding box
    unsigned long long key_hi[3];
    double origin[3];
    int dims[3];
    int n_cells;                     // 0 when the grid is invalid (error raised)
};

// where the LME solve of k_lme starts, and what it records:
//   kLmePlain: at the stored lambda; lam_prev := the solution (initial supports, refresh)
//   kLmeStep : at 4 lambda_n - 6 lambda_{n-1} + 4 lambda_{n-2} - lambda_{n-3} (cubic extrapolation
//              in time); lam_prev3, lam_prev2, lam_prev := lambda_{n-2}, lambda_{n-1}, lambda_n
//   kLmeKeep : at the stored lambda; lam_prev kept (snapshot restore)
//   kLmeRetry: the repeated solve after node insertion: as kLmeKeep, except that the MPs flagged
//              in lme_fail (solved again from lambda_n) restart their history as in kLmePlain
constexpr int kLmePlain = 0, kLmeStep = 1, kLmeKeep = 2, kLmeRetry = 3;

// constants of the support search, derived once on the host from the cell size and r_s^2
struct SearchConst {
    double cell, rs2;
    float cf;              // cell size in FP32 (round to nearest)
    float rs;              // sqrt(rs2) in FP32 (correctly rounded sqrt, then round to nearest)
    float rs2_rd, rs2_ru;  // rs2 rounded down / up to FP32
};

SearchConst make_search_const(double cell, double rs2);

struct Dev {
    // sizes and parameters
    int64_t nn, nm;
    int S;                           // pair slots per MP
    int precision;
    int max_cells;
    double h, beta, rs2, cell, dt, tol_abs, eps_stab;
    SearchConst sc;
    int max_newton;
    int wall, tool, allow_erode;
    int insert_mode;                 // 1: an MP whose LME solve fails is flagged for node insertion
    int lme_mode;                    // start of the LME solve, see k_lme (kLmePlain / kLmeStep / kLmeKeep)
    double wall_p[3], wall_n[3];
    double tool_x0, tool_tip_y, tool_rake, tool_clear, tool_v, friction;
    otm_material mat[4];

    // nodes
    double4_32a *x, *x_prev, *du, *mr;   // mr = (mass, force xyz) of the last node update
    float4 *du32;
    uint8_t *nflags;
    int64_t *ngid;
    int32_t *ncount, *noff;          // influence counts (atomics) and node-major offsets
    // linked cell
    GridDev *grid;
    int32_t *cell_count, *cell_start, *node_cell, *node_rank, *sorted;
    double4_32a *spos;               // node positions in (cell, ID) order, w = ID bits
    float4 *spos32;                  // the same relative to the grid origin in FP32, w = ID bits
    // material points
    double4_32a *xp, *xp_prev;       // position and the position of the previous step
    double *F, *dF, *be, *sig, *vol, *mass, *ebar, *T, *rate, *lam, *logz, *logz_in;
    double *lam_prev, *lam_prev2, *lam_prev3;   // lambda of the three steps before (start extrapolation)
    double *Qe;                      // eigenvectors of b^e from the last return map (9, row-major)
    double *Kinv;                    // J^-1 of the last LME solve (6: xx, yy, zz, xy, yz, xz), see k_lme
    int32_t *mat_id, *cnt, *newton_it;
    uint8_t *failed;                 // fracture flags of the step
    uint8_t *lme_fail;               // LME failures of the step (node insertion)
    int32_t *n_fail;                 // their count
    int32_t *lme_defer;              // MPs whose support exceeds k_lme's shared-memory rows
    int32_t *n_defer;                // their count (k_lme_wide solves them)
    int32_t *flag;                   // one int of scratch for host-read checks (argument validation)
    int64_t *mgid;
    // pairs: MP-major padded rows (ids, shape, rank) and node-major contributions
    int32_t *ids;
    double4_32a *shape;
    double4_32a *contrib64;
    float4 *contrib32;
    uint16_t *rank;
    // status: (first offending id << 8) | (-code), atomicMin
    unsigned long long *err;
    int *emax;                       // largest binary exponent of the mass / force terms (2 ints)
    char *stage;                     // staging for state transfers of pitched fields
    size_t stage_bytes;
};

// scratch of the stand-alone support search (carved from caller memory)
struct SearchScratch {
    GridDev *g;
    double4_32a *x4, *spos;
    float4 *spos32;
    int32_t *cell_count, *cell_start, *node_cell, *node_rank, *sorted;
    unsigned long long *err;
    int max_cells;
};

// adjoint state and the copies of state n used by one backward step (otm_adjoint.cu)
struct AdjDev {
    // adjoint state (of state n+1 on entry, of state n on exit)
    double4_32a *xb, *dub, *rb;        // nodes; rb = (dL/dr_I, dL/dm_I)
    double *Fb, *beb, *ebb, *Tb, *vb, *sigb, *dFb, *thb;   // MPs (thb: 5 per MP, accumulated)
    double4_32a *xpb;
    double4_32a *pb_cur, *pb_prev;     // pairs: (dL/dN, dL/dgradN) of shape n+1 / shape n
    // copies of state n taken before the step is recomputed
    double4_32a *du_n;
    double *F_n, *be_n, *ebar_n, *T_n, *vol_n, *sig_n;
    double4_32a *shape_n;              // shape rows (N, N d) of state n
    double4_32a *shape_next;           // shape rows of state n+1 kept from the previous backward step
    double *K_n, *K_next;              // the matching J^-1 per MP (grad N_a = -J^-1 N_a d_a)
    int32_t *ids_n, *cnt_n, *noff_n;
    uint16_t *rank_n;
    // per-pair node contributions in node-major order
    double4_32a *sc1, *sc3a, *sc3b;
};


// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void raise_error(unsigned long long *err, int code, long long id)
{
    unsigned long long key = ((unsigned long long)id << 8) | (unsigned long long)((-code) & 0xff);
    atomicMin(err, key);
}

__device__ __forceinline__ bool has_error(const unsigned long long *err)
{
    return *((volatile const unsigned long long *)err) != ~0ULL;
}

// order-preserving map of doubles to unsigned 64-bit integers (for exact min/max atomics)
__device__ __forceinline__ unsigned long long dkey(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

__device__ __forceinline__ double dkey_inv(unsigned long long k)
{
    unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Reduce-scatter of 16 per-lane values over a warp in 16 additions per lane (instead of 5 per
// value): after it, lanes 2j and 2j+1 hold the warp total of value j. Unused values may be 0.
__device__ __forceinline__ double warp_reduce_scatter16(const double (&v)[16], int lane)
{
    double a[8], b[4], c[2], d;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const bool up = lane & 16;
        const double mine = up ? v[8 + i] : v[i], other = up ? v[i] : v[8 + i];
        a[i] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const bool up = lane & 8;
        const double mine = up ? a[4 + i] : a[i], other = up ? a[i] : a[4 + i];
        b[i] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const bool up = lane & 4;
        const double mine = up ? b[2 + i] : b[i], other = up ? b[i] : b[2 + i];
        c[i] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
    }
    {
        const bool up = lane & 2;
        const double mine = up ? c[1] : c[0], other = up ? c[0] : c[1];
        d = mine + __shfl_xor_sync(0xffffffffu, other, 2);
    }
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// Reduce-scatter of 12 per-lane values in 13 additions per lane. Afterwards lane L holds the
// warp total of value rs12_value(L) = 6 [L & 16] + 3 [L & 8] + (1 if L & 2, else 2 if L & 4,
// else 0); every value is held by lane pairs (2k, 2k+1), and rs12_writer(L) picks one lane per
// value.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter12(const T (&v)[12], int lane)
{
    T a[6], b[3];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const bool up = lane & 16;
        const T mine = up ? v[6 + i] : v[i], other = up ? v[i] : v[6 + i];
        a[i] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const bool up = lane & 8;
        const T mine = up ? a[3 + i] : a[i], other = up ? a[i] : a[3 + i];
        b[i] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
    }
    const bool up4 = lane & 4;
    const T c0 = (up4 ? b[2] : b[0]) + __shfl_xor_sync(0xffffffffu, up4 ? b[0] : b[2], 4);
    const T c1 = b[1] + __shfl_xor_sync(0xffffffffu, b[1], 4);
    const bool up2 = lane & 2;
    const T d = (up2 ? c1 : c0) + __shfl_xor_sync(0xffffffffu, up2 ? c0 : c1, 2);
    return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

// Reduce-scatter of 10 per-lane values in 12 additions per lane. Afterwards lane L holds the
// warp total of value rs10_value(L); rs10_writer(L) picks one lane per value, and value j can
// be read from lane {0, 2, 4, 8, 10, 16, 18, 20, 24, 26}[j].
__device__ __forceinline__ double warp_reduce_scatter10(const double (&v)[10], int lane)
{
    double a[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const bool up = lane & 16;
        const double mine = up ? v[5 + i] : v[i], other = up ? v[i] : v[5 + i];
        a[i] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    }
    const bool up8 = lane & 8;
    const double b0 = (up8 ? a[3] : a[0]) + __shfl_xor_sync(0xffffffffu, up8 ? a[0] : a[3], 8);
    const double b1 = (up8 ? a[4] : a[1]) + __shfl_xor_sync(0xffffffffu, up8 ? a[1] : a[4], 8);
    const double b2 = a[2] + __shfl_xor_sync(0xffffffffu, a[2], 8);
    const bool up4 = lane & 4;
    const double c0 = (up4 ? b2 : b0) + __shfl_xor_sync(0xffffffffu, up4 ? b0 : b2, 4);
    const double c1 = b1 + __shfl_xor_sync(0xffffffffu, b1, 4);
    const bool up2 = lane & 2;
    const double dd = (up2 ? c1 : c0) + __shfl_xor_sync(0xffffffffu, up2 ? c0 : c1, 2);
    return dd + __shfl_xor_sync(0xffffffffu, dd, 1);
}

__device__ __forceinline__ int rs10_value(int lane)
{
    const int base = (lane & 16) ? 5 : 0;
    if (lane & 2) return base + ((lane & 8) ? 4 : 1);
    return (lane & 4) ? base + 2 : base + ((lane & 8) ? 3 : 0);
}

__device__ __forceinline__ bool rs10_writer(int lane)
{
    return (lane & 1) == 0 && (lane & 14) != 12 && (lane & 6) != 6;
}

__device__ __forceinline__ int rs12_value(int lane)
{
    return ((lane & 16) ? 6 : 0) + ((lane & 8) ? 3 : 0) + ((lane & 2) ? 1 : ((lane & 4) ? 2 : 0));
}

__device__ __forceinline__ bool rs12_writer(int lane) { return (lane & 1) == 0 && (lane & 6) != 6; }

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// linked-cell coordinate: floor((x - o) / c) in correctly rounded FP64 (bit-identical to any
// IEEE implementation of the same expression), optionally clamped to the grid.
__device__ __forceinline__ int cell_coord(double x, double o, double c, int n, bool clamp)
{
    double f = floor(__ddiv_rn(__dsub_rn(x, o), c));
    if (clamp) {
        f = fmin(fmax(f, 0.0), (double)(n - 1));
    } else {
        f = fmin(fmax(f, -4.0), (double)(n + 3));
    }
    return (int)f;
}

// |a - b|^2 with the fixed order ((dx*dx) + (dy*dy)) + (dz*dz) and no contraction
__device__ __forceinline__ double dist2_exact(double ax, double ay, double az, double bx, double by,
                                             double bz)
{
    double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// bitonic sort (ascending) of a[0..n2) in shared memory by one warp; n2 a power of two
template <typename T>
__device__ __forceinline__ void warp_bitonic_sort(T *a, int n2, int lane)
{
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = lane; i < n2; i += kWarp) {
                int ixj = i ^ j;
                if (ixj > i) {
                    T ai = a[i], aj = a[ixj];
                    bool up = ((i & k) == 0);
                    if ((ai > aj) == up) {
                        a[i] = aj;
                        a[ixj] = ai;
                    }
                }
            }
            __syncwarp();
        }
    }
}

__host__ __device__ __forceinline__ int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// ------------------------------------------------------------------ host-side launchers
// Each returns cudaGetLastError() of its launches; `launches` counts kernels enqueued.
cudaError_t launch_grid_build(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_search(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_kin_search(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_lme(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_node_offsets(const Dev &D, int32_t *tmp, cudaStream_t s, long long *launches);
cudaError_t exp_table_setup(bool verify = false);
cudaError_t launch_exp_selftest(const double *x, int64_t n, double *mine, double *ref, cudaStream_t s);
cudaError_t launch_node_update(const Dev &D, double t_next, cudaStream_t s, long long *launches);
cudaError_t launch_rows_to_dense(const void *src, size_t pitch, size_t width, int64_t rows, void *dst, cudaStream_t s);
cudaError_t launch_rows_from_dense(const void *src, size_t pitch, size_t width, int64_t rows, void *dst,
                                   cudaStream_t s);
cudaError_t launch_pack3to4(const double *x3, int64_t n, double4_32a *x4, cudaStream_t s, long long *launches);
cudaError_t launch_init_state(const Dev &D, double T0, cudaStream_t s, long long *launches);
cudaError_t launch_du_to_f32(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_kinematics(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_return_map(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_exclusive_scan_tmp(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp,
                                      cudaStream_t s, long long *launches);
size_t scan_tmp_ints(int64_t n);
bool carve_search_scratch(void *base, size_t bytes, int64_t nn, SearchScratch *S);
cudaError_t build_search_grid(const double *node_x, int64_t nn, double cell, SearchScratch *S,
                              double *grid_out, cudaStream_t s);
size_t lme_smem_bytes(int S, int warps);
cudaError_t launch_adjoint_backward(const Dev &D, const AdjDev &A, cudaStream_t s, long long *launches);
cudaError_t launch_rebuild_ranks(const Dev &D, cudaStream_t s, long long *launches);
cudaError_t launch_csr_gather(const Dev &D, const int32_t *off, int32_t *ids, cudaStream_t s, long long *launches);
cudaError_t launch_csr_check(const int32_t *off, const int32_t *ids, int64_t nm, int S, int64_t len, int64_t nn,
                             int32_t *bad, cudaStream_t s, long long *launches);
cudaError_t launch_csr_scatter(const Dev &D, const int32_t *off, const int32_t *ids, cudaStream_t s,
                               long long *launches);
cudaError_t insert_nodes(Dev &D, int32_t *scan_tmp, int64_t n_fail, int64_t next_gid, cudaStream_t s,
                         long long *launches);
cudaError_t raise_flagged(const Dev &D, int code, cudaStream_t s, long long *launches);
cudaError_t erode_mps(Dev &D, int32_t *scan_tmp, int64_t *n_drop_host, cudaStream_t s, long long *launches);
cudaError_t remove_orphan_nodes(Dev &D, int32_t *scan_tmp, int64_t *n_drop_host, cudaStream_t s,
                                long long *launches);

// stand-alone entry points reuse these
cudaError_t launch_search_only(const double *node_x, int64_t nn, const double *mp_x, int64_t nm,
                               double rs2, double cell, int S, int32_t *ids, int32_t *counts,
                               void *scratch, size_t scratch_bytes, double *grid_out,
                               int32_t *status, cudaStream_t s);
size_t search_scratch_bytes(int64_t nn);
cudaError_t launch_lme_only(const double *node_x, const double *mp_x, int64_t nm,
                            const int32_t *ids, const int32_t *counts, int S, double beta,
                            double tol_abs, int max_newton, double *lam, double *shape,
                            int32_t *iters, int32_t *status, cudaStream_t s);
cudaError_t launch_return_map_only(const otm_material *mat, double dt, int64_t nm, const double *dF,
                                   const double *F_new, double *be, double *ebar, double *T,
                                   double *sigma, double *rate, uint8_t *failed, int32_t *status,
                                   cudaStream_t s);

}  // namespace otm
