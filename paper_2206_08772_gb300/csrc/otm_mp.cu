// otm_mp.cu -- material-point kernels (sm_103a):
//   k_kinematics : Eq. 9-13, warp per MP: x_p = sum N x_I, dF = 1 + sum du_I (x) grad N_I,
//                  F <- dF F, v <- det(dF) v
//   k_return_map : Sec. 4.1 / 4.2, thread per MP: Hencky exponential-map radial return (J2
//                  linear hardening closed form, Johnson-Cook safeguarded Newton), heating,
//                  fracture flag, sigma = tau / J
//   k_search_lme : Algorithm 3 + Eq. 14, warp per MP: linked-cell candidate scan with the
//                  exact FP64 support test, ascending-ID sort, LME Newton for lambda, N and
//                  grad N = -N J^-1 d, per-pair force / mass contributions for the next node
//                  update, influence-list counting (integer atomics)
#include "otm_dev.cuh"

namespace otm {

// ======================================================================== LME (Eq. 14)
struct LmeEval {
    double Z, logZ, rnorm;
    double r0, r1, r2;
    double j00, j11, j22, j01, j12, j02;   // J = sum N d d^T - r r^T
};

// one evaluation at lambda with weights exp(f_a - shift); w[] keeps the unnormalised weights
__device__ __forceinline__ void lme_eval(const double *dx, const double *dy, const double *dz,
                                         const double *q, double *w, int n, double l0, double l1,
                                         double l2, double shift, int lane, LmeEval &E)
{
    double Z = 0, r0 = 0, r1 = 0, r2 = 0, a00 = 0, a11 = 0, a22 = 0, a01 = 0, a12 = 0, a02 = 0;
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double f = q[k] + (l0 * x + l1 * y + l2 * z);
        const double wk = exp(f - shift);
        w[k] = wk;
        Z += wk;
        const double wx = wk * x, wy = wk * y, wz = wk * z;
        r0 += wx; r1 += wy; r2 += wz;
        a00 += wx * x; a11 += wy * y; a22 += wz * z;
        a01 += wx * y; a12 += wy * z; a02 += wx * z;
    }
    Z = warp_sum(Z);
    r0 = warp_sum(r0); r1 = warp_sum(r1); r2 = warp_sum(r2);
    a00 = warp_sum(a00); a11 = warp_sum(a11); a22 = warp_sum(a22);
    a01 = warp_sum(a01); a12 = warp_sum(a12); a02 = warp_sum(a02);
    const double iZ = 1.0 / Z;
    E.Z = Z;
    E.logZ = shift + log(Z);
    E.r0 = r0 * iZ; E.r1 = r1 * iZ; E.r2 = r2 * iZ;
    E.j00 = a00 * iZ - E.r0 * E.r0;
    E.j11 = a11 * iZ - E.r1 * E.r1;
    E.j22 = a22 * iZ - E.r2 * E.r2;
    E.j01 = a01 * iZ - E.r0 * E.r1;
    E.j12 = a12 * iZ - E.r1 * E.r2;
    E.j02 = a02 * iZ - E.r0 * E.r2;
    E.rnorm = sqrt(E.r0 * E.r0 + E.r1 * E.r1 + E.r2 * E.r2);
}

__device__ __forceinline__ double lme_fmax(const double *dx, const double *dy, const double *dz,
                                           const double *q, int n, double l0, double l1, double l2,
                                           int lane)
{
    double m = -INFINITY;
    for (int k = lane; k < n; k += kWarp) m = fmax(m, q[k] + (l0 * dx[k] + l1 * dy[k] + l2 * dz[k]));
    return warp_max(m);
}

__device__ __forceinline__ void lme_eval_safe(const double *dx, const double *dy, const double *dz,
                                              const double *q, double *w, int n, double l0, double l1,
                                              double l2, double shift, int lane, LmeEval &E)
{
    lme_eval(dx, dy, dz, q, w, n, l0, l1, l2, shift, lane, E);
    if (!(E.Z > 0.0) || !isfinite(E.Z)) {   // weights over/underflowed: shift by the max exponent
        double fm = lme_fmax(dx, dy, dz, q, n, l0, l1, l2, lane);
        lme_eval(dx, dy, dz, q, w, n, l0, l1, l2, fm, lane, E);
    }
}

// symmetric 3x3 inverse by cofactors; returns false if singular / non-finite
__device__ __forceinline__ bool sym_inv3(double j00, double j11, double j22, double j01, double j12,
                                         double j02, double inv[6])
{
    double c00 = j11 * j22 - j12 * j12;
    double c01 = j02 * j12 - j01 * j22;
    double c02 = j01 * j12 - j02 * j11;
    double c11 = j00 * j22 - j02 * j02;
    double c12 = j01 * j02 - j00 * j12;
    double c22 = j00 * j11 - j01 * j01;
    double det = j00 * c00 + j01 * c01 + j02 * c02;
    if (!(det > 0.0) || !isfinite(det)) return false;
    double id = 1.0 / det;
    inv[0] = c00 * id; inv[1] = c11 * id; inv[2] = c22 * id;
    inv[3] = c01 * id; inv[4] = c12 * id; inv[5] = c02 * id;   // (xx, yy, zz, xy, yz, xz)
    return true;
}

// Damped Newton on the convex log Z(lambda): step -J^-1 r, halved until log Z or |r| drops.
// On return w[] holds the weights of the accepted evaluation E. Warp-uniform.
__device__ int lme_newton(const double *dx, const double *dy, const double *dz, const double *q, double *w,
                          int n, double &l0, double &l1, double &l2, double tol, int max_it, int lane,
                          LmeEval &E, int &iters)
{
    iters = 0;
    if (n <= 0) return OTM_ERR_LME_NOCONV;
    double fm = lme_fmax(dx, dy, dz, q, n, l0, l1, l2, lane);
    lme_eval(dx, dy, dz, q, w, n, l0, l1, l2, fm, lane, E);
    for (;;) {
        if (!isfinite(E.rnorm)) return OTM_ERR_LME_NOCONV;
        if (E.rnorm <= tol) return OTM_OK;
        if (iters >= max_it) return OTM_ERR_LME_NOCONV;
        iters++;
        double inv[6];
        if (!sym_inv3(E.j00, E.j11, E.j22, E.j01, E.j12, E.j02, inv)) return OTM_ERR_LME_NOCONV;
        const double s0 = -(inv[0] * E.r0 + inv[3] * E.r1 + inv[5] * E.r2);
        const double s1 = -(inv[3] * E.r0 + inv[1] * E.r1 + inv[4] * E.r2);
        const double s2 = -(inv[5] * E.r0 + inv[4] * E.r1 + inv[2] * E.r2);
        double t = 1.0;
        bool accepted = false;
        LmeEval Et;
        double m0 = l0, m1 = l1, m2 = l2;
        for (int halving = 0; halving < 40; halving++) {
            m0 = l0 + t * s0; m1 = l1 + t * s1; m2 = l2 + t * s2;
            lme_eval_safe(dx, dy, dz, q, w, n, m0, m1, m2, E.logZ, lane, Et);
            if (isfinite(Et.logZ) && (Et.logZ < E.logZ || Et.rnorm < E.rnorm)) {
                accepted = true;
                break;
            }
            t *= 0.5;
        }
        if (!accepted) return OTM_ERR_LME_NOCONV;
        l0 = m0; l1 = m1; l2 = m2;
        E = Et;
    }
}

// ======================================================================== support search
// Candidate scan of the +-2 cell stencil (rows of 5 cells are contiguous in the sorted node
// array). Accepted IDs go to list[0..min(count, S)); returns the full count. Warp-uniform.
__device__ int warp_support_search(const GridDev *__restrict__ g, const int32_t *__restrict__ cell_start,
                                   const double4_32a *__restrict__ spos, double cell, double rs2, double px,
                                   double py, double pz, int32_t *list, int S, int lane)
{
    if (g->n_cells == 0) return 0;
    const int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int cx = cell_coord(px, g->origin[0], cell, nx, false);
    const int cy = cell_coord(py, g->origin[1], cell, ny, false);
    const int cz = cell_coord(pz, g->origin[2], cell, nz, false);
    const int x0 = max(cx - 2, 0), x1 = min(cx + 2, nx - 1);
    int cnt = 0;
    if (x0 > x1) return 0;
    const int z0 = max(cz - 2, 0), z1 = min(cz + 2, nz - 1);
    const int y0 = max(cy - 2, 0), y1 = min(cy + 2, ny - 1);
    for (int kz = z0; kz <= z1; kz++) {
        for (int ky = y0; ky <= y1; ky++) {
            const int rowc = (kz * ny + ky) * nx;
            const int s0 = cell_start[rowc + x0], s1 = cell_start[rowc + x1 + 1];
            for (int b = s0; b < s1; b += kWarp) {
                const int s = b + lane;
                bool acc = false;
                int id = 0;
                if (s < s1) {
                    const double4_32a a = spos[s];
                    acc = dist2_exact(px, py, pz, a.x, a.y, a.z) <= rs2;
                    id = (int)__double_as_longlong(a.w);
                }
                const unsigned m = __ballot_sync(0xffffffffu, acc);
                if (acc) {
                    const int pos = cnt + __popc(m & ((1u << lane) - 1u));
                    if (pos < S) list[pos] = id;
                }
                cnt += __popc(m);
            }
        }
    }
    return cnt;
}

// unbiased binary exponent (-2000 for zero / subnormal)
__device__ __forceinline__ int fexp64(double v)
{
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7ff);
    return e == 0 ? -2000 : e - 1023;
}

__device__ __forceinline__ int fexp32(float v)
{
    const int e = (int)((__float_as_uint(v) >> 23) & 0xff);
    return e == 0 ? -2000 : e - 127;
}

// per-warp shared-memory layout for search + LME
struct WarpSmem {
    int32_t *list;   // next_pow2(S) ints
    double *dx, *dy, *dz, *q, *w;
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char *base, int S, int warp)
{
    const int P2 = next_pow2(S);
    const size_t per = (size_t)P2 * sizeof(int32_t) + 5 * (size_t)S * sizeof(double);
    unsigned char *b = base + (size_t)warp * per;
    WarpSmem W;
    W.dx = (double *)b;
    W.dy = W.dx + S;
    W.dz = W.dy + S;
    W.q = W.dz + S;
    W.w = W.q + S;
    W.list = (int32_t *)(W.w + S);
    return W;
}

size_t search_lme_smem_bytes(int S, int warps)
{
    return (size_t)warps * ((size_t)next_pow2(S) * sizeof(int32_t) + 5 * (size_t)S * sizeof(double));
}

// ======================================================================== k_search_lme
// mode 0: initialisation (contributions with the current sigma, v); mode 1: a step.
template <bool MIXED>
__global__ void __launch_bounds__(kSearchWarps * kWarp) k_search_lme(const Dev D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    const int S = D.S;
    WarpSmem W = warp_smem(smem_raw, S, warp);
    const double4_32a xp = D.xp[p];

    // ---- Algorithm 3: linked-cell support search at the current configuration
    int cnt = warp_support_search(D.grid, D.cell_start, D.spos, D.cell, D.rs2, xp.x, xp.y, xp.z, W.list, S,
                                  lane);
    if (cnt > S) {
        if (lane == 0) {
            raise_error(D.err, OTM_ERR_CAPACITY, D.mgid[p]);
            D.cnt[p] = 0;
        }
        return;
    }
    const int P2 = next_pow2(max(cnt, 1));
    for (int k = cnt + lane; k < P2; k += kWarp) W.list[k] = 0x7fffffff;
    __syncwarp();
    warp_bitonic_sort(W.list, P2, lane);

    // ---- d_a = x_p - x_a and the prior exponent -beta |d_a|^2
    const double beta = D.beta;
    for (int k = lane; k < cnt; k += kWarp) {
        const double4_32a a = D.x[W.list[k]];
        const double x = xp.x - a.x, y = xp.y - a.y, z = xp.z - a.z;
        W.dx[k] = x; W.dy[k] = y; W.dz[k] = z;
        W.q[k] = -beta * (x * x + y * y + z * z);
    }
    __syncwarp();

    // ---- Eq. 14: Newton for lambda, warm-started from the previous step
    double l0 = D.lam[3 * p], l1 = D.lam[3 * p + 1], l2 = D.lam[3 * p + 2];
    LmeEval E;
    int iters = 0;
    int st = lme_newton(W.dx, W.dy, W.dz, W.q, W.w, cnt, l0, l1, l2, D.tol_abs, D.max_newton, lane, E, iters);
    double inv[6];
    if (st == OTM_OK && !sym_inv3(E.j00, E.j11, E.j22, E.j01, E.j12, E.j02, inv)) st = OTM_ERR_LME_NOCONV;
    if (lane == 0) {
        D.cnt[p] = (st == OTM_OK) ? cnt : 0;
        D.newton_it[p] = iters;
        if (st == OTM_OK) {
            D.lam[3 * p] = l0; D.lam[3 * p + 1] = l1; D.lam[3 * p + 2] = l2;
        } else {
            raise_error(D.err, st, D.mgid[p]);
        }
    }
    if (st != OTM_OK) return;

    // ---- N_a = w_a / Z, grad N_a = -N_a J^-1 d_a; contributions for Eq. 5 of the next step
    const double iZ = 1.0 / E.Z;
    const double mp = D.mass[p], vp = D.vol[p];
    const double *sg = D.sig + 6 * p;
    const double sxx = sg[0], syy = sg[1], szz = sg[2], sxy = sg[3], syz = sg[4], sxz = sg[5];
    const int64_t base = p * (int64_t)S;
    int em = -2000, ef = -2000;   // largest binary exponents of the stored mass / force terms
    for (int k = lane; k < cnt; k += kWarp) {
        const double N = W.w[k] * iZ;
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        const double gx = -N * (inv[0] * x + inv[3] * y + inv[5] * z);
        const double gy = -N * (inv[3] * x + inv[1] * y + inv[4] * z);
        const double gz = -N * (inv[5] * x + inv[4] * y + inv[2] * z);
        const int id = W.list[k];
        D.ids[base + k] = id;
        D.shape[base + k] = make_double4_32a(N, gx, gy, gz);
        const double cm = mp * N;
        const double fx = -vp * (sxx * gx + sxy * gy + sxz * gz);
        const double fy = -vp * (sxy * gx + syy * gy + syz * gz);
        const double fz = -vp * (sxz * gx + syz * gy + szz * gz);
        if (MIXED) {
            const float4 c = make_float4((float)cm, (float)fx, (float)fy, (float)fz);
            D.contrib32[base + k] = c;
            em = max(em, fexp32(c.x));
            ef = max(ef, max(fexp32(c.y), max(fexp32(c.z), fexp32(c.w))));
        } else {
            D.contrib64[base + k] = make_double4_32a(cm, fx, fy, fz);
            em = max(em, fexp64(cm));
            ef = max(ef, max(fexp64(fx), max(fexp64(fy), fexp64(fz))));
        }
        const int r = atomicAdd(&D.ncount[id], 1);
        if (r > 0xffff) raise_error(D.err, OTM_ERR_CAPACITY, D.ngid[id]);
        D.rank[base + k] = (uint16_t)r;
    }
    em = __reduce_max_sync(0xffffffffu, em);
    ef = __reduce_max_sync(0xffffffffu, ef);
    if (lane == 0) {
        atomicMax(&D.emax[0], em);
        atomicMax(&D.emax[1], ef);
    }
}

cudaError_t launch_search_lme(const Dev &D, bool init, cudaStream_t s, long long *launches)
{
    (void)init;
    const size_t smem = search_lme_smem_bytes(D.S, kSearchWarps);
    const unsigned blocks = (unsigned)((D.nm + kSearchWarps - 1) / kSearchWarps);
    if (blocks == 0) return cudaSuccess;
    cudaError_t e;
    if (D.precision == OTM_PRECISION_MIXED) {
        e = cudaFuncSetAttribute(k_search_lme<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_search_lme<true><<<blocks, kSearchWarps * kWarp, smem, s>>>(D);
    } else {
        e = cudaFuncSetAttribute(k_search_lme<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_search_lme<false><<<blocks, kSearchWarps * kWarp, smem, s>>>(D);
    }
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ======================================================================== k_kinematics
template <bool MIXED>
__global__ void __launch_bounds__(128) k_kinematics(const Dev D)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    const int n = D.cnt[p];
    const int64_t base = p * (int64_t)D.S;
    double x0 = 0, x1 = 0, x2 = 0;
    double a00 = 0, a01 = 0, a02 = 0, a10 = 0, a11 = 0, a12 = 0, a20 = 0, a21 = 0, a22 = 0;
    for (int k = lane; k < n; k += kWarp) {
        const int id = D.ids[base + k];
        const double4_32a sh = D.shape[base + k];
        const double4_32a xa = D.x[id];
        double u0, u1, u2;
        if (MIXED) {
            const float4 u = D.du32[id];
            u0 = u.x; u1 = u.y; u2 = u.z;
        } else {
            const double4_32a u = D.du[id];
            u0 = u.x; u1 = u.y; u2 = u.z;
        }
        x0 += sh.x * xa.x; x1 += sh.x * xa.y; x2 += sh.x * xa.z;
        a00 += u0 * sh.y; a01 += u0 * sh.z; a02 += u0 * sh.w;
        a10 += u1 * sh.y; a11 += u1 * sh.z; a12 += u1 * sh.w;
        a20 += u2 * sh.y; a21 += u2 * sh.z; a22 += u2 * sh.w;
    }
    x0 = warp_sum(x0); x1 = warp_sum(x1); x2 = warp_sum(x2);
    a00 = warp_sum(a00); a01 = warp_sum(a01); a02 = warp_sum(a02);
    a10 = warp_sum(a10); a11 = warp_sum(a11); a12 = warp_sum(a12);
    a20 = warp_sum(a20); a21 = warp_sum(a21); a22 = warp_sum(a22);
    if (lane != 0) return;
    const double d[9] = {1.0 + a00, a01, a02, a10, 1.0 + a11, a12, a20, a21, 1.0 + a22};
    const double det = d[0] * (d[4] * d[8] - d[5] * d[7]) - d[1] * (d[3] * d[8] - d[5] * d[6]) +
                       d[2] * (d[3] * d[7] - d[4] * d[6]);
    D.xp[p] = make_double4_32a(x0, x1, x2, 0.0);
    double *dF = D.dF + 9 * p;
    for (int i = 0; i < 9; i++) dF[i] = d[i];
    if (!(det > 0.0)) {
        raise_error(D.err, OTM_ERR_JACOBIAN, D.mgid[p]);
        return;
    }
    double *F = D.F + 9 * p;
    double Fo[9];
    for (int i = 0; i < 9; i++) Fo[i] = F[i];
    double Fn[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            Fn[3 * i + j] = d[3 * i] * Fo[j] + d[3 * i + 1] * Fo[3 + j] + d[3 * i + 2] * Fo[6 + j];
    for (int i = 0; i < 9; i++) F[i] = Fn[i];
    D.vol[p] *= det;
    D.Jdet[p] = Fn[0] * (Fn[4] * Fn[8] - Fn[5] * Fn[7]) - Fn[1] * (Fn[3] * Fn[8] - Fn[5] * Fn[6]) +
                Fn[2] * (Fn[3] * Fn[7] - Fn[4] * Fn[6]);
    if (!isfinite(x0) || !isfinite(x1) || !isfinite(x2)) raise_error(D.err, OTM_ERR_NONFINITE, D.mgid[p]);
}

cudaError_t launch_kinematics(const Dev &D, cudaStream_t s, long long *launches)
{
    const unsigned blocks = (unsigned)((D.nm * 32 + 127) / 128);
    if (blocks == 0) return cudaSuccess;
    if (D.precision == OTM_PRECISION_MIXED)
        k_kinematics<true><<<blocks, 128, 0, s>>>(D);
    else
        k_kinematics<false><<<blocks, 128, 0, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ======================================================================== return map
// cyclic Jacobi (Golub & Van Loan Sec. 8.5) on a symmetric 3x3, rotations applied in place
__device__ void jacobi_sym3(double A[3][3], double V[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) V[i][j] = (i == j) ? 1.0 : 0.0;
    double nrm = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) nrm += A[i][j] * A[i][j];
    nrm = sqrt(nrm);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = sqrt(2.0 * (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2]));
        if (off <= 1e-15 * nrm) break;
        for (int r = 0; r < 3; r++) {
            const int p = (r == 2) ? 1 : 0, q = (r == 0) ? 1 : 2;
            const double apq = A[p][q];
            if (apq == 0.0) continue;
            const double app = A[p][p], aqq = A[q][q];
            const double th = (aqq - app) / (2.0 * apq);
            const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            const int k = 3 - p - q;
            const double akp = A[k][p], akq = A[k][q];
            A[k][p] = A[p][k] = c * akp - s * akq;
            A[k][q] = A[q][k] = s * akp + c * akq;
            A[p][p] = c * c * app - 2.0 * c * s * apq + s * s * aqq;
            A[q][q] = s * s * app + 2.0 * c * s * apq + c * c * aqq;
            A[p][q] = A[q][p] = 0.0;
            for (int i = 0; i < 3; i++) {
                const double vp = V[i][p], vq = V[i][q];
                V[i][p] = c * vp - s * vq;
                V[i][q] = s * vp + c * vq;
            }
        }
    }
}

__device__ __forceinline__ void jc_sigma_y(const otm_material &M, double ebar_n, double x, double dt,
                                           double T, double &sy, double &dsy)
{
    const double ebar = ebar_n + x;
    const double tstar = fmin(fmax((T - M.T_room) / (M.T_melt - M.T_room), 0.0), 1.0);
    const double therm = 1.0 - pow(tstar, M.m);
    const double rstar = (x / dt) / M.eps_dot0;
    double rate = 1.0, drate = 0.0;
    if (rstar > 1.0) {
        rate = 1.0 + M.C * log(rstar);
        drate = M.C / x;
    }
    const double hard = M.A + M.B * pow(ebar, M.n);
    const double dhard = (ebar > 0.0) ? M.B * M.n * pow(ebar, M.n - 1.0) : INFINITY;
    sy = hard * rate * therm;
    dsy = (dhard * rate + hard * drate) * therm;
}

struct RmIn {
    double dF[9], be[6], ebar, T, J;
};
struct RmOut {
    double sig[6], be[6], ebar, T, rate;
    bool failed;
};

// returns OTM_OK or an error code
__device__ int return_map_point(const otm_material &M, double dt, const RmIn &in, RmOut &out)
{
    const double K = M.E / (3.0 * (1.0 - 2.0 * M.nu));
    const double mu = M.E / (2.0 * (1.0 + M.nu));
    // trial b = dF b_n dF^T
    const double b[3][3] = {{in.be[0], in.be[3], in.be[5]}, {in.be[3], in.be[1], in.be[4]},
                            {in.be[5], in.be[4], in.be[2]}};
    double t[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            t[i][j] = in.dF[3 * i] * b[0][j] + in.dF[3 * i + 1] * b[1][j] + in.dF[3 * i + 2] * b[2][j];
    double A[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            A[i][j] = t[i][0] * in.dF[3 * j] + t[i][1] * in.dF[3 * j + 1] + t[i][2] * in.dF[3 * j + 2];
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++) A[i][j] = A[j][i] = 0.5 * (A[i][j] + A[j][i]);
    double Q[3][3];
    jacobi_sym3(A, Q);
    double e[3];
    for (int a = 0; a < 3; a++) {
        if (!(A[a][a] > 0.0)) return OTM_ERR_JACOBIAN;
        e[a] = 0.5 * log(A[a][a]);
    }
    const double tr = e[0] + e[1] + e[2];
    double s[3], sn2 = 0.0;
    for (int a = 0; a < 3; a++) {
        s[a] = 2.0 * mu * (e[a] - tr / 3.0);
        sn2 += s[a] * s[a];
    }
    const double sn = sqrt(sn2);
    const double q_tr = 1.2247448713915890491 * sn;   // sqrt(3/2) |s|
    double dep = 0.0;
    if (M.model == 0) {
        const double f_tr = sn - 0.81649658092772603273 * (M.sigma_y0 + M.H * in.ebar);
        if (f_tr > 0.0) dep = 0.81649658092772603273 * f_tr / (2.0 * mu + 2.0 * M.H / 3.0);
    } else {
        double sy0, dsy0;
        jc_sigma_y(M, in.ebar, 0.0, dt, in.T, sy0, dsy0);
        if (q_tr - sy0 > 0.0) {
            double lo = 0.0, hi = q_tr / (3.0 * mu), x = 0.5 * hi;
            const double tol = 1e-12 * q_tr;
            bool ok = false;
            for (int it = 0; it < 300; it++) {
                double sy, dsy;
                jc_sigma_y(M, in.ebar, x, dt, in.T, sy, dsy);
                const double g = q_tr - 3.0 * mu * x - sy;
                if (fabs(g) <= tol) { ok = true; break; }
                if (g > 0.0) lo = x; else hi = x;
                if (hi - lo <= 4e-16 * hi) { ok = true; break; }
                double xn = x - g / (-3.0 * mu - dsy);
                if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
                x = xn;
            }
            if (!ok) return OTM_ERR_RETURNMAP_NOCONV;
            dep = x;
        }
    }
    const double dgamma = 1.2247448713915890491 * dep;
    const double qn = q_tr - 3.0 * mu * dep;
    double tau[3], eb2[3];
    for (int a = 0; a < 3; a++) {
        const double na = (sn > 0.0) ? s[a] / sn : 0.0;
        e[a] -= dgamma * na;
        tau[a] = K * tr + 2.0 * mu * (e[a] - tr / 3.0);
        eb2[a] = exp(2.0 * e[a]);
    }
    const double iJ = 1.0 / in.J;
    const int I[6] = {0, 1, 2, 0, 1, 0}, Jx[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        const int i = I[c], j = Jx[c];
        double vb = 0.0, vs = 0.0;
        for (int a = 0; a < 3; a++) {
            const double qq = Q[i][a] * Q[j][a];
            vb += eb2[a] * qq;
            vs += tau[a] * qq;
        }
        out.be[c] = vb;
        out.sig[c] = vs * iJ;
    }
    out.ebar = in.ebar + dep;
    out.rate = dep / dt;
    out.T = in.T;
    if (M.model == 1 && M.chi > 0.0 && dep > 0.0) out.T = in.T + M.chi * qn * dep / (M.rho0 * M.cp);
    out.failed = false;
    if (M.model == 1 && M.fracture && out.ebar > 0.0) {
        const double pr = K * tr * iJ;
        const double sv = qn * iJ;
        const double eta = (sv > 0.0) ? pr / sv : 0.0;
        const double rstar = out.rate / M.eps_dot0;
        const double lr = (rstar > 1.0) ? log(rstar) : 0.0;
        const double tstar = fmin(fmax((out.T - M.T_room) / (M.T_melt - M.T_room), 0.0), 1.0);
        const double ef = (M.d1 + M.d2 * exp(M.d3 * eta)) * (1.0 + M.d4 * lr) * (1.0 + M.d5 * tstar);
        out.failed = (out.ebar >= ef);
    }
    for (int c = 0; c < 6; c++)
        if (!isfinite(out.sig[c])) return OTM_ERR_NONFINITE;
    return OTM_OK;
}

__global__ void __launch_bounds__(128) k_return_map(const Dev D)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    RmIn in;
    for (int i = 0; i < 9; i++) in.dF[i] = D.dF[9 * p + i];
    for (int i = 0; i < 6; i++) in.be[i] = D.be[6 * p + i];
    in.ebar = D.ebar[p];
    in.T = D.T[p];
    in.J = D.Jdet[p];
    RmOut o;
    const int st = return_map_point(D.mat[D.mat_id[p]], D.dt, in, o);
    if (st != OTM_OK) {
        raise_error(D.err, st, D.mgid[p]);
        return;
    }
    for (int i = 0; i < 6; i++) {
        D.be[6 * p + i] = o.be[i];
        D.sig[6 * p + i] = o.sig[i];
    }
    D.ebar[p] = o.ebar;
    D.T[p] = o.T;
    D.rate[p] = o.rate;
    D.failed[p] = (uint8_t)(o.failed && D.allow_erode);
}

cudaError_t launch_return_map(const Dev &D, cudaStream_t s, long long *launches)
{
    const unsigned blocks = (unsigned)((D.nm + 127) / 128);
    if (blocks == 0) return cudaSuccess;
    k_return_map<<<blocks, 128, 0, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ======================================================================== stand-alone kernels
__global__ void __launch_bounds__(kSearchWarps * kWarp)
    k_search_only(const GridDev *g, const int32_t *cell_start, const double4_32a *spos, double cell, double rs2,
                  const double *mp_x, int64_t nm, int S, int32_t *ids, int32_t *counts, int32_t *status,
                  const unsigned long long *grid_err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (p >= nm) return;
    const int P2 = next_pow2(S);
    int32_t *list = (int32_t *)smem_raw + (size_t)warp * P2;
    if (*grid_err != ~0ULL) {
        if (lane == 0) {
            atomicCAS(status, 0, (int)(-(int)(*grid_err & 0xff)));
            counts[p] = 0;
        }
        return;
    }
    const double px = mp_x[3 * p], py = mp_x[3 * p + 1], pz = mp_x[3 * p + 2];
    const int cnt = warp_support_search(g, cell_start, spos, cell, rs2, px, py, pz, list, S, lane);
    const int n = min(cnt, S);
    const int Q2 = next_pow2(max(n, 1));
    for (int k = n + lane; k < Q2; k += kWarp) list[k] = 0x7fffffff;
    __syncwarp();
    warp_bitonic_sort(list, Q2, lane);
    for (int k = lane; k < n; k += kWarp) ids[p * (int64_t)S + k] = list[k];
    if (lane == 0) {
        counts[p] = cnt;
        if (cnt > S) atomicCAS(status, 0, OTM_ERR_CAPACITY);
    }
}

cudaError_t launch_search_only(const double *node_x, int64_t nn, const double *mp_x, int64_t nm, double rs2,
                               double cell, int S, int32_t *ids, int32_t *counts, void *scratch,
                               size_t scratch_bytes, double *grid_out, int32_t *status, cudaStream_t s)
{
    SearchScratch V;
    if (!carve_search_scratch(scratch, scratch_bytes, nn, &V)) return cudaErrorInvalidValue;
    cudaError_t e = build_search_grid(node_x, nn, cell, &V, grid_out, s);
    if (e != cudaSuccess) return e;
    const size_t smem = (size_t)kSearchWarps * next_pow2(S) * sizeof(int32_t);
    const unsigned blocks = (unsigned)((nm + kSearchWarps - 1) / kSearchWarps);
    if (blocks == 0) return cudaSuccess;
    e = cudaFuncSetAttribute(k_search_only, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_search_only<<<blocks, kSearchWarps * kWarp, smem, s>>>(V.g, V.cell_start, V.spos, cell, rs2, mp_x, nm, S,
                                                             ids, counts, status, V.err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kSearchWarps * kWarp)
    k_lme_only(const double *node_x, const double *mp_x, int64_t nm, const int32_t *ids, const int32_t *counts,
               int S, double beta, double tol, int max_newton, double *lam, double *shape, int32_t *iters_out,
               int32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (p >= nm) return;
    WarpSmem W = warp_smem(smem_raw, S, warp);
    const int n = counts[p];
    if (n > S || n <= 0) {
        if (lane == 0) atomicCAS(status, 0, n > S ? OTM_ERR_CAPACITY : OTM_ERR_LME_NOCONV);
        return;
    }
    const double px = mp_x[3 * p], py = mp_x[3 * p + 1], pz = mp_x[3 * p + 2];
    const int64_t base = p * (int64_t)S;
    for (int k = lane; k < n; k += kWarp) {
        const int id = ids[base + k];
        const double x = px - node_x[3 * (int64_t)id], y = py - node_x[3 * (int64_t)id + 1],
                     z = pz - node_x[3 * (int64_t)id + 2];
        W.dx[k] = x; W.dy[k] = y; W.dz[k] = z;
        W.q[k] = -beta * (x * x + y * y + z * z);
    }
    __syncwarp();
    double l0 = lam[3 * p], l1 = lam[3 * p + 1], l2 = lam[3 * p + 2];
    LmeEval E;
    int iters = 0;
    int st = lme_newton(W.dx, W.dy, W.dz, W.q, W.w, n, l0, l1, l2, tol, max_newton, lane, E, iters);
    double inv[6];
    if (st == OTM_OK && !sym_inv3(E.j00, E.j11, E.j22, E.j01, E.j12, E.j02, inv)) st = OTM_ERR_LME_NOCONV;
    if (lane == 0) {
        if (iters_out) iters_out[p] = iters;
        if (st != OTM_OK) atomicCAS(status, 0, st);
        lam[3 * p] = l0; lam[3 * p + 1] = l1; lam[3 * p + 2] = l2;
    }
    if (st != OTM_OK) return;
    const double iZ = 1.0 / E.Z;
    for (int k = lane; k < n; k += kWarp) {
        const double N = W.w[k] * iZ;
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        double *o = shape + 4 * (base + k);
        o[0] = N;
        o[1] = -N * (inv[0] * x + inv[3] * y + inv[5] * z);
        o[2] = -N * (inv[3] * x + inv[1] * y + inv[4] * z);
        o[3] = -N * (inv[5] * x + inv[4] * y + inv[2] * z);
    }
}

cudaError_t launch_lme_only(const double *node_x, const double *mp_x, int64_t nm, const int32_t *ids,
                            const int32_t *counts, int S, double beta, double tol_abs, int max_newton, double *lam,
                            double *shape, int32_t *iters, int32_t *status, cudaStream_t s)
{
    const size_t smem = search_lme_smem_bytes(S, kSearchWarps);
    const unsigned blocks = (unsigned)((nm + kSearchWarps - 1) / kSearchWarps);
    if (blocks == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_lme_only, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_lme_only<<<blocks, kSearchWarps * kWarp, smem, s>>>(node_x, mp_x, nm, ids, counts, S, beta, tol_abs,
                                                          max_newton, lam, shape, iters, status);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128)
    k_return_map_only(const otm_material M, double dt, int64_t nm, const double *dF, const double *F_new, double *be,
                      double *ebar, double *T, double *sigma, double *rate, uint8_t *failed, int32_t *status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nm) return;
    RmIn in;
    for (int i = 0; i < 9; i++) in.dF[i] = dF[9 * p + i];
    for (int i = 0; i < 6; i++) in.be[i] = be[6 * p + i];
    in.ebar = ebar[p];
    in.T = T[p];
    const double *Fn = F_new + 9 * p;
    in.J = Fn[0] * (Fn[4] * Fn[8] - Fn[5] * Fn[7]) - Fn[1] * (Fn[3] * Fn[8] - Fn[5] * Fn[6]) +
           Fn[2] * (Fn[3] * Fn[7] - Fn[4] * Fn[6]);
    RmOut o;
    const int st = return_map_point(M, dt, in, o);
    if (st != OTM_OK) {
        atomicCAS(status, 0, st);
        return;
    }
    for (int i = 0; i < 6; i++) {
        be[6 * p + i] = o.be[i];
        sigma[6 * p + i] = o.sig[i];
    }
    ebar[p] = o.ebar;
    T[p] = o.T;
    if (rate) rate[p] = o.rate;
    if (failed) failed[p] = (uint8_t)o.failed;
}

cudaError_t launch_return_map_only(const otm_material *mat, double dt, int64_t nm, const double *dF,
                                   const double *F_new, double *be, double *ebar, double *T, double *sigma,
                                   double *rate, uint8_t *failed, int32_t *status, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((nm + 127) / 128);
    if (blocks == 0) return cudaSuccess;
    k_return_map_only<<<blocks, 128, 0, s>>>(*mat, dt, nm, dF, F_new, be, ebar, T, sigma, rate, failed, status);
    return cudaGetLastError();
}

}  // namespace otm
