// otm_mp.cu -- material-point kernels (sm_103a):
//   k_search     : Algorithm 3 steps 2-3, warp per MP: candidates of the linked-cell stencil
//                  tested in FP32 against an error band; only candidates inside the band take
//                  the exact FP64 test, so the support (d^2 <= r_s^2 in FP64) is bit-exact.
//                  Ascending-ID sort, influence counting (integer atomics -> rank).
//   k_lme        : Eq. 14, warp per MP: damped Newton for lambda (warm start, exponent shift from
//                  the previous log Z), N and grad N = -N J^-1 d, per-pair contributions
//                  (m_p N, -v sigma grad N) written straight into node-major order.
//   k_kinematics : Eq. 9-13, warp per MP: x_p = sum N x_I, dF = 1 + sum du_I (x) grad N_I,
//                  F <- dF F, v <- det(dF) v
//   k_return_map : Sec. 4.1 / 4.2, thread per MP: Hencky exponential-map radial return (J2
//                  linear hardening closed form, Johnson-Cook safeguarded Newton), heating,
//                  fracture flag, sigma = tau / J
#include <cmath>
#include <mutex>

#include "otm_dev.cuh"
#include "otm_rm.cuh"

namespace otm {

// ======================================================================== double-float arithmetic
// FP32 pairs hi + lo, about 2^-47 relative (the exp's polynomial, the mixed path's Hessian sums)
// An FP64 value split into two FP32 values with integer operations on its bits (GB300 charges a
// conversion instruction an FP64-pipe slot): hi = the leading 24 significant bits, lo = the next
// 24 of the remaining 29 (truncated), so v = hi + lo to 2^-47 relative. Values outside the normal
// FP32 range give hi = lo = 0 (the Hessian sums only see weights in [1e-30, 1e30], checked by the
// caller, and differences of about h).
__device__ __forceinline__ void df_split(double v, float &hi, float &lo)
{
    const int vh = __double2hiint(v);
    const unsigned vl = (unsigned)__double2loint(v);
    const int e = ((vh >> 20) & 0x7ff) - 1023;
    const unsigned sgn = (unsigned)vh & 0x80000000u;
    const bool ok = e > -126 && e < 128;
    hi = ok ? __uint_as_float(sgn | ((unsigned)(e + 127) << 23) | ((unsigned)(vh & 0xfffff) << 3) | (vl >> 29))
            : 0.f;
    const unsigned r = vl & 0x1fffffffu;   // significand bits 28..0 below hi, weight 2^(e - 52)
    const int lz = __clz(r);               // >= 3 when r != 0
    const int el = e - 52 + (31 - lz);     // exponent of r's leading bit
    lo = (ok && r != 0 && el > -126) ? __uint_as_float(sgn | ((unsigned)(el + 127) << 23) | (((r << lz) << 1) >> 9))
                                     : 0.f;
}

// exact widening of an FP32 value to FP64 with integer operations (zero and normal values)
__device__ __forceinline__ double df_widen(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ef = (b >> 23) & 0xff;
    if (ef == 0) return 0.0;
    return __hiloint2double((int)((b & 0x80000000u) | ((ef - 127 + 1023) << 20) | ((b & 0x7fffffu) >> 3)),
                            (int)(b << 29));
}

// (p, e) ~ (ah + al)(bh + bl): the product and its error, the al bl term dropped
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &p, float &e)
{
    p = ah * bh;
    e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
}

// (sh, sl) += (q, f) with an error-free sum of the leading parts
__device__ __forceinline__ void df_add(float &sh, float &sl, float q, float f)
{
    const float s = sh + q;
    const float t = s - sh;
    const float err = (sh - (s - t)) + (q - t);
    sl = sl + (err + f);
    sh = s;
}

// ======================================================================== FP64 exponential
// exp(f) by a table-driven method after P. T. P. Tang ("Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989), with the
// argument scaling folded into the caller: the argument arrives as y = f * 1024 / ln 2 (the LME
// scales lambda and the prior term instead of every exponent), and
//   y = n + s, n = round(y), |s| <= 1/2 and exact (integer operations on y's bits, see below),
//   exp(f) = 2^(n >> 10) * 2^((n & 1023) / 1024) * exp(s ln2 / 1024),
// with exp(t) - 1 for |t| <= ln2/2048 by its Taylor polynomial of degree 3 (truncation below
// 5.5e-16 relative). The 1024-entry table 2^(j/1024) is computed once on the host (C library
// exp2) into g_exp2_table; the LME step kernel reads it through L1, the stand-alone kernels stage
// it into shared memory. Valid for f in about
// [-707, 708]; below it returns 0 (a weight below 1e-307 of the largest), above +inf (the caller
// then re-shifts). The scaling rounds y like any FP64 argument, so the result carries
// |f| * 2^-53 relative error from it, plus about 3 ulps.
constexpr int kExpTable = 1024;
constexpr double kExpScale = 0x1.71547652b82fep+10;   // 1024 / ln 2
constexpr double kExpC1 = 0x1.62e42fefa39efp-11;      // ln 2 / 1024
constexpr double kExpC1lo = 0x1.abc9e3b39803fp-66;    // ln 2 / 1024 - kExpC1
constexpr double kExpC2 = 0x1.ebfbdff82c58fp-23;      // kExpC1^2 / 2
constexpr double kExpC3 = 0x1.c6b08d704a0c0p-35;      // kExpC1^3 / 6
constexpr double kExpShifter = 0x1.8p52;
constexpr int kExpNmin = -1020 * 1024;                 // 2^(n >> 10) stays normal with margin
constexpr int kExpNmax = 1021 * 1024 + 1023;

static __device__ double g_exp2_table[kExpTable];

// Fill g_exp2_table on the current device (first call per device; a synchronous copy, so it
// belongs before any stream capture: otm_init and the stand-alone entries call it). With
// `verify`, a device whose table was already filled is checked again (a synchronous 8-byte read
// of 2^0 = 1): module data is lost when the device or its primary context is reset, and the
// table is then filled anew. otm_init verifies; the stand-alone entries, which must stay free of
// synchronisation once set up, do not.
cudaError_t exp_table_setup(bool verify)
{
    static std::mutex mu;
    static bool done[64];
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev] && verify) {
        double t0 = 0.0;
        e = cudaMemcpyFromSymbol(&t0, g_exp2_table, sizeof(double));
        if (e != cudaSuccess) return e;
        if (t0 != 1.0) done[dev] = false;
    }
    if (done[dev]) return cudaSuccess;
    double host[kExpTable];
    for (int j = 0; j < kExpTable; j++) host[j] = std::exp2((double)j / (double)kExpTable);
    e = cudaMemcpyToSymbol(g_exp2_table, host, sizeof(host));
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

// copy the table into shared memory (block-wide; ends with a barrier)
__device__ __forceinline__ void exp_table_load(double *T)
{
    for (int j = threadIdx.x; j < kExpTable; j += blockDim.x) T[j] = g_exp2_table[j];
    __syncthreads();
}

// the polynomial's coefficients as double-float pairs (C3 needs FP32 only: its term is below 7e-12)
constexpr float kExpC1h = (float)kExpC1;
constexpr float kExpC1l = (float)((kExpC1 - (double)kExpC1h) + kExpC1lo);
constexpr float kExpC2h = (float)kExpC2;
constexpr float kExpC2l = (float)(kExpC2 - (double)kExpC2h);
constexpr float kExpC3f = (float)kExpC3;

// The polynomial p(s) = exp(s ln2/1024) - 1 (|s| <= 1/2, |p| <= 3.4e-4) runs in double-float on
// the FP32 pipe: s split into two FP32 values with integer operations (2^-48 of |s|), Horner in
// error-free FP32 products and sums (p to about 2^-46 of itself: below 5e-18 absolute, against the
// cubic's own truncation of 5.5e-16), then v = T + T p_hi + T p_lo in two FMAs. The result is as
// accurate as the same cubic in FP64 Horner form, with two FP64 instructions instead of four.
__device__ __forceinline__ double exp_scaled(double y, const double *T)
{
    // y = n + s with n = round(y) and s exact, |s| <= 1/2. For 1 <= |y| < 2^20 (every weight of the
    // LME sums: y <= 0, and |y| < 1 only for a single node that carries nearly all the weight)
    // n and s are formed from y's bits with integer operations, which leaves the FP64 pipe to the
    // polynomial; other arguments take the 1.5 * 2^52 shifter (three FP64 additions).
    const int hi = __double2hiint(y);
    const int E = ((hi >> 20) & 0x7ff) - 1023;
    int n;
    double sr;
    if (E >= 0 && E < 20) {
        // significand M (53 bits) = |y| 2^(52 - E); f = 52 - E fraction bits (33..52)
        const unsigned long long M =
            ((unsigned long long)((hi & 0xfffff) | 0x100000) << 32) | (unsigned)__double2loint(y);
        const int f = 52 - E;
        const unsigned long long na = (M + (1ULL << (f - 1))) >> f;   // |n|, rounded half up
        const long long rem = (long long)(M - (na << f));             // |rem| <= 2^(f-1) < 2^52
        const bool neg = hi < 0;
        n = neg ? -(int)na : (int)na;
        // s = rem 2^-f (sign of y applied): normalised with integer operations, exactly (|rem| has
        // at most 52 significant bits, so the 12 or more leading zeros cover the 11 dropped bits)
        const unsigned long long a = (unsigned long long)(rem < 0 ? -rem : rem);
        if (a == 0) {
            sr = 0.0;
        } else {
            const int lz = __clzll((long long)a);
            const unsigned long long m = (a << lz) >> 11;          // 1.xxx in bits 52..0
            const long long ex = 1023 + 63 - lz - f;
            const bool sneg = (rem < 0) != neg;
            sr = __longlong_as_double((long long)((sneg ? 0x8000000000000000ULL : 0ULL) |
                                                  ((unsigned long long)ex << 52) | (m & 0xFFFFFFFFFFFFFULL)));
        }
    } else {
        const double t = y + kExpShifter;
        const int thi = __double2hiint(t);
        n = __double2loint(t);
        // the high word of t is 0x43380000 for round(y) in [0, 2^32) and 0x4337ffff for
        // [-2^32, 0); a mismatch with the sign of the low word means |y| >= 2^31 (or y is not finite)
        if (thi != (n < 0 ? 0x4337ffff : 0x43380000)) return (y > 0.0) ? INFINITY : 0.0;
        sr = y - (t - kExpShifter);
    }
    if (n < kExpNmin || n > kExpNmax) return (y > 0.0) ? INFINITY : 0.0;
    const double Tj = T[n & (kExpTable - 1)];
    float sh, sl;
    df_split(sr, sh, sl);
    float ah = kExpC2h, al = kExpC2l;
    df_add(ah, al, kExpC3f * sh, 0.f);            // C2 + C3 s
    float bh, bl;
    df_mul(ah, al, sh, sl, bh, bl);               // (C2 + C3 s) s
    float ch = kExpC1h, cl = kExpC1l;
    df_add(ch, cl, bh, bl);                       // C1 + (C2 + C3 s) s
    float ph, pl;
    df_mul(ch, cl, sh, sl, ph, pl);               // p
    const double v = fma(Tj, df_widen(pl), fma(Tj, df_widen(ph), Tj));
    return __hiloint2double(__double2hiint(v) + ((n >> 10) << 20), __double2loint(v));
}

// ======================================================================== LME (Eq. 14)
// Sums of one evaluation at lambda with weights w_a = exp(f_a - shift), f_a = q_a + lambda . d_a:
// Z = sum w, r = sum w d, A = sum w d d^T (unnormalised). Then N = w / Z, the residual of the
// consistency condition is r / Z and the Hessian of log Z is J = A / Z - (r/Z)(r/Z)^T = J' / Z
// with J' = A - r r^T / Z.
struct LmeSums {
    double Z, r0, r1, r2, a00, a11, a22, a01, a12, a02;
    double shift;
};

// q[] and the multipliers passed here are in exponent units of ln2/1024 (see exp_scaled)
template <bool SHIFTED>
__device__ __forceinline__ void lme_accumulate(const double *dx, const double *dy, const double *dz, const double *q,
                                               double *w, int n, double l0, double l1, double l2, double qs,
                                               int lane, const double *T, double (&v)[16])
{
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double qk = SHIFTED ? q[k] + qs : q[k];
        const double f = fma(l2, z, fma(l1, y, fma(l0, x, qk)));
        const double wk = exp_scaled(f, T);
        w[k] = wk;
        const double wx = wk * x, wy = wk * y, wz = wk * z;
        v[0] += wk;
        v[1] += wx; v[2] += wy; v[3] += wz;
        v[4] = fma(wx, x, v[4]); v[5] = fma(wy, y, v[5]); v[6] = fma(wz, z, v[6]);
        v[7] = fma(wx, y, v[7]); v[8] = fma(wy, z, v[8]); v[9] = fma(wx, z, v[9]);
    }
}

__device__ __forceinline__ void lme_sums(const double *dx, const double *dy, const double *dz, const double *q,
                                         double *w, int n, double l0, double l1, double l2, double shift,
                                         double q0shift, int lane, const double *T, LmeSums &E)
{
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = 0.0;
    // q[] holds (prior exponent - the solve's first shift) * 1024/ln2; a different shift (only
    // after an over/underflow) is applied as a difference
    const double qs = (q0shift - shift) * kExpScale;
    const double s0 = l0 * kExpScale, s1 = l1 * kExpScale, s2 = l2 * kExpScale;
    if (qs == 0.0)
        lme_accumulate<false>(dx, dy, dz, q, w, n, s0, s1, s2, qs, lane, T, v);
    else
        lme_accumulate<true>(dx, dy, dz, q, w, n, s0, s1, s2, qs, lane, T, v);
    const double t = warp_reduce_scatter16(v, lane);   // value j at lanes 2j, 2j+1
    E.Z = __shfl_sync(0xffffffffu, t, 0);
    E.r0 = __shfl_sync(0xffffffffu, t, 2);
    E.r1 = __shfl_sync(0xffffffffu, t, 4);
    E.r2 = __shfl_sync(0xffffffffu, t, 6);
    E.a00 = __shfl_sync(0xffffffffu, t, 8);
    E.a11 = __shfl_sync(0xffffffffu, t, 10);
    E.a22 = __shfl_sync(0xffffffffu, t, 12);
    E.a01 = __shfl_sync(0xffffffffu, t, 14);
    E.a12 = __shfl_sync(0xffffffffu, t, 16);
    E.a02 = __shfl_sync(0xffffffffu, t, 18);
    E.shift = shift;
}

__device__ __forceinline__ double lme_fmax(const double *dx, const double *dy, const double *dz,
                                           const double *q, int n, double l0, double l1, double l2,
                                           double q0shift, int lane)
{
    const double s0 = l0 * kExpScale, s1 = l1 * kExpScale, s2 = l2 * kExpScale;
    double m = -INFINITY;
    for (int k = lane; k < n; k += kWarp) m = fmax(m, q[k] + (s0 * dx[k] + s1 * dy[k] + s2 * dz[k]));
    return warp_max(m) * (1.0 / kExpScale) + q0shift;
}

// evaluation with the given shift; if the weights over- or underflow, again with max f
__device__ __forceinline__ void lme_sums_safe(const double *dx, const double *dy, const double *dz,
                                              const double *q, double *w, int n, double l0, double l1,
                                              double l2, double shift, double q0shift, int lane, const double *T,
                                              LmeSums &E)
{
    lme_sums(dx, dy, dz, q, w, n, l0, l1, l2, shift, q0shift, lane, T, E);
    if (!(E.Z > 1e-200) || !(E.Z < 1e200)) {
        const double fm = lme_fmax(dx, dy, dz, q, n, l0, l1, l2, q0shift, lane);
        lme_sums(dx, dy, dz, q, w, n, l0, l1, l2, fm, q0shift, lane, T, E);
    }
}

__device__ __forceinline__ double rn2(const LmeSums &E) { return E.r0 * E.r0 + E.r1 * E.r1 + E.r2 * E.r2; }

// J' = A - r r^T / Z and its adjugate / determinant (cofactors); false if not positive definite.
// iZ_out (optional) receives 1 / Z.
__device__ __forceinline__ bool lme_jinv(const LmeSums &E, double inv[6], double *iZ_out = nullptr)
{
    const double iZ = 1.0 / E.Z;
    if (iZ_out) *iZ_out = iZ;
    const double s0 = E.r0 * iZ, s1 = E.r1 * iZ, s2 = E.r2 * iZ;
    const double j00 = E.a00 - s0 * E.r0, j11 = E.a11 - s1 * E.r1, j22 = E.a22 - s2 * E.r2;
    const double j01 = E.a01 - s0 * E.r1, j12 = E.a12 - s1 * E.r2, j02 = E.a02 - s0 * E.r2;
    const double c00 = j11 * j22 - j12 * j12;
    const double c01 = j02 * j12 - j01 * j22;
    const double c02 = j01 * j12 - j02 * j11;
    const double c11 = j00 * j22 - j02 * j02;
    const double c12 = j01 * j02 - j00 * j12;
    const double c22 = j00 * j11 - j01 * j01;
    const double det = j00 * c00 + j01 * c01 + j02 * c02;
    if (!(det > 0.0) || !isfinite(det)) return false;
    const double id = 1.0 / det;
    inv[0] = c00 * id; inv[1] = c11 * id; inv[2] = c22 * id;
    inv[3] = c01 * id; inv[4] = c12 * id; inv[5] = c02 * id;   // (xx, yy, zz, xy, yz, xz) of J'^-1
    return true;
}

// log Z(trial) < log Z(current)
__device__ __forceinline__ bool logz_less(const LmeSums &t, const LmeSums &c)
{
    if (t.shift == c.shift) return t.Z < c.Z;
    return t.shift + log(t.Z) < c.shift + log(c.Z);
}

// Damped Newton on the convex log Z(lambda): step -J^-1 (r/Z) = -J'^-1 r, halved until log Z or
// the residual norm drops; stops when |r| / Z <= tol. All evaluations of one solve share the
// initial shift (the previous step's log Z, so w ~ N), which makes the log Z comparison a
// comparison of Z; q[] must hold the prior exponent minus that shift, times 1024/ln2. On return
// w[] holds the weights of the accepted evaluation E. Warp-uniform.
// Newton iterations from an evaluation E already taken at lambda (see lme_newton).
__device__ int lme_newton_loop(const double *dx, const double *dy, const double *dz, const double *q, double *w,
                               int n, double &l0, double &l1, double &l2, double shift, double tol, int max_it,
                               int lane, const double *T, LmeSums &E, int &iters)
{
    const double tol2 = tol * tol;
    for (;;) {
        const double r2 = rn2(E);
        if (!isfinite(r2) || !isfinite(E.Z)) return OTM_ERR_LME_NOCONV;
        if (r2 <= tol2 * E.Z * E.Z) return OTM_OK;
        if (iters >= max_it) return OTM_ERR_LME_NOCONV;
        iters++;
        double inv[6];
        if (!lme_jinv(E, inv)) return OTM_ERR_LME_NOCONV;
        const double s0 = -(inv[0] * E.r0 + inv[3] * E.r1 + inv[5] * E.r2);
        const double s1 = -(inv[3] * E.r0 + inv[1] * E.r1 + inv[4] * E.r2);
        const double s2 = -(inv[5] * E.r0 + inv[4] * E.r1 + inv[2] * E.r2);
        double t = 1.0;
        bool accepted = false;
        LmeSums Et;
        double m0 = l0, m1 = l1, m2 = l2;
        for (int halving = 0; halving < 40; halving++) {
            m0 = fma(t, s0, l0); m1 = fma(t, s1, l1); m2 = fma(t, s2, l2);
            lme_sums_safe(dx, dy, dz, q, w, n, m0, m1, m2, E.shift, shift, lane, T, Et);
            if (isfinite(Et.Z) && (logz_less(Et, E) || rn2(Et) * (E.Z * E.Z) < r2 * (Et.Z * Et.Z))) {
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

// Damped Newton on the convex log Z(lambda): step -J^-1 (r/Z) = -J'^-1 r, halved until log Z or
// the residual norm drops; stops when |r| / Z <= tol. All evaluations of one solve share the
// initial shift (the previous step's log Z, so w ~ N), which makes the log Z comparison a
// comparison of Z; q[] must hold the prior exponent minus that shift, times 1024/ln2. On return
// w[] holds the weights of the accepted evaluation E. Warp-uniform.
__device__ int lme_newton(const double *dx, const double *dy, const double *dz, const double *q, double *w,
                          int n, double &l0, double &l1, double &l2, double shift, double tol, int max_it,
                          int lane, const double *T, LmeSums &E, int &iters)
{
    iters = 0;
    if (n <= 0) return OTM_ERR_LME_NOCONV;
    lme_sums_safe(dx, dy, dz, q, w, n, l0, l1, l2, shift, shift, lane, T, E);
    return lme_newton_loop(dx, dy, dz, q, w, n, l0, l1, l2, shift, tol, max_it, lane, T, E, iters);
}

// ======================================================================== support search
// Search of one MP over the linked-cell rows that cover [x_p - r_s, x_p + r_s] (with a 1e-4
// relative margin), rows of contiguous cells along x. Each candidate is first tested in FP32 on
// coordinates relative to the grid origin; the FP32 value d2f of |x_p - x_a|^2 differs from the
// FP64 value that defines the support by less than `band` (derived below), so a candidate with
// d2f < rs2 - band is inside, one with d2f > rs2 + band is outside, and only the rest take the
// exact FP64 test on the double coordinates. Accepted IDs go to list[0..min(count, S)); returns
// the full count. Warp-uniform.
//
// Band: with u = 2^-24, U >= |x - o| for both points, e = 1.001 u (2U + 1.5 r_s) bounds the
// error of each FP32 difference (two roundings of the coordinates, one of the difference), so
// |d2f - d2| <= e (2 sum|d_i| + 3e) + 3.1 u d2 (three roundings in the fused sum), and the FP64
// d2 is within 7e-16 d2 of the real value. Near the threshold |d_i| <= 1.5 r_s, giving
// band = 1.25 [e (9 r_s + 3e) + 3.1 u rs2] + 1e-15 rs2.
struct SearchGrid {
    const GridDev *g;
    const int32_t *cell_start;
    const float4 *spos32;
    const double4_32a *spos;
};

SearchConst make_search_const(double cell, double rs2)
{
    SearchConst c;
    c.cell = cell;
    c.rs2 = rs2;
    c.cf = (float)cell;
    c.rs = (float)std::sqrt(rs2);
    float lo = (float)rs2, hi = (float)rs2;
    if ((double)lo > rs2) lo = std::nextafterf(lo, -INFINITY);
    if ((double)hi < rs2) hi = std::nextafterf(hi, INFINITY);
    c.rs2_rd = lo;
    c.rs2_ru = hi;
    return c;
}

__device__ int warp_support_search(const SearchGrid &G, const SearchConst &C, double px, double py, double pz,
                                   int32_t *list, int S, int lane)
{
    const GridDev *g = G.g;
    if (g->n_cells == 0) return 0;
    const int nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const double rs2 = C.rs2;
    // position relative to the grid origin, in FP32 (one FP64 subtraction per axis)
    const float X = (float)(px - g->origin[0]), Y = (float)(py - g->origin[1]), Z = (float)(pz - g->origin[2]);
    const float cf = C.cf;
    const float rs = C.rs;
    // cell ranges covering [x - r_s, x + r_s] with a 1e-4 relative margin (which covers the FP32
    // rounding of X and of the quotient; nodes are binned by the exact FP64 floor)
    const float rsm = rs * 1.0001f;
    const int x0 = max((int)fmaxf(floorf((X - rsm) / cf), -1.f), 0);
    const int x1 = min((int)fminf(floorf((X + rsm) / cf), (float)nx), nx - 1);
    const int y0 = max((int)fmaxf(floorf((Y - rsm) / cf), -1.f), 0);
    const int y1 = min((int)fminf(floorf((Y + rsm) / cf), (float)ny), ny - 1);
    const int z0 = max((int)fmaxf(floorf((Z - rsm) / cf), -1.f), 0);
    const int z1 = min((int)fminf(floorf((Z + rsm) / cf), (float)nz), nz - 1);
    int cnt = 0;
    if (x0 > x1 || y0 > y1 || z0 > z1) return 0;
    const float ext = fmaxf(fmaxf((float)nx, (float)ny), (float)nz) * cf;
    const float U = fmaxf(fmaxf(fmaxf(fabsf(X), fabsf(Y)), fabsf(Z)), ext);
    const float u = 0x1p-24f;
    const float e = 1.001f * u * (2.f * U + 1.5f * rs);
    const float band = 1.5f * (1.25f * (e * (9.f * rs + 3.f * e) + 3.1f * u * rs * rs) + 1e-15f * rs * rs);
    const float lo = __fsub_rd(C.rs2_rd, band), hi = __fadd_ru(C.rs2_ru, band);
    // the test of one candidate slot s of a row ending at s1 (its FP32 record already loaded)
    auto test = [&](int s, int s1, const float4 &a, int &id) -> bool {
        if (s >= s1) return false;
        const float dx = X - a.x, dy = Y - a.y, dz = Z - a.z;
        const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        id = __float_as_int(a.w);
        if (d2 <= lo) return true;
        if (d2 > hi) return false;
        const double4_32a q = G.spos[s];   // ambiguity band: exact FP64 test
        return dist2_exact(px, py, pz, q.x, q.y, q.z) <= rs2;
    };
    auto append = [&](bool acc, int id) {
        const unsigned m = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            const int pos = cnt + __popc(m & ((1u << lane) - 1u));
            if (pos < S) list[pos] = id;
        }
        cnt += __popc(m);
    };
    // Rows in (z, y) order, r = (kz - z0) ny' + (ky - y0). The candidate ranges of up to 32 rows
    // are loaded at once, one row per lane, and each row is scanned 64 slots per pass with both
    // chunks' loads in flight; the accepted IDs keep the order of a plain scan (rows, cells,
    // slots).
    const int nyr = y1 - y0 + 1, nrows = nyr * (z1 - z0 + 1);
    for (int g0 = 0; g0 < nrows; g0 += kWarp) {
        int r0 = 0, r1 = 0;
        if (g0 + lane < nrows) {
            const int r = g0 + lane;
            const int rowc = ((z0 + r / nyr) * ny + (y0 + r % nyr)) * nx;
            r0 = G.cell_start[rowc + x0];
            r1 = G.cell_start[rowc + x1 + 1];
        }
        const int ng = min(kWarp, nrows - g0);
        for (int r = 0; r < ng; r++) {
            const int s0 = __shfl_sync(0xffffffffu, r0, r), s1 = __shfl_sync(0xffffffffu, r1, r);
            for (int b = s0; b < s1; b += 2 * kWarp) {
                const int sa = b + lane, sb = b + kWarp + lane;
                float4 qa = make_float4(0.f, 0.f, 0.f, 0.f), qb = qa;
                if (sa < s1) qa = G.spos32[sa];
                if (sb < s1) qb = G.spos32[sb];
                int ida = 0, idb = 0;
                const bool acca = test(sa, s1, qa, ida);
                const bool accb = test(sb, s1, qb, idb);
                append(acca, ida);
                if (b + kWarp < s1) append(accb, idb);
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

// per-warp shared-memory layout for the LME solve
struct WarpSmem {
    double *dx, *dy, *dz, *q, *w;
};

__device__ __forceinline__ WarpSmem warp_smem(unsigned char *base, int S, int warp)
{
    unsigned char *b = base + (size_t)warp * 5 * (size_t)S * sizeof(double);
    WarpSmem W;
    W.dx = (double *)b;
    W.dy = W.dx + S;
    W.dz = W.dy + S;
    W.q = W.dz + S;
    W.w = W.q + S;
    return W;
}

constexpr int kLmeWarps = 4;

// The damped Newton solve of Eq. 14 for the block's MPs, block-synchronous: each round, every
// warp whose MP has an evaluation pending computes the sums (Z, r, A) at its trial lambda (the
// pair loop); then one thread per MP takes the scalar decisions (accept or halve the trial, the
// convergence test, J'^-1, the next Newton step). FP64 instructions cost the pipe the same with
// one active lane as with 32, so doing the scalar work once per MP instead of once per lane of
// a warp saves most of it. State of one MP's solve, in shared memory:
enum : int { kNewtonIdle = 0, kNewtonEval = 1, kNewtonDone = 2, kNewtonFail = 3 };
struct MpNewton {
    double E[11];      // sums of the latest evaluation: Z, r (3), A (6), shift
    double C[11];      // sums at the current (accepted) point
    double lam[3];     // current lambda
    double trial[3];   // lambda of the pending evaluation
    double dir[3];     // Newton direction at the current point
    double ws[3];      // warm start of the solve (for the cold-start retry)
    double t;          // step fraction of the pending trial
    double inv[6];     // J'^-1 at the solution (xx, yy, zz, xy, yz, xz)
    double iZ, logz;
    double ts[3];      // the trial times 1024/ln2 (the exponent units of exp_scaled)
    double sh;         // exponent shift of the pending evaluation
    double qs;         // (solve's first shift - sh) * 1024/ln2, added to the stored prior terms
    double shift0;     // the solve's first shift (the stored prior terms are relative to it)
    int state, have_cur, iters, iters_total, halvings, retried;
};

// the scaled trial and the shift of the pending evaluation: trials share the current point's
// shift, the first evaluation of a start uses the solve's first shift
__device__ __forceinline__ void newton_set_trial(MpNewton &m)
{
    m.sh = m.have_cur ? m.C[10] : m.shift0;
    m.qs = (m.shift0 - m.sh) * kExpScale;
    for (int i = 0; i < 3; i++) m.ts[i] = m.trial[i] * kExpScale;
}

// One evaluation of the block path (Eq. 14 sums at the pending trial of MP state m): weights
// into W.w, the sums into m.E (written by one lane per value), m.E[10] = the shift used. If Z
// over- or underflows, again with the shift at the largest exponent. Warp-uniform.
// One evaluation's sums over the pairs of lane `lane`: Z, r = sum w d and A = sum w d d^T.
// FP64 path (DFH false): all in FP64. Mixed path (DFH true): Z and r in FP64 (r is a cancelling
// sum that decides convergence at 1e-14 h), the Hessian sums A in double-float: they only set
// the Newton step and J^-1, for which their relative accuracy of about 1e-14 is ample, and they
// then leave the FP64 pipe, the kernel's bound, to the weights; the per-lane double-float sums are
// widened to FP64 before the warp reduction.
template <bool SHIFTED, bool DFH>
__device__ __forceinline__ void lme_acc10(const WarpSmem &W, int n, double s0, double s1, double s2, double qs,
                                          int lane, const double *T, double (&v)[10])
{
#pragma unroll
    for (int i = 0; i < 10; i++) v[i] = 0.0;
    if (!DFH) {
        for (int k = lane; k < n; k += kWarp) {
            const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
            const double qk = SHIFTED ? W.q[k] + qs : W.q[k];
            const double wk = exp_scaled(fma(s2, z, fma(s1, y, fma(s0, x, qk))), T);
            W.w[k] = wk;
            const double wx = wk * x, wy = wk * y, wz = wk * z;
            v[0] += wk;
            v[1] += wx; v[2] += wy; v[3] += wz;
            v[4] = fma(wx, x, v[4]); v[5] = fma(wy, y, v[5]); v[6] = fma(wz, z, v[6]);
            v[7] = fma(wx, y, v[7]); v[8] = fma(wy, z, v[8]); v[9] = fma(wx, z, v[9]);
        }
        return;
    }
    float ah[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, al[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = lane; k < n; k += kWarp) {
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        const double qk = SHIFTED ? W.q[k] + qs : W.q[k];
        const double wk = exp_scaled(fma(s2, z, fma(s1, y, fma(s0, x, qk))), T);
        W.w[k] = wk;
        v[0] += wk;
        v[1] = fma(wk, x, v[1]); v[2] = fma(wk, y, v[2]); v[3] = fma(wk, z, v[3]);
        float wh, wl, xh, xl, yh, yl, zh, zl;
        df_split(wk, wh, wl);
        df_split(x, xh, xl);
        df_split(y, yh, yl);
        df_split(z, zh, zl);
        float pxh, pxl, pyh, pyl, pzh, pzl, q, f;
        df_mul(wh, wl, xh, xl, pxh, pxl);
        df_mul(wh, wl, yh, yl, pyh, pyl);
        df_mul(wh, wl, zh, zl, pzh, pzl);
        df_mul(pxh, pxl, xh, xl, q, f); df_add(ah[0], al[0], q, f);
        df_mul(pyh, pyl, yh, yl, q, f); df_add(ah[1], al[1], q, f);
        df_mul(pzh, pzl, zh, zl, q, f); df_add(ah[2], al[2], q, f);
        df_mul(pxh, pxl, yh, yl, q, f); df_add(ah[3], al[3], q, f);
        df_mul(pyh, pyl, zh, zl, q, f); df_add(ah[4], al[4], q, f);
        df_mul(pxh, pxl, zh, zl, q, f); df_add(ah[5], al[5], q, f);
    }
#pragma unroll
    for (int i = 0; i < 6; i++) v[4 + i] = df_widen(ah[i]) + df_widen(al[i]);
}

// The FP64 Hessian sums of one evaluation from its stored weights (the fallback for weights
// outside the double-float range; see lme_eval_block)
__device__ __forceinline__ void lme_hessian64(const WarpSmem &W, int n, int lane, double (&v)[10])
{
    for (int k = lane; k < n; k += kWarp) {
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        const double wk = W.w[k];
        const double wx = wk * x, wy = wk * y, wz = wk * z;
        v[4] = fma(wx, x, v[4]); v[5] = fma(wy, y, v[5]); v[6] = fma(wz, z, v[6]);
        v[7] = fma(wx, y, v[7]); v[8] = fma(wy, z, v[8]); v[9] = fma(wx, z, v[9]);
    }
}

template <bool DFH>
__device__ void lme_eval_block(const WarpSmem &W, int n, MpNewton &m, int lane, const double *T)
{
    const double s0 = m.ts[0], s1 = m.ts[1], s2 = m.ts[2];
    double qs = m.qs, sh = m.sh;
    double v[10];
    if (qs == 0.0) lme_acc10<false, DFH>(W, n, s0, s1, s2, qs, lane, T, v);
    else lme_acc10<true, DFH>(W, n, s0, s1, s2, qs, lane, T, v);
    double t = warp_reduce_scatter10(v, lane);
    double Z = __shfl_sync(0xffffffffu, t, 0);
    if (!(Z > 1e-200) || !(Z < 1e200)) {
        double mx = -INFINITY;
        for (int k = lane; k < n; k += kWarp) mx = fmax(mx, W.q[k] + (s0 * W.dx[k] + s1 * W.dy[k] + s2 * W.dz[k]));
        sh = warp_max(mx) * (1.0 / kExpScale) + m.shift0;
        qs = (m.shift0 - sh) * kExpScale;
        lme_acc10<true, DFH>(W, n, s0, s1, s2, qs, lane, T, v);
        t = warp_reduce_scatter10(v, lane);
        Z = __shfl_sync(0xffffffffu, t, 0);
    }
    if (DFH && !(Z >= 1e-30 && Z <= 1e30)) {
        // weights this far from 1 may leave the FP32 range of the double-float sums: the Hessian
        // sums again in FP64 from the stored weights (Z and r are kept)
#pragma unroll
        for (int i = 4; i < 10; i++) v[i] = 0.0;
        lme_hessian64(W, n, lane, v);
        const double t2 = warp_reduce_scatter10(v, lane);
        if (rs10_value(lane) >= 4) t = t2;
    }
    if (rs10_writer(lane)) m.E[rs10_value(lane)] = t;
    if (lane == 0) m.E[10] = sh;
}

__device__ __forceinline__ LmeSums sums_of(const double *v)
{
    LmeSums e;
    e.Z = v[0]; e.r0 = v[1]; e.r1 = v[2]; e.r2 = v[3];
    e.a00 = v[4]; e.a11 = v[5]; e.a22 = v[6]; e.a01 = v[7]; e.a12 = v[8]; e.a02 = v[9];
    e.shift = v[10];
    return e;
}

// the solve failed from this start: once more from lambda = 0 if the start was not 0
__device__ __forceinline__ void newton_fail(MpNewton &m)
{
    if (!m.retried && (m.ws[0] != 0.0 || m.ws[1] != 0.0 || m.ws[2] != 0.0)) {
        m.retried = 1;
        m.have_cur = 0;
        m.iters = 0;
        m.halvings = 0;
        m.ws[0] = m.ws[1] = m.ws[2] = 0.0;
        m.trial[0] = m.trial[1] = m.trial[2] = 0.0;
        newton_set_trial(m);
        m.state = kNewtonEval;
    } else {
        m.state = kNewtonFail;
    }
}

// the solve has converged at C (whose Hessian sums are FP64): J'^-1, 1/Z and the next shift for
// the outputs
__device__ __forceinline__ void newton_finish(MpNewton &m)
{
    const LmeSums c = sums_of(m.C);
    double inv[6];
    if (!lme_jinv(c, inv, &m.iZ)) {
        newton_fail(m);
        return;
    }
    for (int i = 0; i < 6; i++) m.inv[i] = inv[i];
    // the next solve's shift only has to keep the weights near 1: log Z to within ln 2, from the
    // binary exponent of Z (Z > 0 and finite here)
    const int ez = ((__double2hiint(c.Z) >> 20) & 0x7ff) - 1023;
    m.logz = fma((double)ez, 0x1.62e42fefa39efp-1, c.shift);
    m.state = kNewtonDone;
}

// one scalar round after an evaluation (the damped Newton of lme_newton_loop, as a state machine)
__device__ void newton_round(MpNewton &m, double tol, int max_it)
{
    if (m.state != kNewtonEval) return;
    if (!m.have_cur) {               // the first evaluation of a start is the current point
        for (int i = 0; i < 11; i++) m.C[i] = m.E[i];
        for (int i = 0; i < 3; i++) m.lam[i] = m.trial[i];
        m.have_cur = 1;
    } else {                          // accept if log Z or the residual norm drops, else halve
        const LmeSums e = sums_of(m.E), c = sums_of(m.C);
        if (isfinite(e.Z) && (logz_less(e, c) || rn2(e) * (c.Z * c.Z) < rn2(c) * (e.Z * e.Z))) {
            for (int i = 0; i < 11; i++) m.C[i] = m.E[i];
            for (int i = 0; i < 3; i++) m.lam[i] = m.trial[i];
            m.halvings = 0;
        } else {
            if (++m.halvings >= 40) {
                newton_fail(m);
                return;
            }
            m.t *= 0.5;
            for (int i = 0; i < 3; i++) m.trial[i] = fma(m.t, m.dir[i], m.lam[i]);
            newton_set_trial(m);
            return;
        }
    }
    const LmeSums c = sums_of(m.C);
    const double r2 = rn2(c);
    if (!isfinite(r2) || !isfinite(c.Z)) {
        newton_fail(m);
        return;
    }
    double inv[6];
    if (r2 <= tol * tol * c.Z * c.Z) {   // converged
        newton_finish(m);
        return;
    }
    if (m.iters >= max_it || !lme_jinv(c, inv)) {
        newton_fail(m);
        return;
    }
    m.iters++;
    m.iters_total++;
    m.dir[0] = -(inv[0] * c.r0 + inv[3] * c.r1 + inv[5] * c.r2);
    m.dir[1] = -(inv[3] * c.r0 + inv[1] * c.r1 + inv[4] * c.r2);
    m.dir[2] = -(inv[5] * c.r0 + inv[4] * c.r1 + inv[2] * c.r2);
    m.t = 1.0;
    for (int i = 0; i < 3; i++) m.trial[i] = fma(m.t, m.dir[i], m.lam[i]);
    newton_set_trial(m);
}

// shared memory of the stand-alone LME kernel (k_lme_only): the exp table and rows of S slots
size_t lme_smem_bytes(int S, int warps)
{
    return kExpTable * sizeof(double) + (size_t)warps * 5 * (size_t)S * sizeof(double) +
           (size_t)warps * sizeof(MpNewton);
}


// The new support of an MP into its row (IDs from the warp's list) and each pair's rank in its
// node's influence list, by counting with atomics; three slots per lane at a time, so that three
// atomics (whose old values are waited for) are in flight together. Any order of the ranks gives
// the same node sums (exact fixed-point sums).
__device__ __forceinline__ void store_support(const Dev &D, const int32_t *list, int64_t base, int cnt, int lane)
{
    for (int k0 = lane; k0 < cnt; k0 += 3 * kWarp) {
        int id[3], r[3];
#pragma unroll
        for (int j = 0; j < 3; j++) id[j] = (k0 + j * kWarp < cnt) ? list[k0 + j * kWarp] : -1;
#pragma unroll
        for (int j = 0; j < 3; j++) r[j] = (id[j] >= 0) ? atomicAdd(&D.ncount[id[j]], 1) : 0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            if (id[j] < 0) continue;
            const int64_t k = base + k0 + j * kWarp;
            D.ids[k] = id[j];
            if (r[j] > 0xffff) raise_error(D.err, OTM_ERR_CAPACITY, D.ngid[id[j]]);
            D.rank[k] = (uint16_t)r[j];
        }
    }
}

// ======================================================================== k_search
__global__ void __launch_bounds__(kSearchWarps * kWarp) k_search(const Dev D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    const int S = D.S;
    int32_t *list = (int32_t *)smem_raw + (size_t)warp * next_pow2(S);
    const double4_32a xp = D.xp[p];
    SearchGrid G{D.grid, D.cell_start, D.spos32, D.spos};
    const int cnt = warp_support_search(G, D.sc, xp.x, xp.y, xp.z, list, S, lane);
    if (cnt > S) {
        if (lane == 0) {
            raise_error(D.err, OTM_ERR_CAPACITY, D.mgid[p]);
            D.cnt[p] = 0;
        }
        return;
    }
    // the list is in linked-cell order (rows, cells, ascending ID within a cell): unique for a
    // given configuration, so no sort is needed for determinism; exports sort it by ID
    __syncwarp();
    const int64_t base = p * (int64_t)S;
    store_support(D, list, base, cnt, lane);
    if (lane == 0) D.cnt[p] = cnt;
}

// ======================================================================== kinematics gathers
// FP64 -> FP32, rounded to nearest (ties away from zero), with integer operations on the bits: a
// conversion instruction takes an FP64-pipe slot on this GPU, integer operations do not. Values
// below the normal FP32 range give a signed zero; |v| < 2^127 is assumed (shape-function values,
// their products with separations, and force contributions).
__device__ __forceinline__ float f32_round_bits(double v)
{
    const unsigned hi = (unsigned)__double2hiint(v), lo = (unsigned)__double2loint(v);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    const unsigned sgn = hi & 0x80000000u;
    const unsigned mag = ((unsigned)(e + 127) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(e < -126 ? sgn : (sgn | (mag + ((lo >> 28) & 1u))));
}

// The 12 sums of the kinematics over MP p's old support (n pairs at row base), reduce-scattered
// (value rs12_value(lane) at each lane): 0-2 the x_p sums, 3-11 G = sum du_a (x) e_a row-major.
//  FP64 path: x_p = sum N_a x_a of the updated node positions (Eq. 9), G from the FP64 increments.
//  Mixed path, in FP32 from the FP32 increments and the pair rows rounded to FP32: with c = the
//  increment of the support's first node, values 0-2 are sum N_a (du_a - c) and G =
//  sum (du_a - c) (x) e_a. Then x_p,n+1 = x_p,n + c + sum N_a (du_a - c), which is Eq. 9 by the
//  partition of unity and the linear reproducibility of the LME functions (sum N_a x_a,n = x_p,n
//  to the Newton tolerance), and G differs from the FP64 sum by c (x) sum e_a = c (x) r / Z, below
//  |c| 1e-14 h. Subtracting c leaves only the deforming part of the increments in the FP32 sums
//  (no cancellation of the rigid translation), so their error is FP32 rounding of the deformation.
template <bool MIXED>
struct KinSum;

template <>
struct KinSum<false> {
    double t;
    __device__ __forceinline__ void gather(const Dev &D, int64_t base, int n, int lane)
    {
        double v[12];
#pragma unroll
        for (int i = 0; i < 12; i++) v[i] = 0.0;
        for (int k = lane; k < n; k += kWarp) {
            const int id = D.ids[base + k];
            const double4_32a sh = D.shape[base + k];
            const double4_32a xa = D.x[id];
            const double4_32a u = D.du[id];
            v[0] = fma(sh.x, xa.x, v[0]); v[1] = fma(sh.x, xa.y, v[1]); v[2] = fma(sh.x, xa.z, v[2]);
            v[3] = fma(u.x, sh.y, v[3]); v[4] = fma(u.x, sh.z, v[4]); v[5] = fma(u.x, sh.w, v[5]);
            v[6] = fma(u.y, sh.y, v[6]); v[7] = fma(u.y, sh.z, v[7]); v[8] = fma(u.y, sh.w, v[8]);
            v[9] = fma(u.z, sh.y, v[9]); v[10] = fma(u.z, sh.z, v[10]); v[11] = fma(u.z, sh.w, v[11]);
        }
        t = warp_reduce_scatter12(v, lane);
    }
    __device__ __forceinline__ double g() const { return t; }
    // x_p,n+1 component i, on the lane that holds value i (lanes 0, 2, 4)
    __device__ __forceinline__ double xp(double, int) const { return t; }
};

template <>
struct KinSum<true> {
    float t;
    float c[3];
    __device__ __forceinline__ void gather(const Dev &D, int64_t base, int n, int lane)
    {
        float v[12];
#pragma unroll
        for (int i = 0; i < 12; i++) v[i] = 0.f;
        float4 c4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n > 0) c4 = D.du32[D.ids[base]];
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z;
#pragma unroll 2
        for (int k = lane; k < n; k += kWarp) {
            const int id = D.ids[base + k];
            const double4_32a sh = D.shape[base + k];
            const float4 u = D.du32[id];
            const float N = f32_round_bits(sh.x), ex = f32_round_bits(sh.y), ey = f32_round_bits(sh.z),
                        ez = f32_round_bits(sh.w);
            const float a0 = u.x - c4.x, a1 = u.y - c4.y, a2 = u.z - c4.z;
            v[0] = fmaf(N, a0, v[0]); v[1] = fmaf(N, a1, v[1]); v[2] = fmaf(N, a2, v[2]);
            v[3] = fmaf(a0, ex, v[3]); v[4] = fmaf(a0, ey, v[4]); v[5] = fmaf(a0, ez, v[5]);
            v[6] = fmaf(a1, ex, v[6]); v[7] = fmaf(a1, ey, v[7]); v[8] = fmaf(a1, ez, v[8]);
            v[9] = fmaf(a2, ex, v[9]); v[10] = fmaf(a2, ey, v[10]); v[11] = fmaf(a2, ez, v[11]);
        }
        t = warp_reduce_scatter12(v, lane);
    }
    __device__ __forceinline__ double g() const { return (double)t; }
    __device__ __forceinline__ double xp(double old, int i) const
    {
        const float ci = i == 0 ? c[0] : (i == 1 ? c[1] : c[2]);
        return old + ((double)ci + (double)t);
    }
};

// ======================================================================== k_kin_search
// Kinematics (Eq. 9, 11) and the support search at the new position (Algorithm 3) in one warp
// per MP: the gather over the old support gives x_p and dF, then the candidate scan builds the
// new support in the same row. Used when no erosion can remove MPs between the two; the
// return map (which only needs dF) follows.
// Occupancy: the mixed kernel is bound by memory latency (the FP32 gather leaves the FP64 pipe
// idle), so 12 blocks per SM (40 registers, a 16-byte spill) beat 10 (48 registers): 14.2 against
// 14.8 ms on the 2.85 M-MP rod; the FP64 kernel is bound by its FP64 gather and takes 8 blocks.
template <bool MIXED>
__global__ void __launch_bounds__(kSearchWarps * kWarp, MIXED ? 12 : 8) k_kin_search(const Dev D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kSearchWarps + warp;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    const int S = D.S;
    const int n = D.cnt[p];
    const int64_t base = p * (int64_t)S;
    KinSum<MIXED> ks;
    ks.gather(D, base, n, lane);
    const int j = rs12_value(lane);
    if (rs12_writer(lane) && j >= 3) D.dF[9 * p + (j - 3)] = ks.g();   // G = sum du (x) e; k_return_map forms dF
    // values 0, 1, 2 (x_p) sit at lanes 0, 2, 4
    double xi = 0.0;
    if (lane < 6 && (lane & 1) == 0) xi = ks.xp(((const double *)&D.xp[p])[lane >> 1], lane >> 1);
    const double px = __shfl_sync(0xffffffffu, xi, 0), py = __shfl_sync(0xffffffffu, xi, 2),
                 pz = __shfl_sync(0xffffffffu, xi, 4);
    if (lane == 0) {
        D.xp_prev[p] = D.xp[p];
        D.xp[p] = make_double4_32a(px, py, pz, 0.0);
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) raise_error(D.err, OTM_ERR_NONFINITE, D.mgid[p]);
    }
    __syncwarp();   // the old row is read completely before the new support overwrites it
    int32_t *list = (int32_t *)smem_raw + (size_t)warp * next_pow2(S);
    SearchGrid G{D.grid, D.cell_start, D.spos32, D.spos};
    const int cnt = warp_support_search(G, D.sc, px, py, pz, list, S, lane);
    if (cnt > S) {
        if (lane == 0) {
            raise_error(D.err, OTM_ERR_CAPACITY, D.mgid[p]);
            D.cnt[p] = 0;
        }
        return;
    }
    __syncwarp();
    store_support(D, list, base, cnt, lane);
    if (lane == 0) D.cnt[p] = cnt;
}

cudaError_t launch_kin_search(const Dev &D, cudaStream_t s, long long *launches)
{
    const size_t smem = (size_t)kSearchWarps * next_pow2(D.S) * sizeof(int32_t);
    const unsigned blocks = (unsigned)((D.nm + kSearchWarps - 1) / kSearchWarps);
    if (blocks == 0) return cudaSuccess;
    if (D.precision == OTM_PRECISION_MIXED)
        k_kin_search<true><<<blocks, kSearchWarps * kWarp, smem, s>>>(D);
    else
        k_kin_search<false><<<blocks, kSearchWarps * kWarp, smem, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_search(const Dev &D, cudaStream_t s, long long *launches)
{
    const size_t smem = (size_t)kSearchWarps * next_pow2(D.S) * sizeof(int32_t);
    const unsigned blocks = (unsigned)((D.nm + kSearchWarps - 1) / kSearchWarps);
    if (blocks == 0) return cudaSuccess;
    k_search<<<blocks, kSearchWarps * kWarp, smem, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

// ======================================================================== k_lme
// store the solution lambda of MP p, and the lambda it replaces where the mode says so
__device__ __forceinline__ void lme_record(const Dev &D, int64_t p, double l0, double l1, double l2)
{
    if (D.lme_mode == kLmeStep) {
        for (int i = 0; i < 3; i++) {
            D.lam_prev3[3 * p + i] = D.lam_prev2[3 * p + i];
            D.lam_prev2[3 * p + i] = D.lam_prev[3 * p + i];
            D.lam_prev[3 * p + i] = D.lam[3 * p + i];
        }
    } else if (D.lme_mode == kLmePlain || (D.lme_mode == kLmeRetry && D.lme_fail[p])) {
        // a plain start, or an MP solved again after node insertion: its previous solutions were
        // not one step apart from this one, so the history restarts at the new solution
        D.lam_prev[3 * p] = D.lam_prev2[3 * p] = D.lam_prev3[3 * p] = l0;
        D.lam_prev[3 * p + 1] = D.lam_prev2[3 * p + 1] = D.lam_prev3[3 * p + 1] = l1;
        D.lam_prev[3 * p + 2] = D.lam_prev2[3 * p + 2] = D.lam_prev3[3 * p + 2] = l2;
    }
    D.lam[3 * p] = l0;
    D.lam[3 * p + 1] = l1;
    D.lam[3 * p + 2] = l2;
}

// Shared-memory rows per MP in k_lme. With 336 slots a block of 4 MPs takes 55 KB and 4 blocks
// fit an SM (3 with full 384-slot rows), which hides more of the FP64 pipe's dependency and
// barrier stalls; the supports of the benchmark rods stay below (at most 316 slots mid-run on the
// 2.85 M-MP rod). MPs with larger supports are deferred to k_lme_wide, which runs the same block
// code with rows of the full capacity S, so either launch gives the same bits.
constexpr int kLmeRows = 336;

__host__ __device__ __forceinline__ int lme_rows(int S) { return S < kLmeRows ? S : kLmeRows; }

// The LME solve of the block's MPs (one per warp; p the warp's MP, active whether it has one),
// shared-memory rows of `rows` slots. Every thread of the block calls it (block barriers inside);
// the exponential's table is read from global memory (L1-resident, 8 KB).
template <bool MIXED, bool STAB>
__device__ __forceinline__ void lme_block(const Dev &D, int64_t p, bool active, int rows, unsigned char *smem_raw)
{
    const double *__restrict__ T = g_exp2_table;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = D.S;
    MpNewton *NS = (MpNewton *)(smem_raw + (size_t)kLmeWarps * 5 * (size_t)rows * sizeof(double));
    // every warp reaches the block barriers below; idle warps skip the work
    WarpSmem W = warp_smem(smem_raw, rows, warp);
    const int64_t base = p * (int64_t)S;
    MpNewton &M = NS[warp];
    int cnt = 0;
    double shift0 = 0;
    if (active) {
        const double4_32a xp = D.xp[p];
        cnt = D.cnt[p];
        // d_a = x_p - x_a and the prior exponent -beta |d_a|^2, minus the Newton solve's shift,
        // in units of ln2/1024
        const double beta_s = D.beta * kExpScale;
        shift0 = D.logz[p];
        const double shift_s = shift0 * kExpScale;
        for (int k = lane; k < cnt; k += kWarp) {
            const double4_32a a = D.x[D.ids[base + k]];
            const double x = xp.x - a.x, y = xp.y - a.y, z = xp.z - a.z;
            W.dx[k] = x; W.dy[k] = y; W.dz[k] = z;
            W.q[k] = fma(-beta_s, fma(z, z, fma(y, y, x * x)), -shift_s);
        }
        if (lane == 0) {
            // Eq. 14: the warm start is the previous step's lambda, or (within a step) the cubic
            // through the last four solutions: while the material deforms smoothly one Newton
            // step from it meets the tolerance
            double l0 = D.lam[3 * p], l1 = D.lam[3 * p + 1], l2 = D.lam[3 * p + 2];
            if (D.lme_mode == kLmeStep) {
                // cubic: 4 l_n - 6 l_{n-1} + 4 l_{n-2} - l_{n-3}
                const double *a1 = D.lam_prev + 3 * p, *a2 = D.lam_prev2 + 3 * p, *a3 = D.lam_prev3 + 3 * p;
                l0 = fma(4.0, l0 + a2[0], -fma(6.0, a1[0], a3[0]));
                l1 = fma(4.0, l1 + a2[1], -fma(6.0, a1[1], a3[1]));
                l2 = fma(4.0, l2 + a2[2], -fma(6.0, a1[2], a3[2]));
            }
            M.trial[0] = M.ws[0] = l0;
            M.trial[1] = M.ws[1] = l1;
            M.trial[2] = M.ws[2] = l2;
            M.t = 1.0;
            M.have_cur = M.iters = M.iters_total = M.halvings = M.retried = 0;
            M.shift0 = shift0;
            newton_set_trial(M);
            M.state = cnt > 0 ? kNewtonEval : kNewtonFail;
        }
    } else if (lane == 0) {
        M.state = kNewtonIdle;
    }
    __syncthreads();
    // rounds: evaluations of the pending trials, then the scalar decisions
    for (;;) {
        if (M.state == kNewtonEval) {
            __syncwarp();
            lme_eval_block<MIXED>(W, cnt, M, lane, T);
        }
        __syncthreads();
        bool pending = false;
        if (warp == 0 && lane < kLmeWarps) {
            newton_round(NS[lane], D.tol_abs, D.max_newton);
            pending = NS[lane].state == kNewtonEval;
        }
        if (!__syncthreads_or(pending)) break;
    }
    if (!active) return;
    const int st = M.state == kNewtonDone ? OTM_OK : OTM_ERR_LME_NOCONV;
    if (lane == 0) {
        D.newton_it[p] = M.iters_total;
        if (st == OTM_OK) {
            lme_record(D, p, M.lam[0], M.lam[1], M.lam[2]);
            D.logz_in[p] = shift0;
            D.logz[p] = M.logz;
        } else if (D.insert_mode && cnt > 0) {
            D.lme_fail[p] = 1;          // node insertion follows (lambda keeps the warm start)
            atomicAdd(D.n_fail, 1);
        } else {
            raise_error(D.err, st, D.mgid[p]);
        }
    }
    double inv[6];
    for (int i = 0; i < 6; i++) inv[i] = M.inv[i];
    const double iZ = M.iZ;
    if (st != OTM_OK) return;

    // N_a = w_a / Z and grad N_a = -N_a J^-1 d_a = -K e_a with e_a = N_a d_a and K = J^-1 = Z J'^-1
    // (one symmetric 3x3 per MP). The pair rows keep (N_a, e_a) and the MP keeps K: whoever needs
    // grad N applies K once per MP (the kinematics gather sums du_a (x) e_a, and dF = 1 - G K
    // follows in the return map), so the per-pair work here is N, e and the contributions.
    // Eq. 5 contributions of the next step, stored at the pair's place in its node's influence
    // list: mass m_p N_a, force -v_p sigma_p grad N_a = (v_p sigma_p K) e_a = Q e_a.
    const double mp = D.mass[p], vp = D.vol[p];
    const double *sg = D.sig + 6 * p;
    double Kc[6], Q[9];
    {
        // lanes 0-5 form K (and store it), lanes 0-8 one entry of Q each; all lanes get both
        const double Zc = M.C[0];
        const double kj = (lane < 6) ? inv[lane] * Zc : 0.0;
        if (lane < 6) D.Kinv[6 * p + lane] = kj;
#pragma unroll
        for (int i = 0; i < 6; i++) Kc[i] = __shfl_sync(0xffffffffu, kj, i);
        // symmetric index of (i, j) in (xx, yy, zz, xy, yz, xz)
        const int li = (lane < 9) ? lane / 3 : 0, lc = (lane < 9) ? lane % 3 : 0;
        auto sym = [](int i, int j) { return i == j ? i : (i + j == 1 ? 3 : (i + j == 3 ? 4 : 5)); };
        const double q = vp * (sg[sym(li, 0)] * Kc[sym(0, lc)] + sg[sym(li, 1)] * Kc[sym(1, lc)] +
                               sg[sym(li, 2)] * Kc[sym(2, lc)]);
#pragma unroll
        for (int i = 0; i < 9; i++) Q[i] = __shfl_sync(0xffffffffu, q, i);
    }
    int em = -2000, ef = -2000;   // largest binary exponents of the stored mass / force terms
    float Qf[9];
#pragma unroll
    for (int i = 0; i < 9; i++) Qf[i] = MIXED ? (float)Q[i] : 0.f;
    const float mpf = MIXED ? (float)mp : 0.f;
    // stabilisation (Eq. 7-8): -eps N_a e_a / |x_a,n-1 - x_p,n-1|,
    // e_a = x_a - x_p - dF (x_a,n-1 - x_p,n-1), with dF the increment that led to this state
    double xq0 = 0, xq1 = 0, xq2 = 0, F00 = 0, F01 = 0, F02 = 0, F10 = 0, F11 = 0, F12 = 0, F20 = 0, F21 = 0, F22 = 0;
    if (STAB) {
        const double4_32a q = D.xp_prev[p];
        xq0 = q.x; xq1 = q.y; xq2 = q.z;
        const double *Fd = D.dF + 9 * p;
        F00 = Fd[0]; F01 = Fd[1]; F02 = Fd[2]; F10 = Fd[3]; F11 = Fd[4]; F12 = Fd[5]; F20 = Fd[6]; F21 = Fd[7];
        F22 = Fd[8];
    }
    for (int k = lane; k < cnt; k += kWarp) {
        const double wk = W.w[k];
        const double N = wk * iZ;
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        double ex, ey, ez;
        float fN = 0.f, fex = 0.f, fey = 0.f, fez = 0.f;
        if (MIXED) {
            // e = N d in FP32 (every consumer of the mixed path's rows rounds them to FP32),
            // stored widened exactly; N stays FP64
            fN = f32_round_bits(N);
            fex = fN * f32_round_bits(x);
            fey = fN * f32_round_bits(y);
            fez = fN * f32_round_bits(z);
            ex = df_widen(fex); ey = df_widen(fey); ez = df_widen(fez);
        } else {
            ex = N * x; ey = N * y; ez = N * z;
        }
        D.shape[base + k] = make_double4_32a(N, ex, ey, ez);
        const int id = D.ids[base + k];
        const int64_t pos = (int64_t)D.noff[id] + D.rank[base + k];
        double sx = 0.0, sy = 0.0, sz = 0.0;
        if (STAB) {
            const double4_32a a = D.x_prev[id];
            const double q0 = a.x - xq0, q1 = a.y - xq1, q2 = a.z - xq2;
            const double len = sqrt(q0 * q0 + q1 * q1 + q2 * q2);
            if (len > 1e-12 * D.h) {
                const double c = -D.eps_stab * N / len;
                sx = c * (-x - (F00 * q0 + F01 * q1 + F02 * q2));
                sy = c * (-y - (F10 * q0 + F11 * q1 + F12 * q2));
                sz = c * (-z - (F20 * q0 + F21 * q1 + F22 * q2));
            }
        }
        if (MIXED) {
            const float c0 = mpf * fN;
            float c1 = fmaf(Qf[2], fez, fmaf(Qf[1], fey, Qf[0] * fex));
            float c2 = fmaf(Qf[5], fez, fmaf(Qf[4], fey, Qf[3] * fex));
            float c3 = fmaf(Qf[8], fez, fmaf(Qf[7], fey, Qf[6] * fex));
            if (STAB) {
                c1 += f32_round_bits(sx);
                c2 += f32_round_bits(sy);
                c3 += f32_round_bits(sz);
            }
            D.contrib32[pos] = make_float4(c0, c1, c2, c3);
            em = max(em, fexp32(c0));
            ef = max(ef, max(fexp32(c1), max(fexp32(c2), fexp32(c3))));
        } else {
            const double cm = mp * N;
            double fx = Q[0] * ex + Q[1] * ey + Q[2] * ez;
            double fy = Q[3] * ex + Q[4] * ey + Q[5] * ez;
            double fz = Q[6] * ex + Q[7] * ey + Q[8] * ez;
            if (STAB) {
                fx += sx;
                fy += sy;
                fz += sz;
            }
            D.contrib64[pos] = make_double4_32a(cm, fx, fy, fz);
            em = max(em, fexp64(cm));
            ef = max(ef, max(fexp64(fx), max(fexp64(fy), fexp64(fz))));
        }
    }
    em = __reduce_max_sync(0xffffffffu, em);
    ef = __reduce_max_sync(0xffffffffu, ef);
    if (lane == 0) {
        atomicMax(&D.emax[0], em);
        atomicMax(&D.emax[1], ef);
    }
}

template <bool MIXED, bool STAB>
__global__ void __launch_bounds__(kLmeWarps * kWarp) k_lme(const Dev D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kLmeWarps + (threadIdx.x >> 5);
    const int rows = lme_rows(D.S);
    bool active = (p < D.nm) && !has_error(D.err);
    if (active && D.cnt[p] > rows) {   // solved by k_lme_wide
        if (lane == 0) D.lme_defer[atomicAdd(D.n_defer, 1)] = (int32_t)p;
        active = false;
    }
    lme_block<MIXED, STAB>(D, p, active, rows, smem_raw);
}

// the deferred MPs, 4 per block and round, with rows of the full capacity S (grid-stride over the
// list, whose length the previous launch left in *n_defer)
template <bool MIXED, bool STAB>
__global__ void __launch_bounds__(kLmeWarps * kWarp) k_lme_wide(const Dev D)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = *D.n_defer;
    for (int g = blockIdx.x; g * kLmeWarps < n; g += gridDim.x) {
        const int i = g * kLmeWarps + (threadIdx.x >> 5);
        const int64_t p = (i < n) ? (int64_t)D.lme_defer[i] : -1;
        lme_block<MIXED, STAB>(D, p, p >= 0 && !has_error(D.err), D.S, smem_raw);
    }
}

static size_t lme_block_smem(int rows)
{
    return (size_t)kLmeWarps * 5 * (size_t)rows * sizeof(double) + (size_t)kLmeWarps * sizeof(MpNewton);
}

template <bool MIXED, bool STAB>
static cudaError_t launch_lme_t(const Dev &D, cudaStream_t s, unsigned blocks)
{
    const size_t smem = lme_block_smem(lme_rows(D.S)), smem_wide = lme_block_smem(D.S);
    cudaError_t e = cudaFuncSetAttribute(k_lme<MIXED, STAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_lme_wide<MIXED, STAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_wide);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(D.n_defer, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_lme<MIXED, STAB><<<blocks, kLmeWarps * kWarp, smem, s>>>(D);
    // one persistent round of blocks over the deferred MPs (none on most steps: the launch then
    // returns at once)
    k_lme_wide<MIXED, STAB><<<152 * 3, kLmeWarps * kWarp, smem_wide, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_lme(const Dev &D, cudaStream_t s, long long *launches)
{
    const unsigned blocks = (unsigned)((D.nm + kLmeWarps - 1) / kLmeWarps);
    if (blocks == 0) return cudaSuccess;
    const bool mixed = D.precision == OTM_PRECISION_MIXED, stab = D.eps_stab > 0.0;
    cudaError_t e = mixed ? (stab ? launch_lme_t<true, true>(D, s, blocks) : launch_lme_t<true, false>(D, s, blocks))
                          : (stab ? launch_lme_t<false, true>(D, s, blocks) : launch_lme_t<false, false>(D, s, blocks));
    if (launches) *launches += 2;
    return e;
}

// (N, grad N) of every slot of a padded row set, for state export: already stored in shape[]
// ======================================================================== k_kinematics
// warp per MP: the 12 sums x_p,i = sum N x_a,i and G_ij = sum du_a,i e_a,j (e_a = N_a d_a, the
// stored pair row) over the old support; lanes 2j write sum j. Eq. 11 is then
// dF = 1 + sum du_a (x) grad N_a = 1 - G K with K = J^-1 of the old support's LME solve, formed
// once per MP in the thread-per-MP return-map kernel with the products with F, det(dF) and the
// volume update.
template <bool MIXED>
__global__ void __launch_bounds__(128) k_kinematics(const Dev D)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    const int n = D.cnt[p];
    const int64_t base = p * (int64_t)D.S;
    KinSum<MIXED> ks;
    ks.gather(D, base, n, lane);
    const int j = rs12_value(lane);
    if (rs12_writer(lane)) {
        if (j < 3) {
            const double old = ((const double *)&D.xp[p])[j];
            const double x = ks.xp(old, j);
            ((double *)&D.xp_prev[p])[j] = old;
            ((double *)&D.xp[p])[j] = x;
            if (!isfinite(x)) raise_error(D.err, OTM_ERR_NONFINITE, D.mgid[p]);
        } else {
            D.dF[9 * p + (j - 3)] = ks.g();   // row-major G = sum du (x) e; k_return_map forms dF
        }
    }
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

__global__ void __launch_bounds__(128) k_return_map(const Dev D)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= D.nm) return;
    if (has_error(D.err)) return;
    RmIn in;
    {   // Eq. 11: dF = 1 + sum du_a (x) grad N_a = 1 - G K (G from the kinematics gather, K = J^-1
        // of the LME solve the gather's shape functions came from)
        double G[9];
        for (int i = 0; i < 9; i++) G[i] = D.dF[9 * p + i];
        const double *k = D.Kinv + 6 * p;
        const double K[9] = {k[0], k[3], k[5], k[3], k[1], k[4], k[5], k[4], k[2]};
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                const double gk = G[3 * i] * K[j] + G[3 * i + 1] * K[3 + j] + G[3 * i + 2] * K[6 + j];
                in.dF[3 * i + j] = (i == j ? 1.0 : 0.0) - gk;
            }
        for (int i = 0; i < 9; i++) D.dF[9 * p + i] = in.dF[i];
    }
    const double *d = in.dF;
    // Eq. 10-12: F_{n+1} = dF F_n, v_{n+1} = det(dF) v_n
    const double det = d[0] * (d[4] * d[8] - d[5] * d[7]) - d[1] * (d[3] * d[8] - d[5] * d[6]) +
                       d[2] * (d[3] * d[7] - d[4] * d[6]);
    if (!(det > 0.0)) {
        raise_error(D.err, OTM_ERR_JACOBIAN, D.mgid[p]);
        return;
    }
    double *F = D.F + 9 * p;
    double Fo[9], Fn[9];
    for (int i = 0; i < 9; i++) Fo[i] = F[i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            Fn[3 * i + j] = d[3 * i] * Fo[j] + d[3 * i + 1] * Fo[3 + j] + d[3 * i + 2] * Fo[6 + j];
    for (int i = 0; i < 9; i++) F[i] = Fn[i];
    D.vol[p] *= det;
    in.J = Fn[0] * (Fn[4] * Fn[8] - Fn[5] * Fn[7]) - Fn[1] * (Fn[3] * Fn[8] - Fn[5] * Fn[6]) +
           Fn[2] * (Fn[3] * Fn[7] - Fn[4] * Fn[6]);
    for (int i = 0; i < 6; i++) in.be[i] = D.be[6 * p + i];
    in.ebar = D.ebar[p];
    in.T = D.T[p];
    in.guess = D.rate[p] * D.dt;   // the previous step's plastic increment
    double Q0[9];
    for (int i = 0; i < 9; i++) Q0[i] = D.Qe[9 * p + i];
    in.Q0 = Q0;
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
    for (int i = 0; i < 9; i++) D.Qe[9 * p + i] = o.Q[i];
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
    k_search_only(const GridDev *g, const int32_t *cell_start, const float4 *spos32, const double4_32a *spos,
                  const SearchConst C, const double *mp_x, int64_t nm, int S, int32_t *ids, int32_t *counts,
                  int32_t *status, const unsigned long long *grid_err)
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
    SearchGrid G{g, cell_start, spos32, spos};
    const int cnt = warp_support_search(G, C, px, py, pz, list, S, lane);
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
    k_search_only<<<blocks, kSearchWarps * kWarp, smem, s>>>(V.g, V.cell_start, V.spos32, V.spos,
                                                             make_search_const(cell, rs2), mp_x, nm, S, ids, counts,
                                                             status, V.err);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kLmeWarps * kWarp)
    k_lme_only(const double *node_x, const double *mp_x, int64_t nm, const int32_t *ids, const int32_t *counts,
               int S, double beta, double tol, int max_newton, double *lam, double *shape, int32_t *iters_out,
               int32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *T = (double *)smem_raw;
    exp_table_load(T);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kLmeWarps + warp;
    if (p >= nm) return;
    WarpSmem W = warp_smem(smem_raw + kExpTable * sizeof(double), S, warp);
    const int n = counts[p];
    if (n > S || n <= 0) {
        if (lane == 0) atomicCAS(status, 0, n > S ? OTM_ERR_CAPACITY : OTM_ERR_LME_NOCONV);
        return;
    }
    const double px = mp_x[3 * p], py = mp_x[3 * p + 1], pz = mp_x[3 * p + 2];
    const int64_t base = p * (int64_t)S;
    for (int k = lane; k < n; k += kWarp) {
        const int64_t id = ids[base + k];
        const double x = px - node_x[3 * id], y = py - node_x[3 * id + 1], z = pz - node_x[3 * id + 2];
        W.dx[k] = x; W.dy[k] = y; W.dz[k] = z;
        W.q[k] = -(beta * kExpScale) * fma(z, z, fma(y, y, x * x));
    }
    __syncwarp();
    double l0 = lam[3 * p], l1 = lam[3 * p + 1], l2 = lam[3 * p + 2];
    const double shift = lme_fmax(W.dx, W.dy, W.dz, W.q, n, l0, l1, l2, 0.0, lane);
    const double shift_s = shift * kExpScale;
    for (int k = lane; k < n; k += kWarp) W.q[k] -= shift_s;
    __syncwarp();
    LmeSums E;
    int iters = 0;
    int st = lme_newton(W.dx, W.dy, W.dz, W.q, W.w, n, l0, l1, l2, shift, tol, max_newton, lane, T, E, iters);
    double inv[6];
    if (st == OTM_OK && !lme_jinv(E, inv)) st = OTM_ERR_LME_NOCONV;
    if (lane == 0) {
        if (iters_out) iters_out[p] = iters;
        if (st != OTM_OK) atomicCAS(status, 0, st);
        lam[3 * p] = l0; lam[3 * p + 1] = l1; lam[3 * p + 2] = l2;
    }
    if (st != OTM_OK) return;
    const double iZ = 1.0 / E.Z;
    for (int k = lane; k < n; k += kWarp) {
        const double wk = W.w[k];
        const double x = W.dx[k], y = W.dy[k], z = W.dz[k];
        double *o = shape + 4 * (base + k);
        o[0] = wk * iZ;
        o[1] = -wk * (inv[0] * x + inv[3] * y + inv[5] * z);
        o[2] = -wk * (inv[3] * x + inv[1] * y + inv[4] * z);
        o[3] = -wk * (inv[5] * x + inv[4] * y + inv[2] * z);
    }
}

cudaError_t launch_lme_only(const double *node_x, const double *mp_x, int64_t nm, const int32_t *ids,
                            const int32_t *counts, int S, double beta, double tol_abs, int max_newton, double *lam,
                            double *shape, int32_t *iters, int32_t *status, cudaStream_t s)
{
    const size_t smem = lme_smem_bytes(S, kLmeWarps);
    const unsigned blocks = (unsigned)((nm + kLmeWarps - 1) / kLmeWarps);
    if (blocks == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_lme_only, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_lme_only<<<blocks, kLmeWarps * kWarp, smem, s>>>(node_x, mp_x, nm, ids, counts, S, beta, tol_abs, max_newton,
                                                       lam, shape, iters, status);
    return cudaGetLastError();
}

// self-test of the table-driven exponential: mine = exp_scaled(y); ref = CUDA's exp of the same
// argument f = y ln2/1024 carried as a + b (a = fl(y c1), b its rounding error plus y times the
// low part of ln2/1024), ref = exp(a) (1 + b)
__global__ void k_exp_selftest(const double *y, int64_t n, double *mine, double *ref)
{
    __shared__ double T[kExpTable];
    exp_table_load(T);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = y[i];
        mine[i] = exp_scaled(v, T);
        const double a = v * kExpC1;
        const double b = fma(v, kExpC1, -a) + v * kExpC1lo;
        const double e = exp(a);
        ref[i] = fma(e, b, e);
    }
}

cudaError_t launch_exp_selftest(const double *x, int64_t n, double *mine, double *ref, cudaStream_t s)
{
    k_exp_selftest<<<152 * 4, 256, 0, s>>>(x, n, mine, ref);
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
    in.guess = 0.0;
    in.Q0 = nullptr;
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
