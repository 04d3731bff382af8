// otm_node.cu -- the node kernel (sm_103a): lumped mass and internal force as a segmented
// reduction over each node's influence list (Eq. 5), the central-difference update (Eq. 4),
// rigid contact (Sec. 4.1 wall, Sec. 4.2 tool) and the position update (Eq. 6).
//
// Determinism without float atomics and without sorting: every pair contribution is converted
// to a fixed-point integer whose least significant bit is 2^(Emax - 110) (FP64 path, 128-bit
// accumulators) or 2^(Emax - 46) (mixed path, 64-bit accumulators), Emax being the largest
// binary exponent of that field over all pairs of the step. Integer addition is associative,
// so the sum is exact and independent of the order in which the influence list was filled.
// Terms below the least significant bit (2^-110, resp. 2^-46, of the largest term) are truncated.
//
// Headroom: a term is below 2^(Emax + 1), i.e. below 2^111 (FP64) or 2^47 (mixed) units, and a
// node has at most 65,536 influences (the search raises OTM_ERR_CAPACITY beyond), so a node sum
// stays below 2^127 resp. 2^63 and fits the signed accumulator whatever the signs.
#include "otm_dev.cuh"

namespace otm {

struct I128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ void add128(I128 &a, const I128 &b)
{
    const unsigned long long lo = a.lo + b.lo;
    a.hi = a.hi + b.hi + (lo < a.lo ? 1 : 0);
    a.lo = lo;
}

// v / 2^(emax - 110) truncated toward zero, as a signed 128-bit integer
__device__ __forceinline__ I128 to_fixed128(double v, int emax)
{
    I128 r = {0ULL, 0LL};
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((b >> 52) & 0x7ff);
    if (ef == 0 || ef == 0x7ff) return r;   // zero / subnormal (negligible); non-finite caught elsewhere
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFULL) | 0x0010000000000000ULL;
    const int sh = (ef - 1023) - emax + 58;  // value = m * 2^(e - 52); lsb = 2^(emax - 110)
    if (sh < -52) return r;
    if (sh < 0) {
        r.lo = m >> (-sh);
    } else if (sh < 64) {
        r.lo = m << sh;
        r.hi = (sh == 0) ? 0 : (long long)(m >> (64 - sh));
    } else {
        r.hi = (long long)(m << (sh - 64));
    }
    if (b >> 63) {   // two's complement negation
        r.lo = ~r.lo + 1ULL;
        r.hi = ~r.hi + (r.lo == 0ULL ? 1 : 0);
    }
    return r;
}

__device__ __forceinline__ double from_fixed128(const I128 &a, int emax)
{
    // value = (hi * 2^64 + lo) * 2^(emax - 110)
    const double v = (double)a.hi * 18446744073709551616.0 + (double)a.lo;
    return ldexp(v, emax - 110);
}

__device__ __forceinline__ I128 warp_sum128(I128 a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        I128 b;
        b.lo = __shfl_xor_sync(0xffffffffu, a.lo, o);
        b.hi = __shfl_xor_sync(0xffffffffu, a.hi, o);
        add128(a, b);
    }
    return a;
}

__device__ __forceinline__ long long to_fixed64(float v, int emax)
{
    const unsigned int b = __float_as_uint(v);
    const int ef = (int)((b >> 23) & 0xff);
    if (ef == 0 || ef == 0xff) return 0;
    const long long m = (long long)((b & 0x007FFFFFu) | 0x00800000u);
    const int sh = (ef - 127) - emax + 23;   // value = m * 2^(e - 23); lsb = 2^(emax - 46)
    long long r;
    if (sh < -23) return 0;
    r = (sh < 0) ? (m >> (-sh)) : (m << sh);
    return (b >> 31) ? -r : r;
}

__device__ __forceinline__ long long warp_sum64(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------- contact
// rigid frictionless wall: project a penetrating node onto the plane
__device__ __forceinline__ void wall_project(const Dev &D, double &x, double &y, double &z)
{
    const double g = (x - D.wall_p[0]) * D.wall_n[0] + (y - D.wall_p[1]) * D.wall_n[1] +
                     (z - D.wall_p[2]) * D.wall_n[2];
    if (g < 0.0) {
        x -= g * D.wall_n[0];
        y -= g * D.wall_n[1];
        z -= g * D.wall_n[2];
    }
}

// rigid tool (wedge between rake and flank faces, moving along -x): normal projection onto the
// nearer face, Coulomb stick/slip of the increment relative to the tool at the penalty limit
__device__ __forceinline__ void tool_project(const Dev &D, double t_next, double ux, double uy, double uz,
                                             double &x, double &y, double &z)
{
    const double xt = D.tool_x0 - D.tool_v * t_next, yt = D.tool_tip_y;
    const double nrx = -cos(D.tool_rake), nry = sin(D.tool_rake);
    const double nfx = sin(D.tool_clear), nfy = -cos(D.tool_clear);
    const double rx = x - xt, ry = y - yt;
    const double gr = rx * nrx + ry * nry, gf = rx * nfx + ry * nfy;
    if (!(gr < 0.0 && gf < 0.0)) return;
    const bool rake = (gr >= gf);
    const double nx = rake ? nrx : nfx, ny = rake ? nry : nfy;
    const double pen = -(rake ? gr : gf);
    x += pen * nx;
    y += pen * ny;
    const double wx = ux + D.tool_v * D.dt, wy = uy, wz = uz;
    const double wn = wx * nx + wy * ny;
    const double tx = wx - wn * nx, ty = wy - wn * ny, tz = wz;
    const double tn = sqrt(tx * tx + ty * ty + tz * tz);
    const double lim = D.friction * pen;
    const double sc = (tn <= lim) ? 1.0 : lim / tn;
    x -= sc * tx;
    y -= sc * ty;
    z -= sc * tz;
}

// ---------------------------------------------------------------------------- node kernel
template <bool MIXED>
__global__ void __launch_bounds__(kNodeWarps * kWarp) k_node_update(const Dev D, double t_next)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= D.nn) return;
    if (has_error(D.err)) return;
    const int b = D.noff[i], L = D.noff[i + 1] - b;
    const int em = D.emax[0], ef = D.emax[1];
    double m, rx, ry, rz;
    if (MIXED) {
        long long sm = 0, sx = 0, sy = 0, sz = 0;
        for (int k = lane; k < L; k += kWarp) {
            const float4 c = D.contrib32[b + k];
            sm += to_fixed64(c.x, em);
            sx += to_fixed64(c.y, ef);
            sy += to_fixed64(c.z, ef);
            sz += to_fixed64(c.w, ef);
        }
        sm = warp_sum64(sm); sx = warp_sum64(sx); sy = warp_sum64(sy); sz = warp_sum64(sz);
        m = ldexp((double)sm, em - 46);
        rx = ldexp((double)sx, ef - 46);
        ry = ldexp((double)sy, ef - 46);
        rz = ldexp((double)sz, ef - 46);
    } else {
        I128 sm = {0, 0}, sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
        for (int k = lane; k < L; k += kWarp) {
            const double4_32a c = D.contrib64[b + k];
            add128(sm, to_fixed128(c.x, em));
            add128(sx, to_fixed128(c.y, ef));
            add128(sy, to_fixed128(c.z, ef));
            add128(sz, to_fixed128(c.w, ef));
        }
        sm = warp_sum128(sm); sx = warp_sum128(sx); sy = warp_sum128(sy); sz = warp_sum128(sz);
        m = from_fixed128(sm, em);
        rx = from_fixed128(sx, ef);
        ry = from_fixed128(sy, ef);
        rz = from_fixed128(sz, ef);
    }
    if (lane != 0) return;
    D.mr[i] = make_double4_32a(m, rx, ry, rz);
    const double4_32a xo = D.x[i];
    double ux, uy, uz;
    const bool fixed = (D.nflags[i] & OTM_FLAG_FIXED) != 0;
    const double dt2 = D.dt * D.dt;
    if (MIXED) {
        float4 u = D.du32[i];
        if (fixed) {
            u = make_float4(0.f, 0.f, 0.f, 0.f);
        } else if (m > 0.0) {
            const float s = (float)(dt2 / m);
            u.x += s * (float)rx;
            u.y += s * (float)ry;
            u.z += s * (float)rz;
        }
        ux = u.x; uy = u.y; uz = u.z;
    } else {
        double4_32a u = D.du[i];
        if (fixed) {
            u = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        } else if (m > 0.0) {
            u.x += dt2 * rx / m;
            u.y += dt2 * ry / m;
            u.z += dt2 * rz / m;
        }
        ux = u.x; uy = u.y; uz = u.z;
    }
    double x = xo.x + ux, y = xo.y + uy, z = xo.z + uz;
    if (!fixed) {
        if (D.wall) wall_project(D, x, y, z);
        if (D.tool) tool_project(D, t_next, ux, uy, uz, x, y, z);
    }
    ux = x - xo.x; uy = y - xo.y; uz = z - xo.z;
    if (MIXED)
        D.du32[i] = make_float4((float)ux, (float)uy, (float)uz, 0.f);
    D.du[i] = make_double4_32a(ux, uy, uz, 0.0);
    D.x_prev[i] = xo;
    D.x[i] = make_double4_32a(x, y, z, 0.0);
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) raise_error(D.err, OTM_ERR_NONFINITE, D.ngid[i]);
}

cudaError_t launch_node_update(const Dev &D, double t_next, cudaStream_t s, long long *launches)
{
    const unsigned blocks = (unsigned)((D.nn * 32 + kNodeWarps * 32 - 1) / (kNodeWarps * 32));
    if (blocks == 0) return cudaSuccess;
    if (D.precision == OTM_PRECISION_MIXED)
        k_node_update<true><<<blocks, kNodeWarps * 32, 0, s>>>(D, t_next);
    else
        k_node_update<false><<<blocks, kNodeWarps * 32, 0, s>>>(D, t_next);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace otm
