// otm_adjoint.cu -- reverse-mode adjoint of one explicit step (sm_103a), topology, wall-contact set
// and elastic/plastic branches frozen at the trajectory being differentiated. One backward step
// takes the adjoint of the state after step n to the adjoint of the state before it:
//   k_adj_lme   : Eq. 14 by the implicit-function theorem (warp per MP, supports of state n+1)
//   k_adj_rm    : Sec. 4.1 / 4.2 return map as isotropic tensor functions of b_tr + Eq. 10-12
//                 (thread per MP)
//   k_adj_kin   : Eq. 9 and Eq. 11 transposed (warp per MP, supports of state n)
//   k_adj_node  : Eq. 4 and Eq. 6 with the frozen wall projection transposed (warp per node; the
//                 per-pair node contributions are summed over the node-major segments)
//   k_adj_force : Eq. 5 transposed (warp per MP, supports of state n)
#include "otm_dev.cuh"
#include "otm_rm.cuh"

namespace otm {

constexpr int kAdjWarps = 4;

// (N, grad N) of a stored pair row (N, e = N d): grad N = -K e with K = J^-1 of the MP's LME
// solve (xx, yy, zz, xy, yz, xz)
__device__ __forceinline__ double4_32a grad_row(const double4_32a r, double k0, double k1, double k2, double k3,
                                                double k4, double k5)
{
    return make_double4_32a(r.x, -(k0 * r.y + k3 * r.z + k5 * r.w), -(k3 * r.y + k1 * r.z + k4 * r.w),
                            -(k5 * r.y + k4 * r.z + k2 * r.w));
}

// ---------------------------------------------------------------------------- LME backward
// d_a = x_p - x_a, N = softmax(f), f_a = -beta |d_a|^2 + lambda . d_a, lambda from
// r = sum N d = 0, grad N_a = -N_a H^-1 d_a, H = sum N d d^T - r r^T.
__global__ void __launch_bounds__(kAdjWarps * kWarp) k_adj_lme(const Dev D, const AdjDev A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kAdjWarps + warp;
    if (p >= D.nm) return;
    const int S = D.S;
    double *sm = (double *)smem_raw + (size_t)warp * 7 * S;
    double *dx = sm, *dy = sm + S, *dz = sm + 2 * S, *Nb = sm + 3 * S, *bx = sm + 4 * S, *by = sm + 5 * S,
           *bz = sm + 6 * S;
    const int n = D.cnt[p];
    const int64_t base = p * (int64_t)S;
    const double4_32a xp = D.xp[p];
    const double l0 = D.lam[3 * p], l1 = D.lam[3 * p + 1], l2 = D.lam[3 * p + 2], beta = D.beta;
    double v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = 0.0;
    for (int k = lane; k < n; k += kWarp) {
        const double4_32a a = D.x[D.ids[base + k]];
        const double x = xp.x - a.x, y = xp.y - a.y, z = xp.z - a.z;
        dx[k] = x; dy[k] = y; dz[k] = z;
        const double N = D.shape[base + k].x;
        v[0] += N * x; v[1] += N * y; v[2] += N * z;
        v[3] += N * x * x; v[4] += N * y * y; v[5] += N * z * z;
        v[6] += N * x * y; v[7] += N * y * z; v[8] += N * x * z;
    }
    double t = warp_reduce_scatter16(v, lane);
    double r0 = __shfl_sync(0xffffffffu, t, 0), r1 = __shfl_sync(0xffffffffu, t, 2), r2 = __shfl_sync(0xffffffffu, t, 4);
    const double h00 = __shfl_sync(0xffffffffu, t, 6) - r0 * r0, h11 = __shfl_sync(0xffffffffu, t, 8) - r1 * r1;
    const double h22 = __shfl_sync(0xffffffffu, t, 10) - r2 * r2, h01 = __shfl_sync(0xffffffffu, t, 12) - r0 * r1;
    const double h12 = __shfl_sync(0xffffffffu, t, 14) - r1 * r2, h02 = __shfl_sync(0xffffffffu, t, 16) - r0 * r2;
    const double c00 = h11 * h22 - h12 * h12, c01 = h02 * h12 - h01 * h22, c02 = h01 * h12 - h02 * h11;
    const double c11 = h00 * h22 - h02 * h02, c12 = h01 * h02 - h00 * h12, c22 = h00 * h11 - h01 * h01;
    const double det = h00 * c00 + h01 * c01 + h02 * c02;
    const double id = 1.0 / det;
    const double i00 = c00 * id, i11 = c11 * id, i22 = c22 * id, i01 = c01 * id, i12 = c12 * id, i02 = c02 * id;
    // pass 1: G_a = -N_a u_a, u_a = H^-1 d_a;  Nb_a = Nbar_a - Gbar_a . u_a;  db_a = w_a = -N_a H^-1 Gbar_a;
    // Hbar = -sum w u^T
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = 0.0;
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double N = D.shape[base + k].x;
        const double4_32a pb = A.pb_cur[base + k];
        const double u0 = i00 * x + i01 * y + i02 * z, u1 = i01 * x + i11 * y + i12 * z, u2 = i02 * x + i12 * y + i22 * z;
        Nb[k] = pb.x - (pb.y * u0 + pb.z * u1 + pb.w * u2);
        const double w0 = -N * (i00 * pb.y + i01 * pb.z + i02 * pb.w);
        const double w1 = -N * (i01 * pb.y + i11 * pb.z + i12 * pb.w);
        const double w2 = -N * (i02 * pb.y + i12 * pb.z + i22 * pb.w);
        bx[k] = w0; by[k] = w1; bz[k] = w2;
        v[0] -= w0 * u0; v[1] -= w0 * u1; v[2] -= w0 * u2;
        v[3] -= w1 * u0; v[4] -= w1 * u1; v[5] -= w1 * u2;
        v[6] -= w2 * u0; v[7] -= w2 * u1; v[8] -= w2 * u2;
    }
    t = warp_reduce_scatter16(v, lane);
    double Hb[9];
#pragma unroll
    for (int i = 0; i < 9; i++) Hb[i] = __shfl_sync(0xffffffffu, t, 2 * i);
    const double s00 = Hb[0], s11 = Hb[4], s22 = Hb[8];
    const double s01 = 0.5 * (Hb[1] + Hb[3]), s12 = 0.5 * (Hb[5] + Hb[7]), s02 = 0.5 * (Hb[2] + Hb[6]);
    const double hr0 = s00 * r0 + s01 * r1 + s02 * r2, hr1 = s01 * r0 + s11 * r1 + s12 * r2,
                 hr2 = s02 * r0 + s12 * r1 + s22 * r2;
    // pass 2: H = sum N d d^T - r r^T contributions; S = sum N Nb
    double Ssum = 0.0;
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double N = D.shape[base + k].x;
        const double hd0 = s00 * x + s01 * y + s02 * z, hd1 = s01 * x + s11 * y + s12 * z, hd2 = s02 * x + s12 * y + s22 * z;
        Nb[k] += (x * hd0 + y * hd1 + z * hd2) - 2.0 * (x * hr0 + y * hr1 + z * hr2);
        bx[k] += 2.0 * N * (hd0 - hr0);
        by[k] += 2.0 * N * (hd1 - hr1);
        bz[k] += 2.0 * N * (hd2 - hr2);
        Ssum += N * Nb[k];
    }
    Ssum = warp_sum(Ssum);
    // pass 3: softmax and the prior exponent; lambda bar
    double lb0 = 0, lb1 = 0, lb2 = 0;
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double N = D.shape[base + k].x;
        const double fb = N * (Nb[k] - Ssum);
        bx[k] += fb * (l0 - 2.0 * beta * x);
        by[k] += fb * (l1 - 2.0 * beta * y);
        bz[k] += fb * (l2 - 2.0 * beta * z);
        lb0 += fb * x; lb1 += fb * y; lb2 += fb * z;
    }
    lb0 = warp_sum(lb0); lb1 = warp_sum(lb1); lb2 = warp_sum(lb2);
    const double m0 = i00 * lb0 + i01 * lb1 + i02 * lb2, m1 = i01 * lb0 + i11 * lb1 + i12 * lb2,
                 m2 = i02 * lb0 + i12 * lb1 + i22 * lb2;
    // pass 4: lambda(d) through r = 0; scatter to the node and to x_p
    double px = 0, py = 0, pz = 0;
    for (int k = lane; k < n; k += kWarp) {
        const double x = dx[k], y = dy[k], z = dz[k];
        const double N = D.shape[base + k].x;
        const double dm = x * m0 + y * m1 + z * m2;
        const double b0 = bx[k] - N * (m0 + (l0 - 2.0 * beta * x) * dm);
        const double b1 = by[k] - N * (m1 + (l1 - 2.0 * beta * y) * dm);
        const double b2 = bz[k] - N * (m2 + (l2 - 2.0 * beta * z) * dm);
        px += b0; py += b1; pz += b2;
        const int nid = D.ids[base + k];
        A.sc1[(int64_t)D.noff[nid] + D.rank[base + k]] = make_double4_32a(b0, b1, b2, 0.0);
    }
    px = warp_sum(px); py = warp_sum(py); pz = warp_sum(pz);
    if (lane == 0) A.xpb[p] = make_double4_32a(px, py, pz, 0.0);
}

// ---------------------------------------------------------------------------- return map backward
struct RmDetail {
    double K, mu, J;
    double lam[3], Q[3][3], e[3], enorm, qtr, x, q, rho, tau[3], bA[3];
    bool plastic;
    double dsy_eb, dsy_x, dsy_T, dsy_th[5], chi_c;
};

__device__ inline void jc_partials_dev(const otm_material &M, double ebar_n, double x, double dt, double T, double &d_eb,
                                       double &d_x, double &d_T, double d_th[5])
{
    const double ebar = ebar_n + x;
    const double span = M.T_melt - M.T_room;
    const double ts_raw = (T - M.T_room) / span;
    const double ts = fmin(fmax(ts_raw, 0.0), 1.0);
    const double therm = 1.0 - pow(ts, M.m);
    const double dtherm = (ts_raw > 0.0 && ts_raw < 1.0) ? -M.m * pow(ts, M.m - 1.0) / span : 0.0;
    const double rstar = (x / dt) / M.eps_dot0;
    double rate = 1.0, drate = 0.0, lr = 0.0;
    if (rstar > 1.0) {
        lr = log(rstar);
        rate = 1.0 + M.C * lr;
        drate = M.C / x;
    }
    const double epn = pow(ebar, M.n);
    const double hard = M.A + M.B * epn;
    const double dhard = (ebar > 0.0) ? M.B * M.n * pow(ebar, M.n - 1.0) : 0.0;
    d_eb = dhard * rate * therm;
    d_x = (dhard * rate + hard * drate) * therm;
    d_T = hard * rate * dtherm;
    d_th[0] = rate * therm;
    d_th[1] = epn * rate * therm;
    d_th[2] = (ebar > 0.0) ? M.B * epn * log(ebar) * rate * therm : 0.0;
    d_th[3] = hard * lr * therm;
    d_th[4] = (ts > 0.0) ? -hard * rate * pow(ts, M.m) * log(ts) : 0.0;
}

// principal tangent: (dlam[3], deb_n, dT_n, dth[5]) -> (dtau[3], db[3], deb', dT')
__device__ inline void principal_tangent(const RmDetail &o, const double dl[3], double deb, double dT,
                                         const double dth[5], double dtau[3], double db[3], double &deb1,
                                         double &dT1)
{
    double deps[3], dtr = 0.0, de[3], den = 0.0;
    for (int a = 0; a < 3; a++) {
        deps[a] = dl[a] / (2.0 * o.lam[a]);
        dtr += deps[a];
    }
    for (int a = 0; a < 3; a++) de[a] = deps[a] - dtr / 3.0;
    if (o.enorm > 0.0)
        for (int a = 0; a < 3; a++) den += o.e[a] * de[a] / o.enorm;
    const double dqtr = 2.4494897427831780982 * o.mu * den;   // sqrt(6) mu d|e|
    double dx = 0.0, drho = 0.0, dq = dqtr;
    if (o.plastic) {
        double dsth = 0.0;
        for (int k = 0; k < 5; k++) dsth += o.dsy_th[k] * dth[k];
        dx = (dqtr - o.dsy_eb * deb - o.dsy_T * dT - dsth) / (3.0 * o.mu + o.dsy_x);
        dq = dqtr - 3.0 * o.mu * dx;
        drho = (dq - o.rho * dqtr) / o.qtr;
    }
    for (int a = 0; a < 3; a++) {
        const double dee = dtr / 3.0 + de[a] * o.rho + o.e[a] * drho;
        dtau[a] = o.K * dtr + 2.0 * o.mu * (de[a] * o.rho + o.e[a] * drho);
        db[a] = 2.0 * o.bA[a] * dee;
    }
    deb1 = deb + dx;
    dT1 = dT + o.chi_c * (dq * o.x + o.q * dx);
}

__device__ inline void mat3mul(const double a[3][3], const double b[3][3], double c[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) c[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j] + a[i][2] * b[2][j];
}

__global__ void __launch_bounds__(128) k_adj_rm(const Dev D, const AdjDev A)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= D.nm) return;
    const otm_material &M = D.mat[D.mat_id[p]];
    double dF[3][3], Fo[3][3], Fn[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            dF[i][j] = D.dF[9 * p + 3 * i + j];
            Fo[i][j] = A.F_n[9 * p + 3 * i + j];
            Fn[i][j] = D.F[9 * p + 3 * i + j];
        }
    const double Jn = Fn[0][0] * (Fn[1][1] * Fn[2][2] - Fn[1][2] * Fn[2][1]) -
                      Fn[0][1] * (Fn[1][0] * Fn[2][2] - Fn[1][2] * Fn[2][0]) +
                      Fn[0][2] * (Fn[1][0] * Fn[2][1] - Fn[1][1] * Fn[2][0]);
    // recompute the return map and its intermediate quantities
    RmIn in;
    for (int i = 0; i < 9; i++) in.dF[i] = dF[i / 3][i % 3];
    for (int i = 0; i < 6; i++) in.be[i] = A.be_n[6 * p + i];
    in.ebar = A.ebar_n[p];
    in.T = A.T_n[p];
    in.J = Jn;
    in.guess = D.rate[p] * D.dt;   // the recomputed step's own increment
    in.Q0 = nullptr;
    RmOut out;
    return_map_point(M, D.dt, in, out);
    RmDetail o;
    o.K = M.E / (3.0 * (1.0 - 2.0 * M.nu));
    o.mu = M.E / (2.0 * (1.0 + M.nu));
    o.J = Jn;
    const double bn[3][3] = {{in.be[0], in.be[3], in.be[5]}, {in.be[3], in.be[1], in.be[4]}, {in.be[5], in.be[4], in.be[2]}};
    double t1[3][3], btr[3][3], dFT[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFT[i][j] = dF[j][i];
    mat3mul(dF, bn, t1);
    mat3mul(t1, dFT, btr);
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++) btr[i][j] = btr[j][i] = 0.5 * (btr[i][j] + btr[j][i]);
    jacobi_sym3(btr, o.Q);
    double tr = 0.0, eps[3];
    for (int a = 0; a < 3; a++) {
        o.lam[a] = btr[a][a];
        eps[a] = 0.5 * log(o.lam[a]);
        tr += eps[a];
    }
    double en2 = 0.0;
    for (int a = 0; a < 3; a++) {
        o.e[a] = eps[a] - tr / 3.0;
        en2 += o.e[a] * o.e[a];
    }
    o.enorm = sqrt(en2);
    o.qtr = 2.4494897427831780982 * o.mu * o.enorm;
    o.x = out.ebar - in.ebar;
    o.plastic = o.x > 0.0;
    o.q = o.qtr - 3.0 * o.mu * o.x;
    o.rho = o.plastic ? o.q / o.qtr : 1.0;
    for (int a = 0; a < 3; a++) {
        const double ee = tr / 3.0 + o.e[a] * o.rho;
        o.tau[a] = o.K * tr + 2.0 * o.mu * o.e[a] * o.rho;
        o.bA[a] = exp(2.0 * ee);
    }
    const bool heating = (M.model == 1 && M.chi > 0.0 && o.plastic);
    o.chi_c = heating ? M.chi / (M.rho0 * M.cp) : 0.0;
    o.dsy_T = 0.0;
    for (int k = 0; k < 5; k++) o.dsy_th[k] = 0.0;
    if (M.model == 0) {
        o.dsy_eb = M.H;
        o.dsy_x = M.H;
    } else {
        jc_partials_dev(M, in.ebar, o.x, D.dt, in.T, o.dsy_eb, o.dsy_x, o.dsy_T, o.dsy_th);
    }
    // incoming adjoints: full symmetric matrices from 6-vector adjoints
    const double *sb6 = A.sigb + 6 * p, *bb6 = A.beb + 6 * p;
    const double Sb[3][3] = {{sb6[0], 0.5 * sb6[3], 0.5 * sb6[5]}, {0.5 * sb6[3], sb6[1], 0.5 * sb6[4]},
                             {0.5 * sb6[5], 0.5 * sb6[4], sb6[2]}};
    const double Bb[3][3] = {{bb6[0], 0.5 * bb6[3], 0.5 * bb6[5]}, {0.5 * bb6[3], bb6[1], 0.5 * bb6[4]},
                             {0.5 * bb6[5], 0.5 * bb6[4], bb6[2]}};
    const double *s6 = D.sig + 6 * p;
    const double Sg[3][3] = {{s6[0], s6[3], s6[5]}, {s6[3], s6[1], s6[4]}, {s6[5], s6[4], s6[2]}};
    double taub[3][3], ss = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            taub[i][j] = Sb[i][j] / Jn;
            ss += Sb[i][j] * Sg[i][j];
        }
    const double Jb = -ss / Jn;
    double QT[3][3], tmp[3][3], Tq[3][3], Bq[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) QT[i][j] = o.Q[j][i];
    mat3mul(QT, taub, tmp);
    mat3mul(tmp, o.Q, Tq);
    mat3mul(QT, Bb, tmp);
    mat3mul(tmp, o.Q, Bq);
    double ctau[10][3], cb[10][3], ceb[10], cT[10];
    for (int c = 0; c < 10; c++) {
        double dl[3] = {0, 0, 0}, dth[5] = {0, 0, 0, 0, 0};
        double deb = 0.0, dT = 0.0;
        if (c < 3) dl[c] = 1.0;
        else if (c == 3) deb = 1.0;
        else if (c == 4) dT = 1.0;
        else dth[c - 5] = 1.0;
        principal_tangent(o, dl, deb, dT, dth, ctau[c], cb[c], ceb[c], cT[c]);
    }
    double g[10];
    for (int c = 0; c < 10; c++) {
        g[c] = A.ebb[p] * ceb[c] + A.Tb[p] * cT[c];
        for (int a = 0; a < 3; a++) g[c] += Tq[a][a] * ctau[c][a] + Bq[a][a] * cb[c][a];
    }
    double Xb[3][3];
    const double lmax = fmax(fabs(o.lam[0]), fmax(fabs(o.lam[1]), fabs(o.lam[2])));
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            if (a == b) {
                Xb[a][a] = g[a];
                continue;
            }
            const double dl = o.lam[a] - o.lam[b];
            double tt, tb;
            if (fabs(dl) > 1e-6 * lmax) {
                tt = (o.tau[a] - o.tau[b]) / dl;
                tb = (o.bA[a] - o.bA[b]) / dl;
            } else {   // repeated eigenvalues: second-order symmetric limit of the divided difference
                tt = 0.5 * ((ctau[a][a] - ctau[b][a]) + (ctau[b][b] - ctau[a][b]));
                tb = 0.5 * ((cb[a][a] - cb[b][a]) + (cb[b][b] - cb[a][b]));
            }
            Xb[a][b] = tt * Tq[a][b] + tb * Bq[a][b];
        }
    double btrb[3][3];
    mat3mul(o.Q, Xb, tmp);
    mat3mul(tmp, QT, btrb);
    // b_tr = dF b dF^T
    double Db[3][3], t2[3][3];
    mat3mul(btrb, dF, tmp);
    mat3mul(tmp, bn, t2);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Db[i][j] = 2.0 * t2[i][j];
    double bbf[3][3];
    mat3mul(dFT, btrb, tmp);
    mat3mul(tmp, dF, bbf);
    // F' = dF F_n (with the J' term), v' = det(dF) v_n
    double Fni[3][3];
    {
        const double c00 = Fn[1][1] * Fn[2][2] - Fn[1][2] * Fn[2][1], c01 = Fn[0][2] * Fn[2][1] - Fn[0][1] * Fn[2][2];
        const double c02 = Fn[0][1] * Fn[1][2] - Fn[0][2] * Fn[1][1], c10 = Fn[1][2] * Fn[2][0] - Fn[1][0] * Fn[2][2];
        const double c11 = Fn[0][0] * Fn[2][2] - Fn[0][2] * Fn[2][0], c12 = Fn[0][2] * Fn[1][0] - Fn[0][0] * Fn[1][2];
        const double c20 = Fn[1][0] * Fn[2][1] - Fn[1][1] * Fn[2][0], c21 = Fn[0][1] * Fn[2][0] - Fn[0][0] * Fn[2][1];
        const double c22 = Fn[0][0] * Fn[1][1] - Fn[0][1] * Fn[1][0];
        const double iJ = 1.0 / Jn;
        Fni[0][0] = c00 * iJ; Fni[0][1] = c01 * iJ; Fni[0][2] = c02 * iJ;
        Fni[1][0] = c10 * iJ; Fni[1][1] = c11 * iJ; Fni[1][2] = c12 * iJ;
        Fni[2][0] = c20 * iJ; Fni[2][1] = c21 * iJ; Fni[2][2] = c22 * iJ;
    }
    const double detD = dF[0][0] * (dF[1][1] * dF[2][2] - dF[1][2] * dF[2][1]) -
                        dF[0][1] * (dF[1][0] * dF[2][2] - dF[1][2] * dF[2][0]) +
                        dF[0][2] * (dF[1][0] * dF[2][1] - dF[1][1] * dF[2][0]);
    double Fbt[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Fbt[i][j] = A.Fb[9 * p + 3 * i + j] + Jb * Jn * Fni[j][i];
    const double vbn = A.vb[p], vnew = D.vol[p];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double fo = 0.0, dbj = 0.0;
            for (int k = 0; k < 3; k++) {
                fo += dF[k][i] * Fbt[k][j];
                dbj += Fbt[i][k] * Fo[j][k];
            }
            A.Fb[9 * p + 3 * i + j] = fo;
            // d det(dF) / d dF = det(dF) dF^-T; det(dF) v_n = v'
            const double dinvT = (dF[(i + 1) % 3][(j + 1) % 3] * dF[(i + 2) % 3][(j + 2) % 3] -
                                  dF[(i + 1) % 3][(j + 2) % 3] * dF[(i + 2) % 3][(j + 1) % 3]) / detD;
            A.dFb[9 * p + 3 * i + j] = Db[i][j] + dbj + vbn * vnew * dinvT;
        }
    A.vb[p] = detD * vbn;
    double *beo = A.beb + 6 * p;
    beo[0] = bbf[0][0]; beo[1] = bbf[1][1]; beo[2] = bbf[2][2];
    beo[3] = bbf[0][1] + bbf[1][0]; beo[4] = bbf[1][2] + bbf[2][1]; beo[5] = bbf[0][2] + bbf[2][0];
    A.ebb[p] = g[3];
    A.Tb[p] = g[4];
    if (D.mat_id[p] == 0)
        for (int k = 0; k < 5; k++) A.thb[5 * p + k] += g[5 + k];
}

// ---------------------------------------------------------------------------- kinematics backward
// dF = 1 + sum du'_a (x) G_a, x_p' = sum N_a x'_a over the supports of state n
__global__ void __launch_bounds__(kAdjWarps * kWarp) k_adj_kin(const Dev D, const AdjDev A)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kAdjWarps + warp;
    if (p >= D.nm) return;
    const int S = D.S;
    const int n = A.cnt_n[p];
    const int64_t base = p * (int64_t)S;
    double Db[9];
    for (int i = 0; i < 9; i++) Db[i] = A.dFb[9 * p + i];
    const double4_32a xpb = A.xpb[p];
    const double *K = A.K_n + 6 * p;
    const double k0 = K[0], k1 = K[1], k2 = K[2], k3 = K[3], k4 = K[4], k5 = K[5];
    for (int k = lane; k < n; k += kWarp) {
        const int id = A.ids_n[base + k];
        const double4_32a sh = grad_row(A.shape_n[base + k], k0, k1, k2, k3, k4, k5);
        const double4_32a u = D.du[id], xa = D.x[id];
        const double ub0 = Db[0] * sh.y + Db[1] * sh.z + Db[2] * sh.w;
        const double ub1 = Db[3] * sh.y + Db[4] * sh.z + Db[5] * sh.w;
        const double ub2 = Db[6] * sh.y + Db[7] * sh.z + Db[8] * sh.w;
        const int64_t pos = (int64_t)A.noff_n[id] + A.rank_n[base + k];
        A.sc3a[pos] = make_double4_32a(sh.x * xpb.x, sh.x * xpb.y, sh.x * xpb.z, 0.0);
        A.sc3b[pos] = make_double4_32a(ub0, ub1, ub2, 0.0);
        const double g0 = Db[0] * u.x + Db[3] * u.y + Db[6] * u.z;
        const double g1 = Db[1] * u.x + Db[4] * u.y + Db[7] * u.z;
        const double g2 = Db[2] * u.x + Db[5] * u.y + Db[8] * u.z;
        A.pb_prev[base + k] = make_double4_32a(xpb.x * xa.x + xpb.y * xa.y + xpb.z * xa.z, g0, g1, g2);
    }
}

// ---------------------------------------------------------------------------- node backward
// x' = P(x + du_t), du' = x' - x, du_t = du + dt^2 r / m (fixed nodes: x' = x, du' = 0)
__global__ void __launch_bounds__(128) k_adj_node(const Dev D, const AdjDev A)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= D.nn) return;
    // sums over the node-major segments: -d_bar (state n+1 supports), N x_p_bar and dF_bar G (state n)
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0.0;
    const int b1 = D.noff[i], e1 = D.noff[i + 1];
    for (int k = b1 + lane; k < e1; k += kWarp) {
        const double4_32a c = A.sc1[k];
        v[0] -= c.x; v[1] -= c.y; v[2] -= c.z;
    }
    const int b0 = A.noff_n[i], e0 = A.noff_n[i + 1];
    for (int k = b0 + lane; k < e0; k += kWarp) {
        const double4_32a a = A.sc3a[k], b = A.sc3b[k];
        v[0] += a.x; v[1] += a.y; v[2] += a.z;
        v[3] += b.x; v[4] += b.y; v[5] += b.z;
    }
    const double t = warp_reduce_scatter16(v, lane);
    double s[6];
#pragma unroll
    for (int k = 0; k < 6; k++) s[k] = __shfl_sync(0xffffffffu, t, 2 * k);
    if (lane != 0) return;
    const double4_32a xb1 = A.xb[i], ub1 = A.dub[i];
    const double X[3] = {xb1.x + s[0], xb1.y + s[1], xb1.z + s[2]};   // dL/dx' (direct)
    const double U[3] = {ub1.x + s[3], ub1.y + s[4], ub1.z + s[5]};   // dL/ddu'
    if (D.nflags[i] & OTM_FLAG_FIXED) {
        A.xb[i] = make_double4_32a(X[0], X[1], X[2], 0.0);
        A.dub[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        A.rb[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        return;
    }
    const double4_32a mr = D.mr[i], u0 = A.du_n[i], x0 = D.x_prev[i];
    const double m = mr.x;
    double tot[3] = {X[0] + U[0], X[1] + U[1], X[2] + U[2]};
    if (D.wall) {
        const double dt2m = (m > 0.0) ? D.dt * D.dt / m : 0.0;
        const double ut0 = u0.x + dt2m * mr.y, ut1 = u0.y + dt2m * mr.z, ut2 = u0.z + dt2m * mr.w;
        const double g = (x0.x + ut0 - D.wall_p[0]) * D.wall_n[0] + (x0.y + ut1 - D.wall_p[1]) * D.wall_n[1] +
                         (x0.z + ut2 - D.wall_p[2]) * D.wall_n[2];
        if (g < 0.0) {
            const double tn = tot[0] * D.wall_n[0] + tot[1] * D.wall_n[1] + tot[2] * D.wall_n[2];
            for (int c = 0; c < 3; c++) tot[c] -= tn * D.wall_n[c];
        }
    }
    A.xb[i] = make_double4_32a(tot[0] - U[0], tot[1] - U[1], tot[2] - U[2], 0.0);
    A.dub[i] = make_double4_32a(tot[0], tot[1], tot[2], 0.0);
    if (m > 0.0) {
        const double c = D.dt * D.dt / m;
        const double rdot = mr.y * tot[0] + mr.z * tot[1] + mr.w * tot[2];
        A.rb[i] = make_double4_32a(c * tot[0], c * tot[1], c * tot[2], -c * rdot / m);
    } else {
        A.rb[i] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
    }
}

// ---------------------------------------------------------------------------- force backward
// m_I = sum N m_p, r_I = -sum v_p sigma_p G_pI over the supports of state n
__global__ void __launch_bounds__(kAdjWarps * kWarp) k_adj_force(const Dev D, const AdjDev A)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kAdjWarps + warp;
    if (p >= D.nm) return;
    const int S = D.S;
    const int n = A.cnt_n[p];
    const int64_t base = p * (int64_t)S;
    const double *sg = A.sig_n + 6 * p;
    const double sxx = sg[0], syy = sg[1], szz = sg[2], sxy = sg[3], syz = sg[4], sxz = sg[5];
    const double vp = A.vol_n[p], mp = D.mass[p];
    const double *K = A.K_n + 6 * p;
    const double k0 = K[0], k1 = K[1], k2 = K[2], k3 = K[3], k4 = K[4], k5 = K[5];
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = 0.0;
    for (int k = lane; k < n; k += kWarp) {
        const int id = A.ids_n[base + k];
        const double4_32a sh = grad_row(A.shape_n[base + k], k0, k1, k2, k3, k4, k5);
        const double4_32a rb = A.rb[id];
        double4_32a pb = A.pb_prev[base + k];
        pb.x += rb.w * mp;
        pb.y -= vp * (sxx * rb.x + sxy * rb.y + sxz * rb.z);
        pb.z -= vp * (sxy * rb.x + syy * rb.y + syz * rb.z);
        pb.w -= vp * (sxz * rb.x + syz * rb.y + szz * rb.z);
        A.pb_prev[base + k] = pb;
        const double sgx = sxx * sh.y + sxy * sh.z + sxz * sh.w;
        const double sgy = sxy * sh.y + syy * sh.z + syz * sh.w;
        const double sgz = sxz * sh.y + syz * sh.z + szz * sh.w;
        v[0] -= rb.x * sgx + rb.y * sgy + rb.z * sgz;
        // dL/dsigma_ij (full) = -v rbar_i G_j
        v[1] -= vp * rb.x * sh.y; v[2] -= vp * rb.y * sh.z; v[3] -= vp * rb.z * sh.w;
        v[4] -= vp * (rb.x * sh.z + rb.y * sh.y);
        v[5] -= vp * (rb.y * sh.w + rb.z * sh.z);
        v[6] -= vp * (rb.x * sh.w + rb.z * sh.y);
    }
    const double t = warp_reduce_scatter16(v, lane);
    double s[7];
#pragma unroll
    for (int k = 0; k < 7; k++) s[k] = __shfl_sync(0xffffffffu, t, 2 * k);
    if (lane == 0) {
        A.vb[p] += s[0];
        double *sb = A.sigb + 6 * p;
        sb[0] = s[1]; sb[1] = s[2]; sb[2] = s[3]; sb[3] = s[4]; sb[4] = s[5]; sb[5] = s[6];
    }
}

// ---------------------------------------------------------------------------- host launchers
static unsigned wblocks(int64_t n, int warps) { return (unsigned)((n + warps - 1) / warps); }

cudaError_t launch_adjoint_backward(const Dev &D, const AdjDev &A, cudaStream_t s, long long *launches)
{
    if (D.nm <= 0) return cudaSuccess;
    const size_t smem = (size_t)kAdjWarps * 7 * D.S * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_adj_lme, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adj_lme<<<wblocks(D.nm, kAdjWarps), kAdjWarps * kWarp, smem, s>>>(D, A);
    k_adj_rm<<<(unsigned)((D.nm + 127) / 128), 128, 0, s>>>(D, A);
    k_adj_kin<<<wblocks(D.nm, kAdjWarps), kAdjWarps * kWarp, 0, s>>>(D, A);
    k_adj_node<<<(unsigned)((D.nn * 32 + 127) / 128), 128, 0, s>>>(D, A);
    k_adj_force<<<wblocks(D.nm, kAdjWarps), kAdjWarps * kWarp, 0, s>>>(D, A);
    if (launches) *launches += 5;
    return cudaGetLastError();
}

// rank of every support pair in its node's influence list (integer atomics) and the counts
__global__ void k_rebuild_ranks(const Dev D)
{
    const int64_t total = D.nm * (int64_t)D.S;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = t / D.S;
        const int k = (int)(t - p * D.S);
        if (k >= D.cnt[p]) continue;
        const int r = atomicAdd(&D.ncount[D.ids[t]], 1);
        if (r > 0xffff) raise_error(D.err, OTM_ERR_CAPACITY, D.ngid[D.ids[t]]);
        D.rank[t] = (uint16_t)r;
    }
}

cudaError_t launch_rebuild_ranks(const Dev &D, cudaStream_t s, long long *launches)
{
    int64_t total = D.nm * (int64_t)D.S;
    int64_t b = (total + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    k_rebuild_ranks<<<(unsigned)b, 256, 0, s>>>(D);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace otm
