// otm_rm.cuh -- constitutive update of one material point (Sec. 4.1 J2, Sec. 4.2 Johnson-Cook),
// shared by the forward step kernels and the adjoint kernels.
#pragma once

#include "otm_dev.cuh"

namespace otm {

// ======================================================================== return map
// cyclic Jacobi (Golub & Van Loan Sec. 8.5) on a symmetric 3x3, rotations applied in place
__device__ inline void jacobi_sym3(double A[3][3], double V[3][3])
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

// the thermal softening factor 1 - T*^m of the Johnson-Cook flow stress (T* clamped to [0, 1])
__device__ __forceinline__ double jc_therm(const otm_material &M, double T)
{
    const double tstar = fmin(fmax((T - M.T_room) / (M.T_melt - M.T_room), 0.0), 1.0);
    return 1.0 - pow(tstar, M.m);
}

// Johnson-Cook flow stress at ebar_n + x with plastic rate x / dt, and its derivative in x;
// `therm` from jc_therm (the temperature is held at T_n within the step)
__device__ __forceinline__ void jc_sigma_y(const otm_material &M, double ebar_n, double x, double dt,
                                           double therm, double &sy, double &dsy)
{
    const double ebar = ebar_n + x;
    const double rstar = (x / dt) / M.eps_dot0;
    double rate = 1.0, drate = 0.0;
    if (rstar > 1.0) {
        rate = 1.0 + M.C * log(rstar);
        drate = M.C / x;
    }
    const double pe = pow(ebar, M.n);
    const double hard = M.A + M.B * pe;
    const double dhard = (ebar > 0.0) ? M.B * M.n * pe / ebar : INFINITY;
    sy = hard * rate * therm;
    dsy = (dhard * rate + hard * drate) * therm;
}

struct RmIn {
    double dF[9], be[6], ebar, T, J;
    double guess;      // start of the consistency iteration (e.g. the last step's increment); <= 0: none
    const double *Q0;  // start basis of the eigen solver (row-major, columns the last step's
                       // eigenvectors of b^e) or nullptr
};
struct RmOut {
    double sig[6], be[6], ebar, T, rate;
    double Q[9];       // eigenvectors of the trial b^e (row-major, columns)
    bool failed;
};

// returns OTM_OK or an error code
__device__ inline int return_map_point(const otm_material &M, double dt, const RmIn &in, RmOut &out)
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
    if (in.Q0) {
        // in the last step's eigenbasis the trial b^e is nearly diagonal, so the Jacobi sweeps
        // start close to convergence: A <- Q0^T A Q0, then Q = Q0 V
        double T3[3][3], B[3][3], V[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                T3[i][j] = A[i][0] * in.Q0[j] + A[i][1] * in.Q0[3 + j] + A[i][2] * in.Q0[6 + j];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                B[i][j] = in.Q0[i] * T3[0][j] + in.Q0[3 + i] * T3[1][j] + in.Q0[6 + i] * T3[2][j];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) A[i][j] = (i == j) ? B[i][i] : 0.5 * (B[i][j] + B[j][i]);
        jacobi_sym3(A, V);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++)
                Q[i][j] = in.Q0[3 * i] * V[0][j] + in.Q0[3 * i + 1] * V[1][j] + in.Q0[3 * i + 2] * V[2][j];
    } else {
        jacobi_sym3(A, Q);
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) out.Q[3 * i + j] = Q[i][j];
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
        const double therm = jc_therm(M, in.T);
        double sy0, dsy0;
        jc_sigma_y(M, in.ebar, 0.0, dt, therm, sy0, dsy0);
        if (q_tr - sy0 > 0.0) {
            // g(x) = q_tr - 3 mu x - sigma_y(x) on [0, q_tr / (3 mu)]: Newton safeguarded by
            // bisection, from the given guess when it lies inside the bracket
            double lo = 0.0, hi = q_tr / (3.0 * mu);
            double x = (in.guess > 0.0 && in.guess < hi) ? in.guess : 0.5 * hi;
            const double tol = 1e-12 * q_tr;
            bool ok = false;
            for (int it = 0; it < 300; it++) {
                double sy, dsy;
                jc_sigma_y(M, in.ebar, x, dt, therm, sy, dsy);
                const double g = q_tr - 3.0 * mu * x - sy;
                if (fabs(g) <= tol) { ok = true; break; }
                if (g > 0.0) lo = x; else hi = x;
                if (hi - lo <= 4e-16 * hi) { ok = true; break; }
                double xn = x - g / (-3.0 * mu - dsy);
                if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
                x = xn;
            }
            if (!ok) return OTM_ERR_RETURNMAP_NOCONV;
            {   // one more Newton step: the accepted iterate is fixed only to the tolerance, the
                // step fixes it to rounding, whatever the start (warm or the bracket's midpoint)
                double sy, dsy;
                jc_sigma_y(M, in.ebar, x, dt, therm, sy, dsy);
                const double g = q_tr - 3.0 * mu * x - sy;
                const double xn = x - g / (-3.0 * mu - dsy);
                if (xn > lo && xn < hi) x = xn;
            }
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
        // b^e = Q diag(exp(2 e)) Q^T; without plastic flow e = ln(lambda) / 2 of the trial, so the
        // eigenvalues are the trial's own
        eb2[a] = (dep > 0.0) ? exp(2.0 * e[a]) : A[a][a];
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
        const double sv = fmax(qn, 0.0) * iJ;
        // triaxiality; its limit sign(p) * inf where no deviatoric stress is left (melted point)
        const double eta = (sv > 1e-12 * fabs(pr)) ? pr / sv : (pr > 0.0 ? INFINITY : (pr < 0.0 ? -INFINITY : 0.0));
        const double texp = (M.d3 == 0.0) ? 1.0 : exp(M.d3 * eta);
        const double rstar = out.rate / M.eps_dot0;
        const double lr = (rstar > 1.0) ? log(rstar) : 0.0;
        const double tstar = fmin(fmax((out.T - M.T_room) / (M.T_melt - M.T_room), 0.0), 1.0);
        const double ef = (M.d1 + M.d2 * texp) * (1.0 + M.d4 * lr) * (1.0 + M.d5 * tstar);
        out.failed = (out.ebar >= ef);
    }
    for (int c = 0; c < 6; c++)
        if (!isfinite(out.sig[c])) return OTM_ERR_NONFINITE;
    return OTM_OK;
}


}  // namespace otm
