/*
 * otm_oracle.c -- serial FP64 CPU oracle of the explicit OTM step.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the CUDA library is
 * checked against. Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * it. It shares no code, header, table or helper with the CUDA path.
 *
 * Paper: Kumar, Gosselet, Huang, Weissenfels, Wriggers, "Parallel multiphysics simulation for
 * the stabilized optimal transportation meshfree (OTM) method" (arXiv 2206.08772).
 * Equations are numbered in order of appearance in Sec. 2 and Sec. 4:
 *   Eq. 1 weak form; Eq. 2 meshfree interpolation; Eq. 3 assembled equation of motion;
 *   Eq. 4 central-difference nodal equilibrium; Eq. 5 lumped mass and nodal residual;
 *   Eq. 6 nodal position update; Eq. 7 stabilised residual; Eq. 8 under-integration error;
 *   Eq. 9 material-point position; Eq. 10 F update; Eq. 11 F increment; Eq. 12-13 volume and
 *   density; Eq. 14 LME shape functions (Sec. 2.3); Sec. 4.1 J2 finite plasticity and wall
 *   contact; Sec. 4.2 Johnson-Cook flow (Eq. JC-flow), heating, fracture (Eq. JC-fracture)
 *   and tool contact. Algorithm 1 = the OTM step, Algorithm 3 = linked-cell search.
 *
 * Readings where the paper is silent or garbled are listed at each use; they are:
 *   - support: node a belongs to MP p iff |x_p - x_a|^2 <= rs2, rs2 = ln(1/tol)/beta (host bits)
 *   - LME gradient: grad N_a = -N_a J^-1 d_a, J = sum N d d^T - r r^T (derived from Eq. 14)
 *   - stress back-transform: sigma = J^-1 Q diag(tau) Q^T, tau = K tr(e) + 2 mu dev(e)
 *   - yield check on the deviatoric trial stress; Simo exponential-map radial return
 *   - JC rate term uses max(rate/rate0, 1); T* clamped to [0, 1]
 *   - heating dT = chi * q * d(ebar) / (rho0 cp), isothermal split (flow stress uses T_n)
 *   - fracture: ebar >= eps_f checked only where ebar > 0; eta = (tr sigma / 3) / sigma_v, and
 *     eta = sign(p) * infinity where sigma_v <= 1e-12 |p| (no deviatoric stress left)
 *   - wall contact projects the node onto the plane, keeping the tangential increment
 *   - tool contact: normal projection plus Coulomb stick/slip at the penalty limit m/dt^2
 *   - LME Newton: damped, stops at |r| <= newton_tol * h (1e-14 h in the scenarios); after a
 *     failed warm start one more solve from lambda = 0
 *   - node insertion (max_insert > 0): a node one spacing beyond an MP whose solve fails, away
 *     from its support's centroid (see insert_nodes)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- status codes */
enum {
    ORC_OK = 0,
    ORC_ERR_ARG = -1,
    ORC_ERR_OOM = -3,
    ORC_ERR_LME_NOCONV = -4,
    ORC_ERR_JACOBIAN = -5,
    ORC_ERR_NONFINITE = -6,
    ORC_ERR_RETURNMAP_NOCONV = -7,
    ORC_ERR_CAPACITY = -8
};

/* ---------------------------------------------------------------- parameters */
typedef struct {
    int32_t model;       /* 0: J2 linear isotropic hardening, 1: Johnson-Cook */
    int32_t fracture;    /* 1: Johnson-Cook fracture -> erosion */
    double E, nu, rho0;
    double sigma_y0, H;                      /* J2 */
    double A, B, n, C, m, eps_dot0;          /* JC flow */
    double T_room, T_melt, chi, cp;          /* JC thermal */
    double d1, d2, d3, d4, d5;               /* JC fracture */
} orc_material;

typedef struct {
    double h, beta, rs2, cell_size, dt, T0, newton_tol, eps_stab;
    int32_t max_newton;
    int32_t n_materials;
    int32_t wall, tool;
    double wall_p[3], wall_n[3];
    double tool_x0, tool_tip_y, tool_rake, tool_clear, tool_v, friction;  /* angles in rad */
    int32_t allow_insert, allow_erode;
    orc_material mat[4];
} orc_params;

/* ---------------------------------------------------------------- 3x3 helpers */
/* symmetric 6-vector order: xx, yy, zz, xy, yz, xz */
static void sym_to_full(const double s[6], double a[3][3])
{
    a[0][0] = s[0]; a[1][1] = s[1]; a[2][2] = s[2];
    a[0][1] = a[1][0] = s[3];
    a[1][2] = a[2][1] = s[4];
    a[0][2] = a[2][0] = s[5];
}

static double det3(const double a[3][3])
{
    return a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1])
         - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0])
         + a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
}

/* inverse by cofactors; returns 0 if singular / non-finite */
static int inv3(const double a[3][3], double inv[3][3])
{
    double det = det3(a);
    if (!(fabs(det) > 0.0) || !isfinite(det)) return 0;
    inv[0][0] = (a[1][1] * a[2][2] - a[1][2] * a[2][1]) / det;
    inv[0][1] = (a[0][2] * a[2][1] - a[0][1] * a[2][2]) / det;
    inv[0][2] = (a[0][1] * a[1][2] - a[0][2] * a[1][1]) / det;
    inv[1][0] = (a[1][2] * a[2][0] - a[1][0] * a[2][2]) / det;
    inv[1][1] = (a[0][0] * a[2][2] - a[0][2] * a[2][0]) / det;
    inv[1][2] = (a[0][2] * a[1][0] - a[0][0] * a[1][2]) / det;
    inv[2][0] = (a[1][0] * a[2][1] - a[1][1] * a[2][0]) / det;
    inv[2][1] = (a[0][1] * a[2][0] - a[0][0] * a[2][1]) / det;
    inv[2][2] = (a[0][0] * a[1][1] - a[0][1] * a[1][0]) / det;
    return 1;
}

static void matmul3(const double a[3][3], const double b[3][3], double c[3][3])
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (Golub & Van Loan, Matrix
 * Computations, Sec. 8.5): a = V diag(w) V^T, columns of V are eigenvectors. Sweeps until the
 * off-diagonal Frobenius norm is <= 1e-15 of the matrix norm (or exactly zero). */
static void jacobi_eig3(const double a_in[3][3], double w[3], double V[3][3])
{
    double a[3][3];
    memcpy(a, a_in, sizeof(a));
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) V[i][j] = (i == j) ? 1.0 : 0.0;
    double norm = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) norm += a[i][j] * a[i][j];
    norm = sqrt(norm);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = sqrt(2.0 * (a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2]));
        if (off <= 1e-15 * norm) break;
        static const int P[3] = {0, 0, 1}, Q[3] = {1, 2, 2};
        for (int k = 0; k < 3; k++) {
            int p = P[k], q = Q[k];
            if (a[p][q] == 0.0) continue;
            double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
            double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
            /* rotation R = I except R[p][p]=c, R[p][q]=s, R[q][p]=-s, R[q][q]=c; a <- R^T a R */
            double R[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, RT[3][3], tmp[3][3];
            R[p][p] = c; R[p][q] = s; R[q][p] = -s; R[q][q] = c;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) RT[i][j] = R[j][i];
            matmul3(RT, a, tmp);
            matmul3(tmp, R, a);
            a[p][q] = a[q][p] = 0.0;     /* annihilated by construction */
            matmul3(V, R, tmp);
            memcpy(V, tmp, sizeof(tmp));
        }
    }
    for (int i = 0; i < 3; i++) w[i] = a[i][i];
}

/* ================================================================ linked-cell search
 * Algorithm 3: (1) divide the domain into static cells, (2) find the cells that intersect the
 * support sphere, (3) test the nodes of those cells. Cells are boxes of edge `cell_size`
 * (>= half the support radius) starting at the componentwise node minimum; the stencil is
 * +-2 cells per axis. Nodes are listed per cell in ascending ID. */
typedef struct {
    double origin[3];
    int64_t dims[3];
    int64_t n_cells;
    int64_t *cell_start;   /* n_cells + 1 */
    int32_t *sorted;       /* node IDs ordered by (cell, ID) */
    int64_t *node_cell;    /* cell of each node */
} orc_grid;

static int64_t cell_coord(double x, double o, double c, int64_t n, int clamp)
{
    double f = floor((x - o) / c);
    if (clamp) {
        if (f < 0.0) f = 0.0;
        if (f > (double)(n - 1)) f = (double)(n - 1);
    } else {
        if (f < -4.0) f = -4.0;                 /* far outside: keep it an integer */
        if (f > (double)(n + 3)) f = (double)(n + 3);
    }
    return (int64_t)f;
}

static void grid_free(orc_grid *g)
{
    free(g->cell_start); free(g->sorted); free(g->node_cell);
    memset(g, 0, sizeof(*g));
}

#define ORC_MAX_CELLS (int64_t)(1 << 26)

static int grid_build(orc_grid *g, int64_t nn, const double *x, double c)
{
    memset(g, 0, sizeof(*g));
    if (nn <= 0) return ORC_ERR_ARG;
    double lo[3], hi[3];
    for (int d = 0; d < 3; d++) { lo[d] = x[d]; hi[d] = x[d]; }
    for (int64_t i = 1; i < nn; i++)
        for (int d = 0; d < 3; d++) {
            if (x[3 * i + d] < lo[d]) lo[d] = x[3 * i + d];
            if (x[3 * i + d] > hi[d]) hi[d] = x[3 * i + d];
        }
    for (int d = 0; d < 3; d++) {
        if (!isfinite(lo[d]) || !isfinite(hi[d])) return ORC_ERR_NONFINITE;
        g->origin[d] = lo[d];
        double nd = floor((hi[d] - lo[d]) / c) + 1.0;
        if (nd > (double)ORC_MAX_CELLS) return ORC_ERR_CAPACITY;
        g->dims[d] = (int64_t)nd;
    }
    g->n_cells = g->dims[0] * g->dims[1] * g->dims[2];
    if (g->n_cells > ORC_MAX_CELLS) return ORC_ERR_CAPACITY;
    g->cell_start = calloc((size_t)g->n_cells + 1, sizeof(int64_t));
    g->sorted = malloc((size_t)nn * sizeof(int32_t));
    g->node_cell = malloc((size_t)nn * sizeof(int64_t));
    if (!g->cell_start || !g->sorted || !g->node_cell) { grid_free(g); return ORC_ERR_OOM; }
    for (int64_t i = 0; i < nn; i++) {
        int64_t ix = cell_coord(x[3 * i + 0], g->origin[0], c, g->dims[0], 1);
        int64_t iy = cell_coord(x[3 * i + 1], g->origin[1], c, g->dims[1], 1);
        int64_t iz = cell_coord(x[3 * i + 2], g->origin[2], c, g->dims[2], 1);
        g->node_cell[i] = (iz * g->dims[1] + iy) * g->dims[0] + ix;
        g->cell_start[g->node_cell[i] + 1]++;
    }
    for (int64_t k = 0; k < g->n_cells; k++) g->cell_start[k + 1] += g->cell_start[k];
    int64_t *fill = malloc((size_t)g->n_cells * sizeof(int64_t));
    if (!fill) { grid_free(g); return ORC_ERR_OOM; }
    memcpy(fill, g->cell_start, (size_t)g->n_cells * sizeof(int64_t));
    for (int64_t i = 0; i < nn; i++) g->sorted[fill[g->node_cell[i]]++] = (int32_t)i;  /* ascending ID */
    free(fill);
    return ORC_OK;
}

/* squared distance with a fixed operation order and no fused multiply-add */
static double dist2(const double *a, const double *b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    double xx = dx * dx, yy = dy * dy, zz = dz * dz;
    double s = xx + yy;
    return s + zz;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* support of one MP: all nodes with d^2 <= rs2, ascending ID. Returns the count (which may
 * exceed cap; only the first cap IDs are then stored, unsorted beyond cap). */
static int64_t search_mp(const orc_grid *g, const double *node_x, const double *xp, double rs2,
                         double c, int32_t *out, int64_t cap)
{
    int64_t ci[3];
    for (int d = 0; d < 3; d++) ci[d] = cell_coord(xp[d], g->origin[d], c, g->dims[d], 0);
    int64_t cnt = 0;
    for (int64_t kz = ci[2] - 2; kz <= ci[2] + 2; kz++) {
        if (kz < 0 || kz >= g->dims[2]) continue;
        for (int64_t ky = ci[1] - 2; ky <= ci[1] + 2; ky++) {
            if (ky < 0 || ky >= g->dims[1]) continue;
            for (int64_t kx = ci[0] - 2; kx <= ci[0] + 2; kx++) {
                if (kx < 0 || kx >= g->dims[0]) continue;
                int64_t cell = (kz * g->dims[1] + ky) * g->dims[0] + kx;
                for (int64_t s = g->cell_start[cell]; s < g->cell_start[cell + 1]; s++) {
                    int32_t a = g->sorted[s];
                    if (dist2(xp, node_x + 3 * (int64_t)a) <= rs2) {
                        if (cnt < cap) out[cnt] = a;
                        cnt++;
                    }
                }
            }
        }
    }
    if (cnt <= cap) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

/* ================================================================ LME shape functions
 * Eq. 14: N_a = Z_a / Z, Z_a = exp(-beta |d_a|^2 + lambda . d_a), d_a = x_p - x_a, with lambda
 * chosen so that sum_a N_a d_a = 0 (first-order consistency), solved by Newton-Raphson.
 * log Z(lambda) is convex; its gradient is r = sum N_a d_a and its Hessian is
 * J = sum N_a d_a d_a^T - r r^T. Newton steps are damped by halving until log Z or |r|
 * decreases (damped Newton, Boyd & Vandenberghe Sec. 9.5). Weights are evaluated as
 * exp(f_a - max f) (the shift cancels in N_a). At convergence grad N_a = -N_a J^-1 d_a, which
 * follows from differentiating r(lambda(x), x) = 0 (beta cancels).
 * Stops when |r| <= tol_r; fails after max_it iterations. */
typedef struct {
    double logZ, rnorm, r[3], J[3][3];
} lme_eval_t;

static void lme_evaluate(int64_t n, const double *d, double beta, const double lam[3],
                         double *N, lme_eval_t *e)
{
    double fmax = -INFINITY;
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a;
        double f = -beta * (da[0] * da[0] + da[1] * da[1] + da[2] * da[2])
                 + (lam[0] * da[0] + lam[1] * da[1] + lam[2] * da[2]);
        N[a] = f;
        if (f > fmax) fmax = f;
    }
    double Z = 0.0;
    for (int64_t a = 0; a < n; a++) {
        N[a] = exp(N[a] - fmax);
        Z += N[a];
    }
    e->logZ = fmax + log(Z);
    for (int i = 0; i < 3; i++) {
        e->r[i] = 0.0;
        for (int j = 0; j < 3; j++) e->J[i][j] = 0.0;
    }
    for (int64_t a = 0; a < n; a++) {
        N[a] /= Z;
        const double *da = d + 3 * a;
        for (int i = 0; i < 3; i++) {
            e->r[i] += N[a] * da[i];
            for (int j = 0; j < 3; j++) e->J[i][j] += N[a] * da[i] * da[j];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) e->J[i][j] -= e->r[i] * e->r[j];
    e->rnorm = sqrt(e->r[0] * e->r[0] + e->r[1] * e->r[1] + e->r[2] * e->r[2]);
}

int orc_lme(int64_t n, const double *d, double beta, double tol_r, int32_t max_it,
            double lam[3], double *N, double *dN, int32_t *iters)
{
    if (n <= 0) return ORC_ERR_LME_NOCONV;
    double *Nt = malloc((size_t)n * sizeof(double));
    if (!Nt) return ORC_ERR_OOM;
    lme_eval_t e, et;
    lme_evaluate(n, d, beta, lam, N, &e);
    int32_t it = 0;
    int status = ORC_ERR_LME_NOCONV;
    for (;;) {
        if (!isfinite(e.rnorm)) break;
        if (e.rnorm <= tol_r) { status = ORC_OK; break; }
        if (it >= max_it) break;
        it++;
        double Jinv[3][3];
        if (!inv3(e.J, Jinv)) break;
        double step[3];
        for (int i = 0; i < 3; i++)
            step[i] = -(Jinv[i][0] * e.r[0] + Jinv[i][1] * e.r[1] + Jinv[i][2] * e.r[2]);
        double t = 1.0, lt[3];
        int accepted = 0;
        for (int halving = 0; halving < 40; halving++) {
            for (int i = 0; i < 3; i++) lt[i] = lam[i] + t * step[i];
            lme_evaluate(n, d, beta, lt, Nt, &et);
            if (isfinite(et.logZ) && (et.logZ < e.logZ || et.rnorm < e.rnorm)) { accepted = 1; break; }
            t *= 0.5;
        }
        if (!accepted) break;
        for (int i = 0; i < 3; i++) lam[i] = lt[i];
        memcpy(N, Nt, (size_t)n * sizeof(double));
        e = et;
    }
    free(Nt);
    if (iters) *iters = it;
    if (status != ORC_OK) return status;
    double Jinv[3][3];
    if (!inv3(e.J, Jinv)) return ORC_ERR_LME_NOCONV;
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a;
        for (int i = 0; i < 3; i++)
            dN[3 * a + i] = -N[a] * (Jinv[i][0] * da[0] + Jinv[i][1] * da[1] + Jinv[i][2] * da[2]);
    }
    return ORC_OK;
}

/* ================================================================ constitutive update */
static const double SQRT23 = 0.81649658092772603273;   /* sqrt(2/3) */
static const double SQRT32 = 1.22474487139158904910;   /* sqrt(3/2) */

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Johnson-Cook flow stress (Eq. JC-flow) and its derivative with respect to the plastic
 * strain increment x (ebar = ebar_n + x, rate = x / dt), temperature frozen at T. */
static void jc_flow(const orc_material *M, double ebar_n, double x, double dt, double T,
                    double *sy, double *dsy)
{
    double ebar = ebar_n + x;
    double tstar = clamp01((T - M->T_room) / (M->T_melt - M->T_room));
    double therm = 1.0 - pow(tstar, M->m);
    double rstar = (x / dt) / M->eps_dot0;
    double rate = 1.0, drate = 0.0;
    if (rstar > 1.0) { rate = 1.0 + M->C * log(rstar); drate = M->C / x; }
    double hard = M->A + M->B * pow(ebar, M->n);
    double dhard = (ebar > 0.0) ? M->B * M->n * pow(ebar, M->n - 1.0) : INFINITY;
    *sy = hard * rate * therm;
    *dsy = (dhard * rate + hard * drate) * therm;
}

typedef struct {
    double sig[6], be[6];
    double ebar, T, rate, q, eps_f;
    int failed;
} rm_out_t;

/* Sec. 4.1 / 4.2: multiplicative split, Hencky strain of the trial elastic left Cauchy-Green
 * tensor b_tr = dF b_n dF^T, spectral decomposition b_tr = Q diag(lam2) Q^T, principal
 * trial strains e_A = 1/2 ln lam2_A, Kirchhoff tau = K tr(e) 1 + 2 mu dev(e), von Mises check
 * q_tr = sqrt(3/2) |dev tau| against the flow stress, radial return along n = dev tau / |dev tau|
 * (exponential map: e = e_tr - dgamma n), b_{n+1} = Q diag(exp(2 e)) Q^T, sigma = tau / J. */
static int return_map(const orc_material *M, double dt, const double dF[3][3], const double be_n[6],
                      double ebar_n, double T_n, double J, rm_out_t *o)
{
    double K = M->E / (3.0 * (1.0 - 2.0 * M->nu));
    double mu = M->E / (2.0 * (1.0 + M->nu));
    double b[3][3], t1[3][3], dFT[3][3], btr[3][3];
    sym_to_full(be_n, b);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFT[i][j] = dF[j][i];
    matmul3(dF, b, t1);
    matmul3(t1, dFT, btr);
    for (int i = 0; i < 3; i++)          /* exact symmetry */
        for (int j = i + 1; j < 3; j++) btr[i][j] = btr[j][i] = 0.5 * (btr[i][j] + btr[j][i]);
    double lam2[3], Q[3][3];
    jacobi_eig3(btr, lam2, Q);
    double e[3];
    for (int A = 0; A < 3; A++) {
        if (!(lam2[A] > 0.0)) return ORC_ERR_JACOBIAN;
        e[A] = 0.5 * log(lam2[A]);
    }
    double tr = e[0] + e[1] + e[2];
    double s[3], snorm2 = 0.0;
    for (int A = 0; A < 3; A++) {
        s[A] = 2.0 * mu * (e[A] - tr / 3.0);
        snorm2 += s[A] * s[A];
    }
    double snorm = sqrt(snorm2);
    double q_tr = SQRT32 * snorm;
    double dep = 0.0;   /* increment of the equivalent plastic strain, sqrt(2/3) dgamma */
    if (M->model == 0) {
        /* Eq. von-Mises-yield (linear hardening): f = |s_tr| - 2 mu dgamma
         *   - sqrt(2/3) [sy0 + H (ebar_n + sqrt(2/3) dgamma)] = 0, closed form */
        double f_tr = snorm - SQRT23 * (M->sigma_y0 + M->H * ebar_n);
        if (f_tr > 0.0) {
            double dgamma = f_tr / (2.0 * mu + 2.0 * M->H / 3.0);
            dep = SQRT23 * dgamma;
        }
    } else {
        /* Johnson-Cook: g(x) = q_tr - 3 mu x - sy(ebar_n + x, x/dt, T_n) = 0 on [0, q_tr/(3 mu)],
         * Newton safeguarded by bisection (backward-Euler return mapping) */
        double sy0, dsy0;
        jc_flow(M, ebar_n, 0.0, dt, T_n, &sy0, &dsy0);
        if (q_tr - sy0 > 0.0) {
            double lo = 0.0, hi = q_tr / (3.0 * mu), x = 0.5 * hi;
            double tol = 1e-12 * q_tr;
            int ok = 0;
            for (int it = 0; it < 300; it++) {
                double sy, dsy;
                jc_flow(M, ebar_n, x, dt, T_n, &sy, &dsy);
                double g = q_tr - 3.0 * mu * x - sy;
                if (fabs(g) <= tol) { ok = 1; break; }
                if (g > 0.0) lo = x; else hi = x;
                if (hi - lo <= 4e-16 * hi) { ok = 1; break; }
                double xn = x - g / (-3.0 * mu - dsy);
                if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
                x = xn;
            }
            if (!ok) return ORC_ERR_RETURNMAP_NOCONV;
            /* one more Newton step from the accepted iterate: |g| <= 1e-12 q_tr fixes x only to
             * that tolerance, and the step (quadratic convergence) fixes it to rounding, so the
             * increment does not depend on where the iteration started */
            {
                double sy, dsy;
                jc_flow(M, ebar_n, x, dt, T_n, &sy, &dsy);
                double g = q_tr - 3.0 * mu * x - sy;
                double xn = x - g / (-3.0 * mu - dsy);
                if (xn > lo && xn < hi) x = xn;
            }
            dep = x;
        }
    }
    double dgamma = SQRT32 * dep;
    double q = q_tr - 3.0 * mu * dep;
    double tau[3];
    for (int A = 0; A < 3; A++) {
        double nA = (snorm > 0.0) ? s[A] / snorm : 0.0;
        e[A] -= dgamma * nA;
        tau[A] = K * tr + 2.0 * mu * (e[A] - tr / 3.0);
    }
    double bn[3][3], sg[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double vb = 0.0, vs = 0.0;
            for (int A = 0; A < 3; A++) {
                vb += exp(2.0 * e[A]) * Q[i][A] * Q[j][A];
                vs += tau[A] * Q[i][A] * Q[j][A];
            }
            bn[i][j] = vb;
            sg[i][j] = vs / J;
        }
    o->be[0] = bn[0][0]; o->be[1] = bn[1][1]; o->be[2] = bn[2][2];
    o->be[3] = bn[0][1]; o->be[4] = bn[1][2]; o->be[5] = bn[0][2];
    o->sig[0] = sg[0][0]; o->sig[1] = sg[1][1]; o->sig[2] = sg[2][2];
    o->sig[3] = sg[0][1]; o->sig[4] = sg[1][2]; o->sig[5] = sg[0][2];
    o->ebar = ebar_n + dep;
    o->rate = dep / dt;
    o->q = q;
    o->T = T_n;
    if (M->model == 1 && M->chi > 0.0 && dep > 0.0)        /* adiabatic heating */
        o->T = T_n + M->chi * q * dep / (M->rho0 * M->cp);
    o->failed = 0;
    o->eps_f = INFINITY;
    if (M->model == 1 && M->fracture && o->ebar > 0.0) {   /* Eq. JC-fracture */
        double p = K * tr / J;                /* (1/3) tr sigma */
        double sv = (q > 0.0 ? q : 0.0) / J;  /* von Mises Cauchy stress */
        /* eta = p / sigma_v; with (numerically) no deviatoric stress, e.g. a melted point with
         * zero flow stress, the triaxiality takes its limit sign(p) * infinity */
        double eta;
        if (sv > 1e-12 * fabs(p)) eta = p / sv;
        else eta = (p > 0.0) ? INFINITY : ((p < 0.0) ? -INFINITY : 0.0);
        double texp = (M->d3 == 0.0) ? 1.0 : exp(M->d3 * eta);
        double rstar = o->rate / M->eps_dot0;
        double lr = (rstar > 1.0) ? log(rstar) : 0.0;
        double tstar = clamp01((o->T - M->T_room) / (M->T_melt - M->T_room));
        o->eps_f = (M->d1 + M->d2 * texp) * (1.0 + M->d4 * lr) * (1.0 + M->d5 * tstar);
        o->failed = (o->ebar >= o->eps_f);
    }
    return ORC_OK;
}

/* standalone entry for tests: one MP, principal-space return map */
int orc_return_map(const orc_material *M, double dt, const double *dF9, const double *be_n,
                   double ebar_n, double T_n, double J, double *sig, double *be, double *ebar,
                   double *T, double *q, int32_t *failed)
{
    double dF[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dF[i][j] = dF9[3 * i + j];
    rm_out_t o;
    int st = return_map(M, dt, dF, be_n, ebar_n, T_n, J, &o);
    if (st != ORC_OK) return st;
    memcpy(sig, o.sig, sizeof(o.sig));
    memcpy(be, o.be, sizeof(o.be));
    *ebar = o.ebar; *T = o.T; *q = o.q; *failed = o.failed;
    return ORC_OK;
}

/* ================================================================ contact */
/* Sec. 4.1: frictionless rigid wall; a node with gap g = (x - xbar).n < 0 is placed on the
 * plane, x <- x - g n; its tangential increment is kept. */
static void wall_contact(const orc_params *P, double x[3])
{
    double g = 0.0;
    for (int d = 0; d < 3; d++) g += (x[d] - P->wall_p[d]) * P->wall_n[d];
    if (g < 0.0)
        for (int d = 0; d < 3; d++) x[d] -= g * P->wall_n[d];
}

/* Sec. 4.2: rigid tool = wedge between the rake face (through the cutting edge, tilted by the
 * rake angle from the vertical) and the flank face (rising at the clearance angle behind the
 * edge), moving along -x. A penetrating node is projected onto the nearer face; friction is
 * Coulomb with the penalty limit m/dt^2: the tangential increment relative to the tool is
 * removed (stick) if its size is within mu * penetration, else reduced by mu * penetration
 * (slip). */
static void tool_contact(const orc_params *P, double t_next, const double du_in[3], double x[3])
{
    double xt = P->tool_x0 - P->tool_v * t_next;
    double yt = P->tool_tip_y;
    double nr[3] = {-cos(P->tool_rake), sin(P->tool_rake), 0.0};
    double nf[3] = {sin(P->tool_clear), -cos(P->tool_clear), 0.0};
    double rx = x[0] - xt, ry = x[1] - yt;
    double gr = rx * nr[0] + ry * nr[1];
    double gf = rx * nf[0] + ry * nf[1];
    if (!(gr < 0.0 && gf < 0.0)) return;
    const double *n = (gr >= gf) ? nr : nf;
    double pen = -((gr >= gf) ? gr : gf);
    for (int d = 0; d < 3; d++) x[d] += pen * n[d];
    double w[3] = {du_in[0] + P->tool_v * P->dt, du_in[1], du_in[2]};
    double wn = w[0] * n[0] + w[1] * n[1] + w[2] * n[2];
    double wt[3], wtn = 0.0;
    for (int d = 0; d < 3; d++) { wt[d] = w[d] - wn * n[d]; wtn += wt[d] * wt[d]; }
    wtn = sqrt(wtn);
    double lim = P->friction * pen;
    double scale = (wtn <= lim) ? 1.0 : lim / wtn;
    for (int d = 0; d < 3; d++) x[d] -= scale * wt[d];
}

/* ================================================================ simulation state */
typedef struct {
    orc_params P;
    int64_t nn, nm, cap_nodes, cap_mps;
    /* nodes */
    double *x, *x_prev, *du, *mI, *rI;
    uint8_t *flags;
    int64_t *node_gid;
    /* material points */
    double *xp, *xp_prev, *F, *dF, *be, *sig, *vol, *mass, *ebar, *T, *rate, *lam;
    int32_t *mat, *newton_it;
    int64_t *mp_gid;
    uint8_t *failed;
    /* support CSR (MP-major, IDs ascending) with N and grad N per pair */
    int64_t *off;
    int32_t *ids;
    double *N, *dN;
    int64_t n_pairs, cap_pairs;
    /* run */
    double time;
    int64_t step;
    int64_t next_node_gid;
    int err;
    int64_t err_id;
    int64_t n_eroded_total, n_inserted_total, n_removed_total;
} orc_sim;

static void *xrealloc(void *p, size_t n) { return realloc(p, n ? n : 1); }

static int sim_reserve_pairs(orc_sim *s, int64_t need)
{
    if (need <= s->cap_pairs) return ORC_OK;
    int64_t cap = need + need / 2 + 1024;
    int32_t *ids = xrealloc(s->ids, (size_t)cap * sizeof(int32_t));
    if (!ids) return ORC_ERR_OOM;
    s->ids = ids;
    double *N = xrealloc(s->N, (size_t)cap * sizeof(double));
    if (!N) return ORC_ERR_OOM;
    s->N = N;
    double *dN = xrealloc(s->dN, (size_t)cap * 3 * sizeof(double));
    if (!dN) return ORC_ERR_OOM;
    s->dN = dN;
    s->cap_pairs = cap;
    return ORC_OK;
}

/* the error with the smallest offending ID is kept (one writer at a time in the OpenMP build) */
static void set_err(orc_sim *s, int code, int64_t id)
{
#pragma omp critical(orc_err)
    {
        if (s->err == ORC_OK || id < s->err_id) { s->err = code; s->err_id = id; }
    }
}

/* Steps 5 and 6 of Algorithm 1 for every MP: linked-cell search at the current positions,
 * then the LME Newton solve warm-started from the MP's previous lambda. With lme_fail given, an
 * MP whose Newton solve fails is flagged there (its lambda keeps the warm start) instead of
 * stopping the step; every other error stops it (the smallest offending ID is reported).
 * The MPs are independent: a first pass counts each support, the counts give the CSR offsets,
 * and a second pass searches again into the MP's own slice of the pair arrays and solves for
 * its shape functions (in the OpenMP build both passes run over MPs in parallel). */
static int search_and_shape(orc_sim *s, uint8_t *lme_fail)
{
    const orc_params *P = &s->P;
    const int64_t nm = s->nm;
    orc_grid g;
    int st = grid_build(&g, s->nn, s->x, P->cell_size);
    if (st != ORC_OK) return st;
    const int64_t cap_mp = 4096;
    int64_t *cnt = malloc((size_t)(nm + 1) * sizeof(int64_t));
    s->off = xrealloc(s->off, (size_t)(nm + 1) * sizeof(int64_t));
    if (!cnt || !s->off) { free(cnt); grid_free(&g); return ORC_ERR_OOM; }
    int oom = 0;
#pragma omp parallel
    {
        int32_t *buf = malloc((size_t)cap_mp * sizeof(int32_t));
        if (!buf) {
#pragma omp atomic write
            oom = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < nm; p++)
            cnt[p] = buf ? search_mp(&g, s->x, s->xp + 3 * p, P->rs2, P->cell_size, buf, cap_mp) : 0;
        free(buf);
    }
    if (oom) { free(cnt); grid_free(&g); return ORC_ERR_OOM; }
    s->off[0] = 0;
    for (int64_t p = 0; p < nm; p++) {
        if (cnt[p] > cap_mp) {
            set_err(s, ORC_ERR_CAPACITY, s->mp_gid[p]);
            free(cnt); grid_free(&g);
            return ORC_ERR_CAPACITY;
        }
        s->off[p + 1] = s->off[p] + cnt[p];
    }
    free(cnt);
    if ((st = sim_reserve_pairs(s, s->off[nm])) != ORC_OK) { grid_free(&g); return st; }
    int failed = 0;
#pragma omp parallel
    {
        double *d = malloc((size_t)cap_mp * 3 * sizeof(double));
        if (!d) {
#pragma omp atomic write
            oom = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < nm; p++) {
            if (!d) continue;
            const int64_t base = s->off[p], n = s->off[p + 1] - base;
            search_mp(&g, s->x, s->xp + 3 * p, P->rs2, P->cell_size, s->ids + base, n);
            for (int64_t k = 0; k < n; k++)
                for (int i = 0; i < 3; i++) d[3 * k + i] = s->xp[3 * p + i] - s->x[3 * (int64_t)s->ids[base + k] + i];
            int32_t it = 0, it2 = 0;
            double lam0[3] = {s->lam[3 * p], s->lam[3 * p + 1], s->lam[3 * p + 2]};
            int lst = orc_lme(n, d, P->beta, P->newton_tol * P->h, P->max_newton, s->lam + 3 * p,
                              s->N + base, s->dN + 3 * base, &it);
            if (lst == ORC_ERR_LME_NOCONV && (lam0[0] != 0.0 || lam0[1] != 0.0 || lam0[2] != 0.0)) {
                /* a warm start far from the solution can concentrate the weights on a node or two
                 * (singular Hessian): solve once more from lambda = 0 */
                s->lam[3 * p] = s->lam[3 * p + 1] = s->lam[3 * p + 2] = 0.0;
                lst = orc_lme(n, d, P->beta, P->newton_tol * P->h, P->max_newton, s->lam + 3 * p,
                              s->N + base, s->dN + 3 * base, &it2);
                it += it2;
            }
            s->newton_it[p] = it;
            if (lst == ORC_ERR_LME_NOCONV && lme_fail && n > 0) {
                lme_fail[p] = 1;
                memcpy(s->lam + 3 * p, lam0, sizeof(lam0));
            } else if (lst != ORC_OK) {
                set_err(s, lst, s->mp_gid[p]);
#pragma omp atomic write
                failed = 1;
            }
        }
        free(d);
    }
    grid_free(&g);
    if (oom) return ORC_ERR_OOM;
    if (failed) return s->err;
    s->n_pairs = s->off[nm];
    return ORC_OK;
}

/* ------------------------------------------------------------------ public: create */
orc_sim *orc_sim_create(const orc_params *P, int64_t nn, int64_t nm, const double *node_x,
                        const double *node_du0, const uint8_t *node_flags, const double *mp_x,
                        const double *mp_vol, const double *mp_mass, const int32_t *mp_mat)
{
    orc_sim *s = calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->P = *P;
    s->nn = nn; s->nm = nm;
#define ALLOC(f, n, T) s->f = calloc((size_t)(n) > 0 ? (size_t)(n) : 1, sizeof(T))
    ALLOC(x, 3 * nn, double); ALLOC(x_prev, 3 * nn, double); ALLOC(du, 3 * nn, double);
    ALLOC(mI, nn, double); ALLOC(rI, 3 * nn, double); ALLOC(flags, nn, uint8_t);
    ALLOC(node_gid, nn, int64_t);
    ALLOC(xp, 3 * nm, double); ALLOC(xp_prev, 3 * nm, double); ALLOC(F, 9 * nm, double);
    ALLOC(dF, 9 * nm, double); ALLOC(be, 6 * nm, double); ALLOC(sig, 6 * nm, double);
    ALLOC(vol, nm, double); ALLOC(mass, nm, double); ALLOC(ebar, nm, double); ALLOC(T, nm, double);
    ALLOC(rate, nm, double); ALLOC(lam, 3 * nm, double); ALLOC(mat, nm, int32_t);
    ALLOC(newton_it, nm, int32_t); ALLOC(mp_gid, nm, int64_t); ALLOC(failed, nm, uint8_t);
#undef ALLOC
    s->cap_nodes = nn; s->cap_mps = nm;
    memcpy(s->x, node_x, (size_t)nn * 3 * sizeof(double));
    memcpy(s->x_prev, node_x, (size_t)nn * 3 * sizeof(double));
    memcpy(s->du, node_du0, (size_t)nn * 3 * sizeof(double));
    memcpy(s->flags, node_flags, (size_t)nn);
    for (int64_t i = 0; i < nn; i++) s->node_gid[i] = i;
    s->next_node_gid = nn;
    memcpy(s->xp, mp_x, (size_t)nm * 3 * sizeof(double));
    memcpy(s->xp_prev, mp_x, (size_t)nm * 3 * sizeof(double));
    memcpy(s->vol, mp_vol, (size_t)nm * sizeof(double));
    memcpy(s->mass, mp_mass, (size_t)nm * sizeof(double));
    memcpy(s->mat, mp_mat, (size_t)nm * sizeof(int32_t));
    for (int64_t p = 0; p < nm; p++) {
        s->mp_gid[p] = p;
        for (int i = 0; i < 9; i++) s->F[9 * p + i] = s->dF[9 * p + i] = (i % 4 == 0) ? 1.0 : 0.0;
        s->be[6 * p + 0] = s->be[6 * p + 1] = s->be[6 * p + 2] = 1.0;
        s->T[p] = P->T0;
    }
    /* Algorithm 1 REQUIRE: support domains and shape functions of the initial sets */
    s->err = search_and_shape(s, NULL);
    return s;
}

void orc_sim_destroy(orc_sim *s)
{
    if (!s) return;
    void *ptrs[] = {s->x, s->x_prev, s->du, s->mI, s->rI, s->flags, s->node_gid, s->xp, s->xp_prev,
                    s->F, s->dF, s->be, s->sig, s->vol, s->mass, s->ebar, s->T, s->rate, s->lam,
                    s->mat, s->newton_it, s->mp_gid, s->failed, s->off, s->ids, s->N, s->dN};
    for (size_t i = 0; i < sizeof(ptrs) / sizeof(ptrs[0]); i++) free(ptrs[i]);
    free(s);
}

/* ------------------------------------------------------------------ erosion and node changes */
/* MPs flagged by the fracture criterion leave the body (mass leaves with them). Compaction
 * keeps the surviving MPs in ascending ID order. */
static int64_t erode_mps(orc_sim *s)
{
    int64_t w = 0;
    for (int64_t p = 0; p < s->nm; p++) {
        if (s->failed[p]) continue;
        if (w != p) {
#define MV(f, k) memmove(s->f + (k) * w, s->f + (k) * p, (k) * sizeof(*s->f))
            MV(xp, 3); MV(xp_prev, 3); MV(F, 9); MV(dF, 9); MV(be, 6); MV(sig, 6); MV(vol, 1);
            MV(mass, 1); MV(ebar, 1); MV(T, 1); MV(rate, 1); MV(lam, 3); MV(mat, 1);
            MV(newton_it, 1); MV(mp_gid, 1); MV(failed, 1);
#undef MV
        }
        w++;
    }
    int64_t removed = s->nm - w;
    s->nm = w;
    return removed;
}

/* Nodes that lie in no MP's support after erosion are removed (ascending order kept); the
 * support lists are renumbered (the map is monotone, so lists stay sorted). */
static int64_t remove_orphan_nodes(orc_sim *s)
{
    int64_t nn = s->nn;
    int64_t *cnt = calloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t k = 0; k < s->n_pairs; k++) cnt[s->ids[k]]++;
    int64_t *newid = malloc((size_t)nn * sizeof(int64_t));
    int64_t w = 0;
    for (int64_t i = 0; i < nn; i++) {
        if (cnt[i] == 0) { newid[i] = -1; continue; }
        newid[i] = w;
        if (w != i) {
#define MV(f, k) memmove(s->f + (k) * w, s->f + (k) * i, (k) * sizeof(*s->f))
            MV(x, 3); MV(x_prev, 3); MV(du, 3); MV(flags, 1); MV(node_gid, 1);
#undef MV
        }
        w++;
    }
    for (int64_t k = 0; k < s->n_pairs; k++) s->ids[k] = (int32_t)newid[s->ids[k]];
    int64_t removed = nn - w;
    s->nn = w;
    free(cnt); free(newid);
    return removed;
}

/* Node insertion. The paper adds nodes to the node set during the run (Sec. 1, Sec. 3.2) but
 * gives no rule; the reading taken here: an MP whose LME solve fails at its new position lies
 * outside (or on the boundary of) the convex hull of its support, so a node is inserted one
 * spacing h beyond the MP, away from the centroid c of its support nodes:
 *     x_new = x_p + h u / |u|,   u = x_p - c,
 * which puts x_p strictly inside the hull of the support plus the new node (x_p lies between
 * c and x_new). The new node is free (no flags), its increment is the MP's own increment of
 * the step, du = x_p,n+1 - x_p,n (the interpolation of the old support's increments), and
 * x_prev = x_new - du. New IDs continue the node numbering, in ascending ID of the failing MPs.
 * At most max_insert nodes are inserted over a run (ORC_ERR_CAPACITY beyond that). */
#define ORC_INSERT_ROUNDS 1
static int insert_nodes(orc_sim *s, const uint8_t *lme_fail, int64_t n_fail)
{
    const orc_params *P = &s->P;
    if (s->n_inserted_total + n_fail > P->allow_insert) {
        for (int64_t p = 0; p < s->nm; p++)
            if (lme_fail[p]) { set_err(s, ORC_ERR_CAPACITY, s->mp_gid[p]); break; }
        return ORC_ERR_CAPACITY;
    }
    const int64_t nn = s->nn, nn_new = nn + n_fail;
    if (nn_new > s->cap_nodes) {
#define GROW(f, k) do { void *q_ = xrealloc(s->f, (size_t)(k) * (size_t)nn_new * sizeof(*s->f)); \
                        if (!q_) return ORC_ERR_OOM; s->f = q_; } while (0)
        GROW(x, 3); GROW(x_prev, 3); GROW(du, 3); GROW(mI, 1); GROW(rI, 3); GROW(flags, 1); GROW(node_gid, 1);
#undef GROW
        s->cap_nodes = nn_new;
    }
    int64_t i = nn;
    for (int64_t p = 0; p < s->nm; p++) {
        if (!lme_fail[p]) continue;
        const double *xp = s->xp + 3 * p;
        double c[3] = {0.0, 0.0, 0.0};
        const int64_t n = s->off[p + 1] - s->off[p];
        for (int64_t k = s->off[p]; k < s->off[p + 1]; k++)
            for (int d = 0; d < 3; d++) c[d] += s->x[3 * (int64_t)s->ids[k] + d];
        double u[3], len = 0.0;
        for (int d = 0; d < 3; d++) {
            u[d] = xp[d] - c[d] / (double)n;
            len += u[d] * u[d];
        }
        len = sqrt(len);
        if (!(len > 1e-12 * P->h)) { set_err(s, ORC_ERR_LME_NOCONV, s->mp_gid[p]); return ORC_ERR_LME_NOCONV; }
        for (int d = 0; d < 3; d++) {
            const double xn = xp[d] + P->h * (u[d] / len);
            const double du = xp[d] - s->xp_prev[3 * p + d];
            s->x[3 * i + d] = xn;
            s->du[3 * i + d] = du;
            s->x_prev[3 * i + d] = xn - du;
            s->rI[3 * i + d] = 0.0;
        }
        s->mI[i] = 0.0;
        s->flags[i] = 0;
        s->node_gid[i] = s->next_node_gid++;
        i++;
    }
    s->nn = nn_new;
    s->n_inserted_total += n_fail;
    return ORC_OK;
}

/* ------------------------------------------------------------------ public: one step */
/* Algorithm 1, steps 1-6, in order. Returns ORC_OK or the first error (state then partial). */
int orc_sim_step(orc_sim *s)
{
    const orc_params *P = &s->P;
    if (s->err != ORC_OK) return s->err;
    const double dt = P->dt;
    int64_t nn = s->nn, nm = s->nm;

    /* Step 1 (Eq. 5, Eq. 7): lumped mass m_I = sum_p N_Ip m_p, residual
     * r_I = -sum_p v_p sigma_p grad N_Ip (body force and Neumann loads are zero), optionally
     * stabilised by -eps sum_p N_Ip e_Ip (Eq. 8). Summation over p in ascending MP ID. */
    memset(s->mI, 0, (size_t)nn * sizeof(double));
    memset(s->rI, 0, (size_t)nn * 3 * sizeof(double));
    for (int64_t p = 0; p < nm; p++) {
        const double *sg = s->sig + 6 * p;
        double S[3][3];
        sym_to_full(sg, S);
        for (int64_t k = s->off[p]; k < s->off[p + 1]; k++) {
            int64_t a = s->ids[k];
            const double *g = s->dN + 3 * k;
            s->mI[a] += s->N[k] * s->mass[p];
            for (int i = 0; i < 3; i++)
                s->rI[3 * a + i] -= s->vol[p] * (S[i][0] * g[0] + S[i][1] * g[1] + S[i][2] * g[2]);
            if (P->eps_stab > 0.0) {
                /* Eq. 8: e = [x_I - x_p - dF (x_I,prev - x_p,prev)] / |x_I,prev - x_p,prev| */
                double dp[3], len = 0.0;
                for (int i = 0; i < 3; i++) {
                    dp[i] = s->x_prev[3 * a + i] - s->xp_prev[3 * p + i];
                    len += dp[i] * dp[i];
                }
                len = sqrt(len);
                if (len > 1e-12 * P->h) {
                    const double *D = s->dF + 9 * p;
                    for (int i = 0; i < 3; i++) {
                        double e = s->x[3 * a + i] - s->xp[3 * p + i]
                                 - (D[3 * i + 0] * dp[0] + D[3 * i + 1] * dp[1] + D[3 * i + 2] * dp[2]);
                        s->rI[3 * a + i] -= P->eps_stab * s->N[k] * e / len;
                    }
                }
            }
        }
    }

    /* Step 2 (Eq. 4, Eq. 6): du_{n+1} = du_n + dt^2 r_I / m_I (nodes without mass keep du),
     * fixed nodes du = 0, rigid contact, x_{n+1} = x_n + du_{n+1}. */
    double t_next = s->time + dt;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; i++) {
        double *du = s->du + 3 * i, *x = s->x + 3 * i;
        double xn[3] = {x[0], x[1], x[2]};
        if (s->flags[i] & 1) {
            du[0] = du[1] = du[2] = 0.0;
        } else if (s->mI[i] > 0.0) {
            for (int d = 0; d < 3; d++) du[d] += dt * dt * s->rI[3 * i + d] / s->mI[i];
        }
        double xt[3] = {xn[0] + du[0], xn[1] + du[1], xn[2] + du[2]};
        if (!(s->flags[i] & 1)) {
            if (P->wall) wall_contact(P, xt);
            if (P->tool) tool_contact(P, t_next, du, xt);
        }
        for (int d = 0; d < 3; d++) {
            du[d] = xt[d] - xn[d];
            s->x_prev[3 * i + d] = xn[d];
            x[d] = xt[d];
            if (!isfinite(x[d])) set_err(s, ORC_ERR_NONFINITE, s->node_gid[i]);
        }
    }
    if (s->err != ORC_OK) return s->err;

    /* Step 3 (Eq. 9-13): x_p = sum N_I x_I,n+1; dF = 1 + sum du_I (x) grad N_I;
     * F_{n+1} = dF F_n; v_{n+1} = det(dF) v_n. Step 4: constitutive update. */
    int any_failed = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : any_failed)
    for (int64_t p = 0; p < nm; p++) {
        double xpn[3] = {0, 0, 0}, D[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int64_t k = s->off[p]; k < s->off[p + 1]; k++) {
            int64_t a = s->ids[k];
            for (int i = 0; i < 3; i++) {
                xpn[i] += s->N[k] * s->x[3 * a + i];
                for (int j = 0; j < 3; j++) D[i][j] += s->du[3 * a + i] * s->dN[3 * k + j];
            }
        }
        for (int i = 0; i < 3; i++) {
            s->xp_prev[3 * p + i] = s->xp[3 * p + i];
            s->xp[3 * p + i] = xpn[i];
        }
        double detD = det3(D);
        if (!(detD > 0.0)) { set_err(s, ORC_ERR_JACOBIAN, s->mp_gid[p]); continue; }
        double Fo[3][3], Fn[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Fo[i][j] = s->F[9 * p + 3 * i + j];
        matmul3(D, Fo, Fn);
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                s->F[9 * p + 3 * i + j] = Fn[i][j];
                s->dF[9 * p + 3 * i + j] = D[i][j];
            }
        s->vol[p] *= detD;
        double J = det3(Fn);
        rm_out_t o;
        int st = return_map(&P->mat[s->mat[p]], dt, D, s->be + 6 * p, s->ebar[p], s->T[p], J, &o);
        if (st != ORC_OK) { set_err(s, st, s->mp_gid[p]); continue; }
        memcpy(s->sig + 6 * p, o.sig, sizeof(o.sig));
        memcpy(s->be + 6 * p, o.be, sizeof(o.be));
        s->ebar[p] = o.ebar; s->T[p] = o.T; s->rate[p] = o.rate;
        s->failed[p] = (uint8_t)(o.failed && P->allow_erode);
        any_failed |= s->failed[p];
        for (int i = 0; i < 6; i++)
            if (!isfinite(o.sig[i])) set_err(s, ORC_ERR_NONFINITE, s->mp_gid[p]);
    }
    if (s->err != ORC_OK) return s->err;
    s->time = t_next;
    s->step++;

    /* erosion (fracture): failed MPs leave before the new supports are built */
    if (any_failed) s->n_eroded_total += erode_mps(s);

    /* Steps 5-6: search and shape functions at the new configuration; with insertion on, MPs
     * whose solve fails get a node each and the search and solve are repeated once */
    int st;
    if (P->allow_insert > 0) {
        uint8_t *lme_fail = calloc((size_t)s->nm + 1, 1);
        if (!lme_fail) return ORC_ERR_OOM;
        for (int round = 0;; round++) {
            memset(lme_fail, 0, (size_t)s->nm);
            st = search_and_shape(s, round < ORC_INSERT_ROUNDS ? lme_fail : NULL);
            if (st != ORC_OK || round == ORC_INSERT_ROUNDS) break;
            int64_t n_fail = 0;
            for (int64_t p = 0; p < s->nm; p++) n_fail += lme_fail[p];
            if (n_fail == 0) break;
            if ((st = insert_nodes(s, lme_fail, n_fail)) != ORC_OK) break;
        }
        free(lme_fail);
    } else {
        st = search_and_shape(s, NULL);
    }
    if (st != ORC_OK) return st;
    if (any_failed && P->allow_erode) s->n_removed_total += remove_orphan_nodes(s);
    return ORC_OK;
}

/* ------------------------------------------------------------------ public: accessors */
void orc_sim_counts(const orc_sim *s, int64_t *nn, int64_t *nm, int64_t *np, int64_t *step,
                    int32_t *err, int64_t *err_id)
{
    *nn = s->nn; *nm = s->nm; *np = s->n_pairs; *step = s->step; *err = s->err; *err_id = s->err_id;
}

/* field codes: 0 node_x, 1 node_du, 2 node_mass, 3 node_force, 4 mp_x, 5 F, 6 be, 7 sigma,
 * 8 vol, 9 ebar, 10 T, 11 lambda, 12 offsets, 13 ids, 14 N, 15 dN, 16 node_gid, 17 mp_gid,
 * 18 newton_it, 19 rate */
int orc_sim_get(const orc_sim *s, int32_t field, void *dst, int64_t bytes)
{
    const void *src = NULL;
    int64_t need = 0;
    switch (field) {
    case 0: src = s->x; need = 24 * s->nn; break;
    case 1: src = s->du; need = 24 * s->nn; break;
    case 2: src = s->mI; need = 8 * s->nn; break;
    case 3: src = s->rI; need = 24 * s->nn; break;
    case 4: src = s->xp; need = 24 * s->nm; break;
    case 5: src = s->F; need = 72 * s->nm; break;
    case 6: src = s->be; need = 48 * s->nm; break;
    case 7: src = s->sig; need = 48 * s->nm; break;
    case 8: src = s->vol; need = 8 * s->nm; break;
    case 9: src = s->ebar; need = 8 * s->nm; break;
    case 10: src = s->T; need = 8 * s->nm; break;
    case 11: src = s->lam; need = 24 * s->nm; break;
    case 12: src = s->off; need = 8 * (s->nm + 1); break;
    case 13: src = s->ids; need = 4 * s->n_pairs; break;
    case 14: src = s->N; need = 8 * s->n_pairs; break;
    case 15: src = s->dN; need = 24 * s->n_pairs; break;
    case 16: src = s->node_gid; need = 8 * s->nn; break;
    case 17: src = s->mp_gid; need = 8 * s->nm; break;
    case 18: src = s->newton_it; need = 4 * s->nm; break;
    case 19: src = s->rate; need = 8 * s->nm; break;
    case 20: src = s->xp_prev; need = 24 * s->nm; break;
    case 21: src = s->x_prev; need = 24 * s->nn; break;
    case 22: src = s->dF; need = 72 * s->nm; break;
    default: return ORC_ERR_ARG;
    }
    if (bytes != need) return ORC_ERR_ARG;
    if (need) memcpy(dst, src, (size_t)need);
    return ORC_OK;
}

/* overwrite the node kinematic state (shadow parity: the oracle continues from a given state) */
int orc_sim_set(orc_sim *s, int32_t field, const void *src, int64_t bytes)
{
    void *dst = NULL;
    int64_t need = 0;
    switch (field) {
    case 0: dst = s->x; need = 24 * s->nn; break;
    case 1: dst = s->du; need = 24 * s->nn; break;
    case 4: dst = s->xp; need = 24 * s->nm; break;
    case 5: dst = s->F; need = 72 * s->nm; break;
    case 6: dst = s->be; need = 48 * s->nm; break;
    case 7: dst = s->sig; need = 48 * s->nm; break;
    case 8: dst = s->vol; need = 8 * s->nm; break;
    case 9: dst = s->ebar; need = 8 * s->nm; break;
    case 10: dst = s->T; need = 8 * s->nm; break;
    case 11: dst = s->lam; need = 24 * s->nm; break;
    case 20: dst = s->xp_prev; need = 24 * s->nm; break;
    case 21: dst = s->x_prev; need = 24 * s->nn; break;
    case 22: dst = s->dF; need = 72 * s->nm; break;
    default: return ORC_ERR_ARG;
    }
    if (bytes != need) return ORC_ERR_ARG;
    memcpy(dst, src, (size_t)need);
    return ORC_OK;
}

/* one MP's support row: its node IDs (ascending), N and grad N; returns the row length, or -1 if
 * p is out of range or the row is longer than cap (nothing copied) */
int64_t orc_sim_row(const orc_sim *s, int64_t p, int32_t *ids, double *N, double *dN, int64_t cap)
{
    if (p < 0 || p >= s->nm) return -1;
    const int64_t b = s->off[p], n = s->off[p + 1] - b;
    if (n > cap) return -1;
    memcpy(ids, s->ids + b, (size_t)n * sizeof(int32_t));
    memcpy(N, s->N + b, (size_t)n * sizeof(double));
    memcpy(dN, s->dN + 3 * b, (size_t)n * 3 * sizeof(double));
    return n;
}

/* the tool contact of one node (Sec. 4.2), for tests: x (in/out) is the node's position after
 * the central-difference update, du its increment before contact, t_next the time of the new
 * position */
void orc_tool_contact(const orc_params *P, double t_next, const double *du, double *x)
{
    tool_contact(P, t_next, du, x);
}

/* recompute supports and shape functions from the current positions (after orc_sim_set) */
int orc_sim_refresh(orc_sim *s)
{
    s->err = ORC_OK;
    s->err_id = 0;
    s->err = search_and_shape(s, NULL);
    return s->err;
}

/* ------------------------------------------------------------------ public: standalone pieces */
/* linked-cell grid of a node set: origin (3), dims (3), cell_start (n_cells+1), sorted IDs */
int orc_grid_info(int64_t nn, const double *x, double cell_size, double *origin, int64_t *dims)
{
    orc_grid g;
    int st = grid_build(&g, nn, x, cell_size);
    if (st != ORC_OK) return st;
    for (int d = 0; d < 3; d++) { origin[d] = g.origin[d]; dims[d] = g.dims[d]; }
    grid_free(&g);
    return ORC_OK;
}

int orc_grid_cells(int64_t nn, const double *x, double cell_size, int64_t n_cells,
                   int64_t *cell_start, int32_t *sorted)
{
    orc_grid g;
    int st = grid_build(&g, nn, x, cell_size);
    if (st != ORC_OK) return st;
    if (g.n_cells != n_cells) { grid_free(&g); return ORC_ERR_ARG; }
    memcpy(cell_start, g.cell_start, (size_t)(n_cells + 1) * sizeof(int64_t));
    memcpy(sorted, g.sorted, (size_t)nn * sizeof(int32_t));
    grid_free(&g);
    return ORC_OK;
}

/* supports of a set of points against a node set (Algorithm 3): CSR with ascending IDs.
 * offsets has nm+1 entries; ids has room for cap entries. Returns the total pair count, or a
 * negative status (ORC_ERR_CAPACITY when cap is too small). */
int64_t orc_search(int64_t nn, const double *node_x, int64_t nm, const double *mp_x, double rs2,
                   double cell_size, int64_t *offsets, int32_t *ids, int64_t cap)
{
    orc_grid g;
    int st = grid_build(&g, nn, node_x, cell_size);
    if (st != ORC_OK) return st;
    offsets[0] = 0;
    for (int64_t p = 0; p < nm; p++) {
        int64_t room = cap - offsets[p];
        int64_t cnt = search_mp(&g, node_x, mp_x + 3 * p, rs2, cell_size, ids + offsets[p], room);
        if (cnt > room) { grid_free(&g); return ORC_ERR_CAPACITY; }
        offsets[p + 1] = offsets[p] + cnt;
    }
    grid_free(&g);
    return offsets[nm];
}

/* per-MP kinematic gather (step 3): given the support, N, grad N of one MP and the new nodal
 * positions / increments, return x_p,n+1 and dF (row-major). */
void orc_kinematics(int64_t n, const int32_t *ids, const double *N, const double *dN,
                    const double *node_x, const double *node_du, double *xp, double *dF9)
{
    double D[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    xp[0] = xp[1] = xp[2] = 0.0;
    for (int64_t k = 0; k < n; k++) {
        int64_t a = ids[k];
        for (int i = 0; i < 3; i++) {
            xp[i] += N[k] * node_x[3 * a + i];
            for (int j = 0; j < 3; j++) D[i][j] += node_du[3 * a + i] * dN[3 * k + j];
        }
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dF9[3 * i + j] = D[i][j];
}

int orc_sizeof_params(void) { return (int)sizeof(orc_params); }
int orc_sizeof_material(void) { return (int)sizeof(orc_material); }

/* ================================================================ reference adjoint (test oracle)
 * Reverse-mode derivative of the explicit step (Algorithm 1) with frozen topology: supports,
 * wall-contact set and the elastic/plastic branch of each return map are those of the base
 * trajectory. Objectives are functions of the final node positions; parameters are the
 * Johnson-Cook constants (A, B, n, C, m) of material 0 and the impact velocity (through the
 * initial increments). Derivations:
 *  - LME (Eq. 14), implicit-function theorem on r(lambda, d) = sum N_a d_a = 0:
 *      grad N_a = -N_a H^-1 d_a, H = sum N d d^T - r r^T; dlambda = -H^-1 sum_a (dr/dd_a) dd_a,
 *      dr/dd_a = N_a [1 + d_a (lambda - 2 beta d_a)^T] (at r = 0); N = softmax(f),
 *      f_a = -beta |d_a|^2 + lambda . d_a.
 *  - return map (Sec. 4): isotropic tensor functions of b_tr; principal derivatives by the chain
 *    rule of the radial return (implicit function theorem on the consistency condition), the
 *    off-diagonal part by divided differences (tau_A - tau_B)/(lam_A - lam_B), replaced by the
 *    second-order symmetric limit when the eigenvalues (nearly) coincide.
 *  - kinematics, lumped mass / force and the central-difference update: transposes of the
 *    linear maps (the wall projection acts on the frozen contact set). */

orc_sim *orc_sim_clone(const orc_sim *s)
{
    orc_sim *c = calloc(1, sizeof(orc_sim));
    if (!c) return NULL;
    *c = *s;
#define CP(f, n) do { size_t b_ = (size_t)(n) * sizeof(*s->f); c->f = malloc(b_ ? b_ : 1); if (b_) memcpy(c->f, s->f, b_); } while (0)
    CP(x, 3 * s->nn); CP(x_prev, 3 * s->nn); CP(du, 3 * s->nn); CP(mI, s->nn); CP(rI, 3 * s->nn);
    CP(flags, s->nn); CP(node_gid, s->nn);
    CP(xp, 3 * s->nm); CP(xp_prev, 3 * s->nm); CP(F, 9 * s->nm); CP(dF, 9 * s->nm); CP(be, 6 * s->nm);
    CP(sig, 6 * s->nm); CP(vol, s->nm); CP(mass, s->nm); CP(ebar, s->nm); CP(T, s->nm); CP(rate, s->nm);
    CP(lam, 3 * s->nm); CP(mat, s->nm); CP(newton_it, s->nm); CP(mp_gid, s->nm); CP(failed, s->nm);
    CP(off, s->nm + 1); CP(ids, s->n_pairs); CP(N, s->n_pairs); CP(dN, 3 * s->n_pairs);
#undef CP
    c->cap_pairs = s->n_pairs;
    c->cap_nodes = s->nn;
    c->cap_mps = s->nm;
    return c;
}

/* ---------------------------------------------------------------- LME backward (one MP) */
/* Inputs: d (n x 3) = x_p - x_a, N, G (n x 3) = grad N, lambda, beta; adjoints Nb, Gb.
 * Output: db (n x 3) = dL/dd_a. */
int orc_lme_backward(int64_t n, const double *d, const double *N, const double *G, const double *lam, double beta,
                     const double *Nb_in, const double *Gb, double *db)
{
    (void)G;   /* grad N is recomputed from H below */
    double H[3][3] = {{0}}, r[3] = {0, 0, 0}, Hi[3][3];
    for (int64_t a = 0; a < n; a++)
        for (int i = 0; i < 3; i++) {
            r[i] += N[a] * d[3 * a + i];
            for (int j = 0; j < 3; j++) H[i][j] += N[a] * d[3 * a + i] * d[3 * a + j];
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) H[i][j] -= r[i] * r[j];
    if (!inv3(H, Hi)) return ORC_ERR_LME_NOCONV;
    double *Nb = malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!Nb) return ORC_ERR_OOM;
    /* G_a = -N_a u_a, u_a = H^-1 d_a */
    double Hb[3][3] = {{0}};
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a, *gb = Gb + 3 * a;
        double u[3], w[3];
        for (int i = 0; i < 3; i++) u[i] = Hi[i][0] * da[0] + Hi[i][1] * da[1] + Hi[i][2] * da[2];
        Nb[a] = Nb_in[a] - (gb[0] * u[0] + gb[1] * u[1] + gb[2] * u[2]);
        for (int i = 0; i < 3; i++) w[i] = -N[a] * (Hi[i][0] * gb[0] + Hi[i][1] * gb[1] + Hi[i][2] * gb[2]);
        for (int i = 0; i < 3; i++) {
            db[3 * a + i] = w[i];
            for (int j = 0; j < 3; j++) Hb[i][j] -= w[i] * u[j];
        }
    }
    double Hs[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) Hs[i][j] = 0.5 * (Hb[i][j] + Hb[j][i]);
    /* H = sum N d d^T - r r^T with r = sum N d (r ~ 0 at convergence; kept for consistency) */
    double Hr[3] = {0, 0, 0};   /* Hs r */
    for (int i = 0; i < 3; i++) Hr[i] = Hs[i][0] * r[0] + Hs[i][1] * r[1] + Hs[i][2] * r[2];
    double S = 0.0;
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a;
        double Hd[3];
        for (int i = 0; i < 3; i++) Hd[i] = Hs[i][0] * da[0] + Hs[i][1] * da[1] + Hs[i][2] * da[2];
        /* from sum N d d^T and from -r r^T (r = sum N d): d r r^T -> rbar = -2 Hs r */
        Nb[a] += (da[0] * Hd[0] + da[1] * Hd[1] + da[2] * Hd[2]) - 2.0 * (da[0] * Hr[0] + da[1] * Hr[1] + da[2] * Hr[2]);
        for (int i = 0; i < 3; i++) db[3 * a + i] += 2.0 * N[a] * Hd[i] - 2.0 * N[a] * Hr[i];
        S += N[a] * Nb[a];
    }
    /* softmax: fbar_a = N_a (Nb_a - S); f_a = -beta |d|^2 + lambda.d */
    double lb[3] = {0, 0, 0};
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a;
        double fb = N[a] * (Nb[a] - S);
        for (int i = 0; i < 3; i++) {
            db[3 * a + i] += fb * (lam[i] - 2.0 * beta * da[i]);
            lb[i] += fb * da[i];
        }
    }
    /* lambda(d) from r = 0: mu = H^-1 lb, db_a -= N_a [mu + (lambda - 2 beta d_a)(d_a . mu)] */
    double mu[3];
    for (int i = 0; i < 3; i++) mu[i] = Hi[i][0] * lb[0] + Hi[i][1] * lb[1] + Hi[i][2] * lb[2];
    for (int64_t a = 0; a < n; a++) {
        const double *da = d + 3 * a;
        double dm = da[0] * mu[0] + da[1] * mu[1] + da[2] * mu[2];
        for (int i = 0; i < 3; i++) db[3 * a + i] -= N[a] * (mu[i] + (lam[i] - 2.0 * beta * da[i]) * dm);
    }
    free(Nb);
    return ORC_OK;
}

/* ---------------------------------------------------------------- return map with tangents */
typedef struct {
    double K, mu, dt;
    double lam[3], Q[3][3], eps[3], e[3], enorm, qtr, x, q, rho, ee[3], tau[3], bA[3];
    int plastic, heating;
    double dsy_debar, dsy_dx, dsy_dT, dsy_dth[5], chi_c;   /* sigma_Y partials, chi/(rho0 cp) */
    double J;
} rm_detail_t;

/* JC partials at (ebar_n + x, x/dt, T) with respect to ebar_n, x (total), T and (A, B, n, C, m) */
static void jc_partials(const orc_material *M, double ebar_n, double x, double dt, double T, double *sy,
                        double *d_eb, double *d_x, double *d_T, double d_th[5])
{
    double ebar = ebar_n + x;
    double span = M->T_melt - M->T_room;
    double tstar_raw = (T - M->T_room) / span;
    double tstar = clamp01(tstar_raw);
    double therm = 1.0 - pow(tstar, M->m);
    double dtherm_dT = (tstar_raw > 0.0 && tstar_raw < 1.0) ? -M->m * pow(tstar, M->m - 1.0) / span : 0.0;
    double rstar = (x / dt) / M->eps_dot0;
    double rate = 1.0, drate_dx = 0.0, lr = 0.0;
    if (rstar > 1.0) { lr = log(rstar); rate = 1.0 + M->C * lr; drate_dx = M->C / x; }
    double epn = pow(ebar, M->n);
    double hard = M->A + M->B * epn;
    double dhard = (ebar > 0.0) ? M->B * M->n * pow(ebar, M->n - 1.0) : 0.0;
    *sy = hard * rate * therm;
    *d_eb = dhard * rate * therm;
    *d_x = (dhard * rate + hard * drate_dx) * therm;
    *d_T = hard * rate * dtherm_dT;
    d_th[0] = rate * therm;                                        /* A */
    d_th[1] = epn * rate * therm;                                  /* B */
    d_th[2] = (ebar > 0.0) ? M->B * epn * log(ebar) * rate * therm : 0.0;   /* n */
    d_th[3] = hard * lr * therm;                                   /* C */
    d_th[4] = (tstar > 0.0) ? -hard * rate * pow(tstar, M->m) * log(tstar) : 0.0;   /* m */
}

static int rm_detail(const orc_material *M, double dt, const double dF[3][3], const double be_n[6], double ebar_n,
                     double T_n, double J, rm_detail_t *o)
{
    rm_out_t out;
    int st = return_map(M, dt, dF, be_n, ebar_n, T_n, J, &out);
    if (st != ORC_OK) return st;
    memset(o, 0, sizeof(*o));
    o->K = M->E / (3.0 * (1.0 - 2.0 * M->nu));
    o->mu = M->E / (2.0 * (1.0 + M->nu));
    o->dt = dt;
    o->J = J;
    double b[3][3], t1[3][3], dFT[3][3], btr[3][3];
    sym_to_full(be_n, b);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFT[i][j] = dF[j][i];
    matmul3(dF, b, t1);
    matmul3(t1, dFT, btr);
    for (int i = 0; i < 3; i++)
        for (int j = i + 1; j < 3; j++) btr[i][j] = btr[j][i] = 0.5 * (btr[i][j] + btr[j][i]);
    jacobi_eig3(btr, o->lam, o->Q);
    double tr = 0.0;
    for (int A = 0; A < 3; A++) { o->eps[A] = 0.5 * log(o->lam[A]); tr += o->eps[A]; }
    double en2 = 0.0;
    for (int A = 0; A < 3; A++) { o->e[A] = o->eps[A] - tr / 3.0; en2 += o->e[A] * o->e[A]; }
    o->enorm = sqrt(en2);
    o->qtr = sqrt(6.0) * o->mu * o->enorm;
    o->x = out.ebar - ebar_n;
    o->plastic = o->x > 0.0;
    o->q = o->qtr - 3.0 * o->mu * o->x;
    o->rho = o->plastic ? o->q / o->qtr : 1.0;
    for (int A = 0; A < 3; A++) {
        o->ee[A] = tr / 3.0 + o->e[A] * o->rho;
        o->tau[A] = o->K * tr + 2.0 * o->mu * o->e[A] * o->rho;
        o->bA[A] = exp(2.0 * o->ee[A]);
    }
    o->heating = (M->model == 1 && M->chi > 0.0 && o->plastic);
    o->chi_c = o->heating ? M->chi / (M->rho0 * M->cp) : 0.0;
    if (M->model == 0) {
        o->dsy_debar = M->H;
        o->dsy_dx = M->H;
    } else {
        double sy;
        jc_partials(M, ebar_n, o->x, dt, T_n, &sy, &o->dsy_debar, &o->dsy_dx, &o->dsy_dT, o->dsy_dth);
    }
    return ORC_OK;
}

/* tangent of the principal map: inputs (dlam[3], debar_n, dT_n, dth[5]) ->
 * outputs (dtau[3], db[3], debar', dT') */
static void rm_principal_tangent(const rm_detail_t *o, const double dlam[3], double deb, double dT, const double dth[5],
                                 double dtau[3], double db[3], double *deb1, double *dT1)
{
    double deps[3], dtr = 0.0, de[3], den = 0.0;
    for (int A = 0; A < 3; A++) { deps[A] = dlam[A] / (2.0 * o->lam[A]); dtr += deps[A]; }
    for (int A = 0; A < 3; A++) de[A] = deps[A] - dtr / 3.0;
    if (o->enorm > 0.0)
        for (int A = 0; A < 3; A++) den += o->e[A] * de[A] / o->enorm;
    double dqtr = sqrt(6.0) * o->mu * den;
    double dx = 0.0, drho = 0.0, dq = dqtr;
    if (o->plastic) {
        double dsyth = 0.0;
        for (int k = 0; k < 5; k++) dsyth += o->dsy_dth[k] * dth[k];
        dx = (dqtr - o->dsy_debar * deb - o->dsy_dT * dT - dsyth) / (3.0 * o->mu + o->dsy_dx);
        dq = dqtr - 3.0 * o->mu * dx;
        drho = (dq - o->rho * dqtr) / o->qtr;
    }
    for (int A = 0; A < 3; A++) {
        double dee = dtr / 3.0 + de[A] * o->rho + o->e[A] * drho;
        dtau[A] = o->K * dtr + 2.0 * o->mu * (de[A] * o->rho + o->e[A] * drho);
        db[A] = 2.0 * o->bA[A] * dee;
    }
    *deb1 = deb + dx;
    *dT1 = dT + o->chi_c * (dq * o->x + o->q * dx);
}

/* Backward of one MP's return map. sigb, beb: adjoints of the 6-vectors sigma', b' (d L / d
 * component); ebb, Tb: adjoints of ebar', T'. Outputs: dFb (9, d L / d dF_ij), be_nb (6-vector),
 * ebb_n, Tb_n, Jb (adjoint of J = det F'), thb (5, accumulated). */
static void rm_backward(const rm_detail_t *o, const double dF[3][3], const double be_n[6], const double sig[6],
                        const double sigb[6], const double beb[6], double ebb, double Tb, double dFb[3][3],
                        double be_nb[6], double *ebb_n, double *Tb_n, double *Jb, double thb[5])
{
    /* full symmetric adjoints from 6-vector adjoints (off-diagonal entries count twice) */
    double Sb[3][3], Bb[3][3], S[3][3];
    sym_to_full(sigb, Sb); sym_to_full(beb, Bb); sym_to_full(sig, S);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            if (i != j) { Sb[i][j] *= 0.5; Bb[i][j] *= 0.5; }
    /* sigma = tau / J */
    double taub[3][3], ss = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) { taub[i][j] = Sb[i][j] / o->J; ss += Sb[i][j] * S[i][j]; }
    *Jb = -ss / o->J;
    /* to the eigenbasis */
    double Tq[3][3], Bq[3][3], tmp[3][3], QT[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) QT[i][j] = o->Q[j][i];
    matmul3(QT, taub, tmp); matmul3(tmp, o->Q, Tq);
    matmul3(QT, Bb, tmp); matmul3(tmp, o->Q, Bq);
    /* principal Jacobian columns: 3 eigenvalues, ebar_n, T_n, 5 parameters */
    double col_tau[10][3], col_b[10][3], col_eb[10], col_T[10];
    for (int c = 0; c < 10; c++) {
        double dl[3] = {0, 0, 0}, deb = 0, dTt = 0, dth[5] = {0, 0, 0, 0, 0};
        if (c < 3) dl[c] = 1.0;
        else if (c == 3) deb = 1.0;
        else if (c == 4) dTt = 1.0;
        else dth[c - 5] = 1.0;
        rm_principal_tangent(o, dl, deb, dTt, dth, col_tau[c], col_b[c], &col_eb[c], &col_T[c]);
    }
    double g[10];
    for (int c = 0; c < 10; c++) {
        g[c] = ebb * col_eb[c] + Tb * col_T[c];
        for (int A = 0; A < 3; A++) g[c] += Tq[A][A] * col_tau[c][A] + Bq[A][A] * col_b[c][A];
    }
    /* eigenbasis adjoint of b_tr: diagonal from the principal chain, off-diagonal from divided
     * differences (second-order symmetric limit for close eigenvalues) */
    double Xb[3][3] = {{0}};
    for (int A = 0; A < 3; A++) Xb[A][A] = g[A];
    double lmax = fmax(fabs(o->lam[0]), fmax(fabs(o->lam[1]), fabs(o->lam[2])));
    for (int A = 0; A < 3; A++)
        for (int B = 0; B < 3; B++) {
            if (A == B) continue;
            double th_t, th_b;
            double dl = o->lam[A] - o->lam[B];
            if (fabs(dl) > 1e-6 * lmax) {
                th_t = (o->tau[A] - o->tau[B]) / dl;
                th_b = (o->bA[A] - o->bA[B]) / dl;
            } else {
                th_t = 0.5 * ((col_tau[A][A] - col_tau[B][A]) + (col_tau[B][B] - col_tau[A][B]));
                th_b = 0.5 * ((col_b[A][A] - col_b[B][A]) + (col_b[B][B] - col_b[A][B]));
            }
            Xb[A][B] = th_t * Tq[A][B] + th_b * Bq[A][B];
        }
    double btrb[3][3];
    matmul3(o->Q, Xb, tmp); matmul3(tmp, QT, btrb);
    /* b_tr = dF b dF^T */
    double b[3][3], dFT[3][3], t2[3][3];
    sym_to_full(be_n, b);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFT[i][j] = dF[j][i];
    matmul3(btrb, dF, tmp); matmul3(tmp, b, t2);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFb[i][j] = 2.0 * t2[i][j];
    double bbf[3][3];
    matmul3(dFT, btrb, tmp); matmul3(tmp, dF, bbf);
    be_nb[0] = bbf[0][0]; be_nb[1] = bbf[1][1]; be_nb[2] = bbf[2][2];
    be_nb[3] = bbf[0][1] + bbf[1][0]; be_nb[4] = bbf[1][2] + bbf[2][1]; be_nb[5] = bbf[0][2] + bbf[2][0];
    *ebb_n = g[3];
    *Tb_n = g[4];
    for (int k = 0; k < 5; k++) thb[k] += g[5 + k];
}

/* stand-alone entry for tests: one MP */
int orc_return_map_backward(const orc_material *M, double dt, const double *dF9, const double *be_n, double ebar_n,
                            double T_n, double J, const double *sigb, const double *beb, double ebb, double Tb,
                            double *dFb9, double *be_nb, double *ebb_n, double *Tb_n, double *Jb, double *thb)
{
    double dF[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dF[i][j] = dF9[3 * i + j];
    rm_detail_t o;
    int st = rm_detail(M, dt, dF, be_n, ebar_n, T_n, J, &o);
    if (st != ORC_OK) return st;
    rm_out_t out;
    return_map(M, dt, dF, be_n, ebar_n, T_n, J, &out);
    double Fb[3][3];
    for (int k = 0; k < 5; k++) thb[k] = 0.0;
    rm_backward(&o, dF, be_n, out.sig, sigb, beb, ebb, Tb, Fb, be_nb, ebb_n, Tb_n, Jb, thb);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) dFb9[3 * i + j] = Fb[i][j];
    return ORC_OK;
}

/* ---------------------------------------------------------------- whole-step adjoint */
typedef struct {
    int64_t nn, nm, np;
    double *xb, *dub;               /* nodes: d L / d x, d L / d du of the current state */
    double *Fb, *beb, *ebb, *Tb, *vb, *sigb;   /* MPs */
    double *Nb, *Gb;                /* pairs of the current state's supports */
    double thb[5];                  /* d L / d (A, B, n, C, m) of material 0 */
} orc_adj;

static void adj_free(orc_adj *a)
{
    free(a->xb); free(a->dub); free(a->Fb); free(a->beb); free(a->ebb); free(a->Tb); free(a->vb); free(a->sigb);
    free(a->Nb); free(a->Gb);
}

static int adj_alloc(orc_adj *a, int64_t nn, int64_t nm, int64_t np)
{
    memset(a, 0, sizeof(*a));
    a->nn = nn; a->nm = nm; a->np = np;
    a->xb = calloc((size_t)(3 * nn + 1), 8); a->dub = calloc((size_t)(3 * nn + 1), 8);
    a->Fb = calloc((size_t)(9 * nm + 1), 8); a->beb = calloc((size_t)(6 * nm + 1), 8);
    a->ebb = calloc((size_t)(nm + 1), 8); a->Tb = calloc((size_t)(nm + 1), 8); a->vb = calloc((size_t)(nm + 1), 8);
    a->sigb = calloc((size_t)(6 * nm + 1), 8);
    a->Nb = calloc((size_t)(np + 1), 8); a->Gb = calloc((size_t)(3 * np + 1), 8);
    if (!a->xb || !a->dub || !a->Fb || !a->beb || !a->ebb || !a->Tb || !a->vb || !a->sigb || !a->Nb || !a->Gb) {
        adj_free(a);
        return ORC_ERR_OOM;
    }
    return ORC_OK;
}

orc_adj *orc_adj_create(const orc_sim *s, const double *xb_seed)
{
    orc_adj *a = calloc(1, sizeof(orc_adj));
    if (!a || adj_alloc(a, s->nn, s->nm, s->n_pairs) != ORC_OK) { free(a); return NULL; }
    memcpy(a->xb, xb_seed, (size_t)(3 * s->nn) * 8);
    return a;
}

void orc_adj_destroy(orc_adj *a)
{
    if (!a) return;
    adj_free(a);
    free(a);
}

void orc_adj_result(const orc_adj *a, double *thb, double *dub)
{
    memcpy(thb, a->thb, sizeof(a->thb));
    if (dub) memcpy(dub, a->dub, (size_t)(3 * a->nn) * 8);
}

/* One step backward: a holds adjoints of state s1 (= step(s0)); on return, adjoints of s0.
 * Requires: no erosion in the step (s0 and s1 have the same node and MP sets), J2 or JC. */
int orc_adjoint_step(const orc_sim *s0, const orc_sim *s1, orc_adj *a)
{
    const orc_params *P = &s1->P;
    if (s0->nn != s1->nn || s0->nm != s1->nm) return ORC_ERR_ARG;
    const int64_t nn = s0->nn, nm = s0->nm;
    const double dt = P->dt;
    orc_adj o;   /* adjoints of s0 being built */
    int st = adj_alloc(&o, nn, nm, s0->n_pairs);
    if (st != ORC_OK) return st;
    memcpy(o.thb, a->thb, sizeof(o.thb));
    double *xpb = calloc((size_t)(3 * nm + 1), 8);        /* adjoint of x_p,n+1 */
    double *xb1 = malloc((size_t)(3 * nn + 1) * 8);       /* adjoint of x_n+1 (total) */
    double *dub1 = malloc((size_t)(3 * nn + 1) * 8);      /* adjoint of du_n+1 */
    double *mb = calloc((size_t)(nn + 1), 8), *rb = calloc((size_t)(3 * nn + 1), 8);
    double *d = malloc((size_t)4096 * 3 * 8), *db = malloc((size_t)4096 * 3 * 8);
    if (!xpb || !xb1 || !dub1 || !mb || !rb || !d || !db) { st = ORC_ERR_OOM; goto done; }
    memcpy(xb1, a->xb, (size_t)(3 * nn) * 8);
    memcpy(dub1, a->dub, (size_t)(3 * nn) * 8);

    /* (6)^T LME at the end of the step: shape of s1 from x_p,n+1 and x_n+1 */
    for (int64_t p = 0; p < nm; p++) {
        int64_t b0 = s1->off[p], n = s1->off[p + 1] - b0;
        if (n > 4096) { st = ORC_ERR_CAPACITY; goto done; }
        for (int64_t k = 0; k < n; k++)
            for (int i = 0; i < 3; i++) d[3 * k + i] = s1->xp[3 * p + i] - s1->x[3 * (int64_t)s1->ids[b0 + k] + i];
        st = orc_lme_backward(n, d, s1->N + b0, s1->dN + 3 * b0, s1->lam + 3 * p, P->beta, a->Nb + b0,
                              a->Gb + 3 * b0, db);
        if (st != ORC_OK) goto done;
        for (int64_t k = 0; k < n; k++) {
            int64_t id = s1->ids[b0 + k];
            for (int i = 0; i < 3; i++) {
                xpb[3 * p + i] += db[3 * k + i];
                xb1[3 * id + i] -= db[3 * k + i];
            }
        }
    }
    /* (4)^T return map and (3)^T kinematics, per MP (shape of s0) */
    for (int64_t p = 0; p < nm; p++) {
        double D[3][3], Fo[3][3], Fn[3][3];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                D[i][j] = s1->dF[9 * p + 3 * i + j];
                Fo[i][j] = s0->F[9 * p + 3 * i + j];
                Fn[i][j] = s1->F[9 * p + 3 * i + j];
            }
        double Jn = det3(Fn), detD = det3(D);
        rm_detail_t det;
        st = rm_detail(&P->mat[s0->mat[p]], dt, D, s0->be + 6 * p, s0->ebar[p], s0->T[p], Jn, &det);
        if (st != ORC_OK) goto done;
        double Db[3][3], Jb, ebn, Tn;
        double thb_local[5] = {0, 0, 0, 0, 0};
        rm_backward(&det, D, s0->be + 6 * p, s1->sig + 6 * p, a->sigb + 6 * p, a->beb + 6 * p, a->ebb[p], a->Tb[p],
                    Db, o.beb + 6 * p, &ebn, &Tn, &Jb, thb_local);
        if (s0->mat[p] == 0)
            for (int k = 0; k < 5; k++) o.thb[k] += thb_local[k];
        o.ebb[p] = ebn;
        o.Tb[p] = Tn;
        /* F' = dF F: Fb' total = Fb + Jb J F'^-T */
        double Fni[3][3], Fbt[3][3], Di[3][3];
        if (!inv3(Fn, Fni) || !inv3(D, Di)) { st = ORC_ERR_JACOBIAN; goto done; }
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Fbt[i][j] = a->Fb[9 * p + 3 * i + j] + Jb * Jn * Fni[j][i];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double fo = 0.0, db_ = 0.0;
                for (int k = 0; k < 3; k++) {
                    fo += D[k][i] * Fbt[k][j];        /* dF^T Fb */
                    db_ += Fbt[i][k] * Fo[j][k];      /* Fb F^T */
                }
                o.Fb[9 * p + 3 * i + j] = fo;
                Db[i][j] += db_;
            }
        /* v' = det(dF) v */
        double vnew = s1->vol[p];
        o.vb[p] += detD * a->vb[p];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) Db[i][j] += a->vb[p] * vnew * Di[j][i];
        /* dF = 1 + sum du'_a (x) G_a ; x_p' = sum N_a x'_a  (s0 supports) */
        for (int64_t k = s0->off[p]; k < s0->off[p + 1]; k++) {
            int64_t id = s0->ids[k];
            const double *g = s0->dN + 3 * k;
            const double *u = s1->du + 3 * id;
            for (int i = 0; i < 3; i++) {
                dub1[3 * id + i] += Db[i][0] * g[0] + Db[i][1] * g[1] + Db[i][2] * g[2];
                o.Gb[3 * k + i] += Db[0][i] * u[0] + Db[1][i] * u[1] + Db[2][i] * u[2];
                xb1[3 * id + i] += s0->N[k] * xpb[3 * p + i];
            }
            o.Nb[k] += xpb[3 * p] * s1->x[3 * id] + xpb[3 * p + 1] * s1->x[3 * id + 1] + xpb[3 * p + 2] * s1->x[3 * id + 2];
        }
    }
    /* (2)^T nodes: x' = P(x + du_t), du' = x' - x, du_t = du + dt^2 r / m */
    for (int64_t i = 0; i < nn; i++) {
        double *xb0 = o.xb + 3 * i, *dub0 = o.dub + 3 * i;
        const double *xt1 = xb1 + 3 * i, *ut1 = dub1 + 3 * i;
        if (s0->flags[i] & 1) {   /* fixed: x' = x, du' = 0 */
            for (int c = 0; c < 3; c++) xb0[c] = xt1[c];
            continue;
        }
        double m = s1->mI[i];
        double dut[3], tot[3];
        for (int c = 0; c < 3; c++) {
            dut[c] = s0->du[3 * i + c] + ((m > 0.0) ? dt * dt * s1->rI[3 * i + c] / m : 0.0);
            tot[c] = xt1[c] + ut1[c];
        }
        if (P->wall) {   /* frozen contact set: projection along n removes the normal part */
            double g = 0.0, tn = 0.0;
            for (int c = 0; c < 3; c++) g += (s0->x[3 * i + c] + dut[c] - P->wall_p[c]) * P->wall_n[c];
            if (g < 0.0) {
                for (int c = 0; c < 3; c++) tn += tot[c] * P->wall_n[c];
                for (int c = 0; c < 3; c++) tot[c] -= tn * P->wall_n[c];
            }
        }
        for (int c = 0; c < 3; c++) {
            xb0[c] = tot[c] - ut1[c];
            dub0[c] = tot[c];
        }
        if (m > 0.0) {
            double rdot = 0.0;
            for (int c = 0; c < 3; c++) {
                rb[3 * i + c] = dt * dt / m * tot[c];
                rdot += s1->rI[3 * i + c] * tot[c];
            }
            mb[i] = -dt * dt * rdot / (m * m);
        }
    }
    /* (1)^T lumped mass and internal force (s0 supports, sigma_n, v_n) */
    for (int64_t p = 0; p < nm; p++) {
        const double *sg = s0->sig + 6 * p;
        double S[3][3];
        sym_to_full(sg, S);
        double vp = s0->vol[p], mp = s0->mass[p];
        double Sb[3][3] = {{0}};
        for (int64_t k = s0->off[p]; k < s0->off[p + 1]; k++) {
            int64_t id = s0->ids[k];
            const double *g = s0->dN + 3 * k, *r_ = rb + 3 * id;
            o.Nb[k] += mb[id] * mp;
            for (int i = 0; i < 3; i++) {
                double sg_i = S[i][0] * g[0] + S[i][1] * g[1] + S[i][2] * g[2];
                o.vb[p] -= r_[i] * sg_i;
                o.Gb[3 * k + i] -= vp * (S[0][i] * r_[0] + S[1][i] * r_[1] + S[2][i] * r_[2]);
                for (int j = 0; j < 3; j++) Sb[i][j] -= vp * r_[i] * g[j];
            }
        }
        double *sb = o.sigb + 6 * p;
        sb[0] = Sb[0][0]; sb[1] = Sb[1][1]; sb[2] = Sb[2][2];
        sb[3] = Sb[0][1] + Sb[1][0]; sb[4] = Sb[1][2] + Sb[2][1]; sb[5] = Sb[0][2] + Sb[2][0];
    }
    adj_free(a);
    *a = o;
    memset(&o, 0, sizeof(o));
    st = ORC_OK;
done:
    if (st != ORC_OK) adj_free(&o);
    free(xpb); free(xb1); free(dub1); free(mb); free(rb); free(d); free(db);
    return st;
}
