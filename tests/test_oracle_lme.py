"""Oracle pins for the LME shape functions (Eq. 14, Sec. 2.3).

Pins: (i) the constraints the paper imposes -- partition of unity by normalisation and
first-order consistency sum N_a (x_p - x_a) = 0 by the Newton solve; (ii) the gradient
identities that follow from them, sum grad N_a = 0 and sum (x_a - x_p) (x) grad N_a = -1;
(iii) closed forms: four affinely independent nodes give barycentric coordinates and constant
tetrahedron gradients for any beta; a point-symmetric stencil gives lambda = 0 and the
normalised Gaussian; (iv) central finite differences of N with respect to x_p; (v) the
returned lambda reproduces N through the paper's formula with the +lambda . (x_p - x_a) sign."""
import numpy as np
import pytest

import scenarios


def rod_point_supports(orc, n_pts=60, seed=0):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=8e-3, seed=seed)
    off, ids = orc.search(p.node_x, p.mp_x, p.rs2, p.cell_size)
    rng = np.random.default_rng(seed)
    pick = rng.choice(p.n_mps, n_pts, replace=False)
    pick[0] = 0            # corner of the rod: a surface point
    return p, off, ids, pick


def test_lme_invariants_on_rod(orc):
    p, off, ids, pick = rod_point_supports(orc)
    tol_r = p.newton_tol * p.h
    for q in pick:
        xa = p.node_x[ids[off[q]:off[q + 1]]]
        d = p.mp_x[q] - xa
        st, N, dN, lam, it = orc.lme(d, p.beta, tol_r)
        assert st == 0
        assert abs(N.sum() - 1.0) <= 1e-12
        assert np.linalg.norm(N @ xa - p.mp_x[q]) / p.h <= 1e-12
        assert np.abs(dN.sum(axis=0)).max() * p.h <= 1e-12
        M = (xa - p.mp_x[q]).T @ dN           # sum_a (x_a - x_p) grad N_a^T
        assert np.abs(M - np.eye(3)).max() <= 1e-12
        # lambda reproduces N through Eq. 14 as written (exp(-beta d^2 + lambda . d))
        f = -p.beta * (d * d).sum(axis=1) + d @ lam
        w = np.exp(f - f.max())
        assert np.abs(w / w.sum() - N).max() <= 1e-13
        assert np.all(N > 0)


def test_lme_four_nodes_barycentric(orc):
    rng = np.random.default_rng(3)
    for trial in range(20):
        X = rng.uniform(-1, 1, (4, 3)) * 1e-3
        while np.linalg.cond(np.vstack([X.T, np.ones(4)])) > 2e4:   # well-shaped tets only
            X = rng.uniform(-1, 1, (4, 3)) * 1e-3
        bary = rng.dirichlet(np.ones(4))
        xp = bary @ X
        beta = rng.choice([0.8, 2.0, 4.0]) / (1e-3) ** 2
        st, N, dN, lam, it = orc.lme(xp - X, beta, 1e-13 * 1e-3)
        assert st == 0
        assert np.abs(N - bary).max() <= 1e-12
        # gradients of barycentric coordinates: rows of inv([[x_b - x_0] ...]) arrangement
        Tm = np.vstack([X.T, np.ones(4)])          # 4x4: [x; 1] columns
        G = np.linalg.inv(Tm)[:, :3]                # d(bary_a)/dx
        assert np.abs(dN - G).max() <= 1e-10 * np.abs(G).max()


def test_lme_symmetric_stencil_gaussian(orc):
    h = 1e-3
    g = np.arange(-3, 4) * h
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    X = X[(X * X).sum(1) <= (3.2 * h) ** 2]
    xp = np.array([0.1, -0.2, 0.3])           # point-symmetric stencil around x_p
    beta = 0.8 / h ** 2
    d = -X                                     # x_p - x_a with x_a = x_p + X
    st, N, dN, lam, it = orc.lme(d, beta, 1e-12 * h, lam0=np.array([50.0, -20.0, 10.0]))
    assert st == 0
    assert np.abs(lam).max() * h <= 1e-10
    w = np.exp(-beta * (d * d).sum(1))
    assert np.abs(N - w / w.sum()).max() <= 1e-13


def test_lme_gradient_matches_finite_differences(orc):
    p, off, ids, pick = rod_point_supports(orc, n_pts=12, seed=1)
    tol_r = 1e-14 * p.h
    for q in pick:
        xa = p.node_x[ids[off[q]:off[q + 1]]]
        xp = p.mp_x[q].copy()
        st, N, dN, lam, _ = orc.lme(xp - xa, p.beta, tol_r)
        assert st == 0
        eps = 1e-6 * p.h
        fd = np.zeros_like(dN)
        for j in range(3):
            e = np.zeros(3)
            e[j] = eps
            _, Np, _, _, _ = orc.lme(xp + e - xa, p.beta, tol_r, lam0=lam)
            _, Nm, _, _, _ = orc.lme(xp - e - xa, p.beta, tol_r, lam0=lam)
            fd[:, j] = (Np - Nm) / (2 * eps)
        scale = np.abs(dN).max()
        assert np.abs(fd - dN).max() <= 1e-7 * scale


def test_lme_fails_outside_hull(orc):
    """A point outside the convex hull of its support has no solution: Newton must fail."""
    X = np.random.default_rng(0).uniform(0, 1e-3, (30, 3))
    xp = np.array([2e-3, 0.5e-3, 0.5e-3])
    st, *_ = orc.lme(xp - X, 0.8 / 1e-6, 1e-12 * 1e-3, max_it=50)
    assert st == orc.ERR_LME_NOCONV
