"""Oracle pins for the reference adjoint: every backward piece against central finite
differences of the forward oracle (the forward itself pinned elsewhere)."""
import math

import numpy as np
import pytest

import scenarios

I6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def test_lme_backward_matches_finite_differences(orc):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=4.0e-3)
    off, ids = orc.search(p.node_x, p.mp_x, p.rs2, p.cell_size)
    rng = np.random.default_rng(4)
    tol = 1e-15 * p.h
    for q in (0, 77, 400):
        xa = p.node_x[ids[off[q]:off[q + 1]]]
        d0 = p.mp_x[q] - xa
        st, N, G, lam, _ = orc.lme(d0, p.beta, tol)
        assert st == 0
        Nb = rng.normal(size=N.shape)
        Gb = rng.normal(size=G.shape) * p.h
        db = orc.lme_backward(d0, N, G, lam, p.beta, Nb, Gb)

        def L(d):
            s_, N_, G_, _, _ = orc.lme(d, p.beta, tol, lam0=lam)
            assert s_ == 0
            return (Nb * N_).sum() + (Gb * G_).sum()

        eps = 1e-6 * p.h
        for a in rng.choice(N.size, 6, replace=False):
            for i in range(3):
                dp, dm = d0.copy(), d0.copy()
                dp[a, i] += eps
                dm[a, i] -= eps
                fd = (L(dp) - L(dm)) / (2 * eps)
                assert abs(fd - db[a, i]) <= 1e-6 * np.abs(db).max(), (q, a, i, fd, db[a, i])


@pytest.mark.parametrize("model,stretch", [("jc", 1.03), ("jc", 1.0002), ("j2", 1.02), ("jc_virgin", 1.0001), ("j2_elastic", 1.0001),
                                          ("j2_degenerate", 1.0)])
def test_return_map_backward_matches_finite_differences(orc, model, stretch):
    mat = scenarios.copper_j2() if model.startswith("j2") else scenarios.copper_jc()
    rng = np.random.default_rng(9)
    dt = 5e-9
    s = stretch
    dF = np.diag([s, s ** -0.45, s ** -0.5]) + rng.normal(0, 2e-3 * (s - 1) / 0.03 + 1e-4, (3, 3))
    be = I6 + np.concatenate([rng.normal(0, 1e-3, 3), rng.normal(0, 5e-4, 3)])
    eb, T, J = 0.05, 420.0, 0.998
    if model == "jc_virgin":
        eb = 0.0
    if model in ("j2_elastic", "j2_degenerate"):
        be = I6.copy()
    if model == "j2_degenerate":   # (nearly) repeated eigenvalues: divided-difference limit
        dF = np.eye(3) + rng.normal(0, 1e-9, (3, 3))
    th0 = np.array([mat.A, mat.B, mat.n, mat.C, mat.m])
    sigb = rng.normal(size=6) / 1e9
    beb = rng.normal(size=6)
    ebb, Tb = rng.normal(), rng.normal() / 100

    def fwd(dF_, be_, eb_, T_, J_, th):
        m = scenarios.copper_j2() if model.startswith("j2") else scenarios.copper_jc(*th)
        st, sig, be1, eb1, T1, q, _ = orc.return_map(m, dt, dF_, be_, eb_, T_, J_)
        assert st == 0
        return (sigb * sig).sum() + (beb * be1).sum() + ebb * eb1 + Tb * T1

    dFb, beb_n, ebb_n, Tb_n, Jb, thb = orc.return_map_backward(mat, dt, dF, be, eb, T, J, sigb, beb, ebb, Tb)
    base = fwd(dF, be, eb, T, J, th0)
    checks = []
    for i in range(3):
        for j in range(3):
            h = 1e-7
            a, b_ = dF.copy(), dF.copy()
            a[i, j] += h
            b_[i, j] -= h
            checks.append(((fwd(a, be, eb, T, J, th0) - fwd(b_, be, eb, T, J, th0)) / (2 * h), dFb[i, j]))
    for k in range(6):
        h = 1e-7
        a, b_ = be.copy(), be.copy()
        a[k] += h
        b_[k] -= h
        checks.append(((fwd(dF, a, eb, T, J, th0) - fwd(dF, b_, eb, T, J, th0)) / (2 * h), beb_n[k]))
    if eb > 0:
        checks.append(((fwd(dF, be, eb + 1e-7, T, J, th0) - fwd(dF, be, eb - 1e-7, T, J, th0)) / 2e-7, ebb_n))
    else:   # ebar >= 0 is a constraint: one-sided difference at the virgin state
        h = 1e-10
        fd1 = (fwd(dF, be, h, T, J, th0) - base) / h
        assert abs(fd1 - ebb_n) <= 1e-4 * abs(ebb_n)
    checks.append(((fwd(dF, be, eb, T + 1e-4, J, th0) - fwd(dF, be, eb, T - 1e-4, J, th0)) / 2e-4, Tb_n))
    checks.append(((fwd(dF, be, eb, T, J + 1e-7, th0) - fwd(dF, be, eb, T, J - 1e-7, th0)) / 2e-7, Jb))
    if not model.startswith("j2"):
        for k in range(5):
            h = 1e-6 * th0[k]
            a, b_ = th0.copy(), th0.copy()
            a[k] += h
            b_[k] -= h
            checks.append(((fwd(dF, be, eb, T, J, a) - fwd(dF, be, eb, T, J, b_)) / (2 * h), thb[k]))
    scale = max(abs(c[1]) for c in checks)
    for fd, an in checks:
        assert abs(fd - an) <= 2e-6 * scale + 1e-7 * abs(an), (fd, an, scale)
    assert abs(base) > 0


def _jc_rod(theta=None, h=0.8e-3, L=4.0e-3):
    A, B, n, C, m, v0 = theta if theta is not None else (90e6, 292e6, 0.31, 0.025, 1.09, 227.0)
    mat = scenarios.copper_jc(A=A, B=B, n=n, C=C, m=m)
    p = scenarios.taylor_rod(h=h, R=3.2e-3, L=L, material=mat, v0=v0)
    return p


def _run(orc, theta, steps):
    p = _jc_rod(theta)
    s = orc.Sim(p)
    trace = []
    for _ in range(steps):
        assert s.step(1) == 0
        trace.append((s.get("offsets").copy(), s.get("ids").copy(), s.get("ebar") > 0,
                      s.get("node_x")[:, 2] <= 0.0))
    return s, p, trace


def test_reference_adjoint_matches_central_differences(orc):
    """End-to-end: reverse-mode gradients of final length and footprint radius with respect to
    (A, B, n, C, m, v0) against central differences (step 1e-6 relative) of the forward oracle;
    the perturbed runs must keep the base topology, plastic set and contact set."""
    theta0 = np.array([90e6, 292e6, 0.31, 0.025, 1.09, 227.0])
    steps = 6
    p = _jc_rod(theta0)
    vals, grads, argm = orc.reference_adjoint(p, steps)
    base, _, tr0 = _run(orc, theta0, steps)
    assert grads[0, 5] != 0 and grads[1, 5] != 0
    for k in range(6):
        hk = 1e-6 * abs(theta0[k])
        fv = []
        for sgn in (1, -1):
            th = theta0.copy()
            th[k] += sgn * hk
            s, pp, tr = _run(orc, th, steps)
            for (o0, i0, pl0, c0), (o1, i1, pl1, c1) in zip(tr0, tr):
                assert np.array_equal(o0, o1) and np.array_equal(i0, i1), "topology changed under perturbation"
                assert np.array_equal(pl0, pl1) and np.array_equal(c0, c1), "plastic / contact set changed"
            x = s.get("node_x")
            i_len, i_rad = argm
            fv.append((x[i_len, 2], np.hypot(x[i_rad, 0], x[i_rad, 1])))
        fd = [(fv[0][o] - fv[1][o]) / (2 * hk) for o in range(2)]
        for o in range(2):
            # central differences carry a rounding error of about eps |f| / h
            fd_noise = 20 * np.finfo(float).eps * abs(vals[o]) / hk
            assert abs(fd[o] - grads[o, k]) <= 1e-6 * abs(grads[o, k]) + fd_noise, (k, o, fd[o], grads[o, k])
