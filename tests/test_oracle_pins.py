"""Pins of three oracle parts against independent restatements (CPU only):

  - Eq. 7-8, the stabilised nodal residual: r_stab = r - eps sum_p N_Ip e_Ip with
    e_Ip = [x_I,n - x_p,n - dF_p,n (x_I,n-1 - x_p,n-1)] / |x_I,n-1 - x_p,n-1|, written out in
    numpy from the oracle's exported state after a non-affine increment (so e != 0) and with
    F_n != 1 (so dF and F differ); the term is linear in eps.
  - Sec. 4.2 tool contact as a penalty at its limit c = m/dt^2: normal force t_N = c * pen along
    the face's outward normal, tangential trial t_T = c * (relative tangential increment),
    Coulomb cap |t_T| <= mu |t_N| (stick below it, slip on it), position correction
    (t_N n - t_T) / c. Stick and slip on the rake face, a flank-face case, a node outside.
  - Sec. 4.2 adiabatic heating along the isochoric uniaxial path: with the rate term off, the
    consistency 3 mu (eps - ebar) = sigma_Y(ebar, T) and dT/d(ebar) = chi sigma_Y / (rho0 cp)
    integrated by scipy's solve_ivp; the oracle's incremental update (isothermal split, one
    return map per strain increment) converges to it at first order in the increment.
"""
import copy
import math

import numpy as np
import pytest

import scenarios


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


# ------------------------------------------------------------------ Eq. 7-8
STATE = ["node_x", "node_du", "node_x_prev", "mp_x", "mp_x_prev", "F", "dF", "be", "sigma", "vol", "ebar",
         "T", "lam"]


def sym(s):
    return np.array([[s[0], s[3], s[5]], [s[3], s[1], s[4]], [s[5], s[4], s[2]]])


@pytest.fixture(scope="module")
def stab_case(orc):
    """A short Johnson-Cook rod after one impact step, a random (non-affine) perturbation of the
    nodal increments, and a second step: the state every stabilised residual below starts from."""
    p0 = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=4.8e-3, material=scenarios.copper_jc())
    ref = orc.Sim(p0)
    assert ref.step(1) == 0
    rng = np.random.default_rng(11)
    du = ref.get("node_du")
    du += rng.normal(scale=2e-3 * p0.h, size=du.shape)
    ref.set("node_du", du)
    assert ref.step(1) == 0
    S = {f: ref.get(f) for f in STATE}
    return p0, S


def residual_after_one_step(orc, p0, S, eps):
    p = copy.copy(p0)
    p.eps_stab = eps
    sim = orc.Sim(p)
    for f in ("node_x", "node_du", "node_x_prev", "mp_x", "mp_x_prev", "F", "dF", "be", "sigma", "vol",
              "ebar", "T", "lam"):
        sim.set(f, S[f])
    assert sim.refresh() == 0
    sup = (sim.get("offsets"), sim.get("ids"), sim.get("N"), sim.get("dN"))
    assert sim.step(1) == 0
    return sim.get("node_force"), sup


def eq5_and_eq8(S, sup, n_nodes, h):
    """Eq. 5 residual (no body force) and the Eq. 7-8 sum  sum_p N_Ip e_Ip  per node."""
    off, ids, N, dN = sup
    r = np.zeros((n_nodes, 3))
    s8 = np.zeros((n_nodes, 3))
    for p in range(off.size - 1):
        sig = sym(S["sigma"][p])
        dF = S["dF"][p].reshape(3, 3)
        for k in range(off[p], off[p + 1]):
            a = ids[k]
            r[a] -= S["vol"][p] * sig @ dN[k]
            prev = S["node_x_prev"][a] - S["mp_x_prev"][p]
            dist = np.linalg.norm(prev)
            if dist <= 1e-12 * h:
                continue
            e = (S["node_x"][a] - S["mp_x"][p] - dF @ prev) / dist
            s8[a] += N[k] * e
    return r, s8


def test_stabilised_residual_restated_from_eq7_8(orc, stab_case):
    p0, S = stab_case
    assert np.abs(S["F"].reshape(-1, 3, 3) - S["dF"].reshape(-1, 3, 3)).max() > 1e-6   # F_n != dF_n
    r0, sup = residual_after_one_step(orc, p0, S, 0.0)
    r_np, s8 = eq5_and_eq8(S, sup, p0.n_nodes, p0.h)
    assert rel(r0, r_np) <= 1e-12
    assert np.abs(s8).max() > 1e-3          # the increment was not affine: e != 0
    eps = np.abs(r0).max() / np.abs(s8).max()   # a penalty of the size of the internal force
    r1, _ = residual_after_one_step(orc, p0, S, eps)
    assert rel(r1 - r0, -eps * s8) <= 1e-12
    # a flipped sign, the current separation as the normaliser, or F in place of dF all fail
    off, ids, N, dN = sup
    wrong = {"F_for_dF": np.zeros_like(s8), "current_norm": np.zeros_like(s8)}
    for p in range(off.size - 1):
        F = S["F"][p].reshape(3, 3)
        dF = S["dF"][p].reshape(3, 3)
        for k in range(off[p], off[p + 1]):
            a = ids[k]
            prev = S["node_x_prev"][a] - S["mp_x_prev"][p]
            cur = S["node_x"][a] - S["mp_x"][p]
            wrong["F_for_dF"][a] += N[k] * (cur - F @ prev) / np.linalg.norm(prev)
            wrong["current_norm"][a] += N[k] * (cur - dF @ prev) / np.linalg.norm(cur)
    assert rel(r1 - r0, eps * s8) > 1e-3
    for k, v in wrong.items():
        assert rel(r1 - r0, -eps * v) > 1e-9, k


def test_stabilisation_is_linear_in_eps(orc, stab_case):
    p0, S = stab_case
    r0, _ = residual_after_one_step(orc, p0, S, 0.0)
    r1, _ = residual_after_one_step(orc, p0, S, 1e5)
    r2, _ = residual_after_one_step(orc, p0, S, 2e5)
    assert np.abs(r1 - r0).max() > 1e-6 * np.abs(r0).max()
    assert rel(r2 - r1, r1 - r0) <= 1e-10


# ------------------------------------------------------------------ Sec. 4.2 tool contact
@pytest.fixture(scope="module")
def chip():
    return scenarios.chip_block(h=0.02e-3, size=(0.4e-3, 0.2e-3, 0.1e-3), depth=0.06e-3, steps=2)


def penalty_contact(x, du, xt, yt, gamma, v, dt, mu, m=1.0):
    """Rake angle 0: the tool occupies x >= xt (behind the vertical rake face) above the flank
    line y = yt + (x - xt) tan(gamma). A node inside gets the penalty forces at the limit
    c = m / dt^2 from the nearer face; returns its corrected position."""
    d_rake = x[0] - xt
    d_flank = ((x[1] - yt) - (x[0] - xt) * math.tan(gamma)) * math.cos(gamma)
    if not (d_rake > 0 and d_flank > 0):
        return x.copy()
    if d_rake <= d_flank:
        pen, n = d_rake, np.array([-1.0, 0.0, 0.0])
    else:
        pen, n = d_flank, np.array([math.sin(gamma), -math.cos(gamma), 0.0])
    c = m / dt ** 2
    tN = c * pen
    w = du - np.array([-v * dt, 0.0, 0.0])          # increment relative to the tool
    wt = w - (w @ n) * n
    tT = c * wt
    if np.linalg.norm(tT) > mu * tN:
        tT = mu * tN * tT / np.linalg.norm(tT)
    return x + (tN * n - tT) / c


@pytest.mark.parametrize("case", ["rake_stick", "rake_slip", "flank", "outside"])
def test_tool_contact_penalty_limit(orc, chip, case):
    c = chip.contact
    h, dt, v, mu = chip.h, chip.dt, c.tool_velocity, c.friction
    gamma = math.radians(c.tool_clearance_deg)
    assert c.tool_rake_deg == 0.0 and mu > 0
    t_next = 3 * dt
    xt, yt = c.tool_x0 - v * t_next, c.tool_tip_y
    z = 0.05e-3
    if case == "rake_stick":
        x = np.array([xt + 0.3 * h, yt + 2 * h, z])
        du = np.array([-v * dt + 0.1 * h, 0.05 * h, 0.02 * h])
    elif case == "rake_slip":
        x = np.array([xt + 0.3 * h, yt + 2 * h, z])
        du = np.array([-v * dt + 0.1 * h, 0.5 * h, 0.2 * h])
    elif case == "flank":
        x = np.array([xt + 3 * h, yt + 3 * h * math.tan(gamma) + 0.1 * h / math.cos(gamma), z])
        du = np.array([0.3 * h, -0.2 * h, 0.1 * h])
    else:
        x = np.array([xt - 0.2 * h, yt + h, z])
        du = np.array([0.1 * h, 0.1 * h, 0.0])
    want = penalty_contact(x, du, xt, yt, gamma, v, dt, mu)
    got = orc.tool_contact(chip, t_next, du, x)
    assert np.abs(got - want).max() <= 1e-12 * h
    if case == "outside":
        assert np.array_equal(got, x)
    else:
        assert np.abs(got - x).max() > 0.05 * h
    if case == "rake_stick":     # stick: no tangential motion relative to the tool remains
        assert abs((got[1] - x[1]) + du[1]) <= 1e-12 * h and abs((got[2] - x[2]) + du[2]) <= 1e-12 * h
    if case == "rake_slip":      # slip: the tangential increment relative to the tool shrinks by mu * pen
        left = np.linalg.norm((got - x + du)[1:])
        assert abs(left - (np.linalg.norm(du[1:]) - mu * 0.3 * h)) <= 1e-12 * h


# ------------------------------------------------------------------ Sec. 4.2 heating
def jc_no_rate(cp=100.0):
    m = scenarios.copper_jc(C=0.0)
    m.cp = cp
    return m


def oracle_uniaxial_path(orc, mat, eps_total, n):
    s = math.exp(eps_total / n)
    dF = np.diag([s, s ** -0.5, s ** -0.5])
    be = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])
    eb, T = 0.0, mat.T_room
    for _ in range(n):
        st, sig, be, eb, T, q, _ = orc.return_map(mat, 1e-6, dF, be, eb, T, 1.0)
        assert st == 0
    return eb, T


def integrated_path(mat, eps_total):
    """ebar and T at total log strain eps_total from the scalar ODE in ebar (rate term off)."""
    from scipy.integrate import solve_ivp
    from scipy.optimize import brentq
    mu = mat.E / (2 * (1 + mat.nu))

    def sig_y(eb, T):
        ts = min(max((T - mat.T_room) / (mat.T_melt - mat.T_room), 0.0), 1.0)
        return (mat.A + mat.B * eb ** mat.n) * (1.0 - ts ** mat.m)

    sol = solve_ivp(lambda eb, T: [mat.chi * sig_y(eb, T[0]) / (mat.rho0 * mat.cp)], (0.0, eps_total),
                    [mat.T_room], rtol=1e-12, atol=1e-10, dense_output=True, method="DOP853")
    g = lambda eb: 3 * mu * (eps_total - eb) - sig_y(eb, float(sol.sol(eb)[0]))
    eb = brentq(g, 1e-15, eps_total, xtol=1e-15, rtol=1e-15)
    return eb, float(sol.sol(eb)[0])


def test_jc_heating_converges_to_the_integrated_uniaxial_path(orc):
    pytest.importorskip("scipy")
    mat = jc_no_rate()
    eps_total = 1.0
    eb_ref, T_ref = integrated_path(mat, eps_total)
    assert T_ref - mat.T_room > 200.0                       # strong heating: softening matters
    errs = []
    for n in (2000, 4000):
        eb, T = oracle_uniaxial_path(orc, mat, eps_total, n)
        errs.append((abs(eb - eb_ref) / eb_ref, abs(T - T_ref) / (T_ref - mat.T_room)))
    for k in range(2):
        assert errs[1][k] <= 2e-3
        ratio = errs[1][k] / errs[0][k]
        assert 0.4 <= ratio <= 0.6, (k, errs)               # first order in the increment
