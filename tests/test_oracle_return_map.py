"""Oracle pins for the constitutive update (Sec. 4.1 J2 finite plasticity, Sec. 4.2 Johnson-Cook).

Pins: the isochoric uniaxial path F = diag(s, s^-1/2, s^-1/2) has a closed form for the
exponential-map radial return with linear hardening (q = sigma_y0 + H ebar, ebar =
max(0, (3 mu |ln s| - sigma_y0)/(3 mu + H)), zero pressure), and it is path independent for
monotonic loading; hyperelastic Hencky response and rotation covariance below yield; the JC
consistency equation solved independently by a bracketing library root finder; the heating
law checked in the paper's form (Cauchy von Mises stress, current density); the fracture
strain evaluated from the returned Cauchy stress."""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import scenarios

I6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def full(s6):
    return np.array([[s6[0], s6[3], s6[5]], [s6[3], s6[1], s6[4]], [s6[5], s6[4], s6[2]]])


def rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


@pytest.mark.parametrize("s", [1.02, 0.97, 1.3, 0.6, 1.0005])
def test_j2_uniaxial_isochoric_closed_form(orc, s):
    m = scenarios.copper_j2()
    mu, K = m.mu, m.K
    F = np.diag([s, s ** -0.5, s ** -0.5])
    st, sig, be, eb, T, q, failed = orc.return_map(m, 1e-8, F, I6, 0.0, 298.0, 1.0)
    assert st == 0
    ls = math.log(s)
    ep = max(0.0, (3 * mu * abs(ls) - m.sigma_y0) / (3 * mu + m.H))
    q_ref = 3 * mu * abs(ls) if ep == 0 else m.sigma_y0 + m.H * ep
    assert abs(eb - ep) <= 1e-12 * max(1.0, ep) + 1e-15
    assert abs(q - q_ref) <= 1e-12 * q_ref
    sg = math.copysign(1.0, ls)
    S = full(sig)
    ref = np.diag([sg * 2 * q_ref / 3, -sg * q_ref / 3, -sg * q_ref / 3])
    assert np.abs(S - ref).max() <= 1e-12 * q_ref
    # elastic left Cauchy-Green: exp(2 (e_tr - dgamma n)), n = sg (2,-1,-1)/sqrt(6)
    ee = np.array([ls - sg * ep, -0.5 * ls + sg * ep / 2, -0.5 * ls + sg * ep / 2])
    assert np.abs(full(be) - np.diag(np.exp(2 * ee))).max() <= 1e-12


def test_j2_uniaxial_path_independent(orc):
    m = scenarios.copper_j2()
    s_final, k = 1.25, 40
    ds = s_final ** (1.0 / k)
    dF = np.diag([ds, ds ** -0.5, ds ** -0.5])
    be, eb, T = I6.copy(), 0.0, 298.0
    F = np.eye(3)
    for _ in range(k):
        F = dF @ F
        st, sig, be, eb, T, q, _ = orc.return_map(m, 1e-8, dF, be, eb, T, np.linalg.det(F))
        assert st == 0
    st, sig1, be1, eb1, *_ = orc.return_map(m, 1e-8, np.diag([s_final, s_final ** -0.5, s_final ** -0.5]),
                                            I6, 0.0, 298.0, 1.0)
    assert abs(eb - eb1) <= 1e-12
    assert np.abs(sig - sig1).max() <= 1e-9 * np.abs(sig1).max()
    assert np.abs(be - be1).max() <= 1e-11


def test_hencky_elastic_and_rotation_covariance(orc):
    m = scenarios.copper_j2()
    m.sigma_y0 = 1e30            # elastic
    lam = np.array([1.003, 0.998, 1.001])
    for ax, ang in [((1, 2, 3), 0.7), ((0, 0, 1), 1.1), ((1, -1, 0.5), 2.9)]:
        R = rot(ax, ang)
        F = R @ np.diag(lam) @ R.T
        J = np.prod(lam)
        st, sig, be, eb, T, q, _ = orc.return_map(m, 1e-8, F, I6, 0.0, 298.0, J)
        assert st == 0 and eb == 0.0
        e = np.log(lam)
        tau = m.K * e.sum() + 2 * m.mu * (e - e.sum() / 3)
        ref = R @ np.diag(tau / J) @ R.T
        assert np.abs(full(sig) - ref).max() <= 1e-11 * np.abs(ref).max()
        assert np.abs(full(be) - R @ np.diag(lam ** 2) @ R.T).max() <= 1e-13


def test_rotation_of_plastic_state(orc):
    """Objectivity: rotating the deformation rotates the stress, also past yield."""
    m = scenarios.copper_j2()
    F0 = np.array([[1.05, 0.02, 0.0], [0.01, 0.97, 0.03], [0.0, -0.02, 0.99]])
    R = rot((0.3, 1.0, -0.2), 0.9)
    st, s0, b0, e0, *_ = orc.return_map(m, 1e-8, F0, I6, 0.0, 298.0, np.linalg.det(F0))
    st1, s1, b1, e1, *_ = orc.return_map(m, 1e-8, R @ F0, I6, 0.0, 298.0, np.linalg.det(F0))
    assert st == 0 and st1 == 0 and e0 > 0
    assert abs(e0 - e1) <= 1e-13
    assert np.abs(full(s1) - R @ full(s0) @ R.T).max() <= 1e-10 * np.abs(s0).max()


@pytest.mark.parametrize("C,Tn", [(0.0, 298.0), (0.025, 298.0), (0.025, 700.0)])
def test_jc_consistency_vs_bracketing_root(orc, C, Tn):
    m = scenarios.copper_jc(C=C)
    m.chi = 0.0
    mu = m.mu
    dt = 1e-8
    s = 1.05
    F = np.diag([s, s ** -0.5, s ** -0.5])
    st, sig, be, eb, T, q, _ = orc.return_map(m, dt, F, I6, 0.0, Tn, 1.0)
    assert st == 0
    q_tr = 3 * mu * math.log(s)
    tstar = min(max((Tn - m.T_room) / (m.T_melt - m.T_room), 0), 1)

    def g(x):
        rate = x / dt / m.eps_dot0
        return q_tr - 3 * mu * x - (m.A + m.B * x ** m.n) * (1 + C * math.log(max(rate, 1.0))) * (1 - tstar ** m.m)

    x = brentq(g, 0.0, q_tr / (3 * mu), xtol=1e-300, rtol=4 * np.finfo(float).eps, maxiter=500)
    assert abs(eb - x) <= 1e-10 * x
    assert abs(q - (q_tr - 3 * mu * x)) <= 1e-10 * q


def test_jc_heating_in_paper_form(orc):
    """dT = chi sigma_v d(ebar) / (rho C_p) with the Cauchy von Mises stress and rho = rho0/J."""
    m = scenarios.copper_jc()
    a, s = 0.98, 1.04          # volumetric compression plus isochoric stretch
    F = np.diag([s * a, a / math.sqrt(s), a / math.sqrt(s)])
    J = np.linalg.det(F)
    st, sig, be, eb, T, q, _ = orc.return_map(m, 1e-8, F, I6, 0.0, 400.0, J)
    assert st == 0 and eb > 0
    S = full(sig)
    dev = S - np.trace(S) / 3 * np.eye(3)
    sv = math.sqrt(1.5 * (dev * dev).sum())
    rho = m.rho0 / J
    assert abs((T - 400.0) - m.chi * sv * eb / (rho * m.cp)) <= 1e-12 * (T - 400.0)
    assert abs(np.trace(S) / 3 - m.K * 3 * math.log(a) / J) <= 1e-10 * abs(np.trace(S))


def test_jc_fracture_strain_from_cauchy_stress(orc):
    m = scenarios.ti64_jc()
    dt = 1e-9
    for a in (1.004, 0.998):   # tension and compression triaxiality
        lo, hi = 1.0, 3.0
        for _ in range(60):     # bisect the stretch at which the fracture flag flips
            s = 0.5 * (lo + hi)
            F = np.diag([s * a, a / math.sqrt(s), a / math.sqrt(s)])
            st, sig, be, eb, T, q, failed = orc.return_map(m, dt, F, I6, 0.0, 298.15, np.linalg.det(F))
            assert st == 0
            if failed:
                hi = s
            else:
                lo = s
        F = np.diag([hi * a, a / math.sqrt(hi), a / math.sqrt(hi)])
        st, sig, be, eb, T, q, failed = orc.return_map(m, dt, F, I6, 0.0, 298.15, np.linalg.det(F))
        S = full(sig)
        p = np.trace(S) / 3
        dev = S - p * np.eye(3)
        sv = math.sqrt(1.5 * (dev * dev).sum())
        eta = p / sv
        d1, d2, d3, d4, d5 = m.d
        rate = eb / dt / m.eps_dot0
        tstar = (T - m.T_room) / (m.T_melt - m.T_room)
        ef = (d1 + d2 * math.exp(d3 * eta)) * (1 + d4 * math.log(max(rate, 1))) * (1 + d5 * tstar)
        assert failed and abs(eb - ef) <= 1e-9 * ef
        assert (eta > 0) == (a > 1)


def test_jc_fracture_of_melted_point_follows_pressure_sign(orc):
    """Above the melting temperature the flow stress vanishes, so no deviatoric stress is left and
    the triaxiality p / sigma_v is taken at its limit sign(p) * inf: hydrostatic tension fails
    (eps_f -> d1 (...) < 0), hydrostatic compression does not (eps_f -> +inf)."""
    m = scenarios.ti64_jc()
    for a, want in ((1.002, True), (0.998, False)):
        s = 1.05
        F = np.diag([s * a, a / math.sqrt(s), a / math.sqrt(s)])
        st, sig, be, eb, T, q, failed = orc.return_map(m, 1e-9, F, I6, 0.0, m.T_melt + 50.0, np.linalg.det(F))
        assert st == 0 and eb > 0
        assert abs(q) <= 1e-6 * m.E
        assert failed == want
