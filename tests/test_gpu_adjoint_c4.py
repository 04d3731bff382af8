"""The adjoint at its configured size and horizon: the Johnson-Cook Taylor rod at h 0.29 mm
(38,181 nodes, 202,752 MPs), 500 explicit steps from the impact, checkpoints every
ceil(sqrt(500)) = 23 steps, objectives final length and footprint radius, parameters
theta = (A, B, n, C, m, v0).

  - all twelve gradients of the GPU adjoint against central differences of the GPU forward
    (relative step 1e-6) in which every step replays the base trajectory's supports: the base
    run records each step's supports as a compact CSR in device memory (otm_supports_export,
    about 0.2 GB per step, 108 GB for the run) and the perturbed runs take them with
    otm_step_with_supports_csr, so that no support change enters the difference, as none
    enters the adjoint (1e-6 relative, plus the measured rounding noise of the difference);
  - the same gradients over the first 3 steps against the oracle's FP64 reference adjoint
    (orc_adjoint_step) on the same rod, and over 200 steps on a 4,992-MP rod (1e-10)."""
import math

import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA0 = np.array([90e6, 292e6, 0.31, 0.025, 1.09, 227.0])
H = 0.29e-3


def make(theta):
    A, B, n, C, m, v0 = theta
    return scenarios.taylor_rod(h=H, material=scenarios.copper_jc(A=A, B=B, n=n, C=C, m=m), v0=v0)


def adjoint_gradients(steps, every):
    from paper_2206_08772_gb300.adjoint import rod_objectives
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    vals = rod_objectives(th, make, steps, every)
    g = [torch.autograd.grad(vals[o], th, retain_graph=True)[0].numpy().copy() for o in range(2)]
    return [v.item() for v in vals], g


def test_adjoint_500_steps_against_replayed_finite_differences():
    """Central differences (relative step 1e-6) of the 500-step forward with the base run's
    supports replayed, against the GPU adjoint: |fd - g| <= 1e-6 |g| + 4 eta / h for each of the
    twelve gradients, eta the rounding noise of the objective after 500 steps, measured here as
    the largest change of the objective under relative perturbations of 1e-13 of each parameter
    (far too small to move the objective otherwise). The noise term is what a central difference
    can resolve: the final length changes by 1.5e-4 of itself when A doubles, so a 1e-6 step
    resolves dL/dA only to about 1e-4; the sensitive gradients are held to 1e-6 by the same rule."""
    from paper_2206_08772_gb300.adjoint import objectives_and_seeds
    from paper_2206_08772_gb300.otm import OTM
    torch.cuda.empty_cache()
    steps = 500
    every = int(math.ceil(math.sqrt(steps)))
    vals, g = adjoint_gradients(steps, every)
    torch.cuda.empty_cache()
    base = OTM(make(THETA0))
    rec = []
    for _ in range(steps):
        assert base.step(1) == 0, base.error()
        rec.append(base.supports_export())
    x = base.get("node_x")
    (L0, R0), _, (i_len, i_rad) = objectives_and_seeds(x, base.get("node_mass"), H)
    assert abs(L0 - vals[0]) <= 1e-13 * L0 and abs(R0 - vals[1]) <= 1e-13 * R0
    base.close()
    del base

    def replay(theta):
        s = OTM(make(theta))
        for j in range(steps):
            assert s.step_with_supports_csr(*rec[j]) == 0, s.error()
        xs = s.get("node_x")
        s.close()
        return np.array([xs[i_len, 2], math.hypot(xs[i_rad, 0], xs[i_rad, 1])])

    f0 = replay(THETA0)
    assert np.array_equal(f0, np.array([L0, R0]))          # the replay reproduces the base run
    eta = np.zeros(2)
    for k in range(6):
        t = THETA0.copy()
        t[k] *= 1.0 + 1e-13
        eta = np.maximum(eta, np.abs(replay(t) - f0))
    print("rounding noise of (L, R) after 500 steps:", eta)
    for k in range(6):
        hk = 1e-6 * THETA0[k]
        tp, tm = THETA0.copy(), THETA0.copy()
        tp[k] += hk
        tm[k] -= hk
        fd = (replay(tp) - replay(tm)) / (2 * hk)
        for o in range(2):
            err = abs(fd[o] - g[o][k])
            tol = 1e-6 * abs(g[o][k]) + 4 * eta[o] / hk
            print(f"theta {k} objective {o}: adjoint {g[o][k]:.10e} fd {fd[o]:.10e} rel {err / abs(g[o][k]):.2e} "
                  f"tol {tol / abs(g[o][k]):.2e}")
            assert err <= tol, (k, o, fd[o], g[o][k], tol)
    del rec
    torch.cuda.empty_cache()


def test_adjoint_over_200_steps_matches_the_cpu_reference_adjoint(orc):
    """A long horizon against the independent FP64 reference adjoint (same derivative, no
    finite-difference noise): a Johnson-Cook rod of 4,992 MPs (R 3.2, L 12.8 mm, h 0.8 mm), 200
    steps through the impact, checkpoints every 15 steps; values and all twelve gradients 1e-10."""
    def make_s(theta):
        A, B, n, C, m, v0 = theta
        return scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=12.8e-3,
                                    material=scenarios.copper_jc(A=A, B=B, n=n, C=C, m=m), v0=v0)
    from paper_2206_08772_gb300.adjoint import rod_objectives
    steps = 200
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    vals = rod_objectives(th, make_s, steps, 15)
    g = [torch.autograd.grad(vals[o], th, retain_graph=True)[0].numpy().copy() for o in range(2)]
    ref_vals, ref_grads, _ = orc.reference_adjoint(make_s(THETA0), steps)
    for o in range(2):
        assert abs(vals[o].item() - ref_vals[o]) <= 1e-10 * abs(ref_vals[o])
        scale = np.abs(ref_grads[o] * THETA0)
        print("200 steps, objective", o, "gpu", g[o], "cpu", ref_grads[o])
        assert np.all(np.abs(g[o] - ref_grads[o]) * THETA0 <= 1e-10 * scale.max() + 1e-8 * scale), (g[o], ref_grads[o])


def test_adjoint_first_steps_match_the_cpu_reference_adjoint(orc):
    steps = 3
    vals, g = adjoint_gradients(steps, 2)
    ref_vals, ref_grads, _ = orc.reference_adjoint(make(THETA0), steps)
    assert abs(vals[0] - ref_vals[0]) <= 1e-10 * abs(ref_vals[0])
    assert abs(vals[1] - ref_vals[1]) <= 1e-10 * abs(ref_vals[1])
    for o in range(2):
        scale = np.abs(ref_grads[o] * THETA0)
        assert np.all(np.abs(g[o] - ref_grads[o]) * THETA0 <= 1e-10 * scale.max() + 1e-8 * scale), (g[o], ref_grads[o])
