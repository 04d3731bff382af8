"""GPU adjoint (reverse mode through the C ABI, with step checkpointing) against the FP64 CPU
reference adjoint (1e-10 relative) and against central finite differences of the GPU forward
(1e-6 relative, topology frozen by construction of the small perturbation)."""
import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THETA0 = np.array([90e6, 292e6, 0.31, 0.025, 1.09, 227.0])


def make_rod(theta, L=4.0e-3):
    A, B, n, C, m, v0 = theta
    mat = scenarios.copper_jc(A=A, B=B, n=n, C=C, m=m)
    return scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=L, material=mat, v0=v0)


@pytest.mark.parametrize("steps,every", [(6, 2), (16, 4)])
def test_gpu_adjoint_matches_cpu_reference(orc, steps, every):
    from paper_2206_08772_gb300.adjoint import rod_objectives
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    vals = rod_objectives(th, make_rod, steps, every)
    ref_vals, ref_grads, _ = orc.reference_adjoint(make_rod(THETA0), steps)
    assert abs(vals[0].item() - ref_vals[0]) <= 1e-10 * abs(ref_vals[0])
    assert abs(vals[1].item() - ref_vals[1]) <= 1e-10 * abs(ref_vals[1])
    for o in range(2):
        g, = torch.autograd.grad(vals[o], th, retain_graph=True)
        g = g.numpy()
        print("adjoint", steps, o, g, ref_grads[o])
        scale = np.abs(ref_grads[o] * THETA0)
        assert np.all(np.abs(g - ref_grads[o]) * THETA0 <= 1e-10 * scale.max() + 1e-8 * scale), (g, ref_grads[o])


def test_gpu_adjoint_matches_finite_differences():
    from paper_2206_08772_gb300.adjoint import rod_objectives
    from paper_2206_08772_gb300.otm import OTM
    steps = 8
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    L, R = rod_objectives(th, make_rod, steps)
    (gL,) = torch.autograd.grad(L, th)
    base = OTM(make_rod(THETA0))
    assert base.step(steps) == 0
    x0 = base.get("node_x")
    i_len = int(np.argmin(np.abs(x0[:, 2] - L.item())))
    for k in (0, 2, 3, 5):
        h = 1e-6 * THETA0[k]
        f = []
        for sg in (1, -1):
            t = THETA0.copy()
            t[k] += sg * h
            s = OTM(make_rod(t))
            assert s.step(steps) == 0
            f.append(s.get("node_x")[i_len, 2])
        fd = (f[0] - f[1]) / (2 * h)
        noise = 20 * np.finfo(float).eps * abs(L.item()) / h
        assert abs(fd - gL[k].item()) <= 1e-6 * abs(gL[k].item()) + noise, (k, fd, gL[k].item())


def test_gpu_adjoint_against_finite_differences_with_replayed_supports():
    """Central differences of the GPU forward with the base trajectory's supports replayed at
    every step (otm_step_with_supports), so that no support change can enter the difference:
    all six parameters, both objectives, against the GPU adjoint (1e-6 relative)."""
    from paper_2206_08772_gb300.adjoint import objectives_and_seeds, rod_objectives
    from paper_2206_08772_gb300.otm import OTM
    steps = 10
    th = torch.tensor(THETA0, dtype=torch.float64, requires_grad=True)
    vals = rod_objectives(th, make_rod, steps)
    grads = [torch.autograd.grad(vals[o], th, retain_graph=True)[0].numpy() for o in range(2)]
    base = OTM(make_rod(THETA0))
    rec = []
    for _ in range(steps):
        assert base.step(1) == 0
        rec.append((base.get("support_count"), base.get("support_ids")))
    _, _, (i_len, i_rad) = objectives_and_seeds(base.get("node_x"), base.get("node_mass"), 0.8e-3)
    for k in range(6):
        hk = 1e-6 * THETA0[k]
        f = []
        for sg in (1, -1):
            t = THETA0.copy()
            t[k] += sg * hk
            s = OTM(make_rod(t))
            for j in range(steps):
                assert s.step_with_supports(*rec[j]) == 0
            x = s.get("node_x")
            f.append((x[i_len, 2], np.hypot(x[i_rad, 0], x[i_rad, 1])))
        for o in range(2):
            fd = (f[0][o] - f[1][o]) / (2 * hk)
            noise = 20 * np.finfo(float).eps * abs(vals[o].item()) / hk
            assert abs(fd - grads[o][k]) <= 1e-6 * abs(grads[o][k]) + noise, (k, o, fd, grads[o][k])


def test_backward_from_snapshots_equals_backward_by_recompute():
    """The backward steps that load state n+1 from the segment's snapshots (with the shape
    functions of state n+1 kept from the previous backward step) give the same gradient as
    backward steps that recompute step n."""
    import math
    from paper_2206_08772_gb300.adjoint import backward_pass, objectives_and_seeds
    from paper_2206_08772_gb300.otm import OTM
    steps, every = 9, 3
    p = make_rod(THETA0)
    out = []
    for recompute in (False, True):
        sim = OTM(p)
        checkpoints = {0: sim.snapshot()}
        for k in range(steps):
            assert sim.step(1) == 0
            if (k + 1) % every == 0 and k + 1 < steps:
                checkpoints[k + 1] = sim.snapshot()
        final = sim.snapshot()
        _, seeds, _ = objectives_and_seeds(sim.get("node_x"), sim.get("node_mass"), p.h)
        out.append(backward_pass(sim, p, steps, every, checkpoints, final, seeds[0] + seeds[1],
                                 recompute=recompute))
    scale = np.abs(out[1] * THETA0)
    assert np.all(np.abs(out[0] - out[1]) * THETA0 <= 1e-13 * scale.max() + 1e-12 * scale), out
    assert math.isfinite(out[0][5]) and out[0][5] != 0.0
