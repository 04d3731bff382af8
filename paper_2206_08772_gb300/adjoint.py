"""Gradients of Taylor-rod objectives through the GPU adjoint, as a torch.autograd.Function.

theta = (A, B, n, C, m, v0): the Johnson-Cook flow-stress constants of the rod and its impact
velocity. The objectives are the final rod length (largest z over nodes with mass) and the
footprint radius (largest radial distance over nodes within 1e-3 h of the wall), with their
arg-max nodes, supports, wall-contact set and plastic set frozen at the forward trajectory.

The backward pass uses step checkpointing: the forward keeps a snapshot every `every` steps
(default ceil(sqrt(steps))); the backward recomputes one segment at a time from its snapshot,
keeping that segment's per-step snapshots, and runs the library's backward step (which itself
recomputes the step, then applies the transposed kernels) from the last step to the first.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .otm import OTM

THETA_NAMES = ("A", "B", "n", "C", "m", "v0")


def objectives_and_seeds(x: np.ndarray, node_mass: np.ndarray, h: float):
    act = np.nonzero(node_mass > 0)[0]
    i_len = int(act[np.argmax(x[act, 2])])
    foot = np.nonzero(x[:, 2] <= 1e-3 * h)[0]
    i_rad = int(foot[np.argmax(np.hypot(x[foot, 0], x[foot, 1]))])
    L = float(x[i_len, 2])
    R = float(math.hypot(x[i_rad, 0], x[i_rad, 1]))
    gL = np.zeros_like(x)
    gL[i_len, 2] = 1.0
    gR = np.zeros_like(x)
    gR[i_rad, 0], gR[i_rad, 1] = x[i_rad, 0] / R, x[i_rad, 1] / R
    return (L, R), (gL, gR), (i_len, i_rad)


class RodObjectives(torch.autograd.Function):
    """(L, R) = f(theta); backward by the hand-written adjoint on the GPU."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, make_problem, steps: int, every: int | None):
        th = theta.detach().cpu().double().numpy()
        prob = make_problem(th)
        sim = OTM(prob, precision="fp64")
        every = every or max(1, int(math.ceil(math.sqrt(steps))))
        checkpoints = {0: sim.snapshot()}
        for k in range(steps):
            st = sim.step(1)
            if st != 0:
                raise RuntimeError(f"forward step {k} failed: {st} {sim.error()}")
            if (k + 1) % every == 0 and k + 1 < steps:
                checkpoints[k + 1] = sim.snapshot()
        x = sim.get("node_x")
        vals, seeds, argm = objectives_and_seeds(x, sim.get("node_mass"), prob.h)
        ctx.sim, ctx.prob, ctx.steps, ctx.every = sim, prob, steps, every
        ctx.checkpoints, ctx.seeds, ctx.final = checkpoints, seeds, sim.snapshot()
        return torch.tensor(vals, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        g = gout.detach().cpu().double().numpy()
        grad = backward_pass(ctx.sim, ctx.prob, ctx.steps, ctx.every, ctx.checkpoints, ctx.final,
                             g[0] * ctx.seeds[0] + g[1] * ctx.seeds[1])
        return torch.from_numpy(grad), None, None, None


def backward_pass(sim: OTM, prob, steps: int, every: int, checkpoints: dict, final, xbar: np.ndarray,
                  recompute: bool = False) -> np.ndarray:
    """d objective / d theta for the seed xbar = d objective / d final node positions. Each
    backward step gets state n+1 from the recomputed segment's snapshots, or (recompute=True)
    recomputes step n itself."""
    sim.restore(final)
    sim.adjoint_begin(xbar)
    seg_starts = sorted(checkpoints)
    for s0 in reversed(seg_starts):
        s1 = min(s0 + every, steps)
        # recompute the segment, keeping the state before each of its steps
        sim.restore(checkpoints[s0])
        states = [sim.snapshot()]
        for _ in range(s0, s1 - 1):
            if sim.step(1) != 0:
                raise RuntimeError("recompute failed")
            states.append(sim.snapshot())
        end = checkpoints[s1] if s1 in checkpoints else final    # state s1
        for k in range(s1 - 1, s0 - 1, -1):
            sim.restore(states[k - s0])
            if recompute:
                sim.adjoint_step()
            else:
                sim.adjoint_step(states[k + 1 - s0] if k + 1 - s0 < len(states) else end)
        del states
    # du_0 = (0, 0, -v0 dt) on every node: d(du_0)/d(v0) = (0, 0, -dt)
    du0_dv0 = np.zeros((prob.n_nodes, 3))
    du0_dv0[:, 2] = -prob.dt
    thb, _ = sim.adjoint_result(du0_dv0)
    return thb


def rod_objectives(theta: torch.Tensor, make_problem, steps: int, every: int | None = None) -> torch.Tensor:
    """(final length, footprint radius) with gradients through the GPU adjoint."""
    return RodObjectives.apply(theta, make_problem, steps, every)
