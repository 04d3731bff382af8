"""One-step shadow parity on the benchmark workload at full size, in the middle of its run.

The Johnson-Cook Taylor rod at h 0.12 mm (501,189 nodes, 2,854,368 MPs; FP64, 384 support
slots, the benchmark's launch configuration) runs on the GPU; at steps 10, 100 and 500 (the
benchmark times the steps after 500) its state is handed to the oracle for two slabs of the rod:
the impact zone at the wall and a block at mid-length, each with every node and the slab's MPs.
The oracle (OpenMP build, the serial arithmetic) rebuilds the supports and shape functions at
that state (Algorithm 3, Eq. 14), then the GPU and the oracle each take one step (Algorithm 1).
Compared, on the slab's interior (MPs whose supports only hold nodes whose influence domains lie
inside the slab, so that the oracle's truncated slab does not enter):
  - at step n: support lists of sampled MPs bit-exact, their N and grad N to 1e-10;
  - at step n + 1: nodal position, increment, mass and force, and every MP field (x_p, F,
    sigma, b^e, v, ebar, T, lambda) to 1e-10 (max |gpu - oracle| over the interior relative to
    the field's largest value over the rod); support
    lists of sampled MPs bit-exact and their shape functions to 1e-10.
The linked-cell grid of all nodes at step n (origin, dims, cell starts, (cell, ID) order) is
compared bit-exactly with the oracle's. The GPU starts its Newton solves, its Johnson-Cook
consistency iteration and its eigen solver from extrapolated or previous-step values, the
oracle from the plain starts, so this is where a difference in those starts would show."""
import copy
import math

import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MP_FIELDS = ["mp_x", "F", "sigma", "be", "vol", "ebar", "T", "lam"]
NODE_FIELDS = ["node_x", "node_du", "node_mass", "node_force"]
SAMPLE = 3000


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.fixture(scope="module")
def rod():
    from paper_2206_08772_gb300.otm import OTM
    p = scenarios.config_taylor_jc(h=0.12e-3)
    sim = OTM(p, precision="fp64", max_support=384)
    yield p, sim
    sim.close()


def slab_problem(p, sel):
    s = copy.copy(p)
    s.mp_x = p.mp_x[sel].copy()
    s.mp_vol = p.mp_vol[sel].copy()
    s.mp_mass = p.mp_mass[sel].copy()
    s.mp_material = p.mp_material[sel].copy()
    return s


def compare_rows(orc_sim, sim, rows_local, rows_global, what):
    ids_g = sim.get_rows("support_ids", rows_global)
    sh_g = sim.get_rows("shape", rows_global)
    cnt_g = sim.get_rows("support_count", rows_global)
    worst = 0.0
    for r, (ql, qg) in enumerate(zip(rows_local, rows_global)):
        ids_o, N_o, dN_o = orc_sim.row(ql)
        n = cnt_g[r]
        assert n == ids_o.size and np.array_equal(ids_g[r, :n], ids_o), (what, qg)
        worst = max(worst, rel(sh_g[r, :n, 0], N_o), rel(sh_g[r, :n, 1:], dN_o))
    assert worst <= 1e-10, (what, worst)
    return worst


@pytest.mark.parametrize("n", [10, 100, 500])
def test_shadow_step(orc, rod, n):
    p, sim = rod
    cur = sim.counts()["step"]
    assert cur <= n
    if n > cur:
        assert sim.step(n - cur) == 0, sim.error()
    # the linked-cell grid of all nodes at step n
    node_x = sim.get("node_x")
    origin, dims, cs, srt = sim.grid_cells()
    o_origin, o_dims, o_cs, o_srt = orc.grid(node_x, p.cell_size)
    assert np.array_equal(origin, o_origin) and np.array_equal(dims.astype(np.int64), o_dims)
    assert np.array_equal(cs.astype(np.int64), o_cs) and np.array_equal(srt, o_srt)

    S = {f: sim.get(f) for f in ["node_du"] + MP_FIELDS}
    S["node_x"] = node_x
    rs = math.sqrt(p.rs2)
    zp = S["mp_x"][:, 2]
    zc = 0.5 * (zp.min() + zp.max())
    slabs = {"impact": (-np.inf, 4.0e-3), "mid": (zc - 2.5e-3, zc + 2.5e-3)}
    rng = np.random.default_rng(n)
    oracles = {}
    for name, (z0, z1) in slabs.items():
        sel = np.nonzero((zp >= z0) & (zp <= z1))[0]
        o = orc.Sim(slab_problem(p, sel), omp=True)
        o.set("node_x", S["node_x"])
        o.set("node_du", S["node_du"])
        for f in MP_FIELDS:
            o.set(f, S[f][sel])
        assert o.refresh() == 0, o.counts()
        # interior: MPs at least 2.4 r_s inside the slab's cut faces, nodes at least 1.2 r_s
        zs = zp[sel]
        inner = np.nonzero((zs >= z0 + 2.4 * rs) & (zs <= z1 - 2.4 * rs))[0]
        assert inner.size > 100_000
        xn = S["node_x"][:, 2]
        nodes = np.nonzero((xn >= z0 + 1.2 * rs) & (xn <= z1 - 1.2 * rs))[0]
        smp = np.sort(rng.choice(inner, SAMPLE, replace=False))
        if name == "impact":   # all the sampled rows within 0.5 mm of the wall too
            low = inner[zs[inner] <= 0.5e-3]
            smp = np.union1d(smp, rng.choice(low, min(1000, low.size), replace=False))
        compare_rows(o, sim, smp, sel[smp], f"{name} step {n}")
        oracles[name] = (o, sel, inner, nodes, smp)

    # one step of each; errors relative to the field's largest value over the whole rod (in the
    # mid-rod slab at step 10 the material still translates rigidly and its stress is rounding)
    assert sim.step(1) == 0, sim.error()
    G = {f: sim.get(f) for f in MP_FIELDS + NODE_FIELDS}
    scale = {f: max(np.abs(v).max(), 1e-300) for f, v in G.items()}
    for name, (o, sel, inner, nodes, smp) in oracles.items():
        assert o.step(1) == 0, o.counts()
        errs = {}
        for f in NODE_FIELDS:
            errs[f] = np.abs(G[f][nodes] - o.get(f)[nodes]).max() / scale[f]
        for f in MP_FIELDS:
            errs[f] = np.abs(G[f][sel[inner]] - o.get(f)[inner]).max() / scale[f]
        errs["shape"] = compare_rows(o, sim, smp, sel[smp], f"{name} step {n + 1}")
        print(f"shadow step {n} -> {n + 1}, {name} slab ({sel.size} MPs, {inner.size} interior, {nodes.size} "
              f"nodes): " + ", ".join(f"{k} {v:.1e}" for k, v in errs.items()))
        for f, e in errs.items():
            assert e <= 1e-10, (name, n, f, e)
        del o
    oracles.clear()
