"""Parity at the benchmark's full size (Taylor JC rod, h 0.12 mm: 501,189 nodes, 2,854,368 MPs),
in the benchmark's launch configuration (FP64, 384 support slots), on sampled outputs that the
oracle recomputes one by one from the GPU's own state of the previous step:
  - supports of sampled MPs against a brute-force search (bit-exact)
  - LME shape functions of sampled MPs (1e-10)
  - kinematics (x_p, dF) and return map (sigma, b^e, ebar, T) of sampled MPs (1e-10)
  - lumped mass and internal force of sampled nodes from the sampled influence domains (1e-10)
and properties that hold at any size: sum m_I = sum m_p, sum r_I = 0."""
import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def brute_support(node_x, xp, rs2):
    d = xp[None, :] - node_x
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return np.nonzero(d2 <= rs2)[0].astype(np.int32)


@pytest.fixture(scope="module")
def run():
    from paper_2206_08772_gb300.otm import OTM
    p = scenarios.config_taylor_jc(h=0.12e-3)
    sim = OTM(p, precision="fp64", max_support=384)
    assert sim.step(1) == 0
    rng = np.random.default_rng(0)
    x1 = sim.get("node_x")
    mp1 = sim.get("mp_x")
    near_wall = np.nonzero(mp1[:, 2] < 0.3e-3)[0]
    rows = np.unique(np.concatenate([rng.choice(p.n_mps, 24, replace=False), rng.choice(near_wall, 24, replace=False)]))
    st1 = {k: sim.get(k) for k in ("be", "ebar", "T", "sigma", "vol", "F")}
    st1["ids"] = sim.get_rows("support_ids", rows)
    st1["shape"] = sim.get_rows("shape", rows)
    st1["cnt"] = sim.get("support_count")
    st1["x"], st1["mp_x"] = x1, mp1
    assert sim.step(1) == 0
    st2 = {k: sim.get(k) for k in ("node_x", "node_du", "node_mass", "node_force", "mp_x", "dF", "F", "be",
                                   "sigma", "ebar", "T", "lam")}
    st2["ids"] = sim.get_rows("support_ids", rows)
    st2["shape"] = sim.get_rows("shape", rows)
    st2["cnt"] = sim.get("support_count")
    return p, sim, rows, st1, st2


def test_fullsize_supports_and_lme(orc, run):
    p, sim, rows, st1, st2 = run
    for r, q in enumerate(rows):
        n = st2["cnt"][q]
        ids = st2["ids"][r, :n]
        assert np.array_equal(ids, brute_support(st2["node_x"], st2["mp_x"][q], p.rs2))
        d = st2["mp_x"][q] - st2["node_x"][ids]
        s_, N, dN, lam, _ = orc.lme(d, p.beta, p.newton_tol * p.h)
        assert s_ == 0
        assert rel(st2["shape"][r, :n, 0], N) <= 1e-10
        assert rel(st2["shape"][r, :n, 1:], dN) <= 1e-10


def test_fullsize_kinematics_and_return_map(orc, run):
    p, sim, rows, st1, st2 = run
    mat = p.materials[0]
    plastic = 0
    for r, q in enumerate(rows):
        n = st1["cnt"][q]
        ids = st1["ids"][r, :n]
        xp, dF = orc.kinematics(ids, st1["shape"][r, :n, 0], st1["shape"][r, :n, 1:], st2["node_x"], st2["node_du"])
        assert np.abs(xp - st2["mp_x"][q]).max() <= 1e-10 * np.abs(st2["mp_x"]).max()
        assert np.abs(dF - st2["dF"][q].reshape(3, 3)).max() <= 1e-12
        st, sig, be, eb, T, _, _ = orc.return_map(mat, p.dt, st2["dF"][q].reshape(3, 3), st1["be"][q], st1["ebar"][q],
                                                  st1["T"][q], np.linalg.det(st2["F"][q].reshape(3, 3)))
        assert st == 0
        assert np.abs(sig - st2["sigma"][q]).max() <= 1e-10 * max(np.abs(st2["sigma"]).max(), 1.0)
        assert np.abs(be - st2["be"][q]).max() <= 1e-12
        assert abs(eb - st2["ebar"][q]) <= 1e-12
        assert abs(T - st2["T"][q]) <= 1e-10 * T
        plastic += eb > 0
    assert plastic > 0


def test_fullsize_node_mass_and_force(orc, run):
    p, sim, rows, st1, st2 = run
    m, f = st2["node_mass"], st2["node_force"]
    assert abs(m.sum() - p.mp_mass.sum()) <= 1e-12 * p.mp_mass.sum()
    assert np.abs(f.sum(0)).max() <= 1e-10 * np.abs(f).sum()
    # sampled nodes near the wall: influence domain by brute force at state 1, then the sums
    near = np.nonzero(st1["x"][:, 2] < 1.5e-3)[0]          # all nodes any of these MPs can reach
    cand = np.nonzero(st1["x"][:, 2] < 0.25e-3)[0]
    rng = np.random.default_rng(3)
    for i in rng.choice(cand, 3, replace=False):
        infl = brute_support(st1["mp_x"], st1["x"][i], p.rs2)   # MPs within r_s of node i
        mass = 0.0
        force = np.zeros(3)
        for q in infl:
            sup = near[brute_support(st1["x"][near], st1["mp_x"][q], p.rs2)]
            d = st1["mp_x"][q] - st1["x"][sup]
            s_, N, dN, _, _ = orc.lme(d, p.beta, p.newton_tol * p.h)
            assert s_ == 0
            k = int(np.searchsorted(sup, i))
            assert sup[k] == i
            mass += N[k] * p.mp_mass[q]
            S = st1["sigma"][q]
            Sm = np.array([[S[0], S[3], S[5]], [S[3], S[1], S[4]], [S[5], S[4], S[2]]])
            force -= st1["vol"][q] * (Sm @ dN[k])
        assert abs(m[i] - mass) <= 1e-10 * mass
        assert np.abs(f[i] - force).max() <= 1e-10 * np.abs(f).max()
