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


def chip_full(embed_h):
    h = 1.0e-3 / 68
    return scenarios.chip_block(h=h, embed=embed_h * h, steps=2)


def test_fullsize_chip_mixed_with_erosion(orc):
    """Chip block at full size (4 x 1 x 0.4 mm, h = 1/68 mm: 527,436 nodes, 2,996,352 MPs), mixed
    path, tool embedded 1.5 h. Before step 1 the plastic strain of a chosen set of MPs (5000 at
    rest far from the tool, and every MP within 6 h of the corner (0, L_y, 0)) is raised to 1:
    at rest the Johnson-Cook fracture strain is (d1 + d2)(1 + 0)(1 + 0) = 0.16, so exactly that
    set is eroded in step 1, and the corner nodes left with no MP within r_s are removed.
    Checked: the surviving MP and node IDs (bit-exact, orphans by brute force over the corner);
    then, through step 2 (support IDs renumbered by the compaction), sampled survivors re-derived
    by the oracle from the GPU's own state: kinematics (to the FP32 gather of the mixed path: x_p
    within 1e-6 of the support's largest increment, dF within 1e-6 of the MP's strain increment),
    return map, supports (bit-exact), LME (N 1e-10; grad N 1e-6, its e = N d being FP32)."""
    from paper_2206_08772_gb300.otm import OTM
    p = chip_full(1.5)
    h, Lx, Ly = p.h, p.meta["size"][0], p.meta["size"][1]
    sim = OTM(p, precision="mixed", max_support=384)
    rng = np.random.default_rng(1)
    far = np.nonzero(p.mp_x[:, 0] < 0.5 * Lx)[0]
    corner = np.array([0.0, Ly, 0.0])
    in_corner = np.nonzero(np.linalg.norm(p.mp_x - corner, axis=1) <= 6 * h)[0]
    E = np.union1d(rng.choice(far, 5000, replace=False), in_corner)
    ebar = np.zeros(p.n_mps)
    ebar[E] = 1.0
    sim.set("ebar", ebar)
    assert sim.step(1) == 0, sim.error()
    gid1 = sim.get("mp_gid")
    assert np.array_equal(gid1, np.setdiff1d(np.arange(p.n_mps), E))
    mp1 = sim.get("mp_x")
    # orphans: nodes near the corner with no surviving MP within r_s (the search's distance test)
    cand = np.nonzero(np.linalg.norm(p.node_x - corner, axis=1) <= 10 * h)[0]
    near = np.nonzero(np.linalg.norm(mp1 - corner, axis=1) <= 16 * h)[0]
    x1 = sim.get("node_x")
    ngid1 = sim.get("node_gid")
    orphan = [i for i in cand if brute_support(mp1[near], p.node_x[i], p.rs2).size == 0]
    assert len(orphan) > 0
    assert np.array_equal(ngid1, np.setdiff1d(np.arange(p.n_nodes), orphan))
    st1 = {k: sim.get(k) for k in ("be", "ebar", "T")}
    near_tool = np.nonzero(mp1[:, 0] > p.contact.tool_x0 - 0.1e-3)[0]
    by_corner = np.nonzero(np.linalg.norm(mp1 - corner, axis=1) <= 9 * h)[0]
    rows1 = np.unique(np.concatenate([rng.choice(near_tool, 16, replace=False),
                                      rng.choice(by_corner, 8, replace=False),
                                      rng.choice(gid1.size, 8, replace=False)]))
    ids1 = sim.get_rows("support_ids", rows1)
    shape1 = sim.get_rows("shape", rows1)
    cnt1 = sim.get("support_count")[rows1]
    assert sim.step(1) == 0, sim.error()
    gid2 = sim.get("mp_gid")
    assert np.all(np.diff(gid2) > 0) and np.all(np.diff(sim.get("node_gid")) > 0)
    st2 = {k: sim.get(k) for k in ("node_x", "node_du", "mp_x", "dF", "F", "be", "sigma", "ebar", "T")}
    ngid2 = sim.get("node_gid")
    pos2 = {g: i for i, g in enumerate(gid2)}
    mat = p.materials[0]
    checked = plastic = 0
    for r, q1 in enumerate(rows1):
        g = gid1[q1]
        if g not in pos2:
            continue                      # eroded by the fracture criterion in step 2
        q2 = pos2[g]
        nid1 = ngid1[ids1[r, :cnt1[r]]]
        n2 = np.searchsorted(ngid2, nid1)
        assert np.array_equal(ngid2[n2], nid1)
        xp, dF = orc.kinematics(n2.astype(np.int32), shape1[r, :cnt1[r], 0], shape1[r, :cnt1[r], 1:],
                                st2["node_x"], st2["node_du"])
        # the mixed path gathers the MP displacement and G = sum du (x) e in FP32 (relative to one
        # node's increment): x_p carries FP32 rounding of the support's increments, dF of the MP's
        # own strain increment
        du_sup = np.abs(st2["node_du"][n2]).max()
        assert np.abs(xp - st2["mp_x"][q2]).max() <= 1e-10 * np.abs(st2["mp_x"]).max() + 1e-6 * du_sup
        assert np.abs(dF - st2["dF"][q2].reshape(3, 3)).max() <= 1e-6 * np.abs(dF - np.eye(3)).max() + 1e-13
        st, sig, be, eb, T, _, failed = orc.return_map(mat, p.dt, st2["dF"][q2].reshape(3, 3), st1["be"][q1],
                                                       st1["ebar"][q1], st1["T"][q1],
                                                       np.linalg.det(st2["F"][q2].reshape(3, 3)))
        assert st == 0 and not failed
        assert np.abs(sig - st2["sigma"][q2]).max() <= 1e-10 * np.abs(st2["sigma"]).max()
        assert abs(eb - st2["ebar"][q2]) <= 1e-10 * max(1.0, eb)
        plastic += eb > 0
        row = sim.get_rows("support_ids", [q2])[0]
        n = sim.get_rows("support_count", [q2])[0]
        sup = brute_support(st2["node_x"], st2["mp_x"][q2], p.rs2)
        assert np.array_equal(row[:n], sup)
        s_, N, dN, _, _ = orc.lme(st2["mp_x"][q2] - st2["node_x"][sup], p.beta, p.newton_tol * p.h)
        assert s_ == 0
        shp = sim.get_rows("shape", [q2])[0]
        # N in FP64; the mixed path forms e = N d, hence grad N = -J^-1 e, in FP32
        assert rel(shp[:n, 0], N) <= 1e-10 and rel(shp[:n, 1:], dN) <= 1e-6
        checked += 1
    assert checked >= 24 and plastic > 0


def test_fullsize_chip_degenerate_embedding_fails_like_the_oracle():
    """With the tool embedded 3 h at full resolution, the contact projection of step 1 flattens
    the node layers in front of the rake face so that one MP ends outside the hull of its new
    support: the Newton solve for lambda cannot converge. The GPU must stop with the same status
    and the same MP ID as the oracle (stored by tests/golden/make_chip_embedding_failure.py)."""
    import json
    import pathlib
    from paper_2206_08772_gb300.otm import OTM
    ref = json.loads((pathlib.Path(__file__).parent / "golden" / "chip_embed3h_failure.json").read_text())
    sim = OTM(chip_full(ref["embed_h"]), precision="fp64", max_support=384)
    st = sim.step(ref["steps"])
    assert st == ref["status"]
    assert sim.error() == (ref["status"], ref["mp_id"])


def test_fullsize_adjoint_rod_against_finite_differences():
    """The adjoint configuration's rod (h 0.29 mm: 38,181 nodes, 202,752 MPs, Johnson-Cook): the
    GPU adjoint's d(final length, footprint radius)/d(A, B, C, v0) against central differences of
    the GPU forward (1e-6 relative step) at the forward's arg-max nodes."""
    from paper_2206_08772_gb300.adjoint import objectives_and_seeds, rod_objectives
    from paper_2206_08772_gb300.otm import OTM

    def make(theta):
        A, B, n, C, m, v0 = theta
        return scenarios.taylor_rod(h=0.29e-3, material=scenarios.copper_jc(A=A, B=B, n=n, C=C, m=m), v0=v0)

    theta0 = np.array([90e6, 292e6, 0.31, 0.025, 1.09, 227.0])
    steps = 12
    th = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    vals = rod_objectives(th, make, steps)
    g = [torch.autograd.grad(vals[o], th, retain_graph=True)[0].numpy() for o in range(2)]
    base = OTM(make(theta0))
    assert base.step(steps) == 0
    _, _, (i_len, i_rad) = objectives_and_seeds(base.get("node_x"), base.get("node_mass"), 0.29e-3)
    for k in (0, 1, 3, 5):
        hk = 1e-6 * theta0[k]
        f = []
        for sg in (1, -1):
            t = theta0.copy()
            t[k] += sg * hk
            s = OTM(make(t))
            assert s.step(steps) == 0
            x = s.get("node_x")
            f.append((x[i_len, 2], np.hypot(x[i_rad, 0], x[i_rad, 1])))
        for o in range(2):
            fd = (f[0][o] - f[1][o]) / (2 * hk)
            noise = 20 * np.finfo(float).eps * abs(vals[o].item()) / hk
            assert abs(fd - g[o][k]) <= 1e-6 * abs(g[o][k]) + noise, (k, o, fd, g[o][k])
