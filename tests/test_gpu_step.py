"""GPU parity of the whole explicit step (Algorithm 1) against the oracle, through the C ABI.

FP64 path: neighbour lists bit-exact and every field within 1e-10 relative of the oracle
(max |gpu - oracle| / max |oracle|) after a multi-step trajectory. Mixed path: errors per field
against the FP64 oracle within stated bounds. Determinism: two runs bit-identical."""
import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS_NODE = ["node_x", "node_du"]
FIELDS_MP = ["mp_x", "F", "sigma", "be", "vol", "ebar", "T", "lam"]


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.fixture(scope="module")
def OTM():
    import paper_2206_08772_gb300 as g
    g.load()
    from paper_2206_08772_gb300.otm import OTM
    return OTM


def compare(sim_g, sim_o, fields_tol):
    errs = {}
    for f in FIELDS_NODE + FIELDS_MP:
        g = sim_g.get(f)
        o = sim_o.get(f)
        errs[f] = rel(g, o)
    bad = {f: e for f, e in errs.items() if e > fields_tol.get(f, fields_tol["default"])}
    return errs, bad


def supports_equal(sim_g, sim_o):
    off_g, ids_g = sim_g.supports()
    off_o, ids_o = sim_o.get("offsets"), sim_o.get("ids")
    return np.array_equal(off_g, off_o) and np.array_equal(ids_g, ids_o)


@pytest.mark.parametrize("name,steps", [("taylor_j2_short", 30), ("taylor_jc_short", 30)])
def test_fp64_trajectory_matches_oracle(orc, OTM, name, steps):
    mat = scenarios.copper_j2() if "j2" in name else scenarios.copper_jc()
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=mat)
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    assert supports_equal(sim_g, sim_o)
    for k in range(steps):
        assert sim_o.step(1) == 0
        assert sim_g.step(1) == 0, sim_g.error()
        assert supports_equal(sim_g, sim_o), f"step {k + 1}"
    errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    print(name, errs)
    assert not bad, bad
    assert sim_o.get("ebar").max() > 0


def test_fp64_config1_full_100_steps(orc, OTM):
    """The plain Taylor rod (R 3.2 mm, L 25.4 mm, h 0.8 mm, J2, 100 steps)."""
    p = scenarios.config_taylor_j2()
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    assert sim_g.step(p.steps) == 0, sim_g.error()
    assert sim_o.step(p.steps) == 0
    assert supports_equal(sim_g, sim_o)
    errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    print("config1", errs)
    assert not bad, bad
    m = sim_g.get("node_mass")
    assert abs(m.sum() - p.mp_mass.sum()) <= 1e-12 * p.mp_mass.sum()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_supports_beyond_the_lme_shared_rows(orc, OTM, precision):
    """The LME kernel keeps 336 of the 384 support slots per MP in shared memory; MPs with larger
    supports are solved by a second launch with full rows. With a support tolerance of 3e-7
    (r_s = 4.33 h) a rod of R 4.8 mm has 672 of its 8,064 MPs above 336 nodes at the start: after
    12 steps the FP64 path matches the oracle (supports bit-exact, every field 1e-10), the mixed
    path within its own bounds, and supports above 336 are still present."""
    p = scenarios.taylor_rod(h=0.8e-3, R=4.8e-3, L=9.6e-3, material=scenarios.copper_jc(), support_tol=3e-7)
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision=precision)
    assert np.diff(sim_o.get("offsets")).max() > 336
    assert sim_g.step(12) == 0, sim_g.error()
    assert sim_o.step(12) == 0
    cnt = np.diff(sim_g.supports()[0])
    assert 336 < cnt.max() <= 384
    if precision == "fp64":
        assert supports_equal(sim_g, sim_o)
        errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    else:
        errs, bad = compare(sim_g, sim_o, {"default": 1e-4, "node_x": 1e-7, "mp_x": 1e-7})
    print("wide supports", precision, int((cnt > 336).sum()), errs)
    assert not bad, bad


def test_mixed_path_error_table(orc, OTM):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc())
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="mixed")
    steps = 30
    assert sim_g.step(steps) == 0, sim_g.error()
    assert sim_o.step(steps) == 0
    errs, bad = compare(sim_g, sim_o, {"default": 1e-4, "node_x": 1e-7, "mp_x": 1e-7})
    print("mixed", errs)
    assert not bad, bad


def test_per_field_error_through_the_impact(orc, OTM):
    """The error of each output field against the FP64 oracle (its OpenMP build, the same
    arithmetic as the serial one), max |gpu - oracle| / max |oracle| over the field, for both GPU
    paths on the Johnson-Cook rod at h 0.6 mm (R 3.2, L 25.4 mm, 22,176 MPs) at steps 50, 100 and
    200 of the impact. FP64 path: 1e-10 at step 50; over the longer plastic history the two FP64
    implementations drift apart to a few 1e-10 in the node increments and the stress (measured
    2.9e-10 and 3.3e-10; one-step parity from any state stays at 1e-11), held here to 1e-9. The
    trajectory itself amplifies rounding-level differences that much: the oracle against itself
    with the initial node positions changed by 1e-13 moves by 3.4e-10 in the node increments at
    step 150. Mixed path: 1e-4 (positions 1e-7), its error set by the FP32 force contributions and
    kinematics gather."""
    p = scenarios.taylor_rod(h=0.6e-3, material=scenarios.copper_jc())
    sim_o = orc.Sim(p, omp=True)
    g64 = OTM(p, precision="fp64")
    g32 = OTM(p, precision="mixed")
    table = {"fp64": {}, "mixed": {}}
    bad_all = []
    done = 0
    for n in (50, 100, 200):
        assert sim_o.step(n - done) == 0
        assert g64.step(n - done) == 0, g64.error()
        assert g32.step(n - done) == 0, g32.error()
        done = n
        for name, sim in (("fp64", g64), ("mixed", g32)):
            if name == "fp64":
                tol = {"default": 1e-10 if n <= 50 else 1e-9}
            else:
                tol = {"default": 1e-4, "node_x": 1e-7, "mp_x": 1e-7}
            errs, bad = compare(sim, sim_o, tol)
            table[name][n] = errs
            if bad:
                bad_all.append((name, n, bad))
    for name in ("fp64", "mixed"):
        for n, errs in table[name].items():
            print("per-field error", name, "step", n, " ".join(f"{f} {e:.1e}" for f, e in errs.items()))
    assert not bad_all, bad_all


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_determinism(OTM, precision):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, material=scenarios.copper_jc())
    outs = []
    for _ in range(2):
        s = OTM(p, precision=precision)
        assert s.step(10) == 0
        outs.append([s.get(f).copy() for f in FIELDS_NODE + FIELDS_MP])
        s.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def chip_case(embed_h):
    h = 0.02e-3
    return scenarios.chip_block(h=h, size=(0.4e-3, 0.2e-3, 0.1e-3), depth=0.06e-3, embed=embed_h * h, steps=8)


@pytest.mark.parametrize("embed_h,steps", [(1.5, 6), (3.0, 8)])
def test_chip_tool_contact_erosion_compaction(orc, OTM, embed_h, steps):
    """Chip block with the rigid tool (Coulomb friction) embedded in the work piece: with
    3 h of embedding the Johnson-Cook fracture criterion erodes material points from the second
    step on and orphan nodes are removed; the GPU compaction must keep exactly the oracle's
    survivors, in the same order, with matching supports and fields."""
    p = chip_case(embed_h)
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    eroded = 0
    for k in range(steps):
        assert sim_o.step(1) == 0
        assert sim_g.step(1) == 0, sim_g.error()
        co, cg = sim_o.counts(), sim_g.counts()
        assert (cg["n_mps"], cg["n_nodes"]) == (co["n_mps"], co["n_nodes"]), f"step {k + 1}"
        assert np.array_equal(sim_g.get("mp_gid"), sim_o.get("mp_gid"))
        assert np.array_equal(sim_g.get("node_gid"), sim_o.get("node_gid"))
        assert supports_equal(sim_g, sim_o), f"step {k + 1}"
        eroded = p.n_mps - co["n_mps"]
    errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    print("chip", embed_h, eroded, errs)
    assert not bad, bad
    if embed_h >= 3.0:
        assert eroded > 100
        assert sim_o.counts()["n_nodes"] < p.n_nodes


def test_sweep_mixed_vs_fp64_final_geometry(orc, OTM):
    """Sweep of small rods of uneven size (h, v0 and the JC constants A, B varied from a seed):
    final length and footprint radius of the FP64 and mixed GPU paths against the FP64 oracle."""
    import math
    rng = np.random.default_rng(5)
    rows = []
    for k, h in enumerate((0.6e-3, 0.7e-3, 0.8e-3)):
        v0 = rng.uniform(150, 300)
        A, B = 90e6 * rng.uniform(0.9, 1.1), 292e6 * rng.uniform(0.9, 1.1)
        p = scenarios.taylor_rod(h=h, R=3.2e-3, L=6.4e-3, v0=v0, material=scenarios.copper_jc(A=A, B=B))
        steps = 25
        so = orc.Sim(p)
        assert so.step(steps) == 0
        xo = so.get("node_x")
        act = so.get("node_mass") > 0
        Lo = xo[act, 2].max()
        foot = xo[:, 2] <= 1e-3 * p.h
        Ro = np.hypot(xo[foot, 0], xo[foot, 1]).max()
        errs = {}
        for prec in ("fp64", "mixed"):
            g = OTM(p, precision=prec)
            assert g.step(steps) == 0
            x = g.get("node_x")
            Lg = x[act, 2].max()
            Rg = np.hypot(x[foot, 0], x[foot, 1]).max()
            errs[prec] = (abs(Lg - Lo) / Lo, abs(Rg - Ro) / Ro)
        rows.append((h, v0, errs))
        assert max(errs["fp64"]) <= 1e-12
        assert max(errs["mixed"]) <= 1e-7
    print("sweep", rows)


def test_stabilised_residual_matches_oracle(orc, OTM):
    """Eq. 7-8: the residual with the under-integration penalty, eps = 1e-3 E h^2."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, material=scenarios.copper_jc())
    p.eps_stab = 1e-3 * p.materials[0].E * p.h ** 2
    sim_o = orc.Sim(p)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-4)):
        sim_g = OTM(p, precision=prec)
        if prec == "fp64":
            assert sim_o.step(20) == 0
        assert sim_g.step(20) == 0, sim_g.error()
        errs, bad = compare(sim_g, sim_o, {"default": tol, "node_x": tol * 1e-3 if prec == "mixed" else tol,
                                           "mp_x": tol * 1e-3 if prec == "mixed" else tol})
        print("stab", prec, errs)
        assert not bad, bad
    # the term changes the trajectory: compare with the unstabilised run
    q = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, material=scenarios.copper_jc())
    plain = orc.Sim(q)
    assert plain.step(20) == 0
    assert np.abs(plain.get("node_x") - sim_o.get("node_x")).max() > 1e-9


def insertion_rod(max_insert=200):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, v0=2000.0, material=scenarios.copper_jc())
    p.max_insert = max_insert
    return p


def test_node_insertion_matches_oracle(orc, OTM):
    """Node insertion: at 2000 m/s the rod's foot spreads until MPs leave the hull of their
    supports (step 34); each gets a node one spacing beyond it. GPU and oracle agree at every step
    on the node set (IDs bit-exact, inserted ones included), the supports (bit-exact) and, after
    40 steps, every field (1e-10). The mixed path runs through the same insertions."""
    p = insertion_rod()
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    sim_m = OTM(p, precision="mixed")
    for k in range(40):
        assert sim_o.step(1) == 0
        assert sim_g.step(1) == 0, (k + 1, sim_g.error())
        assert sim_m.step(1) == 0, (k + 1, sim_m.error())
        co, cg = sim_o.counts(), sim_g.counts()
        assert (cg["n_nodes"], cg["n_mps"]) == (co["n_nodes"], co["n_mps"]), f"step {k + 1}"
        assert np.array_equal(sim_g.get("node_gid"), sim_o.get("node_gid"))
        assert supports_equal(sim_g, sim_o), f"step {k + 1}"
    assert sim_o.counts()["n_nodes"] > p.n_nodes
    assert sim_m.counts()["n_nodes"] == sim_o.counts()["n_nodes"]
    errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    print("insertion", errs)
    assert not bad, bad


def test_node_insertion_capacity(orc, OTM):
    """One node slot for two failing MPs: both stop at step 34 with CAPACITY at the same MP."""
    p = insertion_rod(max_insert=1)
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    assert sim_o.step(34) == -8
    assert sim_g.step(34) == -8
    co = sim_o.counts()
    assert sim_g.error() == (co["err"], co["err_id"])


def test_chip_deep_tool_embedding_inserts_nodes(orc, OTM):
    """Tool embedded 6 h into the small chip block: the contact projection of step 1 leaves MPs
    outside their supports' hulls; nodes are inserted (and MPs eroded) in the same step. Node
    and MP sets, supports and fields agree with the oracle after step 1."""
    h = 0.02e-3
    p = scenarios.chip_block(h=h, size=(0.4e-3, 0.2e-3, 0.1e-3), depth=0.06e-3, embed=6 * h, steps=2)
    p.max_insert = 64
    sim_o = orc.Sim(p)
    sim_g = OTM(p, precision="fp64")
    assert sim_o.step(1) == 0
    assert sim_g.step(1) == 0, sim_g.error()
    co, cg = sim_o.counts(), sim_g.counts()
    assert (cg["n_nodes"], cg["n_mps"]) == (co["n_nodes"], co["n_mps"])
    assert co["n_nodes"] > p.n_nodes and co["n_mps"] < p.n_mps
    assert np.array_equal(sim_g.get("node_gid"), sim_o.get("node_gid"))
    assert np.array_equal(sim_g.get("mp_gid"), sim_o.get("mp_gid"))
    assert supports_equal(sim_g, sim_o)
    errs, bad = compare(sim_g, sim_o, {"default": 1e-10})
    print("chip insertion", errs)
    assert not bad, bad


@pytest.mark.parametrize("host", [False, True])
def test_snapshot_restore_continues_bit_exactly(OTM, host):
    """Checkpoint / resume: a snapshot (device or page-locked host memory) taken at step 12 and
    loaded back reproduces the uninterrupted run bit for bit, including the time-extrapolated
    LME start (the previous lambda is part of the state)."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc(), v0=400.0)
    a = OTM(p)
    assert a.step(12) == 0
    snap = a.snapshot(host=host)
    assert a.step(10) == 0
    ref = {f: a.get(f) for f in FIELDS_NODE + FIELDS_MP}
    b = OTM(p)
    b.restore(snap)
    assert b.step(10) == 0
    for f in FIELDS_NODE + FIELDS_MP:
        assert np.array_equal(b.get(f), ref[f]), f


def test_snapshot_loads_across_precisions(orc, OTM):
    """A snapshot of the FP64 path loads into a mixed-path handle (the FP32 increments are rebuilt
    from the FP64 ones): the restored state equals the saved one, and the mixed path continues
    within its stated error of the FP64 oracle."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc())
    a = OTM(p, precision="fp64")
    assert a.step(10) == 0
    snap = a.snapshot()
    m = OTM(p, precision="mixed")
    m.restore(snap)
    for f in ("node_x", "node_du", "mp_x", "F", "sigma", "lam"):
        assert np.array_equal(m.get(f), a.get(f)), f
    assert m.step(10) == 0
    o = orc.Sim(p)
    assert o.step(20) == 0
    assert rel(m.get("node_x"), o.get("node_x")) <= 1e-8
    assert rel(m.get("sigma"), o.get("sigma")) <= 1e-3


def test_mixed_lme_hessian_sums_against_fp64(OTM):
    """The mixed path accumulates the LME Newton's Hessian sums in double-float (FP32 pairs);
    its weights, Z and residual stay FP64, and it forms the rows' e = N d in FP32. Loaded from the
    same FP64-path snapshot, the mixed handle regenerates the same supports, bit-identical N
    (w / Z, FP64), J^-1 within 1e-11 of the FP64 path's (from the double-float sums), and
    grad N = -J^-1 e within the FP32 rounding of e."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc())
    a = OTM(p, precision="fp64")
    assert a.step(12) == 0
    snap = a.snapshot()
    m = OTM(p, precision="mixed")
    m.restore(snap)
    oa, ia = a.supports()
    om, im = m.supports()
    assert np.array_equal(oa, om) and np.array_equal(ia, im)
    Na, dNa = a.shape_functions()
    Nm, dNm = m.shape_functions()
    assert np.array_equal(Na, Nm)
    eK = rel(m.get("kinv"), a.get("kinv"))
    e = rel(dNm, dNa)
    print("J^-1, double-float Hessian sums vs FP64:", eK, "grad N with FP32 e:", e)
    assert 0.0 < eK <= 1e-11
    assert e <= 1e-6


def test_mixed_kinematics_gather_against_fp64(OTM):
    """The mixed path gathers the MP displacement (Eq. 9) and G = sum du (x) e (Eq. 11) in FP32
    from the FP32 increments, relative to the increment of one support node. From the same
    FP64-path snapshot, one step of each path: the step's MP displacement and the strain increment
    dF - 1 agree with the FP64 path's within 1e-5 of their largest values (the FP32 rounding of the
    increments and of the force contributions)."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc())
    a = OTM(p, precision="fp64")
    assert a.step(12) == 0
    snap = a.snapshot()
    m = OTM(p, precision="mixed")
    m.restore(snap)
    x0 = a.get("mp_x")
    assert a.step(1) == 0, a.error()
    assert m.step(1) == 0, m.error()
    I = np.eye(3).reshape(1, 9)
    e_dx = rel(m.get("mp_x") - x0, a.get("mp_x") - x0)
    e_g = rel(m.get("dF") - I, a.get("dF") - I)
    print("mixed vs FP64, one step: MP displacement", e_dx, "dF - 1", e_g)
    assert 0.0 < e_dx <= 1e-5 and 0.0 < e_g <= 1e-5


def test_pitched_state_transfer_round_trip(OTM):
    """otm_state / otm_set_state of the fields stored with padding (node x, du, mass, force, MP x)
    move exact bytes in both directions."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc())
    s = OTM(p)
    assert s.step(3) == 0
    rng = np.random.default_rng(4)
    for f in ("node_x", "node_du", "mp_x"):
        v = s.get(f)
        w = v + rng.standard_normal(v.shape) * 1e-9
        s.set(f, w)
        assert np.array_equal(s.get(f), w), f
        s.set(f, v)
        assert np.array_equal(s.get(f), v), f
    m, fr = s.get("node_mass"), s.get("node_force")
    assert m.shape == (p.n_nodes,) and fr.shape == (p.n_nodes, 3)
    assert abs(m.sum() - p.mp_mass.sum()) <= 1e-12 * p.mp_mass.sum()


def test_replayed_supports_reproduce_the_base_run(OTM):
    """otm_step_with_supports: a run that takes, at every step, the supports a base run found
    (instead of searching) reproduces the base run; here the impact changes the supports, so
    the replay is not trivially the frozen initial topology."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc(), v0=400.0)
    base = OTM(p)
    first = base.get("support_ids")
    rec = []
    for _ in range(12):
        assert base.step(1) == 0
        rec.append((base.get("support_count"), base.get("support_ids")))
    assert not np.array_equal(rec[-1][1], first)
    rep = OTM(p)
    for k in range(12):
        assert rep.step_with_supports(*rec[k]) == 0, rep.error()
        assert np.array_equal(rep.get("support_ids"), rec[k][1])
    for f in FIELDS_NODE + FIELDS_MP:
        assert rel(rep.get(f), base.get(f)) <= 1e-12, f


def test_frozen_topology_keeps_the_supports(OTM):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc(), v0=400.0)
    s = OTM(p)
    ids0, cnt0 = s.get("support_ids"), s.get("support_count")
    s.freeze_topology(True)
    assert s.step(12) == 0
    assert np.array_equal(s.get("support_ids"), ids0) and np.array_equal(s.get("support_count"), cnt0)
    bad = np.full(ids0.shape, p.n_nodes + 5, np.int32)
    assert s.step_with_supports(np.minimum(cnt0, 1), bad) == -1     # out-of-range index: refused
    e = OTM(scenarios.chip_block(h=0.02e-3, size=(0.4e-3, 0.2e-3, 0.1e-3), depth=0.06e-3, steps=2))
    with pytest.raises(Exception):
        e.freeze_topology(True)                                      # eroding problem: refused


def test_lme_cold_start_after_a_failed_warm_start(orc, OTM):
    """A far warm start makes the first Newton solve fail; the kernel solves again from
    lambda = 0 and reaches the shape functions of a fresh solve (as the oracle does)."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=4.0e-3, wall=False)
    g = OTM(p)
    shape0 = g.get("shape")
    g.set("lam", np.tile(np.array([3.0e5, -2.0e5, 4.0e5]), (p.n_mps, 1)))
    assert g.refresh() == 0, g.error()
    assert rel(g.get("shape"), shape0) <= 1e-12
    o = orc.Sim(p)
    assert rel(g.get("lam"), o.get("lam")) <= 1e-10
