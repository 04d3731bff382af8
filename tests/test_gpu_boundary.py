"""The C ABI's failure paths and state-transfer entries on the GPU:
  - bad state injected from the host (otm_set_state) gives the error code and the smallest
    offending ID that the oracle gives for the same state: a NaN in one MP's F -> NONFINITE
    with that MP's ID; a nodal increment that inverts the neighbourhood of some MPs ->
    JACOBIAN (det dF <= 0, Eq. 11-12); an MP pushed out of the rod -> LME_NOCONV (Eq. 14);
  - otm_keep_last_good: a failing step is undone, the state is that of the last good step bit
    for bit, the error stays recorded, and a refresh resumes the run;
  - a node far away on all three axes makes the linked-cell grid (Algorithm 3) too large:
    CAPACITY, not a fault;
  - otm_grid_cells: the device counting sort's (cell, ID) order equals the oracle's linked cell;
  - otm_supports_export / otm_step_with_supports_csr: a device-resident record of a run's
    supports replays it bit for bit, and a malformed CSR is refused before anything runs."""
import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ["node_x", "node_du", "mp_x", "F", "sigma", "be", "vol", "ebar", "T", "lam"]


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


def short_rod():
    return scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=4.8e-3, material=scenarios.copper_jc())


def both_after(orc, OTM, p, steps):
    g, o = OTM(p), orc.Sim(p)
    assert g.step(steps) == 0 and o.step(steps) == 0
    return g, o


def test_nan_in_F_reports_nonfinite_with_the_mp_id(orc, OTM):
    p = short_rod()
    g, o = both_after(orc, OTM, p, 2)
    q = 777
    for sim in (g, o):
        F = sim.get("F")
        F[q, 4] = np.nan
        sim.set("F", F)
    st_g = g.step(1)
    st_o = o.step(1)
    assert st_g == -6 and st_o == -6
    assert g.error() == (-6, q)
    c = o.counts()
    assert (c["err"], c["err_id"]) == (-6, q)


def test_inverted_neighbourhood_reports_jacobian_like_the_oracle(orc, OTM):
    """One interior node gets an increment of 30 h along x: every MP whose support holds it gets
    dF = 1 + du (x) grad N_a + ... (Eq. 11), and det dF ~ 1 + du . grad N_a <= 0 for MPs on the
    node's far side. The GPU must name the same smallest offending MP as the oracle."""
    p = short_rod()
    g, o = both_after(orc, OTM, p, 1)
    x = g.get("node_x")
    c = np.array([0.0, 0.0, 2.4e-3])
    a = int(np.argmin(np.linalg.norm(x - c, axis=1)))
    for sim in (g, o):
        du = sim.get("node_du")
        du[a, 0] += 30.0 * p.h
        sim.set("node_du", du)
    assert g.step(1) == -5
    assert o.step(1) == -5
    cnt = o.counts()
    code, fid = g.error()
    assert code == -5 and fid == cnt["err_id"]
    # the offending MP had the moved node in its support (the oracle stops before its search, so
    # it still holds the supports the failing step started from)
    off, ids = o.get("offsets"), o.get("ids")
    assert a in ids[off[fid]:off[fid + 1]]


def test_point_outside_the_rod_reports_lme_noconv_with_its_id(orc, OTM):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=4.0e-3, wall=False)
    g, o = OTM(p), orc.Sim(p)
    q = 7
    for sim in (g, o):
        xp = sim.get("mp_x")
        xp[q] += np.array([5.0e-3, 0.0, 0.0])     # 5 mm out of a rod of radius 3.2 mm
        sim.set("mp_x", xp)
    assert g.refresh() == -4
    assert g.error() == (-4, q)
    assert o.refresh() == -4
    assert (o.counts()["err"], o.counts()["err_id"]) == (-4, q)


@pytest.mark.parametrize("host", [False, True])
def test_keep_last_good_undoes_the_failing_step(OTM, host):
    p = short_rod()
    g = OTM(p)
    g.keep_last_good(True, host=host)
    assert g.step(3) == 0
    q = 500
    F = g.get("F")
    F_good = F.copy()
    F[q, 0] = np.nan
    g.set("F", F)
    before = {f: g.get(f) for f in FIELDS}
    before["support_ids"] = g.get("support_ids")
    before["shape"] = g.get("shape")
    assert g.step(2) == -6
    assert g.error() == (-6, q)
    assert g.counts()["step"] == 3
    for f, v in before.items():
        assert np.array_equal(g.get(f), v, equal_nan=True), f
    assert g.step(1) == -6                     # the error stays recorded
    # resume: repair the state, rebuild the supports, step on; compare with an undisturbed run
    g.set("F", F_good)
    assert g.refresh() == 0
    assert g.step(2) == 0
    ref = OTM(p)
    assert ref.step(5) == 0
    for f in FIELDS:
        assert rel(g.get(f), ref.get(f)) <= 1e-10, f


def test_adjoint_refuses_a_mixed_path_handle(OTM):
    """The adjoint differentiates the FP64 step: otm_adjoint_begin on a mixed-path handle is
    OTM_ERR_ARG, and the same problem in FP64 starts."""
    from paper_2206_08772_gb300._lib import ERR_ARG, OTMError
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=6.4e-3, material=scenarios.copper_jc())
    m = OTM(p, precision="mixed")
    assert m.step(2) == 0
    xbar = np.zeros((p.n_nodes, 3))
    with pytest.raises(OTMError) as ei:
        m.adjoint_begin(xbar)
    assert ei.value.code == ERR_ARG
    a = OTM(p, precision="fp64")
    assert a.step(2) == 0
    a.adjoint_begin(xbar)


def test_far_node_makes_the_grid_too_large_not_a_fault(OTM):
    """200,000 nodes in a small box plus one node 3000 m away on every axis: each axis has
    about 3e6 cells of 1 mm, within the per-axis limit (16 n + 65536 cells), but their product
    (2.7e19) exceeds both the limit and a signed 64-bit integer. The grid must report CAPACITY."""
    from paper_2206_08772_gb300.otm import support_search
    rng = np.random.default_rng(5)
    n = 200_000
    nx = rng.uniform(0.0, 0.05, size=(n, 3))
    nx[-1] = [3000.0, 3000.0, 3000.0]
    mx = rng.uniform(0.0, 0.05, size=(64, 3))
    node_x = torch.tensor(nx, dtype=torch.float64, device="cuda")
    mp_x = torch.tensor(mx, dtype=torch.float64, device="cuda")
    ids, counts, grid, status = support_search(node_x, mp_x, rs2=4e-6, cell_size=1e-3, max_support=64)
    torch.cuda.synchronize()
    assert int(status.item()) == -8
    assert int(counts.sum().item()) == 0


def test_grid_cell_order_matches_the_oracle(orc, OTM):
    p = short_rod()
    g = OTM(p)
    assert g.step(4) == 0
    origin, dims, cs, srt = g.grid_cells()
    o_origin, o_dims, o_cs, o_srt = orc.grid(g.get("node_x"), p.cell_size)
    assert np.array_equal(origin, o_origin)
    assert np.array_equal(dims.astype(np.int64), o_dims)
    assert np.array_equal(cs.astype(np.int64), o_cs)
    assert np.array_equal(srt, o_srt)


def test_device_support_record_replays_the_run_bit_for_bit(OTM):
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=9.6e-3, material=scenarios.copper_jc(), v0=400.0)
    base = OTM(p)
    rec = []
    for _ in range(10):
        assert base.step(1) == 0
        off, ids = base.supports_export()
        rec.append((off.clone(), ids.clone()))
    rep = OTM(p)
    for k in range(10):
        assert rep.step_with_supports_csr(*rec[k]) == 0, rep.error()
    for f in FIELDS:
        assert np.array_equal(rep.get(f), base.get(f)), f
    for a, b in zip(rep.supports() + rep.shape_functions(), base.supports() + base.shape_functions()):
        assert np.array_equal(a, b)
    # malformed records are refused before anything runs
    s = OTM(p)
    off, ids = rec[0]
    bad_ids = ids.clone()
    bad_ids[17] = p.n_nodes
    assert s.step_with_supports_csr(off, bad_ids) == -1
    bad_off = off.clone()
    bad_off[5] = 1 << 30
    assert s.step_with_supports_csr(bad_off, ids) == -1
    assert s.counts()["step"] == 0
    assert s.step_with_supports_csr(off, ids) == 0
