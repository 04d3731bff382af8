"""GPU parity of the individual kernels, called through the C ABI, against the oracle.

Bars: neighbour lists, counts and linked-cell grid bit-exact; FP64 fields within 1e-10 relative
(max |gpu - oracle| / max |oracle| per field); LME invariants to 1e-12 on the GPU output."""
import math

import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    d = np.abs(a - b).max() if a.size else 0.0
    s = np.abs(b).max() if b.size else 1.0
    return d / (s if s > 0 else 1.0)


@pytest.fixture(scope="module")
def otm():
    import paper_2206_08772_gb300 as g
    g.load()
    from paper_2206_08772_gb300 import otm as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("seed,nn,nm,r,S", [(1, 300, 500, 0.21, 256), (2, 5000, 3000, 0.11, 384),
                                            (3, 40, 100, 0.6, 64), (4, 20000, 1000, 0.05, 128)])
def test_search_bit_exact(orc, otm, seed, nn, nm, r, S):
    node_x, mp_x = scenarios.random_cloud(nn, nm, seed)
    mp_x = np.vstack([mp_x, [[-0.3, 0.5, 0.5], [9.0, 9.0, 9.0]]])   # points outside the node box
    rs2 = r * r
    cell = 0.5 * r * (1 + 2 ** -20)
    ids, counts, grid, status = otm.support_search(dev(node_x), dev(mp_x), rs2, cell, S)
    torch.cuda.synchronize()
    off, ref = orc.search(node_x, mp_x, rs2, cell)
    cnt_ref = np.diff(off)
    counts = counts.cpu().numpy()
    assert np.array_equal(counts, cnt_ref)
    ids = ids.cpu().numpy()
    over = cnt_ref > S
    assert (status.item() == -8) == bool(over.any())
    for p in np.nonzero(~over)[0]:
        assert np.array_equal(ids[p, :counts[p]], ref[off[p]:off[p + 1]])
    origin, dims, _, _ = orc.grid(node_x, cell)
    g = grid.cpu().numpy()
    assert np.array_equal(g[:3], origin) and np.array_equal(g[3:].astype(np.int64), dims)


def test_search_ties_exact(orc, otm):
    r = 0.25
    rs2 = r * r
    rng = np.random.default_rng(7)
    node_x = rng.uniform(0, 1, (400, 3))
    mp = []
    for k in range(60):
        p = node_x[k].copy()
        p[k % 3] += r if p[k % 3] + r <= 1.5 else -r
        mp.append(p)
    mp_x = np.array(mp)
    cell = 0.5 * r * (1 + 2 ** -20)
    ids, counts, _, _ = otm.support_search(dev(node_x), dev(mp_x), rs2, cell, 256)
    off, ref = orc.search(node_x, mp_x, rs2, cell)
    ids, counts = ids.cpu().numpy(), counts.cpu().numpy()
    for p in range(len(mp)):
        assert np.array_equal(ids[p, :counts[p]], ref[off[p]:off[p + 1]])


def rod_supports(orc, h=0.8e-3, L=8e-3):
    p = scenarios.taylor_rod(h=h, R=3.2e-3, L=L)
    off, ids = orc.search(p.node_x, p.mp_x, p.rs2, p.cell_size)
    return p, off, ids


def test_lme_vs_oracle_and_invariants(orc, otm):
    p, off, ref_ids = rod_supports(orc)
    S = 384
    ids, counts, _, st = otm.support_search(dev(p.node_x), dev(p.mp_x), p.rs2, p.cell_size, S)
    assert st.item() == 0
    tol = p.newton_tol * p.h
    shape, lam, iters, status = otm.lme(dev(p.node_x), dev(p.mp_x), ids, counts, p.beta, tol)
    assert status.item() == 0
    shape, lam = shape.cpu().numpy(), lam.cpu().numpy()
    counts = counts.cpu().numpy()
    for q in range(0, p.n_mps, 17):
        n = counts[q]
        xa = p.node_x[ref_ids[off[q]:off[q + 1]]]
        d = p.mp_x[q] - xa
        s_, N, dN, lr, _ = orc.lme(d, p.beta, tol)
        assert s_ == 0
        Ng, dNg = shape[q, :n, 0], shape[q, :n, 1:]
        assert rel(Ng, N) <= 1e-10
        assert rel(dNg, dN) <= 1e-10
        assert rel(lam[q], lr) <= 1e-8 or np.abs(lam[q] - lr).max() * p.h <= 1e-10
        assert abs(Ng.sum() - 1) <= 1e-12
        assert np.linalg.norm(Ng @ xa - p.mp_x[q]) / p.h <= 1e-12
        assert np.abs(dNg.sum(0)).max() * p.h <= 1e-12
        assert np.abs((xa - p.mp_x[q]).T @ dNg - np.eye(3)).max() <= 1e-12


def test_lme_outside_hull_reports_noconv(otm):
    X = np.random.default_rng(0).uniform(0, 1e-3, (30, 3))
    xp = np.array([[2e-3, 0.5e-3, 0.5e-3], [0.5e-3, 0.5e-3, 0.5e-3]])
    ids = np.tile(np.arange(30, dtype=np.int32), (2, 1))
    ids = np.pad(ids, ((0, 0), (0, 2)), constant_values=0)
    counts = np.array([30, 30], np.int32)
    shape, lam, iters, status = otm.lme(dev(X), dev(xp), dev(ids), dev(counts), 0.8e6, 1e-16, 50)
    assert status.item() == -4


@pytest.mark.parametrize("model", ["j2", "jc", "jc_frac"])
def test_return_map_vs_oracle(orc, otm, model):
    mat = {"j2": scenarios.copper_j2, "jc": scenarios.copper_jc, "jc_frac": scenarios.ti64_jc}[model]()
    rng = np.random.default_rng(5)
    n = 600
    dt = 5e-9
    dF = np.eye(3)[None] + rng.normal(0, 0.02, (n, 3, 3))
    F = dF @ (np.eye(3)[None] + rng.normal(0, 0.03, (n, 3, 3)))
    be = np.tile([1.0, 1, 1, 0, 0, 0], (n, 1)) + np.concatenate([rng.normal(0, 0.002, (n, 3)),
                                                                rng.normal(0, 0.001, (n, 3))], 1)
    ebar = np.abs(rng.normal(0, 0.05, n))
    T = 298 + np.abs(rng.normal(0, 80, n))
    dF_t, F_t = dev(dF.reshape(n, 9)), dev(F.reshape(n, 9))
    be_t, eb_t, T_t = dev(be.copy()), dev(ebar.copy()), dev(T.copy())
    sig, rate, failed, status = otm.return_map(mat, dt, dF_t, F_t, be_t, eb_t, T_t)
    assert status.item() == 0
    sig, be_g, eb_g, T_g = sig.cpu().numpy(), be_t.cpu().numpy(), eb_t.cpu().numpy(), T_t.cpu().numpy()
    failed = failed.cpu().numpy()
    ref = [orc.return_map(mat, dt, dF[k], be[k], ebar[k], T[k], np.linalg.det(F[k])) for k in range(n)]
    assert all(r[0] == 0 for r in ref)
    assert rel(sig, np.array([r[1] for r in ref])) <= 1e-10
    assert rel(be_g, np.array([r[2] for r in ref])) <= 1e-10
    assert rel(eb_g, np.array([r[3] for r in ref])) <= 1e-10
    assert rel(T_g, np.array([r[4] for r in ref])) <= 1e-10
    assert np.array_equal(failed.astype(bool), np.array([r[6] for r in ref]))
    assert (eb_g > ebar).any()     # the sample crosses the yield surface


def test_empty_point_sets(otm):
    """Zero points: the stand-alone search, LME and return map launch nothing and report OK."""
    nodes = dev(np.random.default_rng(0).uniform(0, 1, (50, 3)))
    empty = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    ids, counts, grid, status = otm.support_search(nodes, empty, 0.04, 0.2, max_support=64)
    torch.cuda.synchronize()
    assert ids.shape == (0, 64) and counts.numel() == 0 and int(status.item()) == 0
    shape, lam, iters, st = otm.lme(nodes, empty, ids, counts, beta=20.0, tol_abs=1e-14)
    torch.cuda.synchronize()
    assert shape.shape == (0, 64, 4) and int(st.item()) == 0
    z = torch.empty((0, 9), dtype=torch.float64, device="cuda")
    sig, rate, failed, st = otm.return_map(scenarios.copper_jc(), 1e-8, z, z.clone(),
                                           torch.empty((0, 6), dtype=torch.float64, device="cuda"),
                                           torch.empty(0, dtype=torch.float64, device="cuda"),
                                           torch.empty(0, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert sig.shape == (0, 6) and int(st.item()) == 0


def test_lme_degenerate_supports(orc, otm):
    """Degenerate cases of Eq. 14. One node, or a point on the far side of a plane of nodes: no
    finite lambda puts the point inside the hull, so the solve fails (LME_NOCONV) on both sides.
    Four affinely independent nodes: N are the barycentric coordinates and grad N the constant
    tetrahedron gradients for any beta (the consistency conditions fix them), on the GPU to 1e-12."""
    beta, tol = 0.8 / 0.01 ** 2, 1e-14 * 0.01
    tet = np.array([[0.0, 0.0, 0.0], [0.01, 0.0, 0.0], [0.0, 0.01, 0.0], [0.0, 0.0, 0.01]])
    cases = {"one_node": (tet[:1], np.array([0.002, 0.001, 0.0])),
             "outside_plane": (tet[1:], np.array([0.0, 0.0, -0.001])),
             "tet": (tet, np.array([0.002, 0.003, 0.001]))}
    for name, (nx, xp) in cases.items():
        n = nx.shape[0]
        ids = torch.full((1, 32), -1, dtype=torch.int32, device="cuda")
        ids[0, :n] = torch.arange(n, dtype=torch.int32, device="cuda")
        counts = torch.tensor([n], dtype=torch.int32, device="cuda")
        shape, lam, iters, st = otm.lme(dev(nx), dev(xp[None, :]), ids, counts, beta=beta, tol_abs=tol)
        torch.cuda.synchronize()
        so, No, dNo, _, _ = orc.lme(xp[None, :] - nx, beta, tol)
        if name == "tet":
            assert int(st.item()) == 0 and so == 0
            A = np.vstack([np.ones(4), nx.T])                      # barycentric: A N = (1, x_p)
            N = np.linalg.solve(A, np.concatenate([[1.0], xp]))
            G = np.linalg.inv(A)[:, 1:]                            # dN/dx_p, constant
            sh = shape.cpu().numpy()[0, :4]
            assert np.abs(sh[:, 0] - N).max() <= 1e-12
            assert np.abs(sh[:, 1:] - G).max() <= 1e-12 * np.abs(G).max()
            assert rel(sh[:, 0], No) <= 1e-12 and rel(sh[:, 1:], dNo) <= 1e-12
        else:
            assert int(st.item()) == -4 and so == -4, name


def test_internal_exp_against_cuda_exp():
    """The LME weights use the library's table-driven FP64 exp (after Tang 1989, its polynomial
    in double-float) on a scaled argument y = f 1024/ln2; it must agree with CUDA's exp of the
    same f to a few ulps over the whole range it serves, including the table's breakpoints and the
    range limits."""
    import ctypes as C
    import paper_2206_08772_gb300 as g
    L = g.load()
    rng = np.random.default_rng(11)
    K = 1024 / np.log(2)
    y = np.concatenate([rng.uniform(-700, 700, 200000) * K, rng.uniform(-40, 5, 800000) * K,
                        np.arange(-2048, 2049, dtype=np.float64), np.arange(-2048, 2049) + 0.5,
                        [0.0, -0.0, 1e-300, -1e-300, 700.0 * K, -700.0 * K, -1020.0 * 1024, 1021.0 * 1024 + 1023]])
    yt = torch.from_numpy(y).cuda()
    mine, ref = torch.empty_like(yt), torch.empty_like(yt)
    assert L.otm_exp_selftest(C.c_void_p(yt.data_ptr()), y.size, C.c_void_p(mine.data_ptr()),
                              C.c_void_p(ref.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    m, r = mine.cpu().numpy(), ref.cpu().numpy()
    relerr = np.abs(m - r) / r
    assert relerr.max() <= 1.1e-15, relerr.max()   # 5 ulp: 2.5 from the cubic, table and reference roundings
    # against numpy on the range the LME uses (the argument's own rounding: |f| 2^-53)
    f = y * (np.log(2) / 1024)
    sel = np.abs(f) <= 60
    assert (np.abs(m[sel] - np.exp(f[sel])) / np.exp(f[sel])).max() <= 2e-14
    # out of range: zero below, infinity above
    out = torch.tensor([-1.0e7, 1.0e7, -3.0e9, 3.0e9, -1e300, 1e300], dtype=torch.float64).cuda()
    mo, ro = torch.empty_like(out), torch.empty_like(out)
    assert L.otm_exp_selftest(C.c_void_p(out.data_ptr()), out.numel(), C.c_void_p(mo.data_ptr()),
                              C.c_void_p(ro.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    assert mo.cpu().numpy().tolist() == [0.0, np.inf, 0.0, np.inf, 0.0, np.inf]
