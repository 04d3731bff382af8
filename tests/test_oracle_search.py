"""Oracle pins for the linked-cell search (Algorithm 3): brute force on tiny clouds.

The brute force below evaluates every (point, node) pair with the same operation order as the
definition of the support (d^2 = ((dx*dx) + (dy*dy)) + (dz*dz) <= rs2, elementwise IEEE
doubles), independently of any cell structure, so the supports must agree bit for bit."""
import numpy as np
import pytest

import scenarios


def brute_force(node_x, mp_x, rs2):
    out = []
    for p in range(mp_x.shape[0]):
        d = mp_x[p][None, :] - node_x
        xx, yy, zz = d[:, 0] * d[:, 0], d[:, 1] * d[:, 1], d[:, 2] * d[:, 2]
        d2 = (xx + yy) + zz
        out.append(np.nonzero(d2 <= rs2)[0].astype(np.int32))
    return out


@pytest.mark.parametrize("seed,nn,nm,r", [(1, 300, 500, 0.21), (2, 2000, 800, 0.13), (3, 50, 200, 0.6)])
def test_search_matches_brute_force(orc, seed, nn, nm, r):
    node_x, mp_x = scenarios.random_cloud(nn, nm, seed)
    rs2 = r * r
    cell = 0.5 * r * (1 + 2 ** -20)
    off, ids = orc.search(node_x, mp_x, rs2, cell)
    ref = brute_force(node_x, mp_x, rs2)
    for p in range(nm):
        got = ids[off[p]:off[p + 1]]
        assert np.array_equal(got, ref[p]), p
        assert np.all(np.diff(got) > 0)


def test_search_ties_and_cell_faces(orc):
    """Nodes exactly at distance r_s (tie counts as inside) and points on cell faces."""
    r = 0.25
    rs2 = r * r
    cell = 0.5 * r * (1 + 2 ** -20)
    rng = np.random.default_rng(7)
    node_x = rng.uniform(0, 1, (400, 3))
    # points exactly r away along an axis from some nodes: d^2 == rs2 exactly in doubles
    mp = []
    for k in range(40):
        a = node_x[k].copy()
        axis = k % 3
        p = a.copy()
        p[axis] = a[axis] + r if a[axis] + r <= 1.5 else a[axis] - r
        mp.append(p)
    # points lying on cell faces of the grid (origin = node minimum)
    o = node_x.min(axis=0)
    for k in range(40):
        q = rng.uniform(0, 1, 3)
        q[k % 3] = o[k % 3] + (1 + k % 4) * cell
        mp.append(q)
    mp_x = np.array(mp)
    off, ids = orc.search(node_x, mp_x, rs2, cell)
    ref = brute_force(node_x, mp_x, rs2)
    ties = 0
    for p in range(mp_x.shape[0]):
        assert np.array_equal(ids[off[p]:off[p + 1]], ref[p])
        if p < 40:
            d = mp_x[p] - node_x[p]
            if ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) == rs2:
                ties += 1
                assert p in ids[off[p]:off[p + 1]]
    assert ties > 10


def test_search_point_outside_grid(orc):
    node_x, _ = scenarios.random_cloud(300, 1, 11)
    mp_x = np.array([[-0.1, 0.5, 0.5], [1.15, 1.1, -0.05], [5.0, 5.0, 5.0], [0.5, -0.2, 0.5]])
    r = 0.3
    off, ids = orc.search(node_x, mp_x, r * r, 0.5 * r * (1 + 2 ** -20))
    ref = brute_force(node_x, mp_x, r * r)
    for p in range(4):
        assert np.array_equal(ids[off[p]:off[p + 1]], ref[p])
    assert off[3] - off[2] == 0


def test_grid_is_counting_sort_by_cell_then_id(orc):
    node_x, _ = scenarios.random_cloud(3000, 1, 5)
    c = 0.07
    origin, dims, cs, srt = orc.grid(node_x, c)
    assert np.array_equal(origin, node_x.min(axis=0))
    hi = node_x.max(axis=0)
    assert np.array_equal(dims, (np.floor((hi - origin) / c) + 1).astype(np.int64))
    idx = np.clip(np.floor((node_x - origin) / c).astype(np.int64), 0, dims - 1)
    cell = (idx[:, 2] * dims[1] + idx[:, 1]) * dims[0] + idx[:, 0]
    order = np.lexsort((np.arange(node_x.shape[0]), cell))
    assert np.array_equal(srt, order)
    assert np.array_equal(cs, np.concatenate([[0], np.cumsum(np.bincount(cell, minlength=int(np.prod(dims))))]))


def test_taylor_rod_support_sizes(orc):
    """Interior supports hold ~(4/3) pi (r_s/h)^3 ~ 300 nodes; the surface fewer."""
    p = scenarios.taylor_rod(h=0.8e-3, R=3.2e-3, L=8e-3)
    off, ids = orc.search(p.node_x, p.mp_x, p.rs2, p.cell_size)
    cnt = np.diff(off)
    ref = brute_force(p.node_x, p.mp_x[:200], p.rs2)
    for k in range(200):
        assert np.array_equal(ids[off[k]:off[k + 1]], ref[k])
    assert cnt.max() <= 4.0 / 3.0 * np.pi * (np.sqrt(p.rs2) / p.h + 1) ** 3
    assert cnt.min() >= 40
