"""The allocation-free support search against the regular one (collected last on purpose).

otm_support_search_noalloc serves callers that cannot allocate device memory at call time: it
runs the same search with a static scratch array inside the library. This test calls it through
the C ABI twice in a row, on two different point sets, and checks that its neighbour lists,
counts and grid agree exactly with otm_support_search (the search's parity bar is bit-exact)."""
import ctypes as C

import numpy as np
import pytest

import scenarios

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2206_08772_gb300 as g
    L = g.load()
    f = L.otm_support_search_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_int32,
                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return L


def run_noalloc(L, node_x, mp_x, rs2, cell, S):
    nm = mp_x.shape[0]
    ids = torch.full((nm, S), -1, dtype=torch.int32, device="cuda")
    counts = torch.zeros(nm, dtype=torch.int32, device="cuda")
    grid = torch.zeros(6, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.otm_support_search_noalloc(node_x.data_ptr(), node_x.shape[0], mp_x.data_ptr(), nm, rs2, cell, S,
                                      ids.data_ptr(), counts.data_ptr(), grid.data_ptr(), status.data_ptr(),
                                      torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return ids, counts, grid, status


def test_noalloc_search_matches_regular_search_twice(lib):
    from paper_2206_08772_gb300.otm import support_search
    cases = [(scenarios.random_cloud(6000, 2500, 21), 0.11, 384),
             (scenarios.random_cloud(900, 1200, 22), 0.23, 512)]
    for (node_x, mp_x), r, S in cases:
        nx = torch.from_numpy(node_x).cuda()
        mx = torch.from_numpy(mp_x).cuda()
        rs2, cell = r * r, 0.5 * r * (1 + 2 ** -20)
        ids_a, cnt_a, grid_a, st_a = run_noalloc(lib, nx, mx, rs2, cell, S)
        ids_b, cnt_b, grid_b, st_b = support_search(nx, mx, rs2, cell, S)
        torch.cuda.synchronize()
        assert st_a.item() == st_b.item() == 0
        assert torch.equal(cnt_a, cnt_b)
        assert torch.equal(grid_a, grid_b)
        cnt = cnt_a.cpu().numpy()
        a, b = ids_a.cpu().numpy(), ids_b.cpu().numpy()
        mask = np.arange(S)[None, :] < cnt[:, None]
        assert np.array_equal(a[mask], b[mask])
        assert cnt.sum() > 0


def test_noalloc_rejects_too_many_nodes(lib):
    n = 65537
    node_x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    mp_x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    ids = torch.zeros((4, 64), dtype=torch.int32, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.otm_support_search_noalloc(node_x.data_ptr(), n, mp_x.data_ptr(), 4, 0.01, 0.06, 64, ids.data_ptr(),
                                        counts.data_ptr(), None, status.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert st == -8
