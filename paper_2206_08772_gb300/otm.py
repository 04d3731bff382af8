"""Python face of the CUDA OTM library: a handle that owns a torch-allocated device workspace.

PyTorch provides the device memory (one uint8 tensor) and the stream; every step of the
method runs in the library's kernels (include/otm.h). Argument marshalling only.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib
from ._lib import FIELD, Material, Params, Problem, check

_WIDTH = dict(node_x=(3, np.float64), node_du=(3, np.float64), node_mass=(1, np.float64),
              node_force=(3, np.float64), node_flags=(1, np.uint8), mp_x=(3, np.float64),
              F=(9, np.float64), dF=(9, np.float64), be=(6, np.float64), sigma=(6, np.float64),
              vol=(1, np.float64), ebar=(1, np.float64), T=(1, np.float64), rate=(1, np.float64),
              lam=(3, np.float64), support_count=(1, np.int32), newton_it=(1, np.int32),
              mp_gid=(1, np.int64), node_gid=(1, np.int64), kinv=(6, np.float64))


def material_struct(m) -> Material:
    s = Material()
    s.model = 0 if m.model == "j2" else 1
    s.fracture = 1 if m.fracture else 0
    for k in ("E", "nu", "rho0", "sigma_y0", "H", "A", "B", "n", "C", "m", "eps_dot0",
              "T_room", "T_melt", "chi", "cp"):
        setattr(s, k, float(getattr(m, k)))
    s.d1, s.d2, s.d3, s.d4, s.d5 = (float(v) for v in m.d)
    return s


def make_params(prob, precision: str = "fp64", max_support: int = 384) -> Params:
    """otm_params from a problem description (h, gamma, support_tol, dt, materials, contact)."""
    P = Params()
    P.h, P.beta, P.rs2, P.cell_size = prob.h, prob.beta, prob.rs2, prob.cell_size
    P.dt, P.T0, P.newton_tol, P.eps_stab = prob.dt, prob.T0, prob.newton_tol, prob.eps_stab
    P.max_newton = prob.max_newton
    P.n_materials = len(prob.materials)
    P.precision = _lib.PRECISION_MIXED if precision == "mixed" else _lib.PRECISION_FP64
    c = prob.contact
    P.wall, P.tool = int(c.wall), int(c.tool)
    P.allow_erode = int(any(m.fracture for m in prob.materials))
    for i in range(3):
        P.wall_p[i] = c.wall_point[i]
        P.wall_n[i] = c.wall_normal[i]
    P.tool_x0, P.tool_tip_y = c.tool_x0, c.tool_tip_y
    P.tool_rake, P.tool_clear = math.radians(c.tool_rake_deg), math.radians(c.tool_clearance_deg)
    P.tool_v, P.friction = c.tool_velocity, c.friction
    P.max_support = max_support
    P.max_insert = int(getattr(prob, "max_insert", 0))
    for i, m in enumerate(prob.materials):
        P.mat[i] = material_struct(m)
    return P


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


class OTM:
    """One OTM simulation on one GPU (Algorithm 1 per step, all in CUDA kernels)."""

    def __init__(self, prob, precision: str = "fp64", max_support: int = 384, device=None,
                 stream: torch.cuda.Stream | None = None, host_arrays: dict | None = None):
        L = _lib.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.precision = precision
        self.params = make_params(prob, precision, max_support)
        self.S = max_support
        nbytes = C.c_size_t(0)
        check(L.otm_workspace_bytes(prob.n_nodes, prob.n_mps, C.byref(self.params), C.byref(nbytes)),
              "otm_workspace_bytes")
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        a = host_arrays or {}
        self._host = [np.ascontiguousarray(a.get("node_x", prob.node_x), dtype=np.float64),
                      np.ascontiguousarray(a.get("node_du0", prob.node_du0), dtype=np.float64),
                      np.ascontiguousarray(a.get("node_flags", prob.node_flags), dtype=np.uint8),
                      np.ascontiguousarray(a.get("mp_x", prob.mp_x), dtype=np.float64),
                      np.ascontiguousarray(a.get("mp_vol", prob.mp_vol), dtype=np.float64),
                      np.ascontiguousarray(a.get("mp_mass", prob.mp_mass), dtype=np.float64),
                      np.ascontiguousarray(a.get("mp_material", prob.mp_material), dtype=np.int32)]
        pb = Problem(prob.n_nodes, prob.n_mps, *[h.ctypes.data for h in self._host])
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = L.otm_init(C.byref(pb), C.byref(self.params), C.c_void_p(self.stream.cuda_stream),
                            C.c_void_p(aligned), C.c_size_t(nbytes.value), C.byref(self._h))
        self._host = None
        check(st, "otm_init")
        self.n_nodes, self.n_mps = prob.n_nodes, prob.n_mps

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().otm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stepping
    def step(self, n: int = 1, sync: bool = True) -> int:
        L = _lib.load()
        st = L.otm_step(self._h, n) if sync else L.otm_step_async(self._h, n)
        return st

    def error(self):
        code, fid = C.c_int32(0), C.c_int64(0)
        check(_lib.load().otm_error_detail(self._h, C.byref(code), C.byref(fid)), "otm_error_detail")
        return code.value, fid.value

    def counts(self) -> dict:
        v = [C.c_int64() for _ in range(4)]
        check(_lib.load().otm_counts(self._h, *[C.byref(x) for x in v]), "otm_counts")
        return dict(n_nodes=v[0].value, n_mps=v[1].value, n_pairs=v[2].value, step=v[3].value)

    def launches(self) -> int:
        v = C.c_int64()
        check(_lib.load().otm_kernel_launches(self._h, C.byref(v)), "otm_kernel_launches")
        return v.value

    def phase_timing(self, on: bool = True):
        check(_lib.load().otm_phase_timing(self._h, 1 if on else 0), "otm_phase_timing")

    def phase_times(self) -> dict:
        """{phase: (total ms, launches)} since the previous call (synchronises)."""
        ms = (C.c_double * len(_lib.PHASES))()
        n = (C.c_int64 * len(_lib.PHASES))()
        check(_lib.load().otm_phase_times(self._h, ms, n), "otm_phase_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(_lib.PHASES)}

    # -- snapshots and the adjoint (device buffers are torch uint8 tensors, 256-byte aligned)
    def _aligned(self, nbytes):
        t = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        return t, (t.data_ptr() + 255) & ~255

    def snapshot(self, host: bool = False):
        """The complete state in a new buffer: device memory, or page-locked host memory."""
        L = _lib.load()
        nb = C.c_size_t(0)
        check(L.otm_snapshot_bytes(self._h, C.byref(nb)), "otm_snapshot_bytes")
        if host:
            buf = torch.empty(nb.value + 256, dtype=torch.uint8, pin_memory=True)
            ptr = (buf.data_ptr() + 255) & ~255
        else:
            buf, ptr = self._aligned(nb.value)
        check(L.otm_snapshot_save(self._h, C.c_void_p(ptr)), "otm_snapshot_save")
        return (buf, ptr)

    def keep_last_good(self, on: bool = True, host: bool = False):
        """otm_keep_last_good: every step first saves the state into a buffer kept by this object,
        and a failing step is undone (the state stays at the last good step)."""
        L = _lib.load()
        if not on:
            check(L.otm_keep_last_good(self._h, None, 0), "otm_keep_last_good")
            self._keep = None
            return
        nb = C.c_size_t(0)
        check(L.otm_snapshot_bytes(self._h, C.byref(nb)), "otm_snapshot_bytes")
        if host:
            buf = torch.empty(nb.value + 256, dtype=torch.uint8, pin_memory=True)
            ptr = (buf.data_ptr() + 255) & ~255
        else:
            buf, ptr = self._aligned(nb.value)
        check(L.otm_keep_last_good(self._h, C.c_void_p(ptr), nb.value), "otm_keep_last_good")
        self._keep = buf

    def restore(self, snap):
        check(_lib.load().otm_snapshot_load(self._h, C.c_void_p(snap[1])), "otm_snapshot_load")

    def adjoint_begin(self, xbar: np.ndarray):
        L = _lib.load()
        nb = C.c_size_t(0)
        check(L.otm_adjoint_bytes(self._h, C.byref(nb)), "otm_adjoint_bytes")
        self._adj_buf, self._adj_ptr = self._aligned(nb.value)
        xb = np.ascontiguousarray(xbar, dtype=np.float64)
        check(L.otm_adjoint_begin(self._h, C.c_void_p(self._adj_ptr), nb.value, _ptr(xb)), "otm_adjoint_begin")

    def freeze_topology(self, on: bool = True):
        """Skip the support search in the following steps (see otm_freeze_topology)."""
        check(_lib.load().otm_freeze_topology(self._h, int(on)), "otm_freeze_topology")

    def step_with_supports(self, counts: np.ndarray, ids: np.ndarray) -> int:
        """One step whose new supports are given: counts (n_mps,), ids (n_mps, max_support)."""
        c = np.ascontiguousarray(counts, dtype=np.int32)
        i = np.ascontiguousarray(ids, dtype=np.int32)
        if i.shape != (c.size, self.S):
            raise ValueError("ids must be (n_mps, max_support)")
        return _lib.load().otm_step_with_supports(self._h, _ptr(c), _ptr(i))

    def supports_export(self, offsets: torch.Tensor | None = None, ids: torch.Tensor | None = None):
        """The current supports as device tensors (offsets [n_mps + 1], ids [n_pairs], int32) in
        the library's row order; given buffers are filled (ids must be large enough)."""
        L = _lib.load()
        nm = self.counts()["n_mps"]
        if offsets is None:
            offsets = torch.empty(nm + 1, dtype=torch.int32, device=self.device)
        npairs = C.c_int64(0)
        if ids is None:
            probe = torch.empty(1, dtype=torch.int32, device=self.device)
            st = L.otm_supports_export(self._h, C.c_void_p(offsets.data_ptr()), C.c_void_p(probe.data_ptr()), 0,
                                       C.byref(npairs))
            if st not in (0, _lib.ERR_CAPACITY):
                check(st, "otm_supports_export")
            ids = torch.empty(max(npairs.value, 1), dtype=torch.int32, device=self.device)
        assert offsets.dtype == torch.int32 and ids.dtype == torch.int32 and offsets.numel() == nm + 1
        check(L.otm_supports_export(self._h, C.c_void_p(offsets.data_ptr()), C.c_void_p(ids.data_ptr()),
                                    ids.numel(), C.byref(npairs)), "otm_supports_export")
        return offsets, ids[:npairs.value]

    def step_with_supports_csr(self, offsets: torch.Tensor, ids: torch.Tensor) -> int:
        """One step whose new supports are the given device CSR (see otm_step_with_supports_csr)."""
        assert offsets.is_cuda and ids.is_cuda and offsets.dtype == torch.int32 and ids.dtype == torch.int32
        assert offsets.is_contiguous() and ids.is_contiguous()
        return _lib.load().otm_step_with_supports_csr(self._h, C.c_void_p(offsets.data_ptr()),
                                                      C.c_void_p(ids.data_ptr()), ids.numel())

    def grid_cells(self):
        """The linked-cell grid of the current node positions: (origin[3], dims[3], cell_start
        [n_cells + 1], sorted node indices [n_nodes])."""
        L = _lib.load()
        origin = np.zeros(3)
        dims = np.zeros(3, np.int32)
        nc = C.c_int64(0)
        check(L.otm_grid_cells(self._h, _ptr(origin), _ptr(dims), C.byref(nc), None, 0, None), "otm_grid_cells")
        cs = np.zeros(nc.value + 1, np.int32)
        srt = np.zeros(self.counts()["n_nodes"], np.int32)
        check(L.otm_grid_cells(self._h, _ptr(origin), _ptr(dims), C.byref(nc), _ptr(cs), cs.size, _ptr(srt)),
              "otm_grid_cells")
        return origin, dims, cs, srt

    def adjoint_step(self, next_snapshot=None):
        """One backward step from state n (held); next_snapshot (optional) holds state n+1."""
        nxt = C.c_void_p(next_snapshot[1]) if next_snapshot is not None else C.c_void_p(0)
        check(_lib.load().otm_adjoint_step(self._h, C.c_void_p(self._adj_ptr), nxt), "otm_adjoint_step")

    def adjoint_result(self, du0_ds: np.ndarray | None = None):
        """(theta_bar[6], dL/d du): gradients w.r.t. (A, B, n, C, m) and, with du0_ds (the
        derivative of the initial increments w.r.t. a scalar s), w.r.t. s (see otm_adjoint_result)."""
        thb = np.zeros(6)
        dub = np.zeros((self.counts()["n_nodes"], 3))
        d = None if du0_ds is None else np.ascontiguousarray(du0_ds, dtype=np.float64)
        if d is not None and d.shape != dub.shape:
            raise ValueError("du0_ds must be (n_nodes, 3)")
        check(_lib.load().otm_adjoint_result(self._h, C.c_void_p(self._adj_ptr),
                                             _ptr(d) if d is not None else None, _ptr(thb), _ptr(dub)),
              "otm_adjoint_result")
        return thb, dub

    def refresh(self) -> int:
        return _lib.load().otm_refresh(self._h)

    # -- state transfer (host copies, ID order)
    def get(self, name: str, out: np.ndarray | None = None) -> np.ndarray:
        c = None
        if name == "support_ids":
            shape, dt = (self.counts()["n_mps"], self.S), np.int32
        elif name == "shape":
            shape, dt = (self.counts()["n_mps"], self.S, 4), np.float64
        else:
            w, dt = _WIDTH[name]
            c = self.counts()
            rows = c["n_nodes"] if name.startswith("node") else c["n_mps"]
            shape = (rows, w) if w > 1 else (rows,)
        if out is None:
            out = np.empty(shape, dtype=dt)
        check(_lib.load().otm_state(self._h, FIELD[name], _ptr(out), out.nbytes), f"otm_state({name})")
        del c
        return out

    def get_rows(self, name: str, rows) -> np.ndarray:
        """Selected rows of a per-MP (or per-node) field; support rows ordered by node ID."""
        r = np.ascontiguousarray(rows, dtype=np.int64)
        if name == "support_ids":
            out = np.empty((r.size, self.S), np.int32)
        elif name == "shape":
            out = np.empty((r.size, self.S, 4), np.float64)
        else:
            w, dt = _WIDTH[name]
            out = np.empty((r.size, w) if w > 1 else (r.size,), dt)
        check(_lib.load().otm_state_rows(self._h, FIELD[name], _ptr(r), r.size, _ptr(out), out.nbytes),
              f"otm_state_rows({name})")
        return out

    def n_current(self):
        c = self.counts()
        return c["n_nodes"], c["n_mps"]

    def set(self, name: str, value: np.ndarray):
        w, dt = _WIDTH[name]
        v = np.ascontiguousarray(value, dtype=dt)
        check(_lib.load().otm_set_state(self._h, FIELD[name], _ptr(v), v.nbytes), f"otm_set_state({name})")

    def supports(self):
        """(offsets, ids) CSR of the current supports, IDs ascending per MP."""
        cnt = self.get("support_count").astype(np.int64)
        ids = self.get("support_ids")
        off = np.concatenate([[0], np.cumsum(cnt)])
        mask = np.arange(self.S)[None, :] < cnt[:, None]
        return off, ids[mask]

    def shape_functions(self):
        """(N, dN) per pair in CSR order."""
        cnt = self.get("support_count").astype(np.int64)
        sh = self.get("shape")
        mask = np.arange(self.S)[None, :] < cnt[:, None]
        s = sh[mask]
        return s[:, 0].copy(), s[:, 1:].copy()


# ---------------------------------------------------------------------- stand-alone kernels

def support_search(node_x: torch.Tensor, mp_x: torch.Tensor, rs2: float, cell_size: float,
                   max_support: int = 384, stream=None):
    """Device linked-cell search: returns (ids [nm, S] int32, counts [nm] int32, grid [6], status)."""
    L = _lib.load()
    assert node_x.is_cuda and node_x.dtype == torch.float64 and node_x.is_contiguous()
    assert mp_x.is_cuda and mp_x.dtype == torch.float64 and mp_x.is_contiguous()
    nn, nm = node_x.shape[0], mp_x.shape[0]
    dev = node_x.device
    nb = C.c_size_t(0)
    check(L.otm_search_scratch_bytes(nn, C.byref(nb)), "otm_search_scratch_bytes")
    scratch = torch.empty(nb.value + 256, dtype=torch.uint8, device=dev)
    sp = (scratch.data_ptr() + 255) & ~255
    ids = torch.full((nm, max_support), -1, dtype=torch.int32, device=dev)
    counts = torch.zeros(nm, dtype=torch.int32, device=dev)
    grid = torch.zeros(6, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    check(L.otm_support_search(C.c_void_p(node_x.data_ptr()), nn, C.c_void_p(mp_x.data_ptr()), nm, rs2,
                               cell_size, max_support, C.c_void_p(ids.data_ptr()),
                               C.c_void_p(counts.data_ptr()), C.c_void_p(sp), C.c_size_t(nb.value),
                               C.c_void_p(grid.data_ptr()), C.c_void_p(status.data_ptr()),
                               C.c_void_p(s.cuda_stream)), "otm_support_search")
    return ids, counts, grid, status


def lme(node_x: torch.Tensor, mp_x: torch.Tensor, ids: torch.Tensor, counts: torch.Tensor, beta: float,
        tol_abs: float, max_newton: int = 50, lam0: torch.Tensor | None = None, stream=None):
    """Device LME shape functions: returns (shape [nm, S, 4], lambda [nm, 3], iters [nm], status)."""
    L = _lib.load()
    nm, S = ids.shape
    dev = node_x.device
    lam = (lam0.clone() if lam0 is not None else torch.zeros(nm, 3, dtype=torch.float64, device=dev)).contiguous()
    shape = torch.zeros(nm, S, 4, dtype=torch.float64, device=dev)
    iters = torch.zeros(nm, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    check(L.otm_lme(C.c_void_p(node_x.data_ptr()), C.c_void_p(mp_x.data_ptr()), nm, C.c_void_p(ids.data_ptr()),
                    C.c_void_p(counts.data_ptr()), S, beta, tol_abs, max_newton, C.c_void_p(lam.data_ptr()),
                    C.c_void_p(shape.data_ptr()), C.c_void_p(iters.data_ptr()), C.c_void_p(status.data_ptr()),
                    C.c_void_p(s.cuda_stream)), "otm_lme")
    return shape, lam, iters, status


def return_map(mat, dt: float, dF: torch.Tensor, F_new: torch.Tensor, be: torch.Tensor, ebar: torch.Tensor,
               T: torch.Tensor, stream=None):
    """Device constitutive update of n points (in place on be, ebar, T); returns (sigma, rate, failed, status)."""
    L = _lib.load()
    n = dF.shape[0]
    dev = dF.device
    m = material_struct(mat) if not isinstance(mat, Material) else mat
    sigma = torch.zeros(n, 6, dtype=torch.float64, device=dev)
    rate = torch.zeros(n, dtype=torch.float64, device=dev)
    failed = torch.zeros(n, dtype=torch.uint8, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    check(L.otm_return_map(C.byref(m), dt, n, C.c_void_p(dF.data_ptr()), C.c_void_p(F_new.data_ptr()),
                           C.c_void_p(be.data_ptr()), C.c_void_p(ebar.data_ptr()), C.c_void_p(T.data_ptr()),
                           C.c_void_p(sigma.data_ptr()), C.c_void_p(rate.data_ptr()),
                           C.c_void_p(failed.data_ptr()), C.c_void_p(status.data_ptr()),
                           C.c_void_p(s.cuda_stream)), "otm_return_map")
    return sigma, rate, failed, status
