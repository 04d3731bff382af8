"""Serial FP64 CPU oracle of the OTM explicit step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
this package. The product path (the CUDA library and its binding) never touches it, and it
imports nothing from the product: it is a plain C file compiled with gcc and driven through
ctypes.

Functions and the passages they follow (paper: arXiv 2206.08772):
  search / grid_info / grid_cells  -- Algorithm 3 (linked-cell search), Sec. 3.5
  lme                              -- Eq. 14 (local max-ent shape functions, Newton for lambda)
  kinematics                       -- Eq. 9, Eq. 11 (MP position and F increment)
  return_map                       -- Sec. 4.1 J2 finite plasticity, Sec. 4.2 Johnson-Cook flow,
                                      heating and fracture
  Sim                              -- Algorithm 1, the whole explicit step (Eq. 4-13 + the above)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "otm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OK = 0
ERR_ARG, ERR_OOM, ERR_LME_NOCONV, ERR_JACOBIAN = -1, -3, -4, -5
ERR_NONFINITE, ERR_RETURNMAP_NOCONV, ERR_CAPACITY = -6, -7, -8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no floating-point contraction) twice: serial
    (liboracle.so, the reference) and with OpenMP over independent material points and nodes
    (liboracle_omp.so: the same arithmetic per point, so the same results)."""
    for lib_path, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
            tmp = lib_path + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, lib_path)
    return _LIB


class Material(C.Structure):
    _fields_ = [("model", C.c_int32), ("fracture", C.c_int32),
                ("E", C.c_double), ("nu", C.c_double), ("rho0", C.c_double),
                ("sigma_y0", C.c_double), ("H", C.c_double),
                ("A", C.c_double), ("B", C.c_double), ("n", C.c_double), ("C", C.c_double),
                ("m", C.c_double), ("eps_dot0", C.c_double),
                ("T_room", C.c_double), ("T_melt", C.c_double), ("chi", C.c_double), ("cp", C.c_double),
                ("d1", C.c_double), ("d2", C.c_double), ("d3", C.c_double), ("d4", C.c_double),
                ("d5", C.c_double)]


class Params(C.Structure):
    _fields_ = [("h", C.c_double), ("beta", C.c_double), ("rs2", C.c_double),
                ("cell_size", C.c_double), ("dt", C.c_double), ("T0", C.c_double),
                ("newton_tol", C.c_double), ("eps_stab", C.c_double),
                ("max_newton", C.c_int32), ("n_materials", C.c_int32),
                ("wall", C.c_int32), ("tool", C.c_int32),
                ("wall_p", C.c_double * 3), ("wall_n", C.c_double * 3),
                ("tool_x0", C.c_double), ("tool_tip_y", C.c_double), ("tool_rake", C.c_double),
                ("tool_clear", C.c_double), ("tool_v", C.c_double), ("friction", C.c_double),
                ("allow_insert", C.c_int32), ("allow_erode", C.c_int32),
                ("mat", Material * 4)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib(omp: bool = False):
    """The serial oracle library, or (omp=True) its OpenMP build."""
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is None:
            build()
            L = _bind(C.CDLL(_LIB_OMP if omp else _LIB))
            if omp:
                _lib_omp = L
            else:
                _lib = L
    return _lib_omp if omp else _lib


def _bind(L):
    """ctypes signatures of the oracle's entry points."""
    L.orc_lme.restype = C.c_int
    L.orc_lme.argtypes = [C.c_int64, _P, C.c_double, C.c_double, C.c_int32, _P, _P, _P, _P]
    L.orc_return_map.restype = C.c_int
    L.orc_return_map.argtypes = [_P, C.c_double, _P, _P, C.c_double, C.c_double, C.c_double,
                                 _P, _P, _P, _P, _P, _P]
    L.orc_search.restype = C.c_int64
    L.orc_search.argtypes = [C.c_int64, _P, C.c_int64, _P, C.c_double, C.c_double, _P, _P,
                             C.c_int64]
    L.orc_grid_info.restype = C.c_int
    L.orc_grid_info.argtypes = [C.c_int64, _P, C.c_double, _P, _P]
    L.orc_grid_cells.restype = C.c_int
    L.orc_grid_cells.argtypes = [C.c_int64, _P, C.c_double, C.c_int64, _P, _P]
    L.orc_kinematics.restype = None
    L.orc_kinematics.argtypes = [C.c_int64, _P, _P, _P, _P, _P, _P, _P]
    L.orc_sim_create.restype = _P
    L.orc_sim_create.argtypes = [_P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, _P]
    L.orc_sim_destroy.restype = None
    L.orc_sim_destroy.argtypes = [_P]
    L.orc_sim_step.restype = C.c_int
    L.orc_sim_step.argtypes = [_P]
    L.orc_sim_counts.restype = None
    L.orc_sim_counts.argtypes = [_P] + [_P] * 6
    L.orc_sim_get.restype = C.c_int
    L.orc_sim_get.argtypes = [_P, C.c_int32, _P, C.c_int64]
    L.orc_sim_set.restype = C.c_int
    L.orc_sim_set.argtypes = [_P, C.c_int32, _P, C.c_int64]
    L.orc_sim_refresh.restype = C.c_int
    L.orc_sim_refresh.argtypes = [_P]
    L.orc_lme_backward.restype = C.c_int
    L.orc_lme_backward.argtypes = [C.c_int64, _P, _P, _P, _P, C.c_double, _P, _P, _P]
    L.orc_return_map_backward.restype = C.c_int
    L.orc_return_map_backward.argtypes = [_P, C.c_double, _P, _P, C.c_double, C.c_double, C.c_double,
                                          _P, _P, C.c_double, C.c_double, _P, _P, _P, _P, _P, _P]
    L.orc_sim_clone.restype = _P
    L.orc_sim_clone.argtypes = [_P]
    L.orc_adj_create.restype = _P
    L.orc_adj_create.argtypes = [_P, _P]
    L.orc_adj_destroy.restype = None
    L.orc_adj_destroy.argtypes = [_P]
    L.orc_adj_result.restype = None
    L.orc_adj_result.argtypes = [_P, _P, _P]
    L.orc_sim_row.restype = C.c_int64
    L.orc_sim_row.argtypes = [_P, C.c_int64, _P, _P, _P, C.c_int64]
    L.orc_tool_contact.restype = None
    L.orc_tool_contact.argtypes = [_P, C.c_double, _P, _P]
    L.orc_adjoint_step.restype = C.c_int
    L.orc_adjoint_step.argtypes = [_P, _P, _P]
    assert L.orc_sizeof_params() == C.sizeof(Params)
    assert L.orc_sizeof_material() == C.sizeof(Material)
    return L


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


def material_struct(m) -> Material:
    """ctypes material from a scenarios.Material."""
    s = Material()
    s.model = 0 if m.model == "j2" else 1
    s.fracture = 1 if m.fracture else 0
    for k in ("E", "nu", "rho0", "sigma_y0", "H", "A", "B", "n", "C", "m", "eps_dot0",
              "T_room", "T_melt", "chi", "cp"):
        setattr(s, k, float(getattr(m, k)))
    s.d1, s.d2, s.d3, s.d4, s.d5 = (float(v) for v in m.d)
    return s


def params_struct(prob) -> Params:
    """ctypes parameters from a scenarios.Problem (all derived values taken from the problem)."""
    P = Params()
    P.h, P.beta, P.rs2, P.cell_size = prob.h, prob.beta, prob.rs2, prob.cell_size
    P.dt, P.T0, P.newton_tol, P.eps_stab = prob.dt, prob.T0, prob.newton_tol, prob.eps_stab
    P.max_newton = prob.max_newton
    P.n_materials = len(prob.materials)
    c = prob.contact
    P.wall, P.tool = int(c.wall), int(c.tool)
    for i in range(3):
        P.wall_p[i] = c.wall_point[i]
        P.wall_n[i] = c.wall_normal[i]
    P.tool_x0, P.tool_tip_y = c.tool_x0, c.tool_tip_y
    P.tool_rake, P.tool_clear = math.radians(c.tool_rake_deg), math.radians(c.tool_clearance_deg)
    P.tool_v, P.friction = c.tool_velocity, c.friction
    P.allow_insert = int(prob.max_insert)
    P.allow_erode = int(any(m.fracture for m in prob.materials))
    for i, m in enumerate(prob.materials):
        P.mat[i] = material_struct(m)
    return P


# ------------------------------------------------------------------ standalone pieces

def lme(d: np.ndarray, beta: float, tol_r: float, max_it: int = 50, lam0=None):
    """LME shape functions of one point from d_a = x_p - x_a (n x 3). Returns
    (status, N, dN, lambda, iterations)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    lam = np.zeros(3) if lam0 is None else np.array(lam0, dtype=np.float64)
    N = np.zeros(n)
    dN = np.zeros((n, 3))
    it = C.c_int32(0)
    st = lib().orc_lme(n, _ptr(d), beta, tol_r, max_it, _ptr(lam), _ptr(N), _ptr(dN), C.byref(it))
    return st, N, dN, lam, it.value


def return_map(mat, dt: float, dF: np.ndarray, be_n: np.ndarray, ebar_n: float, T_n: float, J: float):
    """One-MP constitutive update. Returns (status, sigma6, be6, ebar, T, q, failed)."""
    m = material_struct(mat) if not isinstance(mat, Material) else mat
    dF = np.ascontiguousarray(dF, dtype=np.float64).reshape(9)
    be_n = np.ascontiguousarray(be_n, dtype=np.float64).reshape(6)
    sig = np.zeros(6)
    be = np.zeros(6)
    eb, T, q = C.c_double(0), C.c_double(0), C.c_double(0)
    failed = C.c_int32(0)
    st = lib().orc_return_map(C.byref(m), dt, _ptr(dF), _ptr(be_n), ebar_n, T_n, J, _ptr(sig), _ptr(be),
                              C.byref(eb), C.byref(T), C.byref(q), C.byref(failed))
    return st, sig, be, eb.value, T.value, q.value, bool(failed.value)


def lme_backward(d, N, G, lam, beta, Nb, Gb):
    """Adjoint of the LME shape functions of one point: dL/dd given dL/dN and dL/d(grad N)."""
    d = np.ascontiguousarray(d, np.float64)
    N = np.ascontiguousarray(N, np.float64)
    G = np.ascontiguousarray(G, np.float64)
    lam = np.ascontiguousarray(lam, np.float64)
    Nb = np.ascontiguousarray(Nb, np.float64)
    Gb = np.ascontiguousarray(Gb, np.float64)
    db = np.zeros_like(d)
    st = lib().orc_lme_backward(d.shape[0], _ptr(d), _ptr(N), _ptr(G), _ptr(lam), beta, _ptr(Nb), _ptr(Gb), _ptr(db))
    if st != OK:
        raise RuntimeError(f"lme_backward {st}")
    return db


def return_map_backward(mat, dt, dF, be_n, ebar_n, T_n, J, sigb, beb, ebb, Tb):
    """Adjoint of one MP's return map. Returns (dFb 3x3, be_nb 6, ebar_nb, T_nb, Jb, thetab 5)."""
    m = material_struct(mat) if not isinstance(mat, Material) else mat
    dF = np.ascontiguousarray(dF, np.float64).reshape(9)
    be_n = np.ascontiguousarray(be_n, np.float64)
    sigb = np.ascontiguousarray(sigb, np.float64)
    beb = np.ascontiguousarray(beb, np.float64)
    dFb, be_nb, thb = np.zeros(9), np.zeros(6), np.zeros(5)
    ebn, Tn, Jb = C.c_double(0), C.c_double(0), C.c_double(0)
    st = lib().orc_return_map_backward(C.byref(m), dt, _ptr(dF), _ptr(be_n), ebar_n, T_n, J, _ptr(sigb), _ptr(beb),
                                       ebb, Tb, _ptr(dFb), _ptr(be_nb), C.byref(ebn), C.byref(Tn), C.byref(Jb),
                                       _ptr(thb))
    if st != OK:
        raise RuntimeError(f"return_map_backward {st}")
    return dFb.reshape(3, 3), be_nb, ebn.value, Tn.value, Jb.value, thb


def search(node_x: np.ndarray, mp_x: np.ndarray, rs2: float, cell_size: float, cap: int | None = None):
    """Linked-cell supports: (offsets int64[nm+1], ids int32[P]), IDs ascending per point."""
    node_x = np.ascontiguousarray(node_x, dtype=np.float64)
    mp_x = np.ascontiguousarray(mp_x, dtype=np.float64)
    nm = mp_x.shape[0]
    if cap is None:
        cap = max(1024, 600 * nm)
    off = np.zeros(nm + 1, np.int64)
    ids = np.zeros(cap, np.int32)
    tot = lib().orc_search(node_x.shape[0], _ptr(node_x), nm, _ptr(mp_x), rs2, cell_size, _ptr(off),
                           _ptr(ids), cap)
    if tot < 0:
        raise RuntimeError(f"oracle search failed: {tot}")
    return off, ids[:tot].copy()


def grid(node_x: np.ndarray, cell_size: float):
    """Linked-cell grid: (origin[3], dims[3], cell_start[n_cells+1], sorted node IDs)."""
    node_x = np.ascontiguousarray(node_x, dtype=np.float64)
    origin = np.zeros(3)
    dims = np.zeros(3, np.int64)
    st = lib().orc_grid_info(node_x.shape[0], _ptr(node_x), cell_size, _ptr(origin), _ptr(dims))
    if st != OK:
        raise RuntimeError(f"oracle grid failed: {st}")
    nc = int(np.prod(dims))
    cs = np.zeros(nc + 1, np.int64)
    srt = np.zeros(node_x.shape[0], np.int32)
    st = lib().orc_grid_cells(node_x.shape[0], _ptr(node_x), cell_size, nc, _ptr(cs), _ptr(srt))
    if st != OK:
        raise RuntimeError(f"oracle grid failed: {st}")
    return origin, dims, cs, srt


def tool_contact(prob, t_next: float, du: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The oracle's tool contact (Sec. 4.2) applied to one node: returns the new position."""
    P = params_struct(prob)
    du = np.ascontiguousarray(du, np.float64)
    out = np.ascontiguousarray(x, np.float64).copy()
    lib().orc_tool_contact(C.byref(P), t_next, _ptr(du), _ptr(out))
    return out


def kinematics(ids, N, dN, node_x, node_du):
    ids = np.ascontiguousarray(ids, np.int32)
    N = np.ascontiguousarray(N, np.float64)
    dN = np.ascontiguousarray(dN, np.float64)
    node_x = np.ascontiguousarray(node_x, np.float64)
    node_du = np.ascontiguousarray(node_du, np.float64)
    xp = np.zeros(3)
    dF = np.zeros(9)
    lib().orc_kinematics(ids.size, _ptr(ids), _ptr(N), _ptr(dN), _ptr(node_x), _ptr(node_du), _ptr(xp),
                         _ptr(dF))
    return xp, dF.reshape(3, 3)


# ------------------------------------------------------------------ the whole step

FIELDS = dict(node_x=(0, 3, np.float64), node_du=(1, 3, np.float64), node_mass=(2, 1, np.float64),
              node_force=(3, 3, np.float64), mp_x=(4, 3, np.float64), F=(5, 9, np.float64),
              be=(6, 6, np.float64), sigma=(7, 6, np.float64), vol=(8, 1, np.float64),
              ebar=(9, 1, np.float64), T=(10, 1, np.float64), lam=(11, 3, np.float64),
              offsets=(12, 1, np.int64), ids=(13, 1, np.int32), N=(14, 1, np.float64),
              dN=(15, 3, np.float64), node_gid=(16, 1, np.int64), mp_gid=(17, 1, np.int64),
              newton_it=(18, 1, np.int32), rate=(19, 1, np.float64), mp_x_prev=(20, 3, np.float64),
              node_x_prev=(21, 3, np.float64), dF=(22, 9, np.float64))


class Sim:
    """The oracle's whole explicit OTM simulation (Algorithm 1) on a scenarios.Problem."""

    def __init__(self, prob, params: Params | None = None, omp: bool = False):
        """omp=True runs the OpenMP build (same results, all host cores)."""
        self._L = L = lib(omp)
        self.prob = prob
        self.params = params if params is not None else params_struct(prob)
        a = [np.ascontiguousarray(v) for v in (
            prob.node_x.astype(np.float64), prob.node_du0.astype(np.float64),
            prob.node_flags.astype(np.uint8), prob.mp_x.astype(np.float64),
            prob.mp_vol.astype(np.float64), prob.mp_mass.astype(np.float64),
            prob.mp_material.astype(np.int32))]
        self._h = L.orc_sim_create(C.byref(self.params), prob.n_nodes, prob.n_mps, *[_ptr(v) for v in a])
        if not self._h:
            raise MemoryError("oracle sim create failed")

    def __del__(self):
        if getattr(self, "_h", None):
            self._L.orc_sim_destroy(self._h)
            self._h = None

    def counts(self):
        v = [C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32(), C.c_int64()]
        self._L.orc_sim_counts(self._h, *[C.byref(x) for x in v])
        return dict(n_nodes=v[0].value, n_mps=v[1].value, n_pairs=v[2].value, step=v[3].value,
                    err=v[4].value, err_id=v[5].value)

    def step(self, n: int = 1) -> int:
        for _ in range(n):
            st = self._L.orc_sim_step(self._h)
            if st != OK:
                return st
        return OK

    def get(self, name: str) -> np.ndarray:
        code, width, dt = FIELDS[name]
        c = self.counts()
        if name.startswith("node"):
            rows = c["n_nodes"]
        elif name == "offsets":
            rows = c["n_mps"] + 1
        elif name in ("ids", "N", "dN"):
            rows = c["n_pairs"]
        else:
            rows = c["n_mps"]
        out = np.zeros((rows, width) if width > 1 else (rows,), dtype=dt)
        st = self._L.orc_sim_get(self._h, code, _ptr(out), out.nbytes)
        if st != OK:
            raise RuntimeError(f"get {name}: {st}")
        return out

    def row(self, p: int, cap: int = 4096):
        """MP p's support: (node IDs ascending, N, grad N)."""
        ids = np.zeros(cap, np.int32)
        N = np.zeros(cap)
        dN = np.zeros((cap, 3))
        n = self._L.orc_sim_row(self._h, int(p), _ptr(ids), _ptr(N), _ptr(dN), cap)
        if n < 0:
            raise IndexError(p)
        return ids[:n].copy(), N[:n].copy(), dN[:n].copy()

    def set(self, name: str, value: np.ndarray):
        code, width, dt = FIELDS[name]
        v = np.ascontiguousarray(value, dtype=dt)
        st = self._L.orc_sim_set(self._h, code, _ptr(v), v.nbytes)
        if st != OK:
            raise RuntimeError(f"set {name}: {st}")

    def refresh(self) -> int:
        return self._L.orc_sim_refresh(self._h)

    def clone(self) -> "Sim":
        c = Sim.__new__(Sim)
        c.prob, c.params, c._L = self.prob, self.params, self._L
        c._h = self._L.orc_sim_clone(self._h)
        if not c._h:
            raise MemoryError("oracle clone failed")
        return c


# ------------------------------------------------------------------ reference adjoint

THETA_NAMES = ("A", "B", "n", "C", "m", "v0")


def objectives(x: np.ndarray, node_mass: np.ndarray, h: float):
    """Final rod length (max z over nodes with mass) and footprint radius (max radial distance
    over nodes within 1e-3 h of the wall), with the arg-max nodes and d(objective)/d(x)."""
    act = np.nonzero(node_mass > 0)[0]
    i_len = int(act[np.argmax(x[act, 2])])
    foot = np.nonzero(x[:, 2] <= 1e-3 * h)[0]
    rad = np.sqrt(x[foot, 0] ** 2 + x[foot, 1] ** 2)
    i_rad = int(foot[np.argmax(rad)])
    L = float(x[i_len, 2])
    R = float(np.sqrt(x[i_rad, 0] ** 2 + x[i_rad, 1] ** 2))
    gL = np.zeros_like(x)
    gL[i_len, 2] = 1.0
    gR = np.zeros_like(x)
    gR[i_rad, 0] = x[i_rad, 0] / R
    gR[i_rad, 1] = x[i_rad, 1] / R
    return (L, R), (gL, gR), (i_len, i_rad)


def reference_adjoint(prob, steps: int):
    """FP64 CPU reverse-mode gradients of (final length, footprint radius) with respect to
    (A, B, n, C, m, v0), topology / contact set / plastic set frozen at the base trajectory.
    Returns (values, gradients [2 x 6], arg-max nodes)."""
    L = lib()
    sims = [Sim(prob)]
    for _ in range(steps):
        nxt = sims[-1].clone()
        st = nxt.step(1)
        if st != OK:
            raise RuntimeError(f"oracle step failed: {st}")
        sims.append(nxt)
    xK = sims[-1].get("node_x")
    vals, seeds, argm = objectives(xK, sims[-1].get("node_mass"), prob.h)
    grads = np.zeros((2, 6))
    for o, seed in enumerate(seeds):
        seed = np.ascontiguousarray(seed)
        a = L.orc_adj_create(sims[-1]._h, _ptr(seed))
        try:
            for k in range(steps - 1, -1, -1):
                st = L.orc_adjoint_step(sims[k]._h, sims[k + 1]._h, a)
                if st != OK:
                    raise RuntimeError(f"adjoint step {k} failed: {st}")
            thb = np.zeros(5)
            dub = np.zeros((sims[0].counts()["n_nodes"], 3))
            L.orc_adj_result(a, _ptr(thb), _ptr(dub))
        finally:
            L.orc_adj_destroy(a)
        grads[o, :5] = thb
        grads[o, 5] = -prob.dt * dub[:, 2].sum()   # du_0 = (0, 0, -v0 dt) on every node
    return vals, grads, argm
