"""Seeded synthetic inputs for the OTM material-point update (shared by the oracle and the GPU path).

This module generates problems only: node and material-point clouds, their masses, volumes,
flags and the run parameters. It contains none of the method's arithmetic (no shape
functions, no search, no constitutive update); both the serial oracle and the CUDA library
consume its output.

Geometry follows the paper's set-up for both applications: the initial domain is meshed
into tetrahedra and one material point is placed at each tetrahedron's barycentre, after
which the mesh is discarded (Sec. 4.1, "Numerical Evaluation"). Here the tetrahedra come
from a structured hexahedral grid of spacing h, each hex split into six Kuhn tetrahedra
around its 0-7 diagonal (corner bit 1 = +x, 2 = +y, 4 = +z).

Jitter: interior nodes (all eight adjacent hexes present) are displaced by U(-0.01 h,
0.01 h) per coordinate, drawn from splitmix64(seed) in node-ID order, x then y then z.
Boundary nodes stay on the flat faces.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# node flags (bit field, same meaning on both sides)
FLAG_FIXED = 1          # Dirichlet node: displacement increment held at zero

# Kuhn split of a hex into 6 tets around the 0-7 diagonal (corner bit 1=x, 2=y, 4=z)
KUHN_TETS = np.array([(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7),
                      (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)], dtype=np.int64)

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """First n outputs of splitmix64 started at `seed` (Steele, Lea, Flood 2014)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Material:
    """Elastic constants and one of two hardening laws (J2 linear or Johnson-Cook)."""
    E: float
    nu: float
    rho0: float
    model: str = "j2"          # "j2" (linear isotropic hardening) or "jc" (Johnson-Cook)
    sigma_y0: float = 0.0      # J2: initial yield stress
    H: float = 0.0             # J2: linear hardening modulus
    A: float = 0.0             # JC flow stress parameters
    B: float = 0.0
    n: float = 1.0
    C: float = 0.0
    m: float = 1.0
    eps_dot0: float = 1.0      # JC reference plastic strain rate [1/s]
    T_room: float = 298.0      # [K]
    T_melt: float = 1356.0     # [K]
    chi: float = 0.0           # Taylor-Quinney coefficient (adiabatic heating)
    cp: float = 385.0          # heat capacity [J/(kg K)]
    fracture: bool = False     # Johnson-Cook fracture -> erosion
    d: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)

    @property
    def K(self) -> float:
        return self.E / (3.0 * (1.0 - 2.0 * self.nu))

    @property
    def mu(self) -> float:
        return self.E / (2.0 * (1.0 + self.nu))

    @property
    def wave_speed(self) -> float:
        return math.sqrt((self.K + 4.0 * self.mu / 3.0) / self.rho0)


@dataclass
class Contact:
    """Rigid contact: an optional frictionless wall and an optional moving tool."""
    wall: bool = False
    wall_point: tuple = (0.0, 0.0, 0.0)
    wall_normal: tuple = (0.0, 0.0, 1.0)
    tool: bool = False
    tool_x0: float = 0.0           # rake-face x position at t = 0
    tool_tip_y: float = 0.0        # cutting-edge height
    tool_rake_deg: float = 0.0
    tool_clearance_deg: float = 7.0
    tool_velocity: float = 0.0     # tool speed along -x [m/s]
    friction: float = 0.0


@dataclass
class Problem:
    """A complete OTM problem: arrays (SI units) + parameters."""
    name: str
    h: float
    node_x: np.ndarray          # (n_nodes, 3) float64
    node_flags: np.ndarray      # (n_nodes,) uint8
    node_du0: np.ndarray        # (n_nodes, 3) float64 initial displacement increment
    mp_x: np.ndarray            # (n_mps, 3) float64
    mp_vol: np.ndarray          # (n_mps,) float64
    mp_mass: np.ndarray         # (n_mps,) float64
    mp_material: np.ndarray     # (n_mps,) int32
    materials: list
    contact: Contact
    dt: float
    gamma: float = 0.8
    support_tol: float = 1e-6
    T0: float = 298.0
    newton_tol: float = 1e-14     # LME residual tolerance, relative to h
    max_newton: int = 50
    eps_stab: float = 0.0
    max_insert: int = 0           # node slots for insertion over the run (0: insertion off)
    steps: int = 100
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.node_x.shape[0])

    @property
    def n_mps(self) -> int:
        return int(self.mp_x.shape[0])

    @property
    def beta(self) -> float:
        return self.gamma / (self.h * self.h)

    @property
    def rs2(self) -> float:
        """Squared support radius: exp(-beta d^2) >= tol  <=>  d^2 <= ln(1/tol)/beta.

        Computed once here so that both implementations receive the same bits."""
        return math.log(1.0 / self.support_tol) / self.beta

    @property
    def cell_size(self) -> float:
        """Linked-cell edge: a hair above half the support radius (search stencil of +-2 cells)."""
        return 0.5 * math.sqrt(self.rs2) * (1.0 + 2.0 ** -20)


def _hex_mesh(keep: np.ndarray, h: float, origin: tuple, seed: int):
    """Nodes, tets and MPs of the kept cells of a structured grid.

    keep: bool array (nk, nj, ni) over cells. Returns node_x, node_cell_counts-derived
    interior mask, MP arrays. Node IDs: lexicographic (k, j, i) over the corners that touch a
    kept cell; MP ID = 6 * (kept-cell rank in (k, j, i) order) + tet."""
    nk, nj, ni = keep.shape
    # corners touched by kept cells, and how many kept cells touch each corner
    touch = np.zeros((nk + 1, nj + 1, ni + 1), dtype=np.int32)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                touch[dk:dk + nk, dj:dj + nj, di:di + ni] += keep
    node_mask = touch > 0
    node_id = -np.ones(touch.shape, dtype=np.int64)
    node_id[node_mask] = np.arange(int(node_mask.sum()))
    kk, jj, ii = np.nonzero(node_mask)          # lexicographic (k, j, i)
    x = np.stack([origin[0] + ii * h, origin[1] + jj * h, origin[2] + kk * h], axis=1).astype(np.float64)
    interior = touch[kk, jj, ii] == 8
    n_int = int(interior.sum())
    u = uniform01(seed, 3 * n_int).reshape(n_int, 3)
    x[interior] += (2.0 * u - 1.0) * (0.01 * h)
    # tets of kept cells
    ck, cj, ci = np.nonzero(keep)
    corners = np.empty((ck.size, 8), dtype=np.int64)
    for c in range(8):
        corners[:, c] = node_id[ck + ((c >> 2) & 1), cj + ((c >> 1) & 1), ci + (c & 1)]
    tets = corners[:, KUHN_TETS].reshape(-1, 4)          # (6 * n_cells, 4)
    p = x[tets]                                          # (n_mps, 4, 3)
    mp_x = p.mean(axis=1)
    e1, e2, e3 = p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]
    vol = np.abs(np.einsum("ij,ij->i", e1, np.cross(e2, e3))) / 6.0
    return x, interior, tets, mp_x, vol


def taylor_rod(h: float = 0.8e-3, R: float = 3.2e-3, L: float = 25.4e-3, v0: float = 227.0,
               material: Material | None = None, cfl: float = 0.3, steps: int = 100,
               seed: int = 0, gamma: float = 0.8, support_tol: float = 1e-6,
               wall: bool = True, name: str = "taylor_rod") -> Problem:
    """Cylinder of radius R along z, z in [0, round(L/h) h], hitting a rigid wall at z = 0.

    Cell (i, j) with centre ((i + 1/2) h, (j + 1/2) h), i, j in [-M, M - 1], M = ceil(R/h), is
    kept iff its centre lies within R of the axis."""
    if material is None:
        material = copper_j2()
    M = int(math.ceil(R / h - 1e-12))
    nk = int(round(L / h))
    c = (np.arange(-M, M) + 0.5) * h
    cy, cx = np.meshgrid(c, c, indexing="ij")
    layer = (cx * cx + cy * cy) <= R * R * (1.0 + 1e-12)
    keep = np.broadcast_to(layer, (nk,) + layer.shape).copy()
    x, interior, tets, mp_x, vol = _hex_mesh(keep, h, (-M * h, -M * h, 0.0), seed)
    n = x.shape[0]
    dt = cfl * h / material.wave_speed
    du0 = np.zeros((n, 3))
    du0[:, 2] = -v0 * dt
    contact = Contact(wall=wall, wall_point=(0.0, 0.0, 0.0), wall_normal=(0.0, 0.0, 1.0))
    return Problem(name=name, h=h, node_x=x, node_flags=np.zeros(n, np.uint8), node_du0=du0,
                   mp_x=mp_x, mp_vol=vol, mp_mass=material.rho0 * vol,
                   mp_material=np.zeros(mp_x.shape[0], np.int32), materials=[material],
                   contact=contact, dt=dt, gamma=gamma, support_tol=support_tol, T0=material.T_room,
                   steps=steps, seed=seed,
                   meta=dict(R=R, L=nk * h, v0=v0, cfl=cfl, interior_nodes=int(interior.sum())))


def chip_block(h: float = 1.0e-3 / 68, size=(4.0e-3, 1.0e-3, 0.4e-3), depth: float = 0.2e-3,
               speed: float = 5.0, material: Material | None = None, cfl: float = 0.3,
               steps: int = 5000, seed: int = 0, embed: float = 0.0, name: str = "chip") -> Problem:
    """Orthogonal cutting: block [0,Lx]x[0,Ly]x[0,Lz] (x = cut direction, y = height, z = width).

    Bottom face (y = 0) fixed. Rigid tool with rake face normal to x, cutting edge at height
    Ly - depth, starting at x = Lx + h (or embedded `embed` into the block) and moving along -x."""
    if material is None:
        material = ti64_jc()
    ni, nj, nk = (int(round(s / h)) for s in size)
    keep = np.ones((nk, nj, ni), dtype=bool)
    x, interior, tets, mp_x, vol = _hex_mesh(keep, h, (0.0, 0.0, 0.0), seed)
    n = x.shape[0]
    flags = np.zeros(n, np.uint8)
    flags[x[:, 1] <= 0.5 * h] = FLAG_FIXED
    dt = cfl * h / material.wave_speed
    Lx = ni * h
    contact = Contact(tool=True, tool_x0=Lx + h - embed, tool_tip_y=nj * h - depth,
                      tool_rake_deg=0.0, tool_clearance_deg=7.0, tool_velocity=speed, friction=0.8)
    return Problem(name=name, h=h, node_x=x, node_flags=flags, node_du0=np.zeros((n, 3)),
                   mp_x=mp_x, mp_vol=vol, mp_mass=material.rho0 * vol,
                   mp_material=np.zeros(mp_x.shape[0], np.int32), materials=[material],
                   contact=contact, dt=dt, T0=material.T_room, steps=steps, seed=seed,
                   meta=dict(size=(ni * h, nj * h, nk * h), depth=depth, speed=speed, cfl=cfl))


def copper_j2() -> Material:
    """Taylor-rod copper with linear isotropic hardening (Sec. 4.1 material data)."""
    return Material(E=117e9, nu=0.35, rho0=8930.0, model="j2", sigma_y0=400e6, H=100e6,
                    T_room=298.0, T_melt=1356.0, cp=385.0)


def copper_jc(A=90e6, B=292e6, n=0.31, C=0.025, m=1.09) -> Material:
    """Johnson-Cook copper (flow-stress constants of the scaled-up Taylor rod), adiabatic heating."""
    return Material(E=117e9, nu=0.35, rho0=8930.0, model="jc", A=A, B=B, n=n, C=C, m=m,
                    eps_dot0=1.0, T_room=298.0, T_melt=1356.0, chi=0.9, cp=385.0)


def ti64_jc() -> Material:
    """Ti-6Al-4V-like Johnson-Cook flow stress and fracture (elastic data and d1..d5 proposed)."""
    return Material(E=113.8e9, nu=0.342, rho0=4430.0, model="jc", A=1098e6, B=1092e6, n=0.93,
                    C=0.014, m=1.1, eps_dot0=1.0, T_room=298.15, T_melt=1903.15, chi=0.9,
                    cp=526.0, fracture=True, d=(-0.09, 0.25, -0.5, 0.014, 3.87))


def random_cloud(n_nodes: int, n_mps: int, seed: int, box: float = 1.0):
    """Uniform random nodes and points in [0, box]^3 (search tests)."""
    u = uniform01(seed, 3 * (n_nodes + n_mps)).reshape(-1, 3) * box
    return u[:n_nodes].copy(), u[n_nodes:].copy()


# ---- the workloads used by the tests and the benchmark ---------------------------------

def config_taylor_j2(seed: int = 0) -> Problem:
    """Plain OTM Taylor rod, FP64: R 3.2 mm, L 25.4 mm, h 0.8 mm, J2 copper, 100 steps."""
    return taylor_rod(h=0.8e-3, material=copper_j2(), steps=100, seed=seed, name="taylor_j2_h0.8")


def config_taylor_jc(h: float = 0.12e-3, seed: int = 0, steps: int = 1000) -> Problem:
    """Scaled-up Johnson-Cook Taylor rod with adiabatic heating, h = 0.12 mm."""
    return taylor_rod(h=h, material=copper_jc(), steps=steps, seed=seed,
                      name=f"taylor_jc_h{h * 1e3:g}")


def config_chip(h: float = 1.0e-3 / 68, seed: int = 0, steps: int = 5000, embed: float = 0.0) -> Problem:
    return chip_block(h=h, steps=steps, seed=seed, embed=embed, name=f"chip_h{h * 1e3:.4g}")
