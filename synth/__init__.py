"""Seeded synthetic inputs for the parabolic-operator solvers.

This module is shared by the oracle tests, the GPU parity tests and the benchmark.  It holds the
input recipe only -- the grid coordinates, the temperature / density / velocity profiles, the
dipole magnetic field evaluated at the grid corners -- and none of the method's arithmetic
(no operator coefficients, no time stepping, no time-step limit).

Array convention: every 3-D field is a float64 array of shape (n_phi, n_theta, n_r) in C order,
so that the r index is fastest in memory and the flat index of cell (i, j, k) is
i + n_r * (j + n_theta * k).

The workloads are stand-ins for the paper's MAS Test 1 / Test 2 states (Sec. 3.2), which are not
available: a dipole field over a radially stratified atmosphere on a nonuniform spherical shell.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 2403_01004
R_INNER = 1.0
R_OUTER = 10.0


@dataclasses.dataclass
class Grid:
    """Face coordinates of a spherical (r, theta, phi) shell grid; phi is uniform and periodic."""

    r_face: np.ndarray  # (n_r + 1,)
    t_face: np.ndarray  # (n_theta + 1,)
    n_phi: int

    @property
    def n_r(self) -> int:
        return len(self.r_face) - 1

    @property
    def n_theta(self) -> int:
        return len(self.t_face) - 1

    @property
    def shape(self) -> tuple[int, int, int]:
        return (self.n_phi, self.n_theta, self.n_r)

    @property
    def size(self) -> int:
        return self.n_r * self.n_theta * self.n_phi


def r_faces(n_r: int, q: float, r0: float = R_INNER, r1: float = R_OUTER) -> np.ndarray:
    """Radial faces with a geometric stretch: dr_{i+1} = q dr_i, spanning [r0, r1]."""
    if q == 1.0:
        dr = np.full(n_r, (r1 - r0) / n_r)
    else:
        dr0 = (r1 - r0) * (q - 1.0) / (q ** n_r - 1.0)
        dr = dr0 * q ** np.arange(n_r)
    f = np.empty(n_r + 1)
    f[0] = r0
    f[1:] = r0 + np.cumsum(dr)
    f[-1] = r1
    return f


def theta_faces(n_t: int) -> np.ndarray:
    """Uniform colatitude faces from pole to pole; cell centres sit half a cell off the poles."""
    return np.pi * np.arange(n_t + 1) / n_t


def make_grid(n_r: int, n_t: int, n_p: int, q: float) -> Grid:
    return Grid(r_faces(n_r, q), theta_faces(n_t), n_p)


def _centres(f: np.ndarray) -> np.ndarray:
    return 0.5 * (f[:-1] + f[1:])


def cell_r(grid: Grid) -> np.ndarray:
    """Radius of every cell centre, broadcast to the field shape."""
    return np.broadcast_to(_centres(grid.r_face)[None, None, :], grid.shape)


def dipole_corners(grid: Grid, m: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Dipole field B = (3 (m.rhat) rhat - m) / r^3 in spherical components at the grid corners.

    Corner [k, j, i] sits at (r_face[i+1], t_face[j+1], (k+1) dphi).  Corners with i = n_r - 1 or
    j = n_theta - 1 lie on the outer boundary / the south pole and carry no flux; they are filled
    anyway so that the arrays are dense.
    """
    if m is None:
        m = np.array([0.0, 0.0, 1.0])
    m = np.asarray(m, dtype=np.float64)
    r = grid.r_face[1:][None, None, :]
    t = grid.t_face[1:][None, :, None]
    p = (2.0 * np.pi / grid.n_phi) * np.arange(1, grid.n_phi + 1)[:, None, None]
    st, ct, sp, cp = np.sin(t), np.cos(t), np.sin(p), np.cos(p)
    m_r = m[0] * st * cp + m[1] * st * sp + m[2] * ct
    m_t = m[0] * ct * cp + m[1] * ct * sp - m[2] * st
    m_p = -m[0] * sp + m[1] * cp + 0.0 * ct
    inv_r3 = 1.0 / r ** 3
    br = np.broadcast_to(2.0 * m_r * inv_r3, grid.shape).copy()
    bt = np.broadcast_to(-m_t * inv_r3, grid.shape).copy()
    bp = np.broadcast_to(-m_p * inv_r3, grid.shape).copy()
    return br, bt, bp


def random_unit_vector(rng: np.random.Generator) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


@dataclasses.dataclass
class TCInputs:
    grid: Grid
    T: np.ndarray        # temperature at cells (also the lagged T0 that sets kappa)
    n: np.ndarray        # number density at cells
    B: tuple             # (B_r, B_theta, B_phi) at corners


def tc_inputs(grid: Grid, seed: int, noise: float = 0.01, m: np.ndarray | None = None,
              profile: str = "exp") -> TCInputs:
    """Thermal-conduction inputs: T = (0.01 + 0.99 exp(-(r-1)/2)) (1 + noise U(-1,1)),
    n = exp(-(r-1)/0.5), dipole B.  profile="jump" gives the transition-region-like
    temperature step of the precision-stress workload instead (see tc_jump_profile)."""
    rng = np.random.default_rng(seed)
    r = cell_r(grid)
    if profile == "exp":
        base = 0.01 + 0.99 * np.exp(-(r - 1.0) / 2.0)
    elif profile == "jump":
        base = tc_jump_profile(grid)
    else:
        raise ValueError(profile)
    T = base * (1.0 + noise * rng.uniform(-1.0, 1.0, size=grid.shape))
    n = np.exp(-(r - 1.0) / 0.5).copy()
    B = dipole_corners(grid, m)
    return TCInputs(grid, np.ascontiguousarray(T), np.ascontiguousarray(n), B)


def tc_jump_profile(grid: Grid, r_jump: float = 1.02, cells: float = 3.0) -> np.ndarray:
    """T rising from 0.01 to 1 over `cells` radial cells around r_jump: the 10%-90% width of
    0.01 + 0.99 (1 + tanh((r - r_jump)/l)) / 2 equals `cells` times the local radial spacing."""
    rf = grid.r_face
    i = int(np.searchsorted(rf, r_jump) - 1)
    i = min(max(i, 0), grid.n_r - 1)
    dr = rf[i + 1] - rf[i]
    ell = cells * dr / (2.0 * np.arctanh(0.8))
    r = cell_r(grid)
    return 0.01 + 0.99 * 0.5 * (1.0 + np.tanh((r - r_jump) / ell))


def staggered_points(grid: Grid, comp: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Coordinates (r, theta, phi) of the points of velocity component `comp` (0 = v_r on interior
    r faces, 1 = v_theta on interior theta faces, 2 = v_phi on phi faces).  Returns 1-D arrays."""
    rc, tc = _centres(grid.r_face), _centres(grid.t_face)
    dphi = 2.0 * np.pi / grid.n_phi
    pc = dphi * (np.arange(grid.n_phi) + 0.5)
    pf = dphi * np.arange(grid.n_phi)
    r = grid.r_face[1:-1] if comp == 0 else rc
    t = grid.t_face[1:-1] if comp == 1 else tc
    p = pf if comp == 2 else pc
    return r, t, p


def staggered_shape(grid: Grid, comp: int) -> tuple[int, int, int]:
    r, t, p = staggered_points(grid, comp)
    return (len(p), len(t), len(r))


@dataclasses.dataclass
class ViscInputs:
    grid: Grid
    v: list              # [v_r, v_theta, v_phi] on their staggered grids
    rho: list            # density at each component's points
    nu: list             # viscosity coefficient at each component's points


def visc_inputs(grid: Grid, seed: int, sigma: float = 0.1) -> ViscInputs:
    """Velocity components ~ N(0, sigma) i.i.d., rho = exp(-(r-1)/0.5), nu = 1e-3 r^2."""
    rng = np.random.default_rng(seed + 7919)
    v, rho, nu = [], [], []
    for comp in range(3):
        r, _, _ = staggered_points(grid, comp)
        shp = staggered_shape(grid, comp)
        rr = np.broadcast_to(r[None, None, :], shp)
        v.append(np.ascontiguousarray(rng.normal(0.0, sigma, size=shp)))
        rho.append(np.ascontiguousarray(np.exp(-(rr - 1.0) / 0.5)))
        nu.append(np.ascontiguousarray(1e-3 * rr ** 2))
    return ViscInputs(grid, v, rho, nu)


def tc_random_inputs(grid: Grid, seed: int) -> TCInputs:
    """Training profiles for the learned PCG guess: the conduction recipe with its shape
    parameters drawn per sample -- temperature scale height H ~ U(1, 4), noise amplitude
    ~ U(0.005, 0.05), density scale height ~ U(0.3, 1), dipole tilted uniformly on the sphere."""
    rng = np.random.default_rng(seed)
    H = rng.uniform(1.0, 4.0)
    eps = rng.uniform(0.005, 0.05)
    hn = rng.uniform(0.3, 1.0)
    m = random_unit_vector(rng)
    r = cell_r(grid)
    T = (0.01 + 0.99 * np.exp(-(r - 1.0) / H)) * (1.0 + eps * rng.uniform(-1.0, 1.0, size=grid.shape))
    n = np.exp(-(r - 1.0) / hn).copy()
    return TCInputs(grid, np.ascontiguousarray(T), np.ascontiguousarray(n), dipole_corners(grid, m))


# ---- workload recipes (sizes, stretch, dt ratios) ------------------------------------------

WORKLOADS = {
    # small FP64 parity case: 32x32x64, q = 1.05, dt = 100 dt_E, untilted dipole
    "shell32": dict(n_r=32, n_t=32, n_p=64, q=1.05, ratio=100.0, seed=SEED_BASE + 0),
    # production-shaped grid: 256x256x512 (33.5M cells), q = 1.01, dt = 1e3 dt_E, TC + viscosity
    "shell256": dict(n_r=256, n_t=256, n_p=512, q=1.01, ratio=1000.0, seed=SEED_BASE + 1),
    # learned-guess BE workload: 192x192x384, dt = 1e4 dt_E
    "shell192": dict(n_r=192, n_t=192, n_p=384, q=1.05, ratio=1e4, seed=SEED_BASE + 3),
    # precision stress: 128x256x512 jump profile, dt = 1e5 dt_E
    "jump128": dict(n_r=128, n_t=256, n_p=512, q=1.05, ratio=1e5, seed=SEED_BASE + 4,
                    profile="jump", noise=0.05),
}


def batched_problems(count: int = 64, seed: int = SEED_BASE + 2):
    """The batched workload: `count` independent conduction problems with n_r, n_theta in
    {16, 32, 64, 128}, n_phi in {n_theta, 2 n_theta}, dt/dt_E log-uniform in [10, 1e4] and a
    dipole tilted uniformly on the sphere.  Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n_r = int(rng.choice([16, 32, 64, 128]))
        n_t = int(rng.choice([16, 32, 64, 128]))
        n_p = int(n_t * rng.choice([1, 2]))
        ratio = float(10.0 ** rng.uniform(1.0, 4.0))
        m = random_unit_vector(rng)
        out.append(dict(n_r=n_r, n_t=n_t, n_p=n_p, q=1.05, ratio=ratio, m=m,
                        seed=int(seed * 1000 + b)))
    return out
