"""Seeded synthetic inputs for the coupled two-fluid system.

This module only builds initial states and problem descriptions. It holds
none of the scheme's arithmetic. Tests and benchmarks hand its output to both
the CUDA library and the CPU oracle, so both sides see the same input.

Geometry. x lies in (-5, 5) and is periodic, with dx = 10/nx. Rows are stacked
bottom to top as slow (S) | buffer (B) | fast (F). S and B are fluid 1 (the
ocean, below the interface at z = 0). F is fluid 2 (the atmosphere, above it).
Cell centres are z = -(n1 - k - 1/2) dz1 for fluid-1 row k, where
n1 = nS + nB, and z = (k - n1 + 1/2) dz2 for fluid-2 rows.

Rest state. This is the neutrally stratified state of the paper's thermal
convection setup (Sec. 5.2) with delta theta = 0: Psi = 1 + g z / c_p with
c_p = 1/(gamma-1) and g = -0.008140864714, T = Psi,
p = Psi^(gamma/(gamma-1)) / gamma and rho = Psi^(1/(gamma-1)).

Perturbations. These are the synthetic stand-ins for the paper's workloads,
whose initial conditions are not given in the paper.
* gaussian_bumps: K bumps with seeded centres and width sigma (in cells).
  They perturb rho by amp*rho0*env, and (u, w) by amp*env along a seeded
  direction. Pressure stays at rest.
* fourier_modes: 10 modes with seeded integer wave numbers kx, kz in [1, 8]
  and seeded phases. Each mode has amplitude amp/10. Independent draws
  perturb rho/rho0, u and w. Pressure stays at rest.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
PR = 0.72
MU1 = 1.0 / 20000.0
MU2 = 1.0 / 5000.0
G_SIGNED = -0.008140864714  # the g of Sec. 5.2 (points down)
SEED0 = 0xC0FFEE


@dataclass
class Grid:
    nx: int
    nS: int
    nB: int
    nF: int
    dx: float = 0.0
    dz1: float = 0.0
    dz2: float = 0.0

    def __post_init__(self):
        if self.dx <= 0.0:
            self.dx = 10.0 / self.nx
        if self.dz1 <= 0.0:
            self.dz1 = self.dx
        if self.dz2 <= 0.0:
            self.dz2 = self.dx

    @property
    def nz(self) -> int:
        return self.nS + self.nB + self.nF

    @property
    def n1(self) -> int:
        return self.nS + self.nB

    def x_centres(self) -> np.ndarray:
        return -5.0 + (np.arange(self.nx) + 0.5) * self.dx

    def z_centres(self) -> np.ndarray:
        k = np.arange(self.nz)
        z1 = -(self.n1 - k - 0.5) * self.dz1
        z2 = (k - self.n1 + 0.5) * self.dz2
        return np.where(k < self.n1, z1, z2)


def conserved(rho, u, w, p, gamma=GAMMA) -> np.ndarray:
    """Stack (rho, rho u, rho w, rho E) from primitive fields of shape [nz][nx]."""
    q = np.empty((4,) + rho.shape)
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * w
    q[3] = p / (gamma - 1.0) + 0.5 * rho * (u * u + w * w)
    return q


def rest_primitives(grid: Grid, gamma=GAMMA, g=G_SIGNED):
    z = grid.z_centres()[:, None] * np.ones((1, grid.nx))
    cp = 1.0 / (gamma - 1.0)
    psi = 1.0 + g * z / cp
    rho = psi ** (1.0 / (gamma - 1.0))
    p = psi ** (gamma / (gamma - 1.0)) / gamma
    return rho, p


def rest_state(grid: Grid, gamma=GAMMA, g=G_SIGNED) -> np.ndarray:
    rho, p = rest_primitives(grid, gamma, g)
    zero = np.zeros_like(rho)
    return conserved(rho, zero, zero, p, gamma)


def gaussian_bumps(grid: Grid, seed: int, k_bumps: int = 4, sigma_cells: float = 4.0,
                   amp: float = 1e-2, gamma=GAMMA, g=G_SIGNED) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rho0, p0 = rest_primitives(grid, gamma, g)
    x = grid.x_centres()[None, :]
    z = grid.z_centres()[:, None]
    zlo = -grid.n1 * grid.dz1
    zhi = (grid.nz - grid.n1) * grid.dz2
    sig = sigma_cells * grid.dx
    drho = np.zeros_like(rho0)
    u = np.zeros_like(rho0)
    w = np.zeros_like(rho0)
    for _ in range(k_bumps):
        xc = rng.uniform(-5.0, 5.0)
        zc = rng.uniform(zlo, zhi)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        ddx = (x - xc + 5.0) % 10.0 - 5.0  # periodic distance in x
        env = np.exp(-(ddx ** 2 + (z - zc) ** 2) / (2.0 * sig * sig))
        drho += amp * env
        u += amp * env * np.cos(phi)
        w += amp * env * np.sin(phi)
    return conserved(rho0 * (1.0 + drho), u, w, p0, gamma)


# ---- three dimensions (App. B in full): state [5][nz][ny][nx] -------------

@dataclass
class Grid3:
    """x-y-z grid: nx x ny columns (both periodic), rows S | B | F in z."""
    nx: int
    ny: int
    nS: int
    nB: int
    nF: int
    dx: float = 0.0
    dy: float = 0.0
    dz1: float = 0.0
    dz2: float = 0.0

    def __post_init__(self):
        if self.dx <= 0.0:
            self.dx = 10.0 / self.nx
        if self.dy <= 0.0:
            self.dy = self.dx
        if self.dz1 <= 0.0:
            self.dz1 = self.dx
        if self.dz2 <= 0.0:
            self.dz2 = self.dx

    @property
    def nz(self) -> int:
        return self.nS + self.nB + self.nF

    @property
    def n1(self) -> int:
        return self.nS + self.nB

    def column_grid(self) -> Grid:
        """The x-z grid of one y column (same rows and cell sizes)."""
        return Grid(self.nx, self.nS, self.nB, self.nF, dx=self.dx, dz1=self.dz1, dz2=self.dz2)

    def y_centres(self) -> np.ndarray:
        return -0.5 * self.ny * self.dy + (np.arange(self.ny) + 0.5) * self.dy


def conserved3(rho, u, v, w, p, gamma=GAMMA) -> np.ndarray:
    """Stack (rho, rho u, rho v, rho w, rho E) from fields of shape [nz][ny][nx]."""
    q = np.empty((5,) + rho.shape)
    q[0] = rho
    q[1] = rho * u
    q[2] = rho * v
    q[3] = rho * w
    q[4] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return q


def rest_state3(grid: Grid3, gamma=GAMMA, g=G_SIGNED) -> np.ndarray:
    rho, p = rest_primitives(grid.column_grid(), gamma, g)
    rho = np.repeat(rho[:, None, :], grid.ny, axis=1)
    p = np.repeat(p[:, None, :], grid.ny, axis=1)
    zero = np.zeros_like(rho)
    return conserved3(rho, zero, zero, zero, p, gamma)


def gaussian_bumps3(grid: Grid3, seed: int, k_bumps: int = 4, sigma_cells: float = 3.0,
                    amp: float = 1e-2, gamma=GAMMA, g=G_SIGNED) -> np.ndarray:
    """The rest state with k seeded Gaussian bumps in density and velocity
    (random direction in 3-D), pressure kept."""
    rng = np.random.default_rng(seed)
    cg = grid.column_grid()
    rho0, p0 = rest_primitives(cg, gamma, g)
    rho0 = np.repeat(rho0[:, None, :], grid.ny, axis=1)
    p0 = np.repeat(p0[:, None, :], grid.ny, axis=1)
    x = cg.x_centres()[None, None, :]
    y = grid.y_centres()[None, :, None]
    z = cg.z_centres()[:, None, None]
    Lx, Ly = grid.nx * grid.dx, grid.ny * grid.dy
    zlo, zhi = -grid.n1 * grid.dz1, (grid.nz - grid.n1) * grid.dz2
    sig = sigma_cells * grid.dx
    drho = np.zeros_like(rho0)
    vel = [np.zeros_like(rho0) for _ in range(3)]
    for _ in range(k_bumps):
        c = (rng.uniform(-Lx / 2, Lx / 2), rng.uniform(-Ly / 2, Ly / 2), rng.uniform(zlo, zhi))
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        ddx = (x - c[0] + Lx / 2) % Lx - Lx / 2  # periodic distances
        ddy = (y - c[1] + Ly / 2) % Ly - Ly / 2
        env = np.exp(-(ddx ** 2 + ddy ** 2 + (z - c[2]) ** 2) / (2.0 * sig * sig))
        drho += amp * env
        for a in range(3):
            vel[a] += amp * env * d[a]
    return conserved3(rho0 * (1.0 + drho), vel[0], vel[1], vel[2], p0, gamma)


def _modes(rng, xi, zeta, n_modes, amp):
    f = np.zeros((zeta.shape[0], xi.shape[1]))
    for _ in range(n_modes):
        kx = int(rng.integers(1, 9))
        kz = int(rng.integers(1, 9))
        ph = rng.uniform(0.0, 2.0 * np.pi)
        ps = rng.uniform(0.0, 2.0 * np.pi)
        f += (amp / n_modes) * np.cos(2.0 * np.pi * kx * xi + ph) * np.cos(np.pi * kz * zeta + ps)
    return f


def fourier_modes(grid: Grid, seed: int, n_modes: int = 10, amp: float = 1e-2,
                  gamma=GAMMA, g=G_SIGNED, periodic_on_grid: bool = False) -> np.ndarray:
    """periodic_on_grid: the x phase runs over the grid's own nx columns,
    (i + 1/2)/nx, so that a strip narrower than (-5, 5) is periodic too;
    otherwise over x in (-5, 5)."""
    rng = np.random.default_rng(seed)
    rho0, p0 = rest_primitives(grid, gamma, g)
    if periodic_on_grid:
        xi = ((np.arange(grid.nx) + 0.5) / grid.nx)[None, :]
    else:
        xi = ((grid.x_centres() + 5.0) / 10.0)[None, :]
    z = grid.z_centres()
    zlo = -grid.n1 * grid.dz1
    zhi = (grid.nz - grid.n1) * grid.dz2
    zeta = ((z - zlo) / (zhi - zlo))[:, None]
    drho = _modes(rng, xi, zeta, n_modes, amp)
    u = _modes(rng, xi, zeta, n_modes, amp)
    w = _modes(rng, xi, zeta, n_modes, amp)
    return conserved(rho0 * (1.0 + drho), u, w, p0, gamma)


def thermal_bubble(grid: Grid, gamma=GAMMA, g=G_SIGNED, theta0=300.0,
                   centre=(0.0, -2.5), radius=2.5, amp=0.25) -> np.ndarray:
    """Warm bubble in fluid 1 of Sec. 5.2: delta theta = amp(1 + cos(pi r)) for
    r <= radius around centre, 0 elsewhere and in fluid 2."""
    return _potential_temperature_state(grid, [(1, centre, radius, amp)], gamma, g, theta0)


def thermal_convection(grid: Grid, gamma=GAMMA, g=G_SIGNED, theta0=300.0) -> np.ndarray:
    """The second thermal-convection case of Sec. 5.2 (the one of Table 6): a
    warm perturbation in fluid 1, delta theta_1 = 1.25 (1 + cos(pi r_1)) for
    r_1 <= 2.5 around (0, -2.5), and a cold one in fluid 2, delta theta_2 =
    -7.5 (1 + cos(pi r_2)) for r_2 <= 1 around (0, 1.5)."""
    return _potential_temperature_state(
        grid, [(1, (0.0, -2.5), 2.5, 1.25), (2, (0.0, 1.5), 1.0, -7.5)], gamma, g, theta0)


def _potential_temperature_state(grid: Grid, bumps, gamma, g, theta0) -> np.ndarray:
    """The initial state of Sec. 5.2 at rest from potential-temperature
    perturbations: T = (1 + dth/theta0) Psi, p = Psi^(gamma/(gamma-1))/gamma,
    rho = theta0/(theta0 + dth) Psi^(1/(gamma-1)), Psi = 1 + g z/(cp (1 +
    dth/theta0)). bumps: (fluid, centre, radius, amplitude) with
    dth = amplitude (1 + cos(pi r)) for r <= radius."""
    x = grid.x_centres()[None, :] * np.ones((grid.nz, 1))
    z = grid.z_centres()[:, None] * np.ones((1, grid.nx))
    k = np.arange(grid.nz)[:, None] * np.ones((1, grid.nx))
    dth = np.zeros((grid.nz, grid.nx))
    for fluid, centre, radius, amp in bumps:
        r = np.sqrt((x - centre[0]) ** 2 + (z - centre[1]) ** 2)
        inside = (k < grid.n1) if fluid == 1 else (k >= grid.n1)
        dth = np.where((r <= radius) & inside, amp * (1.0 + np.cos(np.pi * r)), dth)
    cp = 1.0 / (gamma - 1.0)
    fac = 1.0 + dth / theta0
    psi = 1.0 + g * z / (cp * fac)
    p = psi ** (gamma / (gamma - 1.0)) / gamma
    rho = theta0 / (theta0 + dth) * psi ** (1.0 / (gamma - 1.0))
    zero = np.zeros_like(rho)
    return conserved(rho, zero, zero, p, gamma)


@dataclass
class Workload:
    """One solve: grid, rate ratio, slow steps, precision and initial state recipe."""
    name: str
    grid: Grid
    m: int
    steps: int
    precision: str  # "fp64" or "fp32flux"
    perturbation: str  # "bumps" or "fourier"
    seed: int
    extra: dict = field(default_factory=dict)

    def initial_state(self) -> np.ndarray:
        if self.perturbation == "bumps":
            return gaussian_bumps(self.grid, self.seed)
        if self.perturbation == "fourier":
            return fourier_modes(self.grid, self.seed)
        if self.perturbation == "rest":
            return rest_state(self.grid)
        if self.perturbation == "convection":
            return thermal_convection(self.grid)
        if self.perturbation == "bumps3":
            return gaussian_bumps3(self.grid, self.seed)
        raise ValueError(self.perturbation)

    def cell_stages_per_step(self) -> int:
        """Cell RHS evaluations per slow step: nx (s nS + m s (nB + nF)), s = 2."""
        g = self.grid
        return g.nx * (2 * g.nS + 2 * self.m * (g.nB + g.nF))


def plain_64():
    """64x64 grid, S rows 0-29, B 30-33, F 34-63, m = 4, 100 slow steps, FP64."""
    return Workload("plain_64x64_m4_fp64", Grid(64, 30, 4, 30), 4, 100, "fp64", "bumps", SEED0 + 0)


def large_2048():
    """2048x1024 grid, S 480 / B 64 / F 480 rows, m = 8, 200 slow steps, FP64."""
    return Workload("large_2048x1024_m8_fp64", Grid(2048, 480, 64, 480), 8, 200, "fp64", "fourier",
                    SEED0 + 1)


def mixed_4096():
    """4096x2048 grid, S 960 / B 128 / F 960 rows, m = 8, 500 slow steps, FP32 flux."""
    return Workload("mixed_4096x2048_m8_fp32flux", Grid(4096, 960, 128, 960), 8, 500, "fp32flux",
                    "fourier", SEED0 + 2)


def convection_grid() -> Grid:
    """The thermal-convection mesh of Table 6 (Sec. 5.2, second set-up):
    Omega_1 = (-5,5) x (-7,0) with 100 x 100 cells, Omega_2 = (-5,5) x (0,3)
    with 100 x 200 cells; fluid 1 split into 96 slow and 4 buffer rows."""
    return Grid(100, 96, 4, 200, dx=0.1, dz1=0.07, dz2=0.015)


def convection_100() -> Workload:
    """Table 6's thermal convection: walls on all boundaries, MPRK2 with
    m = 4, dt = 0.025, to t = 2.5 (100 slow steps), FP64."""
    return Workload("convection_100x300_m4_fp64", convection_grid(), 4, 100, "fp64", "convection", 0,
                    extra={"x_walls": 1, "dt": 0.025})


def cube_512() -> Workload:
    """The 3-D model (App. B): 512 x 64 columns, S/B/F = 96/8/96 rows, m = 4,
    seeded bumps, FP64, 20 slow steps."""
    return Workload("cube_512x64x200_m4_fp64", Grid3(512, 64, 96, 8, 96), 4, 20, "fp64", "bumps3",
                    SEED0 + 11)


def batched_256(count: int = 256, seed: int = SEED0 + 3, steps: int = 100):
    """Independent instances: sides log-uniform in [64, 512], m in {2,4,8},
    buffer 4-16 rows, S = (nz-B)//2, F = nz-B-S; Gaussian-bump initial states."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        nx = int(round(np.exp(rng.uniform(np.log(64), np.log(512)))))
        nz = int(round(np.exp(rng.uniform(np.log(64), np.log(512)))))
        m = int(rng.choice([2, 4, 8]))
        nB = int(rng.integers(4, 17))
        nS = (nz - nB) // 2
        nF = nz - nB - nS
        out.append(Workload(f"batch_{j}", Grid(nx, nS, nB, nF), m, steps, "fp64", "bumps",
                            seed * 1000 + j))
    return out


def served_stream(count: int, seed: int = SEED0 + 4, rate_hz: float = 200.0,
                  side_lo: int = 32, side_hi: int = 1024, steps_lo: int = 10, steps_hi: int = 1000):
    """Poisson arrivals (mean rate_hz) of solves with sides log-uniform in
    [side_lo, side_hi], m in {2,4,8}, buffer 4-16 rows, slow steps log-uniform
    in [steps_lo, steps_hi], FP32 flux. Returns (arrival times, workloads)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for j in range(count):
        nx = int(round(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi)))))
        nz = int(round(np.exp(rng.uniform(np.log(max(side_lo, 24)), np.log(side_hi)))))
        nx = max(nx, 8)
        m = int(rng.choice([2, 4, 8]))
        nB = int(rng.integers(4, 17))
        nS = max((nz - nB) // 2, 2)
        nF = max(nz - nB - nS, 2)
        steps = int(round(np.exp(rng.uniform(np.log(steps_lo), np.log(steps_hi)))))
        out.append(Workload(f"req_{j}", Grid(nx, nS, nB, nF), m, steps, "fp32flux", "bumps",
                            seed * 1000 + j))
    return t, out
