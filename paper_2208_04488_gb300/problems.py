"""Seeded synthetic initial conditions shaped like the paper's test problems.

This module is the only input generator shared by the CUDA path and the CPU
oracle. It holds none of the scheme's arithmetic: it produces geometry, the
fluid table and *primitive* initial fields -- the N-1 volume fractions, the
velocity, the pressure and the temperature of every cell -- from which each
side builds its own conservative state (``hrm_set_primitive`` on the GPU,
the oracle's initial-state builder on the CPU), by the p-T equilibrium rule
of Sec. 5 (species densities from the stiffened-gas EOS at the cell's p and T).

Set-up-only thermodynamics kept here: the temperature of a region given its
dominant species' density (Sec. 2, species temperature), and ideal-gas normal
shock relations for post-shock states. Neither is a step of the time
integration.

Fields are SoA ``prim[N + D + 1, ncells]`` with x fastest:
planes 0..N-2 alpha_k, N-1..N+D-2 u_d, N+D-1 p, N+D T.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---------------------------------------------------------------- fluid tables

# Table fluid_properties (Sec. 5): gamma, c_p, p_inf, q. c_v = c_p / gamma.
PAPER_WATER = dict(gamma=3.0, cp=4200.0, pinf=8.533e8, q=-0.1148e7)
PAPER_AIR = dict(gamma=1.4, cp=1007.0, pinf=0.0, q=0.0)
PAPER_SF6 = dict(gamma=1.1, cp=664.0, pinf=0.0, q=0.0)
PAPER_DETONATION = dict(gamma=1.25, cp=1000.0, pinf=0.0, q=0.0)

# Fluids of the benchmark workloads. The paper gives no c_v for this water or
# for helium; the values are a stated choice: water c_v makes rho = 1000 kg/m^3
# at 1e5 Pa and 298 K, helium c_v = R_He / (gamma - 1) with R_He = 2077.3 J/kg/K.
BENCH_WATER = dict(gamma=6.12, cp=6.12 * 224.87, pinf=3.43e8, q=0.0)
BENCH_AIR = dict(gamma=1.4, cp=1007.0, pinf=0.0, q=0.0)
BENCH_HELIUM = dict(gamma=1.67, cp=1.67 * (2077.3 / 0.67), pinf=0.0, q=0.0)

MINOR = 1.0e-8  # minor-phase volume fraction used throughout Sec. 5


@dataclasses.dataclass
class Problem:
    name: str
    gamma: List[float]
    pinf: List[float]
    cv: List[float]
    q: List[float]
    n: List[int]                 # cells per direction (x first)
    lo: List[float]
    hi: List[float]
    bc: List[int]                # 0 transmissive, 1 periodic, 2 Dirichlet; [lo_x, hi_x, lo_y, ...]
    prim: np.ndarray             # (N + D + 1, ncells) float64
    cfl: float = 0.5
    dt: Optional[float] = None   # constant time step, if the problem uses one
    t_end: Optional[float] = None
    nsteps: Optional[int] = None
    extra: dict = dataclasses.field(default_factory=dict)
    # Dirichlet sides (bc 2): {b = 2 d + side: primitive planes of the boundary
    # slice, (N + D + 1, cells of the side), lowest other direction fastest}
    boundary: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.gamma)

    @property
    def D(self) -> int:
        return len(self.n)

    @property
    def M(self) -> int:
        return 2 * self.N + self.D

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def dx(self) -> List[float]:
        return [(self.hi[d] - self.lo[d]) / self.n[d] for d in range(self.D)]

    @property
    def liq(self) -> int:
        return next((k for k in range(self.N) if self.pinf[k] > 0), 0)


def _species(fl: list):
    gamma = [f["gamma"] for f in fl]
    cv = [f["cp"] / f["gamma"] for f in fl]
    pinf = [f["pinf"] for f in fl]
    q = [f["q"] for f in fl]
    return gamma, pinf, cv, q


def cell_centers(n, lo, hi):
    """Cell-centre coordinates (x fastest), each of shape (ncells,)."""
    axes = [lo[d] + (np.arange(n[d]) + 0.5) * (hi[d] - lo[d]) / n[d] for d in range(len(n))]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    return [g.reshape(-1) for g in grids]


def temperature_of(fluid: dict, p: float, rho: float) -> float:
    """Species temperature from p and the species density (Sec. 2)."""
    cv = fluid["cp"] / fluid["gamma"]
    return (p + fluid["pinf"]) / ((fluid["gamma"] - 1.0) * rho * cv)


def normal_shock(gamma: float, p1: float, rho1: float, mach: float):
    """Ideal-gas Rankine-Hugoniot state behind a shock moving at Mach `mach`
    into gas at rest: returns (p2, rho2, u2)."""
    c1 = math.sqrt(gamma * p1 / rho1)
    m2 = mach * mach
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    u2 = mach * c1 * (1.0 - rho1 / rho2)
    return p2, rho2, u2


def _assemble(N, D, alphas, u, p, T):
    nc = p.shape[0]
    prim = np.empty((N + D + 1, nc))
    for k in range(N - 1):
        prim[k] = alphas[k]
    for d in range(D):
        prim[N - 1 + d] = u[d]
    prim[N + D - 1] = p
    prim[N + D] = T
    return prim


def smooth_step(s, width):
    """0.5 (1 - tanh(s / width)): the tanh smoothing of App. A for a signed
    distance s (negative inside); width = C_s dx."""
    return 0.5 * (1.0 - np.tanh(s / width))


# ---------------------------------------------------------------- 1D problems

def shock_tube_1d_baseline(n: int = 400) -> Problem:
    """1D water-air shock tube of the benchmark configuration: 400 cells on
    [0, 1], interface at x = 0.7, water (gamma 6.12, p_inf 3.43e8) at
    rho = 1000, p = 1e9 on the left, air at rho = 50, p = 1e5 on the right,
    u = 0, minor volume fraction 1e-8, CFL 0.4, transmissive, t_end 2.4e-4 s.
    Species order: water, air. T of each side from its dominant species."""
    gamma, pinf, cv, q = _species([BENCH_WATER, BENCH_AIR])
    (x,) = cell_centers([n], [0.0], [1.0])
    TL = temperature_of(BENCH_WATER, 1.0e9, 1000.0)
    TR = temperature_of(BENCH_AIR, 1.0e5, 50.0)
    left = x < 0.7
    a1 = np.where(left, 1.0 - MINOR, MINOR)
    p = np.where(left, 1.0e9, 1.0e5)
    T = np.where(left, TL, TR)
    prim = _assemble(2, 1, [a1], [np.zeros(n)], p, T)
    return Problem("shock_tube_1d_water_air_400", gamma, pinf, cv, q, [n], [0.0], [1.0],
                   [0, 0], prim, cfl=0.4, t_end=2.4e-4)


def shock_tube_1d_paper(n: int = 500, extreme: bool = False) -> Problem:
    """Gas/liquid shock tube of Sec. 5.4 (or the extreme one of Sec. 5.5):
    x in [0, 1.5], interface at 0.8, rho_water = 1000 on the left at 1e9 Pa
    (1e12 Pa when extreme), rho_air = 20 on the right at 1e5 Pa, paper fluids."""
    gamma, pinf, cv, q = _species([PAPER_WATER, PAPER_AIR])
    (x,) = cell_centers([n], [0.0], [1.5])
    pl = 1.0e12 if extreme else 1.0e9
    TL = temperature_of(PAPER_WATER, pl, 1000.0)
    TR = temperature_of(PAPER_AIR, 1.0e5, 20.0)
    left = x < 0.8
    a1 = np.where(left, 1.0 - MINOR, MINOR)
    p = np.where(left, pl, 1.0e5)
    T = np.where(left, TL, TR)
    prim = _assemble(2, 1, [a1], [np.zeros(n)], p, T)
    name = "extreme_shock_tube_1d" if extreme else "shock_tube_1d_paper"
    dt = (8.0e-9 if extreme else 5.0e-7 * 500.0 / n)
    return Problem(name, gamma, pinf, cv, q, [n], [0.0], [1.5], [0, 0], prim, cfl=0.5,
                   dt=dt, t_end=(1.0e-5 if extreme else 3.0e-4),
                   extra=dict(TL=TL, TR=TR))


def shock_interface_1d_3species(n: int = 800) -> Problem:
    """Extreme shock-interface interaction of Sec. 5.6 with water, air and SF6.
    The post-shock liquid state is taken from the table of the paper (its
    velocity and pressure) with the temperature that gives its liquid density."""
    gamma, pinf, cv, q = _species([PAPER_WATER, PAPER_AIR, PAPER_SF6])
    (x,) = cell_centers([n], [0.0], [1.0])
    T0 = 298.0
    # post-shock water: alpha_1 rho_1 = 2.0429330221481357e3 at alpha_1 = 1 - 1e-8, p = 1e12
    rho_ps = 2.0429330221481357e3 / (1.0 - MINOR)
    T_ps = temperature_of(PAPER_WATER, 1.0e12, rho_ps)
    region0 = x < 0.15
    region1 = (x >= 0.15) & (x < 0.3)
    a1 = np.where(x < 0.3, 1.0 - 2.0 * MINOR, MINOR)
    a2 = np.where(x < 0.3, MINOR, 0.5 - 5.0e-9)
    u = np.where(region0, 2.2096204395563851e4, 0.0)
    p = np.where(region0, 1.0e12, 1.01325e5)
    T = np.where(region0, T_ps, T0)
    del region1
    prim = _assemble(3, 1, [a1, a2], [u], p, T)
    return Problem("shock_interface_1d_3species", gamma, pinf, cv, q, [n], [0.0], [1.0],
                   [0, 0], prim, cfl=0.5, dt=6.0e-9 * 800.0 / n, t_end=1.26e-5)


def material_interface_1d(n: int = 500, Cs: Optional[float] = None) -> Problem:
    """Material-interface advection of App. A: periodic [0, 1), water in
    [0.25, 0.75), air elsewhere, u = 100 m/s, p = 101325 Pa, T = 298 K,
    optional tanh smoothing with parameter C_s."""
    gamma, pinf, cv, q = _species([PAPER_WATER, PAPER_AIR])
    (x,) = cell_centers([n], [0.0], [1.0])
    mid, side = 1.0 - MINOR, MINOR
    if Cs is None:
        a1 = np.where((x >= 0.25) & (x < 0.75), mid, side)
    else:
        dx = 1.0 / n
        fs = 0.5 * (np.tanh((x - 0.25) / (Cs * dx)) - np.tanh((x - 0.75) / (Cs * dx)))
        a1 = (mid - side) * fs + side
    prim = _assemble(2, 1, [a1], [np.full(n, 100.0)], np.full(n, 101325.0), np.full(n, 298.0))
    return Problem("material_interface_1d", gamma, pinf, cv, q, [n], [0.0], [1.0], [1, 1], prim,
                   dt=6.25e-7 * 500.0 / n, t_end=0.01)


def advection_1d_smooth(n: int = 64) -> Problem:
    """1D periodic advection of Sec. 5.1 on [-1, 1): alpha_1 = 0.5 + 0.25 sin(pi x),
    u = 10 m/s, p = 101325 Pa, T = 298 K."""
    gamma, pinf, cv, q = _species([PAPER_WATER, PAPER_AIR])
    (x,) = cell_centers([n], [-1.0], [1.0])
    a1 = 0.5 + 0.25 * np.sin(np.pi * x)
    prim = _assemble(2, 1, [a1], [np.full(n, 10.0)], np.full(n, 101325.0), np.full(n, 298.0))
    return Problem("advection_1d_smooth", gamma, pinf, cv, q, [n], [-1.0], [1.0], [1, 1], prim,
                   t_end=0.1)


# ---------------------------------------------------------------- 2D / 3D problems

def advection_2d_smooth(n: int = 64, t: float = 0.0) -> Problem:
    """2D periodic advection of Sec. 5.2 on [-1, 1)^2:
    alpha_1 = 0.5 + 0.25 sin(pi (x + y - 20 t)), u = v = 10 m/s, p = 101325 Pa,
    T = 298 K; dt/dx = 4e-5 s/m, t_end = 1e-4 s."""
    gamma, pinf, cv, q = _species([PAPER_WATER, PAPER_AIR])
    x, y = cell_centers([n, n], [-1.0, -1.0], [1.0, 1.0])
    a1 = 0.5 + 0.25 * np.sin(np.pi * (x + y - 20.0 * t))
    nc = n * n
    prim = _assemble(2, 2, [a1], [np.full(nc, 10.0), np.full(nc, 10.0)], np.full(nc, 101325.0),
                     np.full(nc, 298.0))
    dx = 2.0 / n
    return Problem("advection_2d_smooth", gamma, pinf, cv, q, [n, n], [-1.0, -1.0], [1.0, 1.0],
                   [1, 1, 1, 1], prim, dt=4.0e-5 * dx, t_end=1.0e-4)


def shock_bubble_2d(nx: int = 1024, ny: int = 512, mach: float = 1.5, Cs: float = 2.0) -> Problem:
    """2D shock-bubble interaction with three species (benchmark workload):
    domain [0, 2] x [0, 1], air at 101325 Pa and 298 K, a planar Mach 1.5
    shock at x = 0.25 moving +x, a helium bubble of radius 0.1 at (0.6, 0.65)
    beside a water column of radius 0.1 at (0.6, 0.35), interfaces smoothed by
    tanh over C_s = 2 cells with p and T uniform across them, minor volume
    fraction 1e-8, transmissive boundaries, CFL 0.4.
    Species order: water, air, helium."""
    fl = [BENCH_WATER, BENCH_AIR, BENCH_HELIUM]
    gamma, pinf, cv, q = _species(fl)
    x, y = cell_centers([nx, ny], [0.0, 0.0], [2.0, 1.0])
    dx = 1.0 / ny
    p1, T1 = 101325.0, 298.0
    rho_air = p1 / ((BENCH_AIR["gamma"] - 1.0) * (BENCH_AIR["cp"] / BENCH_AIR["gamma"]) * T1)
    p2, rho2, u2 = normal_shock(1.4, p1, rho_air, mach)
    T2 = T1 * (p2 / p1) * (rho_air / rho2)
    post = x < 0.25
    f_he = smooth_step(np.hypot(x - 0.6, y - 0.65) - 0.1, Cs * dx)
    f_w = smooth_step(np.hypot(x - 0.6, y - 0.35) - 0.1, Cs * dx)
    a_w = MINOR + f_w * (1.0 - 3.0 * MINOR)
    a_he = MINOR + f_he * (1.0 - 3.0 * MINOR)
    nc = nx * ny
    u = np.where(post, u2, 0.0)
    prim = _assemble(3, 2, [a_w, 1.0 - a_w - a_he], [u, np.zeros(nc)],
                     np.where(post, p2, p1), np.where(post, T2, T1))
    return Problem("shock_bubble_2d_3species", gamma, pinf, cv, q, [nx, ny], [0.0, 0.0],
                   [2.0, 1.0], [0, 0, 0, 0], prim, cfl=0.4, nsteps=2000)


def shock_water_column_2d(nx: int = 2048, ny: int = 1024, third_species: bool = True) -> Problem:
    """Shape of the Mach 1.47 shock-water-cylinder problem of Sec. 5.7 with the
    paper's fluids: domain [-10D, 10D] x [-5D, 5D], D = 4.8 mm, water cylinder
    of diameter D at the origin, pre-/post-shock air of the paper's table, the
    shock placed so that it reaches the cylinder after 5 us, constant
    extrapolation at all boundaries. With `third_species`, an SF6 bubble of
    radius D/2 at (3D, 0) is added (the learned-detector workload)."""
    fl = [PAPER_WATER, PAPER_AIR] + ([PAPER_SF6] if third_species else [])
    gamma, pinf, cv, q = _species(fl)
    N = len(fl)
    Dm = 4.8e-3
    x, y = cell_centers([nx, ny], [-10 * Dm, -5 * Dm], [10 * Dm, 5 * Dm])
    p1, T1 = 1.01325e5, 298.0
    u_post, p_post = 228.00747932015310, 2.3855789125e5
    rho_air_post = 2.1397213925906398 / (1.0 - 2 * MINOR if third_species else 1.0 - MINOR)
    T_post = temperature_of(PAPER_AIR, p_post, rho_air_post)
    c1 = math.sqrt(1.4 * p1 / (p1 / ((1.4 - 1.0) * (1007.0 / 1.4) * T1)))
    x_shock = -Dm / 2 - 5.0e-6 * 1.47 * c1
    post = x < x_shock
    f_w = (np.hypot(x, y) < Dm / 2).astype(np.float64)
    nc = nx * ny
    a_w = MINOR + f_w * (1.0 - N * MINOR)
    alphas = [a_w]
    if third_species:
        f_s = (np.hypot(x - 3 * Dm, y) < Dm / 2).astype(np.float64)
        a_s = MINOR + f_s * (1.0 - 3.0 * MINOR)
        alphas.append(1.0 - a_w - a_s)
    u = np.where(post, u_post, 0.0)
    prim = _assemble(N, 2, alphas, [u, np.zeros(nc)], np.where(post, p_post, p1),
                     np.where(post, T_post, T1))
    return Problem("shock_water_column_2d", gamma, pinf, cv, q, [nx, ny], [-10 * Dm, -5 * Dm],
                   [10 * Dm, 5 * Dm], [0, 0, 0, 0], prim, cfl=0.5)


def undex_2d(nx: int = 1536, ny: int = 1920) -> Problem:
    """Three-species extreme underwater explosion of Sec. 5.10 with the paper's
    fluids (water, air, detonation products gamma 1.25, c_p 1000): a 16 L x
    20 L domain, L = 1 m, with the free surface at y = 0 and 6 L of water below
    it (the schematic's proportions; the text's y-range is read as [-6 L, 14 L]),
    a detonation-gas bubble of radius 0.3 L centred at (0, -0.5 L) at 1e12 Pa and
    1250 kg/m^3, water and air at 101325 Pa and 298 K, minor volume fractions
    1e-8, sharp interfaces, constant extrapolation at every boundary."""
    fl = [PAPER_WATER, PAPER_AIR, PAPER_DETONATION]
    gamma, pinf, cv, q = _species(fl)
    x, y = cell_centers([nx, ny], [-8.0, -6.0], [8.0, 14.0])
    bubble = np.hypot(x, y + 0.5) < 0.3
    water = (y < 0.0) & ~bubble
    air = (y >= 0.0) & ~bubble
    a1 = np.where(water, 1.0 - 2.0 * MINOR, MINOR)
    a2 = np.where(air, 1.0 - 2.0 * MINOR, MINOR)
    p_det, rho_det = 1.0e12, 1250.0
    T_det = temperature_of(PAPER_DETONATION, p_det, rho_det)
    p = np.where(bubble, p_det, 101325.0)
    T = np.where(bubble, T_det, 298.0)
    nc = nx * ny
    prim = _assemble(3, 2, [a1, a2], [np.zeros(nc), np.zeros(nc)], p, T)
    return Problem("undex_2d", gamma, pinf, cv, q, [nx, ny], [-8.0, -6.0], [8.0, 14.0], [0, 0, 0, 0], prim,
                   cfl=0.5, t_end=2.5e-4)


def mach100_jet_2d(nx: int = 1024, ny: int = 512) -> Problem:
    """Two-dimensional Mach 100 water jet of Sec. 5.9 with the paper's fluids:
    [0, L] x [-0.25 L, 0.25 L], L = 1 m, essentially pure air at 101325 Pa and
    298 K; a Dirichlet left boundary with a water jet (alpha_1 = 1 - 1e-8,
    u = 1.5e5 m/s) for |y| <= 0.05 L and ambient air elsewhere; constant
    extrapolation at the top, bottom and right."""
    fl = [PAPER_WATER, PAPER_AIR]
    gamma, pinf, cv, q = _species(fl)
    nc = nx * ny
    prim = _assemble(2, 2, [np.full(nc, MINOR)], [np.zeros(nc), np.zeros(nc)], np.full(nc, 101325.0),
                     np.full(nc, 298.0))
    yb = -0.25 + (np.arange(ny) + 0.5) * (0.5 / ny)
    jet = np.abs(yb) <= 0.05
    left = _assemble(2, 2, [np.where(jet, 1.0 - MINOR, MINOR)], [np.where(jet, 1.5e5, 0.0), np.zeros(ny)],
                     np.full(ny, 101325.0), np.full(ny, 298.0))
    return Problem("mach100_jet_2d", gamma, pinf, cv, q, [nx, ny], [0.0, -0.25], [1.0, 0.25], [2, 0, 0, 0], prim,
                   cfl=0.5, boundary={0: left})


def dirichlet_box(n, seed: int = 7) -> Problem:
    """Seeded two-species state (the paper's water and air) on [0, 1]^D, D =
    len(n), with a Dirichlet state on every side: the interior is smooth
    (alpha_1 = 0.5 + 0.4 sin, |u| <= 50 m/s, p in 1e5..2e5 Pa, T in 300..400 K),
    each boundary cell an independent random state, so the stencils next to
    every side see jumps. For the boundary's wiring: ghost layers, sides and
    transverse indices."""
    rng = np.random.default_rng(seed)
    D = len(n)
    fl = [PAPER_WATER, PAPER_AIR]
    gamma, pinf, cv, q = _species(fl)
    X = cell_centers(list(n), [0.0] * D, [1.0] * D)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=(4, D))
    wave = [sum(np.sin(2.0 * math.pi * (d + 1) * X[d] + ph[j, d]) for d in range(D)) / D for j in range(4)]
    prim = _assemble(2, D, [0.5 + 0.4 * wave[0]], [50.0 * wave[1 + (d % 2)] for d in range(D)],
                     1.5e5 + 0.5e5 * wave[3], 350.0 + 50.0 * wave[2])
    nc = int(np.prod(n))
    boundary = {}
    for b in range(2 * D):
        ns = nc // n[b // 2]
        boundary[b] = _assemble(2, D, [rng.uniform(1e-6, 1.0 - 1e-6, ns)],
                                [rng.normal(0.0, 100.0, ns) for _ in range(D)],
                                10.0 ** rng.uniform(5.0, 6.0, ns), rng.uniform(250.0, 600.0, ns))
    return Problem("dirichlet_box_%dd" % D, gamma, pinf, cv, q, list(n), [0.0] * D, [1.0] * D, [2] * (2 * D), prim,
                   cfl=0.45, boundary=boundary)


def interface_3d(n: int = 256, mach: float = 1.5, seed: int = 20221003) -> Problem:
    """3D planar liquid/gas interface with a seeded multimode perturbation
    (benchmark workload): [0, 1]^3, liquid for x > x_i(y, z), a 50/50 mixture
    of the two ideal gases (gamma 1.4 and 1.67) for x < x_i,
    x_i = 0.5 + sum_{4 <= |k| <= 16} a_k cos(2 pi (k_y y + k_z z) + phi_k),
    a_k ~ 1/|k| rescaled to a maximum amplitude of 0.01, a planar shock in the
    gas at x = 0.3 moving +x, periodic in y and z, transmissive in x."""
    fl = [BENCH_WATER, BENCH_AIR, BENCH_HELIUM]
    gamma, pinf, cv, q = _species(fl)
    rng = np.random.default_rng(seed)
    x, y, z = cell_centers([n, n, n], [0.0] * 3, [1.0] * 3)
    modes = [(ky, kz) for ky in range(-16, 17) for kz in range(-16, 17)
             if 4 <= math.hypot(ky, kz) <= 16]
    phis = rng.uniform(0.0, 2.0 * math.pi, size=len(modes))
    yy = (np.arange(n) + 0.5) / n
    Y, Z = np.meshgrid(yy, yy, indexing="xy")
    pert = np.zeros_like(Y)
    for (ky, kz), ph in zip(modes, phis):
        pert += (1.0 / math.hypot(ky, kz)) * np.cos(2 * math.pi * (ky * Y + kz * Z) + ph)
    pert *= 0.01 / np.max(np.abs(pert))
    # Y, Z from meshgrid(indexing="xy") are indexed [z, y]; cells are ordered
    # (z, y, x) with x fastest, so the perturbation broadcasts along x.
    xi = 0.5 + np.broadcast_to(pert[:, :, None], (n, n, n)).reshape(-1)
    gas = x < xi
    p1, T1 = 101325.0, 298.0
    half = 0.5 - 5.0e-9
    # mixture gamma and density of the 50/50 gas for the shock relations
    S = half / 0.4 + half / 0.67
    gbar = 1.0 + 1.0 / S
    rho_mix = sum(half * p1 / ((f["gamma"] - 1.0) * (f["cp"] / f["gamma"]) * T1)
                  for f in fl[1:])
    p2, rho2, u2 = normal_shock(gbar, p1, rho_mix, mach)
    T2 = T1 * (p2 / p1) * (rho_mix / rho2)
    post = x < 0.3
    a_w = np.where(gas, MINOR, 1.0 - 2 * MINOR)
    a_air = np.where(gas, half, MINOR)
    nc = n ** 3
    u = np.where(post, u2, 0.0)
    prim = _assemble(3, 3, [a_w, a_air], [u, np.zeros(nc), np.zeros(nc)],
                     np.where(post, p2, p1), np.where(post, T2, T1))
    return Problem("interface_3d", gamma, pinf, cv, q, [n, n, n], [0.0] * 3, [1.0] * 3,
                   [0, 0, 1, 1, 1, 1], prim, cfl=0.4, nsteps=500)


def batch_instances(count: int = 64, seed: int = 4242, scale: int = 128) -> List[Problem]:
    """Batched workload: `count` seeded 2D shock-droplet/bubble instances with
    uneven grids nx = scale*U{1..8}, ny = scale*U{1..4} clamped to
    [scale, 8 scale] x [scale, 4 scale], shock Mach U[1.2, 3], radius
    U[0.05, 0.2] L_y, two or three species (a water droplet in air and/or a
    helium bubble)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = scale * int(rng.integers(1, 9))
        ny = scale * int(rng.integers(1, 5))
        mach = float(rng.uniform(1.2, 3.0))
        r = float(rng.uniform(0.05, 0.2))
        three = bool(rng.integers(0, 2))
        fl = [BENCH_WATER, BENCH_AIR] + ([BENCH_HELIUM] if three else [])
        gamma, pinf, cv, q = _species(fl)
        N = len(fl)
        Ly = 1.0
        Lx = nx / ny
        x, y = cell_centers([nx, ny], [0.0, 0.0], [Lx, Ly])
        dx = Ly / ny
        p1, T1 = 101325.0, 298.0
        rho_air = p1 / (0.4 * (1007.0 / 1.4) * T1)
        p2, rho2, u2 = normal_shock(1.4, p1, rho_air, mach)
        T2 = T1 * (p2 / p1) * (rho_air / rho2)
        xs = 0.1 * Lx
        rr = min(r, 0.3 * Lx, 0.45 * Ly)
        cx = min(xs + 1.5 * rr + 0.05 * Lx, Lx - 1.1 * rr)
        f_w = smooth_step(np.hypot(x - cx, y - (0.5 * Ly if not three else 0.3 * Ly)) - rr * (1 if not three else 0.6), 2 * dx)
        a_w = MINOR + f_w * (1.0 - N * MINOR)
        alphas = [a_w]
        if three:
            f_he = smooth_step(np.hypot(x - cx, y - 0.72 * Ly) - 0.6 * rr, 2 * dx)
            a_he = MINOR + f_he * (1.0 - N * MINOR)
            alphas.append(1.0 - a_w - a_he)
        post = x < xs
        nc = nx * ny
        prim = _assemble(N, 2, alphas, [np.where(post, u2, 0.0), np.zeros(nc)],
                         np.where(post, p2, p1), np.where(post, T2, T1))
        out.append(Problem(f"batch_{i:02d}", gamma, pinf, cv, q, [nx, ny], [0.0, 0.0], [Lx, Ly],
                           [0, 0, 0, 0], prim, cfl=0.4, extra=dict(mach=mach, radius=r)))
    return out


def random_admissible_states(N: int, D: int, count: int, seed: int, fluids=None):
    """Seeded random primitive states (alpha_k in (0,1), u, p, T) for
    cell-local property tests; returns (prim[N+D+1, count], fluid table)."""
    rng = np.random.default_rng(seed)
    fl = fluids or ([BENCH_WATER, BENCH_AIR, BENCH_HELIUM][:N] if N <= 3 else None)
    gamma, pinf, cv, q = _species(fl)
    a = rng.dirichlet(np.full(N, 0.7), size=count).T  # (N, count)
    a = np.clip(a, 1e-9, None)
    a /= a.sum(axis=0)
    u = rng.normal(0.0, 200.0, size=(D, count))
    p = 10.0 ** rng.uniform(4.0, 9.0, size=count)
    T = rng.uniform(150.0, 2000.0, size=count)
    prim = _assemble(N, D, [a[k] for k in range(N - 1)], [u[d] for d in range(D)], p, T)
    return prim, (gamma, pinf, cv, q)
