"""Seeded synthetic inputs for the dual-porosity oil-water problem.

This module is shared by the CPU oracle (``oracle/``) and the CUDA library
(``paper_1808_04338_gb300``).  It holds none of the method's arithmetic: it
only draws permeability fields, places wells and converts field units to SI.
Everything the method computes from these inputs (transmissibilities, well
indices, properties, residuals, Jacobians, solvers) lives separately on each
side.

Random numbers: SplitMix64 applied to a counter (seed, stream, index) gives a
uniform in (0, 1); Box-Muller on the two uniforms (2*loc, 2*loc+1) gives one
standard normal per grid location.  Permeability fields are lognormal and
uncorrelated per location (the paper gives no geostatistics).

Units: the paper's field units are converted with the constants below
(mD, psi, cP, bbl/day, day, ft, lbm/ft^3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MD = 9.869233e-16          # m^2 per millidarcy
PSI = 6894.757293168       # Pa per psi
CP = 1.0e-3                # Pa s per centipoise
BBL_DAY = 1.840130728e-6   # m^3/s per bbl/day
DAY = 86400.0              # s per day
FT = 0.3048                # m per ft

# Densities of oil and water given for the paper's examples: 58.0 and
# 62.4 lbm/ft^3 (Section 4, Example 1), in kg/m^3.
RHO_O_REF = 929.07
RHO_W_REF = 999.55

WELL_RATE_INJ = 0
WELL_BHP = 1
WELL_OIL_RATE = 2

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def splitmix64_uniform(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Counter-based uniforms in (0, 1): SplitMix64 of (seed, stream, index)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = np.uint64(seed) * _GOLDEN + np.uint64(stream) * _STREAM
        z = key + (idx + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normals(seed: int, stream: int, n: int) -> np.ndarray:
    """One standard normal per location from two counter uniforms (Box-Muller)."""
    loc = np.arange(n, dtype=np.uint64)
    u1 = splitmix64_uniform(seed, stream, 2 * loc)
    u2 = splitmix64_uniform(seed, stream, 2 * loc + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Well:
    kind: int            # WELL_RATE_INJ, WELL_BHP or WELL_OIL_RATE
    i: int
    j: int
    k_top: int
    k_bot: int
    target: float        # m^3/s (injector rate), Pa (BHP) or kg/s of oil (producer rate)
    rw: float = 0.25 * FT
    skin: float = 0.0
    limit: float = 0.0   # BHP limit of a rate-controlled well (Pa), 0: none
    wi: float = 0.0      # given well index (m^3), 0: Peaceman


@dataclass
class Problem:
    """One realisation: grid, rock, fluid, wells and the initial state (SI)."""
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    top_depth: float
    kf: np.ndarray
    km: np.ndarray
    phi_f: np.ndarray
    phi_m: np.ndarray
    sigma: float
    c_rock: float
    p_ref_rock: float
    mu_o: float
    mu_w: float
    c_o: float
    c_w: float
    rho_o_ref: float
    rho_w_ref: float
    p_ref: float
    swc: float
    sor: float
    g: float
    wells: list = field(default_factory=list)
    p0: np.ndarray | None = None
    sw0: np.ndarray | None = None
    bhp0: np.ndarray | None = None
    dt: float = DAY
    nsteps: int = 1
    # capillary pressure p_cow(s_w) per continuum: None, or an (n, 2) array of
    # (s_w, p_cow in Pa) points with s_w strictly ascending
    pc_f: np.ndarray | None = None
    pc_m: np.ndarray | None = None

    def pc_tables(self):
        """(n, contiguous float64 table) of the fracture and matrix curves."""
        out = []
        for t in (self.pc_f, self.pc_m):
            if t is None:
                out.append((0, np.zeros(2)))
            else:
                a = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1, 2))
                out.append((a.shape[0], a.reshape(-1)))
        return out

    @property
    def n_loc(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_cells(self) -> int:
        return 2 * self.n_loc

    @property
    def n_wells(self) -> int:
        return len(self.wells)

    @property
    def n_unknowns(self) -> int:
        return 2 * (self.n_cells + self.n_wells)


def _base(name, nx, ny, nz, kf_md, km_md, phi_f, phi_m, sigma, wells, seed,
          dx=20.0, dy=20.0, dz=5.0, p0_psi=3000.0, sw0=0.2, dt_days=1.0,
          nsteps=1, g=0.0, c_rock_psi=0.0):
    n = nx * ny * nz
    p0 = p0_psi * PSI
    prob = Problem(
        name=name, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
        top_depth=2000.0 * FT,
        kf=np.ascontiguousarray(kf_md * MD, dtype=np.float64),
        km=np.ascontiguousarray(km_md * MD, dtype=np.float64),
        phi_f=np.full(n, phi_f), phi_m=np.full(n, phi_m),
        sigma=sigma, c_rock=c_rock_psi / PSI, p_ref_rock=p0,
        mu_o=2.0 * CP, mu_w=0.5 * CP, c_o=1e-5 / PSI, c_w=1e-5 / PSI,
        rho_o_ref=RHO_O_REF, rho_w_ref=RHO_W_REF, p_ref=p0,
        swc=0.2, sor=0.2, g=g, wells=wells,
        p0=np.full(2 * n, p0), sw0=np.full(2 * n, sw0),
        dt=dt_days * DAY, nsteps=nsteps)
    prob.bhp0 = np.array([w.target if w.kind == WELL_BHP else p0
                          for w in wells], dtype=np.float64)
    prob.seed = seed
    return prob


def five_spot(nx, ny, nz, rate_bbl=100.0, bhp_psi=2500.0):
    """Injectors at the four corners, a BHP producer in the middle; all layers."""
    inj = [(0, 0), (nx - 1, 0), (0, ny - 1), (nx - 1, ny - 1)]
    wells = [Well(WELL_RATE_INJ, i, j, 0, nz - 1, rate_bbl * BBL_DAY) for i, j in inj]
    wells.append(Well(WELL_BHP, nx // 2, ny // 2, 0, nz - 1, bhp_psi * PSI))
    return wells


def tiny(seed: int = 0) -> Problem:
    """10x10x3 grid, 600 cells: lognormal fracture perm (ln 100 mD, sd 1),
    a 100 bbl/d corner injector and a 2500 psi opposite-corner producer,
    ten 1-day steps."""
    nx, ny, nz = 10, 10, 3
    n = nx * ny * nz
    kf = np.exp(math.log(100.0) + 1.0 * normals(seed, 0, n))
    wells = [Well(WELL_RATE_INJ, 0, 0, 0, nz - 1, 100.0 * BBL_DAY),
             Well(WELL_BHP, nx - 1, ny - 1, 0, nz - 1, 2500.0 * PSI)]
    return _base("tiny_10x10x3", nx, ny, nz, kf, np.full(n, 0.1), 0.01, 0.2,
                 0.08, wells, seed, dt_days=1.0, nsteps=10)


def layered(nx=100, ny=100, nz=10, seed: int = 0) -> Problem:
    """100x100x10 grid, 200k cells: lognormal fracture perm (sd 1) whose
    log-mean rises from ln 50 to ln 500 mD over five groups of two layers,
    five-spot wells, thirty 5-day steps."""
    n = nx * ny * nz
    k = np.arange(n) // (nx * ny)
    group = np.minimum(k * 5 // nz, 4)
    mu = math.log(50.0) + (math.log(500.0) - math.log(50.0)) * group / 4.0
    kf = np.exp(mu + 1.0 * normals(seed, 0, n))
    return _base(f"layered_{nx}x{ny}x{nz}", nx, ny, nz, kf, np.full(n, 0.1),
                 0.01, 0.2, 0.08, five_spot(nx, ny, nz), seed, dt_days=5.0,
                 nsteps=30)


def field8m(nx=200, ny=200, nz=50, seed: int = 0) -> Problem:
    """200x200x50 grid, 4M cells, 8M unknowns: fracture perm lognormal
    (ln 100 mD, sd 2), matrix perm lognormal (ln 0.05 mD, sd 0.5), 9 injectors
    on i, j in {50, 100, 150} and 16 producers on i, j in {25, 75, 125, 175}
    (coordinates scaled with nx, ny for smaller grids), all layers."""
    n = nx * ny * nz
    kf = np.exp(math.log(100.0) + 2.0 * normals(seed, 0, n))
    km = np.exp(math.log(0.05) + 0.5 * normals(seed, 2, n))
    wells = []
    for a in (50, 100, 150):
        for b in (50, 100, 150):
            wells.append(Well(WELL_RATE_INJ, a * nx // 200, b * ny // 200, 0,
                              nz - 1, 100.0 * BBL_DAY))
    for a in (25, 75, 125, 175):
        for b in (25, 75, 125, 175):
            wells.append(Well(WELL_BHP, a * nx // 200, b * ny // 200, 0,
                              nz - 1, 2500.0 * PSI))
    return _base(f"field_{nx}x{ny}x{nz}", nx, ny, nz, kf, km, 0.01, 0.2, 0.08,
                 wells, seed, dt_days=5.0, nsteps=1)


def ensemble_member(r: int) -> Problem:
    """Member r of the 64-realisation ensemble: size grows from 20x20x5 to
    80x80x20 with r, its own seed and a shape factor in [0.01, 0.2]."""
    t = r / 63.0
    nxy = int(round(20 + 60 * t))
    nz = int(round(5 + 15 * t))
    n = nxy * nxy * nz
    kf = np.exp(math.log(100.0) + 1.0 * normals(r, 0, n))
    sigma = 0.01 + 0.19 * float(splitmix64_uniform(r, 1, np.array([0]))[0])
    return _base(f"member{r}_{nxy}x{nxy}x{nz}", nxy, nxy, nz, kf,
                 np.full(n, 0.1), 0.01, 0.2, sigma, five_spot(nxy, nxy, nz), r,
                 dt_days=5.0, nsteps=1)


def one_d(nx: int, perm_md: float = 100.0, q_bbl: float = 100.0,
          bhp_psi: float = 2500.0, sigma: float = 0.08) -> Problem:
    """nx x 1 x 1 line for the single-phase incompressible limit: no
    compressibility, no gravity, water-filled (Sw = 1), a rate injector at
    i = 0 and a BHP producer at i = nx - 1."""
    n = nx
    prob = _base(f"line_{nx}", nx, 1, 1, np.full(n, perm_md), np.full(n, 0.1),
                 0.01, 0.2, sigma,
                 [Well(WELL_RATE_INJ, 0, 0, 0, 0, q_bbl * BBL_DAY),
                  Well(WELL_BHP, nx - 1, 0, 0, 0, bhp_psi * PSI)], 0,
                 sw0=1.0, dt_days=1.0, nsteps=1)
    prob.c_o = 0.0
    prob.c_w = 0.0
    prob.c_rock = 0.0
    return prob


CONFIGS = {
    "tiny": tiny,
    "layered": layered,
    "field8m": field8m,
}


def served_member(r: int) -> Problem:
    """Realisation r of the 128 of the served stream: a log-uniform size from
    about 10k to 1M cells (5k to 500k locations, ten layers), its own seed
    (1000 + r), fracture perm lognormal (ln 100 mD, sd 1), a shape factor in
    [0.01, 0.2] and five-spot wells."""
    seed = 1000 + r
    u = float(splitmix64_uniform(seed, 3, np.array([0]))[0])
    n_loc = 5000.0 * 100.0 ** u
    nz = 10
    nxy = max(3, int(round(math.sqrt(n_loc / nz))))
    n = nxy * nxy * nz
    kf = np.exp(math.log(100.0) + 1.0 * normals(seed, 0, n))
    sigma = 0.01 + 0.19 * float(splitmix64_uniform(seed, 1, np.array([0]))[0])
    return _base(f"served{r}_{nxy}x{nxy}x{nz}", nxy, nxy, nz, kf, np.full(n, 0.1), 0.01, 0.2,
                 sigma, five_spot(nxy, nxy, nz), seed, dt_days=5.0, nsteps=1)


def request_stream(n_requests: int = 512, rate_per_s: float = 200.0, n_real: int = 128,
                   seed: int = 7):
    """A seeded Poisson request stream: arrival times (s, exponential gaps of
    mean 1/rate), the realisation of each request (uniform over n_real) and
    its timestep in days (1, 2, 5 or 10, so that Newton counts differ)."""
    k = np.arange(n_requests, dtype=np.uint64)
    gaps = -np.log(splitmix64_uniform(seed, 0, k)) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    real = np.minimum((splitmix64_uniform(seed, 1, k) * n_real).astype(np.int64), n_real - 1)
    dts = np.array([1.0, 2.0, 5.0, 10.0])[
        np.minimum((splitmix64_uniform(seed, 2, k) * 4).astype(np.int64), 3)]
    return arrivals, real, dts


LBM_FT3 = 16.01846337       # kg/m^3 per lbm/ft^3


def paper_example(which: int, days: float = 1.0, nsteps: int = 10, grid=None) -> Problem:
    """The setups of the paper's Examples 1 (10x10x1) and 2 (10x10x3), Section
    4: field units converted to SI, oil density at the reference pressure
    from the stock-tank density and the formation volume factor (58.0 lbm/ft^3
    / 1.036), rock and oil compressibility about 15 psi, gravity with depth,
    fracture and matrix initial states, a water injector with a given well
    index and a maximum BHP, two oil-rate producers with a minimum BHP.
    Not given by the paper, read here: water viscosity 1 cP and
    compressibility 3e-6/psi; Corey curves with no residual saturations;
    transfer through the Kazemi shape factor of the grid block, with the
    matrix's vertical permeability folded into sigma (k_m = k_m,x).
    grid = (nx, ny, nz) gives the same example on another grid (Example 3 is
    Example 1 at 500x500x50): the same cells and rates, the wells in the
    cells at the same relative positions, perforating the top layer as the
    paper's cells [i j 1] do."""
    if which == 1:
        nz, kmz, pm0, pf0, q_inj, q_oil = 1, 10.0, 2000.0, 1980.0, 500.0, 300.0
        inj, prods, h = (4, 0), [(0, 9), (9, 9)], 102.04
    else:
        nz, kmz, pm0, pf0, q_inj, q_oil = 3, 100.0, 800.0, 500.0, 200.0, 500.0
        inj, prods, h = (4, 4), [(0, 0), (9, 9)], 102.0
    nx = ny = 10
    if grid is not None:
        gx, gy, nz = grid
        inj = ((2 * inj[0] + 1) * gx // 20, (2 * inj[1] + 1) * gy // 20)
        prods = [((2 * i + 1) * gx // 20, (2 * j + 1) * gy // 20) for (i, j) in prods]
        nx, ny = gx, gy
    n = nx * ny * nz
    dx = dy = h * FT
    dz = 100.0 * FT
    kmx = 100.0
    sigma = 4.0 * (1.0 / dx ** 2 + 1.0 / dy ** 2 + (kmz / kmx) / dz ** 2)
    rho_o_std = 58.0 * LBM_FT3
    wells = [Well(WELL_RATE_INJ, inj[0], inj[1], 0, 0, q_inj * BBL_DAY, limit=5.0e4 * PSI,
                  wi=200.0 * BBL_DAY * CP / PSI)]
    for (i, j) in prods:
        wells.append(Well(WELL_OIL_RATE, i, j, 0, 0, q_oil * BBL_DAY * rho_o_std,
                          rw=0.25 * FT, limit=15.0 * PSI))
    p0 = np.empty(2 * n)
    p0[0::2], p0[1::2] = pf0 * PSI, pm0 * PSI
    sw0 = np.empty(2 * n)
    sw0[0::2], sw0[1::2] = 0.01, 0.08
    prob = Problem(
        name=f"example{which}" + (f"_{nx}x{ny}x{nz}" if grid is not None else ""),
        nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz,
        top_depth=2000.0 * FT - 0.5 * dz,
        kf=np.full(n, 395.85 * MD), km=np.full(n, kmx * MD),
        phi_f=np.full(n, 0.039585), phi_m=np.full(n, 0.1392),
        sigma=sigma, c_rock=3e-6 / PSI, p_ref_rock=15.0 * PSI,
        mu_o=40.0 * CP, mu_w=1.0 * CP, c_o=1.313e-5 / PSI, c_w=3e-6 / PSI,
        rho_o_ref=rho_o_std / 1.036, rho_w_ref=62.4 * LBM_FT3, p_ref=15.0 * PSI,
        swc=0.0, sor=0.0, g=9.80665, wells=wells, p0=p0, sw0=sw0,
        dt=days * DAY, nsteps=nsteps)
    prob.bhp0 = np.array([pf0 * PSI] * len(wells))
    prob.seed = 0
    return prob

