"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and fills problem descriptions; it holds
none of the method's arithmetic.  The paper's LiPON site geometry and data are
not available, so seeded synthetic films stand in for them: uniform random
stationary sites, Gaussian fixed charge, lognormal density perturbations, with
the grid sizes, radii, packing fractions, well depths and temperatures of the
five workloads below.

Every array is drawn on the host in FP64 with ``numpy.random.default_rng(seed)``
(PCG64).  Draw order: sites (n x 3, uniform over the grid box in grid-index
units), then fields in C order [species][z][y][x].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# boundary types per axis: 'P' periodic, 'D' Dirichlet (z only), 'N' no-flux.
# For the cDFT integrals every non-periodic axis is zero-extended.


@dataclasses.dataclass
class ProblemSpec:
    nx: int
    ny: int
    nz: int
    bc: Tuple[str, str, str] = ("P", "P", "D")
    R: Sequence[float] = (2.0, 2.0)          # hard-sphere radii (h)
    q: Sequence[int] = (1, -1)               # valences
    rho_b: Sequence[float] = (0.0, 0.0)      # bulk densities (h^-3)
    D: Optional[Sequence[float]] = None      # diffusion coefficients (None -> 1)
    depth: Optional[Sequence[float]] = None  # square-well depth per species (kT)
    well_inner: float = 4.0                  # square-well shell inner radius sigma_ab (h)
    well_outer: float = 5.0                  # outer radius sigma_ab + width (h)
    sites: Optional[np.ndarray] = None       # (n, 3) site coordinates, grid-index units
    site_alpha: float = 1.0                  # Gaussian exponent (h^-2)
    rho_f: Optional[np.ndarray] = None       # fixed charge per cell (e h^-3), [nz, ny, nx]
    temperature_K: float = 300.0
    eps_r: float = 16.6
    h_nm: float = 1.0                        # grid spacing in nm
    phi_lo: float = 0.0                      # Dirichlet potential at the z = 0 side (kT/e)
    phi_hi: float = 0.0                      # Dirichlet potential at the z = top side (kT/e)
    lambda_phi: float = 0.3
    lambda_rho: float = 0.3
    rho_mix: int = 0                         # 0 linear, 1 geometric, 2 geometric step-limited
    tol: float = 1e-8
    max_iter: int = 500
    quad_nmu: int = 0                        # FMT quadrature counts (0 = default rule)
    quad_ntheta: int = 0
    quad_nr: int = 0
    well_nmu: int = 0                        # square-well quadrature counts
    well_ntheta: int = 0
    well_nr: int = 0
    sw_half: bool = True                     # keep the 1/2 of the mean-field mu_sh
    fft_len: Tuple[int, int, int] = (0, 0, 0)  # padded FFT lengths for the GPU plan (0 = auto)
    lin_tol: float = 0.0                     # linear-solve relative residual (0 = library default)
    autotune: bool = False                   # GPU plan: time candidate lengths and tiles, keep the fastest
    eq_init: bool = False                    # start the Gummel loop from the equilibrium cDFT state
    eq_tol: float = 0.0                      # its stopping residual (0 = library default)
    eq_max_iter: int = 0                     # its iteration cap (0 = library default)
    screened_poisson: bool = False           # Gummel Poisson step as one screened Newton step
    fmt: int = 0                             # hard-sphere functional: 0 Rosenfeld, 1 White Bear (MFMT)
    msa: bool = False                        # add the MSA electrostatic-correlation term (Sec 2.3.4)
    anderson: int = 0                        # Anderson mixing depth of the Gummel iteration (0 = relaxed only)
    phase_timing: bool = False               # the solve graph sums device time per phase of each iteration

    @property
    def s(self) -> int:
        return len(self.R)

    @property
    def shape(self) -> Tuple[int, int, int]:
        return (self.nz, self.ny, self.nx)

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def bulk_density(eta: float, R: float) -> float:
    """Number density of spheres of radius R at packing fraction eta."""
    return eta / (4.0 / 3.0 * math.pi * R ** 3)


def uniform_sites(rng: np.random.Generator, n: int, nx: int, ny: int, nz: int) -> np.ndarray:
    return rng.uniform(0.0, 1.0, size=(n, 3)) * np.array([nx, ny, nz], dtype=np.float64)


def lognormal_density(spec: ProblemSpec, seed: int, sigma: float = 0.1) -> np.ndarray:
    """rho_i = rho_b,i x lognormal(0, sigma) per cell, species in order."""
    rng = np.random.default_rng(seed)
    out = np.empty((spec.s,) + spec.shape)
    for i in range(spec.s):
        out[i] = spec.rho_b[i] * rng.lognormal(0.0, sigma, size=spec.shape)
    return out


# --------------------------------------------------------------------------
# Gummel solve of a film: grid n^3 (32^3 in the full size), periodic x,y,
# Dirichlet z with phi = 0 / 0.1 kT/e; two species q = +-1 of radius 2h at
# packing fraction 0.2 each; cation square well 1 kT deep, 1h wide, on 64
# uniform sites (seed 0); fixed charge N(0, 0.01^2) per cell (seed 1);
# relaxation 0.3 on phi; residual 1e-8; 300 K.  The density update uses the
# geometric relaxation with lambda_rho = 0.05: at total packing 0.4 the
# linear update with 0.3 is unstable (bulk 1/S(0) = 25 bounds the stable
# Picard step at 2/26).
def film_gummel(nx: int = 32, ny: int = 32, nz: int = 32, nsites: Optional[int] = None,
                seed_sites: int = 0, seed_rhof: int = 1, tol: float = 1e-8,
                max_iter: int = 500, phi_hi: float = 0.1, depth: float = 1.0) -> ProblemSpec:
    if nsites is None:
        nsites = max(1, (nx * ny * nz) // 512)
    R = 2.0
    rb = bulk_density(0.2, R)
    sites = uniform_sites(np.random.default_rng(seed_sites), nsites, nx, ny, nz)
    rho_f = np.random.default_rng(seed_rhof).normal(0.0, 0.01, size=(nz, ny, nx))
    sigma_ab = 2.0 * R   # site diameter taken equal to the cation diameter
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(R, R), q=(1, -1), rho_b=(rb, rb),
                       depth=(depth, 0.0), well_inner=sigma_ab, well_outer=sigma_ab + 1.0,
                       sites=sites, site_alpha=1.0, rho_f=rho_f, temperature_K=300.0,
                       phi_lo=0.0, phi_hi=phi_hi, lambda_phi=0.3, lambda_rho=0.05, rho_mix=1,
                       tol=tol, max_iter=max_iter)


# --------------------------------------------------------------------------
# Single mu_ex evaluation: n^3 grid (128^3 in the full size), zero-extended on
# every axis, three species of radius 1.5h, 2h, 3h at packing fraction 0.1
# each (0.3 total), densities rho_b x lognormal(0, 0.1) (seed 2), hard spheres
# only.  The full-size FFT grid is zero-padded to 2n per axis (256^3).
def mu_microbench(n: int = 128, seed: int = 2, fft_len: int = 0,
                  shape: Optional[Tuple[int, int, int]] = None) -> Tuple[ProblemSpec, np.ndarray]:
    nx, ny, nz = (n, n, n) if shape is None else shape
    R = (1.5, 2.0, 3.0)
    rb = tuple(bulk_density(0.1, r) for r in R)
    L = (fft_len, fft_len, fft_len) if fft_len else (0, 0, 0)
    spec = ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("N", "N", "D"), R=R, q=(1, -1, 0), rho_b=rb,
                       depth=(0.0, 0.0, 0.0), sites=None, rho_f=None, fft_len=L)
    return spec, lognormal_density(spec, seed)


# --------------------------------------------------------------------------
# Film with a third mobile species: nx x ny x nz (128 x 128 x 256 in the full
# size), species +1 (R 2h, eta 0.2), -1 (R 2h) and -1 (R 1h) with the anion
# densities set to half the cation's (bulk electroneutrality); cation wells
# 3 kT deep on 4096 sites (seed 0) at the full size; fixed charge seed 1.
# The box is ~200 Debye lengths long: the plain relaxed Gummel iteration is
# unstable there, so the solve uses the screened Poisson step, the
# equilibrium initial guess and the step-limited geometric relaxation.
def film3(nx: int = 128, ny: int = 128, nz: int = 256, nsites: Optional[int] = None,
          bias: float = 0.0, tol: float = 1e-8, max_iter: int = 2000) -> ProblemSpec:
    if nsites is None:
        nsites = max(1, (nx * ny * nz) // 1024)
    rb1 = bulk_density(0.2, 2.0)
    sites = uniform_sites(np.random.default_rng(0), nsites, nx, ny, nz)
    rho_f = np.random.default_rng(1).normal(0.0, 0.01, size=(nz, ny, nx))
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(2.0, 2.0, 1.0), q=(1, -1, -1),
                       rho_b=(rb1, rb1 / 2, rb1 / 2), depth=(3.0, 0.0, 0.0), well_inner=4.0,
                       well_outer=5.0, sites=sites, rho_f=rho_f, phi_lo=0.0, phi_hi=bias, tol=tol,
                       lambda_phi=0.3, lambda_rho=0.05, rho_mix=2, max_iter=max_iter,
                       screened_poisson=True, eq_init=True)


# --------------------------------------------------------------------------
# Batch of independent solves: grids from {32^3, 48^3, 64^3, 80x80x96, 96^3},
# temperatures U(250, 400) K with well depth 0.3 eV / kT, total packing
# fraction U(0.1, 0.35) split equally over the two ions, fixed-charge seeds
# 100..163, sites at one per 512 cells (seed = fixed-charge seed + 1000).
# Wells 9-14 kT deep on a fluid at packing up to 0.35 need the step-limited
# geometric density relaxation with per-point factors (with one global factor
# the densely packed well shells alternate at the step limit); grids of 64
# planes and more are many Debye lengths long and need the screened Poisson
# step.
BATCH_GRIDS = [(32, 32, 32), (48, 48, 48), (64, 64, 64), (80, 80, 96), (96, 96, 96)]
KB_EV_PER_K = 8.617333262e-5


def batch_specs(count: int = 64, seed: int = 4, grids=None, max_iter: int = 2000,
                tol: float = 1e-8) -> List[ProblemSpec]:
    rng = np.random.default_rng(seed)
    grids = BATCH_GRIDS if grids is None else grids
    out = []
    for j in range(count):
        nx, ny, nz = grids[int(rng.integers(len(grids)))]
        T = float(rng.uniform(250.0, 400.0))
        eta = float(rng.uniform(0.1, 0.35))
        seed_f = 100 + j
        R = 2.0
        rb = bulk_density(eta / 2.0, R)
        sites = uniform_sites(np.random.default_rng(seed_f + 1000), max(1, nx * ny * nz // 512), nx, ny, nz)
        rho_f = np.random.default_rng(seed_f).normal(0.0, 0.01, size=(nz, ny, nx))
        depth = 0.3 / (KB_EV_PER_K * T)
        out.append(ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(R, R), q=(1, -1),
                               rho_b=(rb, rb), depth=(depth, 0.0), well_inner=4.0, well_outer=5.0,
                               sites=sites, rho_f=rho_f, temperature_K=T, phi_lo=0.0, phi_hi=0.1,
                               lambda_phi=0.3, lambda_rho=0.05, rho_mix=3, tol=tol, max_iter=max_iter,
                               screened_poisson=True))
    return out


def _smooth_sizes(lo: int, hi: int) -> List[int]:
    """Even 2^a 3^b 5^c sizes in [lo, hi] (x is periodic and carries the
    two-for-one real transform, so it must be even)."""
    out = []
    for n in range(lo + (lo % 2), hi + 1, 2):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


# --------------------------------------------------------------------------
# Served requests: Poisson arrivals at `rate` per second (seed 5), cubic
# grids with log-uniform edge in [32, 256] rounded to an even 2^a 3^b 5^c size,
# bias U(0, 1) kT/e, temperature U(250, 400) K (well depth 0.3 eV / kT).
def serving_arrivals(count: int = 600, rate: float = 20.0, seed: int = 5, lo: int = 32, hi: int = 256):
    """[(arrival time s, edge n, bias, temperature)]; build each problem with serving_spec."""
    rng = np.random.default_rng(seed)
    sizes = np.array(_smooth_sizes(lo, hi))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        edge = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        n = int(sizes[np.argmin(np.abs(sizes - edge))])
        bias = float(rng.uniform(0.0, 1.0))
        T = float(rng.uniform(250.0, 400.0))
        out.append((t, n, bias, T))
    return out


def serving_spec(n: int, bias: float, T: float, max_iter: int = 2000, tol: float = 1e-8) -> ProblemSpec:
    """The 32^3 film's physics (2 ions, R 2h, packing 0.2 each, 1 kT wells on
    one site per 512 cells, fixed charge) on an n^3 grid at bias and T (which
    sets the Bjerrum length)."""
    spec = film_gummel(n, n, n, tol=tol, max_iter=max_iter, phi_hi=bias)
    spec.temperature_K = T
    spec.rho_mix = 3                  # per-point relaxation factors
    spec.screened_poisson = True      # edges up to 256: many Debye lengths
    return spec
