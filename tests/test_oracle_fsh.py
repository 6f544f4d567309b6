"""Pins of the oracle's square-well free energy F_sh (Sec 2.3.2).

- Uniform mobile densities on a periodic box: sum_r U(r) = (sum_m K_sw[m])
  (sum_r rho_s(r)), so F_sh = -sum_i eps_i rho_i V_shell sum_r rho_s(r) with
  V_shell = 4/3 pi (r_out^3 - r_in^3) (the quadrature's exact volume) and the
  site density summed by numpy from its Gaussian definition.
- Linearity and the functional derivative: F_sh is linear in rho, and its
  derivative with respect to rho_i(r) is the well field -eps_i U(r), twice the
  oracle's mu_sh under the kept factor 1/2.
"""
import math

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density


def spec_wells(bc=("P", "P", "P"), shape=(10, 9, 8)):
    nz, ny, nx = shape
    rng = np.random.default_rng(8)
    R = (1.5, 2.0)
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=bc, R=R, q=(1, -1),
                       rho_b=tuple(bulk_density(0.1, r) for r in R), depth=(1.3, 0.6),
                       well_inner=2.0, well_outer=3.0, site_alpha=0.9,
                       sites=rng.uniform(0, 1, (5, 3)) * np.array([nx, ny, nz]))


def test_uniform_density_closed_form():
    spec = spec_wells()
    nz, ny, nx = spec.shape
    rho = np.stack([np.full(spec.shape, r) for r in spec.rho_b])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rs = np.zeros(spec.shape)
    for s in spec.sites:
        for ix in range(-3, 4):
            for iy in range(-3, 4):
                for iz in range(-3, 4):
                    d2 = ((x - s[0] - nx * ix) ** 2 + (y - s[1] - ny * iy) ** 2 + (z - s[2] - nz * iz) ** 2)
                    rs += np.exp(-spec.site_alpha * d2)
    rs *= (spec.site_alpha / np.pi) ** 1.5
    vshell = 4 / 3 * math.pi * (spec.well_outer ** 3 - spec.well_inner ** 3)
    ref = -sum(e * r for e, r in zip(spec.depth, spec.rho_b)) * vshell * rs.sum()
    assert oracle.square_well_energy(spec, rho) == pytest.approx(ref, rel=1e-12)


def test_linear_with_derivative_twice_mu_sh():
    spec = spec_wells(bc=("P", "P", "D"))
    rng = np.random.default_rng(9)
    a = rng.lognormal(0, 0.3, (2,) + spec.shape) * 0.01
    b = rng.lognormal(0, 0.3, (2,) + spec.shape) * 0.01
    F = lambda r: oracle.square_well_energy(spec, r)
    assert F(2.0 * a - 0.5 * b) == pytest.approx(2.0 * F(a) - 0.5 * F(b), rel=1e-12)
    msh = oracle.mu_sh(spec, oracle.site_density(spec))         # with the kept 1/2
    for i, k in [(0, 17), (1, 300), (0, 555)]:
        e = np.zeros_like(a)
        e.reshape(2, -1)[i, k] = 1.0
        assert F(e) == pytest.approx(2.0 * msh.reshape(2, -1)[i, k], rel=1e-12)
