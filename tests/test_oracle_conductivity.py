"""Pins of the oracle's conductivity (Sec 4.2.1: current density averaged along
the transport axis over the applied field).

- Exact discrete steady state: with uniform densities rho_b, a linear phi
  and no excess chemical potential, the Slotboom flux through every face is
  2 D rho_b tanh(q (phi_k - phi_k+1) / 2) per face (harmonic mean of
  D exp(-q phi)), so the conductivity is
  sum_i q_i^2 D_i rho_b,i tanh(q_i d/2) / (q_i d/2), d = (phi_hi - phi_lo)/(nz+1),
  which tends to the Nernst-Einstein value sum_i q_i^2 D_i rho_b,i.
- SI units: the reduced value times e^2 D / (k_B T h^3), with Table 1's beta
  at 223 K, against the same product written with the SI constants.
"""
import math

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec


def ideal_state(bias, nz=9, q=(1, -1, 2), rho_b=(0.01, 0.006, 0.002), D=(1.0, 0.5, 2.0)):
    spec = ProblemSpec(nx=4, ny=3, nz=nz, bc=("P", "P", "D"), R=(1.0,) * len(q), q=q, rho_b=rho_b, D=D,
                       phi_lo=0.0, phi_hi=bias)
    z = np.arange(1, nz + 1)[:, None, None]
    phi = np.broadcast_to(bias * z / (nz + 1), spec.shape).copy()
    mu = np.zeros(spec.shape)
    flux = []
    for i in range(spec.s):
        rbar = rho_b[i] * np.exp(q[i] * phi)
        flux.append(oracle.np_flux(spec, i, phi, mu, 0.0, rbar))
    return spec, np.array(flux)


@pytest.mark.parametrize("bias", [1e-4, 0.3, -2.0])
def test_exact_steady_state_conductivity(bias):
    spec, flux = ideal_state(bias)
    d = bias / (spec.nz + 1)
    for i in range(spec.s):
        per_face = 2 * spec.D[i] * spec.rho_b[i] * math.tanh(spec.q[i] * -d / 2) * spec.nx * spec.ny
        # rho_bar differences cancel to ~eps / |q d| relative at tiny bias
        np.testing.assert_allclose(flux[i], per_face, rtol=1e-10)
    sigma, _ = oracle.conductivity(spec, flux)
    ref = sum(q * q * Di * r * math.tanh(q * d / 2) / (q * d / 2) for q, Di, r in zip(spec.q, spec.D, spec.rho_b))
    assert sigma == pytest.approx(ref, rel=1e-10)
    ne = sum(q * q * Di * r for q, Di, r in zip(spec.q, spec.D, spec.rho_b))
    if abs(bias) < 1e-3:
        assert sigma == pytest.approx(ne, rel=1e-8)       # Nernst-Einstein limit
    else:
        assert sigma < ne                                 # tanh(x)/x < 1


def test_si_conversion_with_table1_units():
    spec, flux = ideal_state(0.05)
    spec.temperature_K = 223.0
    spec.h_nm = 0.5
    sigma, si = oracle.conductivity(spec, flux, D_m2_per_s=1e-10)     # 1e-6 cm^2/s (Table 1)
    e, kB = 1.602176634e-19, 1.380649e-23
    ref = sigma * e * e * 1e-10 / (kB * 223.0 * (0.5e-9) ** 3) / 100.0
    assert si == pytest.approx(ref, rel=1e-9)
    # beta at 223 K is Table 1's 52.03749 / eV (printed from an older k_B: 1.4e-5 apart)
    assert si == pytest.approx(sigma * e * 52.03749 * 1e-10 / (0.5e-9) ** 3 / 100.0, rel=1e-4)
