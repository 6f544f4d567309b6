"""Pins of the oracle's relaxed Gummel iteration (Sec 3.2) on small, dilute
films (8 x 8 x 10, R = 1h, packing 0.05 per ion, wells on 3 sites, random
fixed charge).

- Zero bias: the converged state is the self-consistent Poisson-Boltzmann-cDFT
  equilibrium rho_i = rho_b,i exp(mu_b,i + q_i phi_face - q_i phi - mu_ex,i)
  with a uniform Slotboom variable, and phi solves Poisson for that rho.
- Nonzero bias: the discrete flux through every z plane is the same (div J = 0)
  and cations drift down the potential.
- Linear and geometric density relaxation reach the same fixed point.
"""
import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density


def film(bias_lo, bias_hi, mix=0, tol=1e-11):
    rng = np.random.default_rng(0)
    shape = (10, 8, 8)
    rb = bulk_density(0.05, 1.0)
    return ProblemSpec(nx=8, ny=8, nz=10, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(1.0, 0.0), well_inner=2.0, well_outer=3.0,
                       sites=rng.uniform(0, 1, (3, 3)) * np.array([8, 8, 10]),
                       rho_f=rng.normal(0, 0.01, shape), phi_lo=bias_lo, phi_hi=bias_hi,
                       lambda_phi=0.3, lambda_rho=0.3, rho_mix=mix, tol=tol, max_iter=400)


@pytest.fixture(scope="module")
def zero_bias():
    spec = film(0.2, 0.2)
    return spec, oracle.gummel(spec)


def test_zero_bias_is_boltzmann(zero_bias):
    spec, r = zero_bias
    assert r["status"] == 0
    mu, bad = oracle.excess_mu(spec, r["rho"])
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    for i in range(2):
        q = spec.q[i]
        ref = spec.rho_b[i] * np.exp(mub[i] + q * 0.2 - q * r["phi"] - mu[i])
        np.testing.assert_allclose(r["rho"][i], ref, rtol=1e-8)


def test_zero_bias_phi_solves_poisson(zero_bias):
    spec, r = zero_bias
    phi, it, rel = oracle.poisson(spec, r["rho"], phi0=r["phi"])
    np.testing.assert_allclose(phi, r["phi"], atol=1e-9)


def test_geometric_relaxation_same_fixed_point(zero_bias):
    spec, r = zero_bias
    r2 = oracle.gummel(film(0.2, 0.2, mix=1))
    assert r2["status"] == 0
    np.testing.assert_allclose(r2["rho"], r["rho"], rtol=1e-8)
    np.testing.assert_allclose(r2["phi"], r["phi"], atol=1e-9)


def test_step_limited_relaxation_same_fixed_point(zero_bias):
    spec, r = zero_bias
    r2 = oracle.gummel(film(0.2, 0.2, mix=2))
    assert r2["status"] == 0
    np.testing.assert_allclose(r2["rho"], r["rho"], rtol=1e-8)


def test_biased_flux_is_conserved():
    spec = film(0.0, 0.6)
    r = oracle.gummel(spec)
    assert r["status"] == 0
    mu, _ = oracle.excess_mu(spec, r["rho"])
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    J = []
    for i in range(2):
        rbar = r["rho"][i] * np.exp(spec.q[i] * r["phi"] + mu[i])
        f = oracle.np_flux(spec, i, r["phi"], mu[i], mub[i], rbar)
        np.testing.assert_allclose(f, f.mean(), rtol=1e-6)
        J.append(f.mean())
    assert J[0] < 0 < J[1]      # cations toward low phi (z = 0 side), anions up


def test_not_converged_status():
    spec = film(0.0, 0.6)
    spec.max_iter = 3
    r = oracle.gummel(spec)
    assert r["status"] == 1 and r["iters"] == 3
