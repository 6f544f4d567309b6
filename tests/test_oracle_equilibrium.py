"""Pins of the oracle's equilibrium cDFT initial guess (Sec 3.2, choice of
initial guess): Boltzmann densities about the reservoirs with the
Poisson-Boltzmann potential, solved by Newton steps on phi and step-limited
geometric relaxation of rho.

1. Debye-Hueckel plates: point-like ions (R = 0.05 h, packing 5e-6), a 0.01
   kT/e bias between Dirichlet planes, periodic x, y.  The linearised discrete
   Poisson-Boltzmann equation (2 phi_k - phi_k-1 - phi_k+1) + kappa^2 phi_k = 0
   with phi_-1 = 0, phi_nz = V has the closed form
   phi_k = V sinh(theta (k+1)) / sinh(theta (nz+1)), cosh theta = 1 + kappa^2/2,
   kappa^2 = 4 pi lB sum q^2 rho_b; the nonlinear and excess terms are O(1e-5).
2. Zero bias: the equilibrium is the zero-flux PNP solution, so the oracle's
   Gummel iteration (linear Poisson + Slotboom Nernst-Planck) must reach the
   same state -- a different algorithm to the same fixed point.
3. With bias, the converged state satisfies its defining relations: the
   Boltzmann law with the oracle's own mu_ex, and the Poisson equation.
4. The Gummel iteration with the screened Poisson step (one Newton step with
   the densities' Boltzmann dependence on phi) is stable on a box many Debye
   lengths long where the plain step blows up, reaches the equilibrium at zero
   bias, and shares the plain iteration's fixed point with a bias.
"""
import numpy as np

from oracle import oracle
from workloads import ProblemSpec, bulk_density, uniform_sites


def dh_spec(phi_hi=0.01, nz=24):
    return ProblemSpec(nx=4, ny=4, nz=nz, bc=("P", "P", "D"), R=(0.05, 0.05), q=(1, -1), rho_b=(0.01, 0.01),
                       depth=(0.0, 0.0), sites=None, rho_f=None, phi_lo=0.0, phi_hi=phi_hi, eps_r=56.0,
                       lambda_rho=0.3)


def test_debye_hueckel_plates():
    spec = dh_spec()
    r = oracle.equilibrium(spec, tol=1e-12, max_iter=500)
    assert r["status"] == 0
    k2 = 4 * np.pi * r["lB"] * (0.01 + 0.01)
    th = np.arccosh(1 + k2 / 2)
    k = np.arange(spec.nz)
    ref = 0.01 * np.sinh(th * (k + 1)) / np.sinh(th * (spec.nz + 1))
    phi = r["phi"]
    for j in range(spec.ny):
        for i in range(spec.nx):
            assert np.abs(phi[:, j, i] - ref).max() <= 1e-4 * 0.01
    # cation depleted and anion enriched where phi > 0 (Boltzmann, not its inverse)
    assert np.abs(r["rho"][0] / 0.01 - np.exp(-phi)).max() <= 1e-4
    assert np.abs(r["rho"][1] / 0.01 - np.exp(phi)).max() <= 1e-4


def small_film(bias):
    rb = bulk_density(0.05, 1.0)
    sites = uniform_sites(np.random.default_rng(7), 2, 6, 6, 8)
    rf = np.random.default_rng(8).normal(0, 0.01, size=(8, 6, 6))
    return ProblemSpec(nx=6, ny=6, nz=8, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(1.0, 0.0), well_inner=1.5, well_outer=2.5, sites=sites, rho_f=rf,
                       phi_lo=0.0, phi_hi=bias, lambda_phi=0.3, lambda_rho=0.3, rho_mix=1, tol=1e-11,
                       max_iter=3000)


def test_zero_bias_equilibrium_is_the_pnp_fixed_point():
    spec = small_film(0.0)
    e = oracle.equilibrium(spec, tol=1e-11, max_iter=3000)
    g = oracle.gummel(spec)
    assert e["status"] == 0 and g["status"] == 0
    rb = spec.rho_b[0]
    # the state is far from uniform (wells, fixed charge), so this is no accident
    assert max(np.abs(g["rho"][i] / rb - 1).max() for i in range(2)) > 0.3
    assert np.abs(e["phi"] - g["phi"]).max() <= 1e-9
    assert max(np.abs(e["rho"][i] - g["rho"][i]).max() / rb for i in range(2)) <= 1e-9


def test_biased_equilibrium_satisfies_boltzmann_and_poisson():
    spec = small_film(0.5)
    e = oracle.equilibrium(spec, tol=1e-12, max_iter=3000)
    assert e["status"] == 0
    mu, bad = oracle.excess_mu(spec, e["rho"])
    assert bad == 0
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    for i in range(2):
        boltz = spec.rho_b[i] * np.exp(mub[i] - mu[i] - spec.q[i] * e["phi"])
        assert np.abs(e["rho"][i] - boltz).max() / spec.rho_b[i] <= 1e-9
    # Poisson residual of the converged potential with these densities
    phi, _, _ = oracle.poisson(spec, e["rho"], phi0=e["phi"], lin_tol=1e-14)
    assert np.abs(phi - e["phi"]).max() <= 1e-8


def long_box():
    rb = bulk_density(0.05, 1.0)
    rf = np.random.default_rng(3).normal(0, 0.02, size=(64, 4, 4))
    return ProblemSpec(nx=4, ny=4, nz=64, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(0.0, 0.0), sites=None, rho_f=rf, phi_lo=0.0, phi_hi=0.0,
                       lambda_phi=0.3, lambda_rho=0.3, rho_mix=1, tol=1e-10, max_iter=400)


def test_screened_poisson_step_is_stable_on_a_long_box():
    """64 planes of ~20 Debye lengths: the relaxed Gummel iteration with the
    plain Poisson solve amplifies the longest charge mode (loop gain
    l_phi l_rho kappa^2 / k^2 ~ 40 >> 1) and blows up; with the screened Newton
    step it converges, at zero bias to the equilibrium state."""
    import dataclasses
    spec = long_box()
    plain = oracle.gummel(spec)
    assert plain["status"] != 0
    scr = oracle.gummel(dataclasses.replace(spec, screened_poisson=True))
    assert scr["status"] == 0
    e = oracle.equilibrium(spec, tol=1e-10, max_iter=3000)
    rb = spec.rho_b[0]
    assert np.abs(scr["phi"] - e["phi"]).max() <= 1e-8
    assert max(np.abs(scr["rho"][i] - e["rho"][i]).max() / rb for i in range(2)) <= 1e-8


def test_screened_and_plain_gummel_share_the_biased_fixed_point():
    """Where both iterations converge (small film, 0.5 kT/e bias, a current
    flows), they reach the same state."""
    import dataclasses
    spec = small_film(0.5)
    a = oracle.gummel(spec)
    b = oracle.gummel(dataclasses.replace(spec, screened_poisson=True))
    assert a["status"] == 0 and b["status"] == 0
    rb = spec.rho_b[0]
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-8
    assert max(np.abs(a["rho"][i] - b["rho"][i]).max() / rb for i in range(2)) <= 1e-8


def test_adaptive_relaxation_shares_the_fixed_point():
    """Per-point adaptive relaxation (rho_mix 3) reaches the state of the
    global step-limited relaxation: only the path differs."""
    import dataclasses
    spec = small_film(0.5)
    a = oracle.gummel(dataclasses.replace(spec, rho_mix=2))
    b = oracle.gummel(dataclasses.replace(spec, rho_mix=3))
    assert a["status"] == 0 and b["status"] == 0
    rb = spec.rho_b[0]
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-8
    assert max(np.abs(a["rho"][i] - b["rho"][i]).max() / rb for i in range(2)) <= 1e-8
