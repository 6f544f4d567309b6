"""Pins of the oracle's White Bear (modified FMT) functional, the variant the
paper names beside Rosenfeld's (Sec 2.3.1):

1. Bulk: for one species the White Bear chemical potential is the
   Carnahan-Starling one, mu_ex = (8 eta - 9 eta^2 + 3 eta^3) / (1 - eta)^3 --
   through the reservoir formula and through the full oracle mu_ex on a
   uniform periodic fluid; for a mixture, the BMCSL equation of state.
2. The ten derivatives against a complex step of an independent numpy Phi.
3. The power series used near n3 = 0 (where the closed form cancels, and n3 is
   exactly 0 off the domain) against the closed form at 50 digits.
4. Reduction: a White Bear fluid differs from a Rosenfeld one (same inputs),
   and both agree at vanishing density.
"""
import numpy as np
import pytest

import brute
from oracle import oracle
from workloads import ProblemSpec, bulk_density


def cs_mu(eta):
    return (8 * eta - 9 * eta ** 2 + 3 * eta ** 3) / (1 - eta) ** 3


@pytest.mark.parametrize("eta", [0.05, 0.2, 0.35, 0.45])
def test_bulk_is_carnahan_starling(eta):
    R = 1.7
    rb = bulk_density(eta, R)
    mu = oracle.bulk_mu([R], [rb], fmt=1)[0]
    assert mu == pytest.approx(cs_mu(eta), rel=1e-13)
    # the Rosenfeld functional gives the Percus-Yevick value instead
    assert abs(oracle.bulk_mu([R], [rb], fmt=0)[0] - mu) > 1e-3 * eta


@pytest.mark.parametrize("eta", [0.1, 0.3])
def test_uniform_periodic_fluid_mu_ex_is_carnahan_starling(eta):
    R = 2.0
    rb = bulk_density(eta, R)
    spec = ProblemSpec(nx=8, ny=8, nz=8, bc=("P", "P", "P"), R=(R,), q=(0,), rho_b=(rb,), fmt=1)
    rho = np.full((1, 8, 8, 8), rb)
    mu, bad = oracle.excess_mu(spec, rho)
    assert bad == 0
    # the quadrature weights integrate a constant exactly, so the discrete
    # weighted densities of a uniform fluid are the continuum ones
    assert np.abs(mu - cs_mu(eta)).max() <= 1e-12 * cs_mu(eta)


def test_dphi_matches_complex_step_of_phi():
    rng = np.random.default_rng(11)
    n = np.zeros((10, 5))
    n[3] = rng.uniform(0.06, 0.6, 5)
    n[2] = rng.uniform(0.1, 2.0, 5)
    n[0] = n[2] / (4 * np.pi * 4.0)
    n[1] = n[2] / (4 * np.pi * 2.0)
    n[4:10] = rng.normal(0, 0.05, (6, 5))
    psi, bad = oracle.dphi(n, fmt=1)
    assert bad == 0
    for a in range(10):
        nc = n.astype(complex)
        nc[a] += 1e-30j
        d = brute.phi_white_bear(nc).imag / 1e-30
        np.testing.assert_allclose(psi[a], d, rtol=1e-12, atol=1e-14)
    # and the free energy itself
    assert oracle.fhs(n, fmt=1) == pytest.approx(np.sum(brute.phi_white_bear(n)), rel=1e-13)


def test_series_near_zero_packing():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50

    def exact(x):
        x = mpmath.mpf(x)
        f = lambda t: (t + (1 - t) ** 2 * mpmath.log(1 - t)) / (t ** 2 * (1 - t) ** 2)
        return f(x), mpmath.diff(f, x)

    # n2 = 1, every other density 0: psi2 = phi3 / (12 pi), psi3 = phi3' / (36 pi)
    xs = [1e-12, 1e-6, 1e-3, 0.02, 0.0499, 0.0501, 0.2]
    n = np.zeros((10, len(xs)))
    n[2] = 1.0
    n[3] = xs
    psi, bad = oracle.dphi(n, fmt=1)
    assert bad == 0
    for k, x in enumerate(xs):
        f, df = exact(x)
        assert psi[2, k] * 12 * np.pi == pytest.approx(float(f), rel=1e-13)
        assert psi[3, k] * 36 * np.pi == pytest.approx(float(df), rel=1e-11)
    # exactly zero packing (off the domain): the series' constant terms
    n[3] = 0.0
    psi, _ = oracle.dphi(n, fmt=1)
    assert psi[2, 0] * 12 * np.pi == pytest.approx(1.5, rel=1e-15)
    assert psi[3, 0] * 36 * np.pi == pytest.approx(8.0 / 3.0, rel=1e-15)


def test_mixture_bulk_is_bmcsl():
    """Three species: the White Bear reservoir chemical potentials equal the
    derivatives of the Boublik-Mansoori-Carnahan-Starling-Leland excess free
    energy density (an equation of state, not a density functional),
    (6/pi) [(xi2^3/xi3^2 - xi0) ln(1 - xi3) + 3 xi1 xi2 / (1 - xi3)
    + xi2^3 / (xi3 (1 - xi3)^2)],  xi_k = (pi/6) sum_i rho_i d_i^k."""
    sp = pytest.importorskip("sympy")
    R = [1.5, 2.0, 3.0]
    eta = [0.1, 0.12, 0.08]
    rb = [e / (4.0 / 3.0 * np.pi * r ** 3) for e, r in zip(eta, R)]
    rho = sp.symbols("r0:3", positive=True)
    xi = [sp.pi / 6 * sum(rho[i] * (2 * R[i]) ** k for i in range(3)) for k in range(4)]
    F = (6 / sp.pi) * ((xi[2] ** 3 / xi[3] ** 2 - xi[0]) * sp.log(1 - xi[3]) + 3 * xi[1] * xi[2] / (1 - xi[3])
                       + xi[2] ** 3 / (xi[3] * (1 - xi[3]) ** 2))
    sub = {rho[i]: rb[i] for i in range(3)}
    ref = [float(sp.diff(F, rho[i]).subs(sub)) for i in range(3)]
    mu = oracle.bulk_mu(R, rb, fmt=1)
    np.testing.assert_allclose(mu, ref, rtol=1e-13)


def test_white_bear_zero_bias_gummel_is_its_equilibrium():
    """With the White Bear functional the Gummel iteration at zero bias and the
    equilibrium solver (two algorithms; the reservoir mu_b of the functional
    enters both through the Dirichlet data) reach the same state, which is
    not the Rosenfeld one."""
    import dataclasses
    from test_oracle_equilibrium import small_film
    spec = dataclasses.replace(small_film(0.0), fmt=1)
    e = oracle.equilibrium(spec, tol=1e-11, max_iter=3000)
    g = oracle.gummel(spec)
    assert e["status"] == 0 and g["status"] == 0
    rb = spec.rho_b[0]
    assert np.abs(e["phi"] - g["phi"]).max() <= 1e-9
    assert max(np.abs(e["rho"][i] - g["rho"][i]).max() / rb for i in range(2)) <= 1e-9
    ros = oracle.equilibrium(dataclasses.replace(spec, fmt=0), tol=1e-11, max_iter=3000)
    assert max(np.abs(ros["rho"][i] - e["rho"][i]).max() / rb for i in range(2)) > 1e-4
