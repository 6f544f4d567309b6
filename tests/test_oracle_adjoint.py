"""Discrete-adjoint pin: with F = h^3 sum_Omega Phi(n(rho)) (h = 1), the
oracle's mu_hs,i(r) must equal dF/drho_i(r) (Sec 2.3.1, functional derivative
of Eq. hs-energy).  The derivative is taken by a complex step through the
independent brute-force forward operator and a numpy Phi, so a wrong sign, a
dropped term in any of the ten printed derivatives, or a transposed
back-convolution fails here.
"""
import numpy as np
import pytest

import brute
from oracle import oracle
from workloads import ProblemSpec, bulk_density


@pytest.mark.parametrize("bc", [("P", "N", "D"), ("P", "P", "P")])
def test_mu_hs_is_gradient_of_free_energy(bc):
    R = (1.5, 2.0)
    rb = tuple(bulk_density(0.15, r) for r in R)
    spec = ProblemSpec(nx=6, ny=6, nz=7, bc=bc, R=R, q=(1, -1), rho_b=rb)
    rng = np.random.default_rng(5)
    rho = np.stack([rb[i] * rng.lognormal(0, 0.4, spec.shape) for i in range(2)])
    n = oracle.weighted_densities(spec, rho)
    psi, bad = oracle.dphi(n)
    assert bad == 0
    mu = oracle.mu_hs(spec, psi)
    B = brute.BruteFMT(spec.shape, tuple(b == "P" for b in bc), R)
    # F from the oracle and from brute force agree
    assert oracle.fhs(n) == pytest.approx(np.sum(brute.phi_rosenfeld(B.weighted(rho))).real, rel=1e-12)
    hstep = 1e-30
    for trial in range(6):
        i = trial % 2
        idx = tuple(int(rng.integers(d)) for d in spec.shape)
        rc = rho.astype(complex)
        rc[(i,) + idx] += 1j * hstep
        dF = np.sum(brute.phi_rosenfeld(B.weighted(rc))).imag / hstep
        assert mu[(i,) + idx] == pytest.approx(dF, rel=1e-11, abs=1e-13)


def test_dphi_matches_complex_step_of_phi():
    """Each printed derivative against a complex step of Phi itself."""
    rng = np.random.default_rng(9)
    n = np.zeros((10, 4))
    n[3] = rng.uniform(0.05, 0.6, 4)
    n[2] = rng.uniform(0.1, 2.0, 4)
    n[0] = n[2] / (4 * np.pi * 4.0)
    n[1] = n[2] / (4 * np.pi * 2.0)
    n[4:10] = rng.normal(0, 0.05, (6, 4))
    psi, bad = oracle.dphi(n)
    for a in range(10):
        nc = n.astype(complex)
        nc[a] += 1e-30j
        d = brute.phi_rosenfeld(nc).imag / 1e-30
        np.testing.assert_allclose(psi[a], d, rtol=1e-13, atol=1e-15)


def test_packing_error_flag():
    n = np.zeros((10, 3))
    n[3] = [0.5, 1.0, 1.2]
    psi, bad = oracle.dphi(n)
    assert bad == 2
