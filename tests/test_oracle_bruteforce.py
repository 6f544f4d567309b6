"""Brute-force pins: the oracle's interpolate-at-every-node sums against an
O(N^2) dense operator built from tabulated kernel values (tests/brute.py).
Covers zero extension on non-periodic axes, wrap on periodic axes, the
back-convolution as the transpose of the forward operator, and mu_sh.
"""
import numpy as np
import pytest

import brute
from oracle import oracle
from workloads import ProblemSpec, bulk_density


def spec_small(shape=(6, 7, 8), bc=("P", "N", "D"), R=(1.5, 2.0)):
    nz, ny, nx = shape
    rb = tuple(bulk_density(0.12, r) for r in R)
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=bc, R=R, q=(1, -1)[:len(R)], rho_b=rb)


def rand_rho(spec, seed=7):
    rng = np.random.default_rng(seed)
    return np.stack([spec.rho_b[i] * rng.lognormal(0, 0.3, spec.shape) for i in range(spec.s)])


@pytest.mark.parametrize("bc", [("P", "N", "D"), ("N", "N", "D"), ("P", "P", "P")])
def test_weighted_densities_match_dense_sums(bc):
    spec = spec_small(bc=bc)
    rho = rand_rho(spec)
    per = tuple(b == "P" for b in bc)
    B = brute.BruteFMT(spec.shape, per, spec.R)
    ref = B.weighted(rho)
    got = oracle.weighted_densities(spec, rho)
    for a in range(10):
        scale = np.abs(ref[a]).max() + 1e-30
        np.testing.assert_allclose(got[a], ref[a], atol=1e-13 * scale, err_msg=f"field {a}")


def test_back_convolution_is_transpose():
    spec = spec_small()
    per = (True, False, False)
    B = brute.BruteFMT(spec.shape, per, spec.R)
    rng = np.random.default_rng(3)
    psi = rng.normal(size=(10,) + spec.shape)
    got = oracle.mu_hs(spec, psi)
    N = int(np.prod(spec.shape))
    P = psi.reshape(10, N)
    for i, (M2, M3, Mv) in enumerate(B.ops):
        R = spec.R[i]
        c0, c1 = 1 / (4 * np.pi * R * R), 1 / (4 * np.pi * R)
        ref = M2.T @ (c0 * P[0] + c1 * P[1] + P[2]) + M3.T @ P[3]
        for c in range(3):
            ref += Mv[:, :, c].T @ (c1 * P[4 + c] + P[7 + c])
        np.testing.assert_allclose(got[i].reshape(-1), ref, atol=1e-12 * np.abs(ref).max())


def test_square_well_and_site_density():
    spec = spec_small(shape=(7, 6, 6), bc=("P", "P", "D"))
    rng = np.random.default_rng(11)
    spec.sites = rng.uniform(0, 1, (5, 3)) * np.array([6, 6, 7])
    spec.site_alpha = 0.8
    spec.depth = (1.3, 0.0)
    spec.well_inner, spec.well_outer = 2.0, 3.0
    rs = oracle.site_density(spec)
    # independent Gaussian sum with explicit periodic images on x, y
    z, y, x = np.meshgrid(np.arange(7), np.arange(6), np.arange(6), indexing="ij")
    ref = np.zeros(spec.shape)
    for s in spec.sites:
        for ix in range(-3, 4):
            for iy in range(-3, 4):
                d2 = (x - s[0] - 6 * ix) ** 2 + (y - s[1] - 6 * iy) ** 2 + (z - s[2]) ** 2
                ref += np.exp(-spec.site_alpha * d2)
    ref *= (spec.site_alpha / np.pi) ** 1.5
    np.testing.assert_allclose(rs, ref, rtol=1e-12, atol=1e-14)
    got = oracle.mu_sh(spec, rs)
    reach = 4
    p, w, u = brute.nodes("thick", 3.0, r_in=2.0)
    K = brute.kernel_table(p, w, u, reach)
    M = brute.dense_operator(K, reach, spec.shape, (True, True, False))
    ref_mu = 0.5 * (-1.3) * (M @ rs.reshape(-1))
    np.testing.assert_allclose(got[0].reshape(-1), ref_mu, atol=1e-13 * np.abs(ref_mu).max())
    assert np.all(got[1] == 0)


def test_invariants():
    spec = spec_small(shape=(6, 6, 6), bc=("P", "P", "P"))
    rho = rand_rho(spec)
    n1 = oracle.weighted_densities(spec, rho)
    # linearity
    n2 = oracle.weighted_densities(spec, 2.5 * rho)
    scale = np.abs(n1).max(axis=(1, 2, 3), keepdims=True)
    np.testing.assert_allclose(n2 / scale, 2.5 * n1 / scale, rtol=0, atol=1e-13)
    # integer shift equivariance on periodic axes
    sh = np.roll(rho, (1, -2, 3), axis=(1, 2, 3))
    ns = oracle.weighted_densities(spec, sh)
    np.testing.assert_allclose(ns / scale, np.roll(n1, (1, -2, 3), axis=(1, 2, 3)) / scale, rtol=0, atol=1e-13)
    # positivity of the packing fraction field
    assert n1[3].min() >= 0


@pytest.mark.parametrize("bc", [("N", "N", "D"), ("P", "P", "D")])
def test_sampled_mu_ex_equals_full_evaluation(bc):
    """oracle.excess_mu_sampled (used for the full-size GPU checks) equals the
    full evaluation at every sampled point, wells included, near faces and in
    the interior."""
    from workloads import film_gummel
    spec = film_gummel(12, 10, 14, nsites=5)
    spec.bc = bc
    spec.well_inner, spec.well_outer = 2.0, 3.0
    rng = np.random.default_rng(17)
    rho = np.stack([spec.rho_b[i] * rng.lognormal(0.0, 0.3, spec.shape) for i in range(spec.s)])
    full, bad = oracle.excess_mu(spec, rho)
    assert bad == 0
    N = spec.npoints
    flat = np.unique(np.concatenate([rng.integers(0, N, 40), [0, N - 1, spec.nx * spec.ny]]))
    got = oracle.excess_mu_sampled(spec, rho, flat)
    ref = full.reshape(spec.s, -1)[:, flat]
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
