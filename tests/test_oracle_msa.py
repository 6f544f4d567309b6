"""Pins of the oracle's electrostatic-correlation term (Sec 2.3.4, MSA).

- Uniform excess densities on a periodic box: the ball quadrature of r^2 C(r)
  (a cubic in r) is exact, so mu_el,i = sum_j c_j 4 pi q_i q_j l_B s^2
  (2B/3 - B^2/4 - 1/2), with B from the textbook MSA screening parameter,
  B = Gamma s / (1 + Gamma s), 2 Gamma s = sqrt(1 + 2 kappa s) - 1 (an
  independent form of the printed B).
- Brute force: dense operators built from numpy's own Gauss-Legendre ball
  nodes and hat functions (tests/brute.py), zero extension on Dirichlet and
  no-flux axes, wrap on periodic ones.
- Plane waves evaluated at the nodes: the radial Fourier transform
  4 pi int r^2 C(r) sin(kr)/(kr) dr by adaptive quadrature (scipy).
- rho = rho_b gives zero; neutral species neither feel nor cause the term.
"""
import math

import numpy as np
import pytest

import brute
from oracle import oracle, units
from workloads import ProblemSpec


def spec_msa(bc=("P", "P", "P"), shape=(9, 8, 10), **kw):
    nz, ny, nx = shape
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=bc, R=(1.0, 1.5, 0.7, 1.2), q=(1, -1, 2, 0),
                       rho_b=(0.004, 0.006, 0.001, 0.003), **kw)


def kappa(spec):
    lB = units.bjerrum_length_h(spec.temperature_K, spec.eps_r, spec.h_nm)
    return math.sqrt(4 * math.pi * lB * sum(r * q * q for r, q in zip(spec.rho_b, spec.q))), lB


def B_gamma(k, s):
    gs = 0.5 * (math.sqrt(1 + 2 * k * s) - 1)
    return gs / (1 + gs)


def C_of_r(r, qq, lB, B, s):
    return -qq * lB * (2 * B / s - (B / s) ** 2 * r - 1 / r)


def test_uniform_excess_closed_form():
    spec = spec_msa()
    c = np.array([0.001, -0.0005, 0.0003, 0.002])
    rho = np.stack([np.full(spec.shape, rb + ci) for rb, ci in zip(spec.rho_b, c)])
    mu = oracle.mu_el(spec, rho)
    k, lB = kappa(spec)
    assert k * 1.0 > 0.1          # screening well away from the small-xi branch
    for i in range(spec.s):
        ref = 0.0
        for j in range(spec.s):
            s = spec.R[i] + spec.R[j]
            B = B_gamma(k, s)
            ref += c[j] * 4 * math.pi * spec.q[i] * spec.q[j] * lB * s * s * (2 * B / 3 - B * B / 4 - 0.5)
        np.testing.assert_allclose(mu[i], ref, rtol=1e-12, atol=1e-15)
    assert np.all(mu[3] == 0.0)                          # neutral species


def test_bulk_gives_zero():
    spec = spec_msa(bc=("N", "P", "D"))
    rho = np.stack([np.full(spec.shape, rb) for rb in spec.rho_b])
    assert np.all(oracle.mu_el(spec, rho) == 0.0)


@pytest.mark.parametrize("bc", [("P", "N", "D"), ("P", "P", "P")])
def test_matches_dense_operator(bc):
    spec = spec_msa(bc=bc, shape=(6, 7, 8))
    rng = np.random.default_rng(4)
    rho = np.stack([rb * rng.lognormal(0, 0.3, spec.shape) for rb in spec.rho_b])
    mu = oracle.mu_el(spec, rho)
    k, lB = kappa(spec)
    per = tuple(b == "P" for b in bc)
    N = int(np.prod(spec.shape))
    for i in range(spec.s):
        ref = np.zeros(N)
        for j in range(spec.s):
            qq = spec.q[i] * spec.q[j]
            if qq == 0:
                continue
            s = spec.R[i] + spec.R[j]
            B = B_gamma(k, s)
            p, w, u = brute.nodes("ball", s)
            r = np.linalg.norm(p, axis=1)
            reach = int(math.ceil(s)) + 1
            K = brute.kernel_table(p, w * C_of_r(r, qq, lB, B, s), u, reach)
            M = brute.dense_operator(K, reach, spec.shape, per)
            ref -= M @ (rho[j] - spec.rho_b[j]).reshape(-1)
        scale = max(np.abs(ref).max(), 1e-30)
        np.testing.assert_allclose(mu[i].reshape(-1), ref, rtol=0, atol=1e-12 * scale)


def test_plane_wave_transform():
    from scipy.integrate import quad
    spec = spec_msa(shape=(5, 6, 7), quad_nmu=40, quad_ntheta=80, quad_nr=40)
    kv = np.array([0.9, -0.4, 0.6])
    amp = np.array([1.0, 0.5, -0.7, 2.0])
    ph = 0.3
    mu = oracle.mu_el(spec, wave=(kv, ph, amp))
    kk, lB = kappa(spec)
    km = np.linalg.norm(kv)
    z, y, x = np.meshgrid(np.arange(spec.nz), np.arange(spec.ny), np.arange(spec.nx), indexing="ij")
    phase = np.cos(kv[0] * x + kv[1] * y + kv[2] * z + ph)
    for i in range(spec.s):
        ref = 0.0
        for j in range(spec.s):
            qq = spec.q[i] * spec.q[j]
            if qq == 0:
                continue
            s = spec.R[i] + spec.R[j]
            B = B_gamma(kk, s)
            f = lambda r: r * r * C_of_r(r, qq, lB, B, s) * math.sin(km * r) / (km * r)
            Ck = 4 * math.pi * quad(f, 0.0, s, epsabs=1e-13, epsrel=1e-12, limit=200)[0]
            ref = ref - amp[j] * Ck * phase
        scale = max(np.abs(ref).max(), 1e-30) if np.ndim(ref) else 1.0
        np.testing.assert_allclose(mu[i], ref, rtol=0, atol=1e-9 * scale)
