"""Pins of the oracle's 7-point finite-difference solves (Sec 3.1).

- Poisson against a dense LU solve of the textbook Laplacian assembled from
  Kronecker products of 1D second-difference matrices.
- Poisson with uniform charge: the discrete solution is the exact quadratic
  phi(z) = phi_lo + (phi_hi - phi_lo) z/Lz + 2 pi lB c z (Lz - z).
- Slotboom Nernst-Planck against a dense LU of the harmonic-mean system
  assembled point by point, the 1D series-resistor closed form, and constant
  flux through every z plane (div J = 0).
"""
import math

import numpy as np
import pytest

from oracle import oracle, units
from workloads import ProblemSpec


def lap1d(n, kind):
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    if kind == "P":
        T[0, -1] -= 1
        T[-1, 0] -= 1
    elif kind == "N":
        T[0, 0] = 1
        T[-1, -1] = 1
    return T


def spec_for(shape, bc, **kw):
    nz, ny, nx = shape
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=bc, R=(1.0, 1.0), q=(1, -1), rho_b=(0.01, 0.01), **kw)


@pytest.mark.parametrize("bc", [("P", "P", "D"), ("N", "P", "D"), ("N", "N", "D")])
def test_poisson_dense_lu(bc):
    shape = (5, 4, 3)
    rng = np.random.default_rng(1)
    spec = spec_for(shape, bc, rho_f=rng.normal(0, 0.01, shape), phi_lo=0.3, phi_hi=-0.2)
    rho = np.abs(rng.normal(0.01, 0.003, (2,) + shape))
    phi, it, rel = oracle.poisson(spec, rho)
    nz, ny, nx = shape
    A = (np.kron(np.eye(nz), np.kron(np.eye(ny), lap1d(nx, bc[0])))
         + np.kron(np.eye(nz), np.kron(lap1d(ny, bc[1]), np.eye(nx)))
         + np.kron(lap1d(nz, "D"), np.eye(ny * nx)))
    lB = units.bjerrum_length_h(spec.temperature_K, spec.eps_r, spec.h_nm)
    b = 4 * np.pi * lB * (spec.rho_f + rho[0] - rho[1])
    b[0] += spec.phi_lo
    b[-1] += spec.phi_hi
    ref = np.linalg.solve(A, b.reshape(-1))
    np.testing.assert_allclose(phi.reshape(-1), ref, atol=1e-11 * np.abs(ref).max())


def test_poisson_uniform_charge_is_quadratic():
    shape = (9, 3, 4)
    c = 0.002
    spec = spec_for(shape, ("P", "P", "D"), rho_f=np.full(shape, c), phi_lo=0.1, phi_hi=0.7)
    rho = np.zeros((2,) + shape)
    phi, it, rel = oracle.poisson(spec, rho)
    lB = units.bjerrum_length_h(spec.temperature_K, spec.eps_r, spec.h_nm)
    Lz = shape[0] + 1
    z = np.arange(1, shape[0] + 1)
    ref = 0.1 + 0.6 * z / Lz + 2 * math.pi * lB * c * z * (Lz - z)
    np.testing.assert_allclose(phi, np.broadcast_to(ref[:, None, None], shape), atol=1e-11 * np.abs(ref).max())


def harmonic(a, b):
    return 2 * a * b / (a + b)


def np_dense(spec, i, phi, mu, mu_b):
    nz, ny, nx = spec.shape
    q = spec.q[i]
    Db = np.exp(-(q * phi + mu))
    Dlo = math.exp(-(q * spec.phi_lo + mu_b))
    Dhi = math.exp(-(q * spec.phi_hi + mu_b))
    rlo = spec.rho_b[i] * math.exp(q * spec.phi_lo + mu_b)
    rhi = spec.rho_b[i] * math.exp(q * spec.phi_hi + mu_b)
    N = nx * ny * nz
    A = np.zeros((N, N))
    b = np.zeros(N)
    idx = lambda k, j, l: (k * ny + j) * nx + l
    for k in range(nz):
        for j in range(ny):
            for l in range(nx):
                p = idx(k, j, l)
                nbrs = []
                for axis, n, bcv in ((0, nx, spec.bc[0]), (1, ny, spec.bc[1])):
                    for d in (-1, 1):
                        c = [l, j][axis] + d
                        if c < 0 or c >= n:
                            if bcv == "N":
                                continue
                            c %= n
                        ll, jj = (c, j) if axis == 0 else (l, c)
                        nbrs.append(idx(k, jj, ll))
                for d in (-1, 1):
                    kk = k + d
                    if kk < 0 or kk >= nz:
                        Dn, rv = (Dlo, rlo) if kk < 0 else (Dhi, rhi)
                        c = harmonic(Db[k, j, l], Dn)
                        A[p, p] += c
                        b[p] += c * rv
                    else:
                        nbrs.append(idx(kk, j, l))
                for qn in nbrs:
                    c = harmonic(Db.reshape(-1)[p], Db.reshape(-1)[qn])
                    A[p, p] += c
                    A[p, qn] -= c
    return np.linalg.solve(A, b).reshape(spec.shape)


@pytest.mark.parametrize("bc", [("P", "P", "D"), ("N", "P", "D")])
def test_np_dense_lu(bc):
    shape = (5, 4, 4)
    rng = np.random.default_rng(2)
    spec = spec_for(shape, bc, phi_lo=0.0, phi_hi=0.8)
    phi = rng.normal(0, 0.5, shape)
    mu = rng.normal(0, 2.0, shape)
    for i in range(2):
        rb, it, rel = oracle.np_solve(spec, i, phi, mu, 1.3)
        ref = np_dense(spec, i, phi, mu, 1.3)
        np.testing.assert_allclose(rb, ref, rtol=1e-10)


def test_np_series_resistor():
    shape = (12, 3, 3)
    rng = np.random.default_rng(3)
    spec = spec_for(shape, ("P", "P", "D"), phi_lo=0.2, phi_hi=1.1)
    phz = rng.normal(0, 0.4, 12)
    muz = rng.normal(0, 3.0, 12)
    phi = np.broadcast_to(phz[:, None, None], shape).copy()
    mu = np.broadcast_to(muz[:, None, None], shape).copy()
    mu_b = 0.7
    i = 0
    q = spec.q[i]
    Dnodes = np.concatenate([[math.exp(-(q * 0.2 + mu_b))], np.exp(-(q * phz + muz)),
                             [math.exp(-(q * 1.1 + mu_b))]])
    c = harmonic(Dnodes[:-1], Dnodes[1:])          # 13 face conductances
    rlo = spec.rho_b[i] * math.exp(q * 0.2 + mu_b)
    rhi = spec.rho_b[i] * math.exp(q * 1.1 + mu_b)
    J = (rlo - rhi) / np.sum(1 / c)
    ref = rlo - J * np.cumsum(1 / c)[:-1]
    rb, it, rel = oracle.np_solve(spec, i, phi, mu, mu_b)
    np.testing.assert_allclose(rb, np.broadcast_to(ref[:, None, None], shape), rtol=1e-11)


def test_np_flux_constant_through_planes():
    shape = (10, 5, 6)
    rng = np.random.default_rng(4)
    spec = spec_for(shape, ("P", "P", "D"), phi_lo=0.0, phi_hi=1.0)
    phi = rng.normal(0, 0.5, shape)
    mu = rng.normal(0, 2.0, shape)
    rb, it, rel = oracle.np_solve(spec, 1, phi, mu, 0.4)
    J = oracle.np_flux(spec, 1, phi, mu, 0.4, rb)
    assert abs(J[0]) > 0
    np.testing.assert_allclose(J, J[0], rtol=1e-9)
