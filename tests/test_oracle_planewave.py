"""Plane-wave pins (analytic Fourier transforms of the weights, Sec 2.3.1).

For rho(r) = cos(k.r + c) evaluated exactly at the quadrature nodes the
weighted densities are, with kR = |k| R and theta = k.r + c,
  n3 = 4 pi (sin kR - kR cos kR)/|k|^3 cos(theta)
  n2 = 4 pi R^2 sin(kR)/(kR) cos(theta)
  vec n2 = -4 pi R^2 j1(kR) khat sin(theta),  j1(x) = (sin x - x cos x)/x^2
(the correlation orientation of Sec 2.3.1 makes vec n2 = grad n3), and
n0 = n2/(4 pi R^2), n1 = n2/(4 pi R), vec n1 = vec n2/(4 pi R).
This pins node positions, weights and the sign of the vector weight.
"""
import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec


def analytic(k, R, pts, c):
    kk = np.linalg.norm(k)
    x = kk * R
    th = pts @ k + c
    n3 = 4 * np.pi * (np.sin(x) - x * np.cos(x)) / kk ** 3 * np.cos(th)
    n2 = 4 * np.pi * R * R * np.sin(x) / x * np.cos(th)
    j1 = (np.sin(x) - x * np.cos(x)) / x ** 2
    v2 = -4 * np.pi * R * R * j1 * (k / kk)[None, :] * np.sin(th)[:, None]
    return n2 / (4 * np.pi * R * R), n2 / (4 * np.pi * R), n2, n3, v2 / (4 * np.pi * R), v2


@pytest.mark.parametrize("R,k", [(2.0, (0.3, -0.2, 0.5)), (1.5, (0.9, 0.4, -0.7)), (3.0, (0.1, 0.2, 0.25))])
def test_plane_wave_weighted_densities(R, k):
    n = 5
    spec = ProblemSpec(nx=n, ny=n, nz=n, bc=("N", "N", "D"), R=(R,), q=(0,), rho_b=(0.0,),
                       quad_nmu=24, quad_ntheta=48, quad_nr=24)
    k = np.array(k)
    c = 0.37
    out = oracle.weighted_densities(spec, wave=(k, c, [1.0]))
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pts = np.stack([x, y, z], -1).reshape(-1, 3).astype(float)
    n0, n1, n2, n3, v1, v2 = analytic(k, R, pts, c)
    got = out.reshape(10, -1)
    scale = 4 * np.pi * R ** 3
    np.testing.assert_allclose(got[0], n0, atol=1e-12)
    np.testing.assert_allclose(got[1], n1, atol=1e-12 * R)
    np.testing.assert_allclose(got[2], n2, atol=1e-12 * scale)
    np.testing.assert_allclose(got[3], n3, atol=1e-12 * scale)
    np.testing.assert_allclose(got[4:7].T, v1, atol=1e-12 * R)
    np.testing.assert_allclose(got[7:10].T, v2, atol=1e-12 * scale)


def test_plane_wave_default_counts_shell():
    """The default angular counts already resolve the shell integrals."""
    R, k = 2.0, np.array([0.5, 0.3, -0.4])
    spec = ProblemSpec(nx=3, ny=3, nz=3, bc=("N", "N", "D"), R=(R,), q=(0,), rho_b=(0.0,))
    out = oracle.weighted_densities(spec, wave=(k, 0.1, [1.0])).reshape(10, -1)
    z, y, x = np.meshgrid(np.arange(3), np.arange(3), np.arange(3), indexing="ij")
    pts = np.stack([x, y, z], -1).reshape(-1, 3).astype(float)
    n0, n1, n2, n3, v1, v2 = analytic(k, R, pts, 0.1)
    np.testing.assert_allclose(out[2], n2, atol=1e-12 * 4 * np.pi * R * R)
    np.testing.assert_allclose(out[7:10].T, v2, atol=1e-12 * 4 * np.pi * R * R)
    # radial rule: 4 Gauss points integrate r^2 j0(kr) to a few 1e-5 at kR ~ 1.4
    np.testing.assert_allclose(out[3], n3, atol=1e-4 * 4 * np.pi * R ** 3 / 3)


def test_grid_mode_converges_second_order():
    """On the grid the trilinear interpolation error is O(h^2): refine h by 2
    at fixed physical radius and wave number (R = 2h -> 4h, one wave across
    16 -> 32 cells) and the shell density error drops about fourfold."""
    errs = []
    for n, R in ((16, 2.0), (32, 4.0)):
        spec = ProblemSpec(nx=n, ny=4, nz=4, bc=("P", "P", "P"), R=(R,), q=(0,), rho_b=(0.0,),
                           quad_nmu=24, quad_ntheta=48, quad_nr=4)
        k = np.array([2 * np.pi / n, 0.0, 0.0])
        z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(n), indexing="ij")
        rho = np.cos(k[0] * x)[None].astype(float)
        got = oracle.weighted_densities(spec, rho=rho)
        pts = np.stack([x, y, z], -1).reshape(-1, 3).astype(float)
        ref = analytic(k, R, pts, 0.0)
        errs.append(np.abs(got[2].reshape(-1) - ref[2]).max() / np.abs(ref[2]).max())
    assert 3.0 < errs[0] / errs[1] < 5.0
