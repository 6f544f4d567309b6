"""Pins of the oracle's quadrature node sets (Sec 3.5 change of variables).

Checked against what the mathematics fixes: Gauss-Legendre nodes/weights equal
numpy's textbook routine, the rules integrate constants and low moments of the
sphere, ball and thick shell exactly, and the node set has the reflection and
x<->y symmetry the reading promises.
"""
import math

import numpy as np
import pytest

from oracle import oracle


@pytest.mark.parametrize("R", [1.0, 1.5, 2.0, 3.0])
def test_shell_nodes_are_gauss_legendre_in_cos_phi(R):
    p, w, u = oracle.nodeset(0, 0.0, R)
    nmu = max(8, math.ceil(2 * math.pi * R))
    ntheta = -(-2 * nmu // 4) * 4
    assert len(w) == nmu * ntheta
    mu_ref, w_ref = np.polynomial.legendre.leggauss(nmu)
    mus = np.unique(np.round(u[:, 2], 14))
    np.testing.assert_allclose(np.sort(mus), np.sort(mu_ref), atol=1e-14)
    # weights of one theta ring reproduce w_b * 2 pi / n_theta * R^2
    ring = np.isclose(u[:, 2], mu_ref[0], atol=1e-13)
    np.testing.assert_allclose(w[ring], R * R * w_ref[0] * 2 * np.pi / ntheta, rtol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(p, R * u, atol=1e-14)


@pytest.mark.parametrize("R", [1.0, 2.0, 3.0])
def test_shell_moments(R):
    p, w, u = oracle.nodeset(0, 0.0, R)
    assert w.sum() == pytest.approx(4 * np.pi * R * R, rel=1e-14)
    np.testing.assert_allclose((w[:, None] * p).sum(0), 0.0, atol=1e-13)
    second = np.einsum("q,qi,qj->ij", w, p, p)
    np.testing.assert_allclose(second, 4 * np.pi * R ** 4 / 3 * np.eye(3), atol=1e-12 * R ** 4)


@pytest.mark.parametrize("R", [1.0, 2.0, 3.0])
def test_ball_moments(R):
    p, w, u = oracle.nodeset(1, 0.0, R)
    assert w.sum() == pytest.approx(4 * np.pi * R ** 3 / 3, rel=1e-14)
    second = np.einsum("q,qi,qj->ij", w, p, p)
    np.testing.assert_allclose(second, 4 * np.pi * R ** 5 / 15 * np.eye(3), atol=1e-12 * R ** 5)


def test_thick_shell_volume():
    a, b = 4.0, 5.0
    p, w, u = oracle.nodeset(2, a, b)
    assert w.sum() == pytest.approx(4 * np.pi * (b ** 3 - a ** 3) / 3, rel=1e-14)
    r = np.linalg.norm(p, axis=1)
    assert r.min() > a and r.max() < b


@pytest.mark.parametrize("R", [1.5, 2.0])
def test_node_set_symmetries(R):
    """Reflections of each axis and the x<->y swap map the node set onto itself
    with equal weights (so the discrete stencils are even/odd as required)."""
    p, w, _ = oracle.nodeset(0, 0.0, R)
    key = {tuple(np.round(x, 12)): ww for x, ww in zip(p, w)}
    for T in (np.diag([-1, 1, 1]), np.diag([1, -1, 1]), np.diag([1, 1, -1]),
              np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]])):
        for x, ww in zip(p @ T.T, w):
            k = tuple(np.round(x, 12))
            assert k in key and key[k] == pytest.approx(ww, rel=1e-14)


def test_explicit_counts_override_rule():
    p, w, u = oracle.nodeset(1, 0.0, 2.0, nmu=10, ntheta=12, nr=5)
    assert len(w) == 10 * 12 * 5
