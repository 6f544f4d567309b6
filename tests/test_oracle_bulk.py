"""Bulk pins: for a uniform fluid on an all-periodic grid every weighted
density is the exact moment of its weight (the rules integrate constants
exactly), so mu_ex must equal the closed forms of the uniform hard-sphere
fluid.  Single species: the Percus-Yevick compressibility result
-ln(1-eta) + eta(14 - 13 eta + 5 eta^2) / (2 (1-eta)^3).  Mixtures: the
scaled-particle-theory chemical potential (Lebowitz-Rowlinson form), a
different algebraic route to the same numbers Rosenfeld FMT gives in bulk.
"""
import math

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density


def py_single(eta):
    return -math.log(1 - eta) + eta * (14 - 13 * eta + 5 * eta ** 2) / (2 * (1 - eta) ** 3)


def spt_mixture(R, rho):
    sig = 2 * np.asarray(R, float)
    rho = np.asarray(rho, float)
    xi = [math.pi / 6 * np.sum(rho * sig ** m) for m in range(4)]
    o = 1 - xi[3]
    betaP = 6 / math.pi * (xi[0] / o + 3 * xi[1] * xi[2] / o ** 2 + 3 * xi[2] ** 3 / o ** 3)
    return (-math.log(o) + (3 * xi[2] * sig + 3 * xi[1] * sig ** 2) / o
            + 9 * xi[2] ** 2 * sig ** 2 / (2 * o ** 2) + betaP * math.pi * sig ** 3 / 6)


def uniform_mu(R, rho_b, n=6):
    spec = ProblemSpec(nx=n, ny=n, nz=n, bc=("P", "P", "P"), R=tuple(R), q=(0,) * len(R),
                       rho_b=tuple(rho_b))
    rho = np.stack([np.full((n, n, n), r) for r in rho_b])
    mu, bad = oracle.excess_mu(spec, rho)
    assert bad == 0
    return mu


@pytest.mark.parametrize("eta,R", [(0.2, 2.0), (0.1, 1.5), (0.3, 1.0), (0.4, 2.0), (0.05, 3.0)])
def test_single_species_percus_yevick(eta, R):
    mu = uniform_mu([R], [bulk_density(eta, R)], n=7)
    np.testing.assert_allclose(mu, py_single(eta), rtol=1e-13)


def test_spt_reduces_to_py():
    for eta in (0.1, 0.3):
        assert spt_mixture([1.0], [bulk_density(eta, 1.0)])[0] == pytest.approx(py_single(eta), rel=1e-14)


@pytest.mark.parametrize("R,eta", [((1.5, 2.0, 3.0), (0.1, 0.1, 0.1)), ((2.0, 2.0), (0.2, 0.2)),
                                   ((2.0, 2.0, 1.0), (0.2, 0.1, 0.0125))])
def test_mixture_spt(R, eta):
    rb = [bulk_density(e, r) for e, r in zip(eta, R)]
    mu = uniform_mu(R, rb, n=8)
    ref = spt_mixture(R, rb)
    for i in range(len(R)):
        np.testing.assert_allclose(mu[i], ref[i], rtol=1e-13)
    np.testing.assert_allclose(oracle.bulk_mu(R, rb), ref, rtol=1e-13)


def test_two_ions_at_total_packing_04():
    """Two species of radius 2h at packing fraction 0.2 each: total 0.4."""
    rb = bulk_density(0.2, 2.0)
    assert rb == pytest.approx(0.0059683103659461, rel=1e-12)
    mu = oracle.bulk_mu([2.0, 2.0], [rb, rb])
    np.testing.assert_allclose(mu, py_single(0.4), rtol=1e-13)
