"""Pins of the oracle's Anderson-accelerated Gummel iteration (an extension of
the paper's relaxed iteration, Sec 3.2): it must reach the same fixed point
as the plain relaxed iteration -- only the path differs -- and it must get
there in far fewer sweeps on the dense film physics.
"""
import numpy as np

from oracle import oracle
from test_oracle_equilibrium import small_film
from workloads import film_gummel


def test_same_fixed_point_as_the_relaxed_iteration():
    spec = small_film(0.5)                 # biased: a current flows
    a = oracle.gummel_anderson(spec, m=3)
    b = oracle.gummel(spec)
    assert a["status"] == 0 and b["status"] == 0
    rb = spec.rho_b[0]
    assert np.abs(a["phi"] - b["phi"]).max() <= 1e-9
    assert max(np.abs(a["rho"][i] - b["rho"][i]).max() / rb for i in range(2)) <= 1e-9
    assert a["iters"] < b["iters"]


def test_dense_film_converges_in_a_fraction_of_the_sweeps():
    """8^3 film (packing 0.2 per ion, wells, lambda_rho 0.05): the plain
    relaxed iteration needs 388 sweeps to 1e-8; depth-3 Anderson about 100."""
    spec = film_gummel(8, 8, 8, tol=1e-8, max_iter=600)
    a = oracle.gummel_anderson(spec, m=3)
    assert a["status"] == 0
    assert a["iters"] <= 150
    # residual history ends below the tolerance
    assert a["hist"][-1] < 1e-8
