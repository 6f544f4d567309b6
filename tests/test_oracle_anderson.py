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


def test_backtracking_converges_where_the_relaxed_iteration_fails():
    """The film physics on 8^3 with the single relaxation 0.3 of the configs
    on both phi and rho (the printed linear form): the relaxed iteration
    overshoots into n3 >= 1 at its second sweep; the plain restart from that
    iterate fails the same way, and only the step halving back toward the
    last clean iterate continues.  Anderson then converges to the relaxed
    iteration's fixed point (here computed with the stable geometric 0.05)."""
    import dataclasses
    spec = film_gummel(8, 8, 8, tol=1e-8, max_iter=300)
    lit = dataclasses.replace(spec, lambda_rho=0.3, rho_mix=0)
    plain = oracle.gummel(lit)
    assert plain["status"] == 2 and plain["iters"] == 2
    a = oracle.gummel_anderson(lit, m=3)
    assert a["status"] == 0 and a["iters"] <= 200
    ref = oracle.gummel_anderson(dataclasses.replace(spec, tol=1e-11, max_iter=600), m=3)
    assert ref["status"] == 0
    assert np.abs(a["phi"] - ref["phi"]).max() <= 1e-6
    for i in range(2):
        assert np.abs(a["rho"][i] - ref["rho"][i]).max() / np.abs(ref["rho"][i]).max() <= 1e-6
