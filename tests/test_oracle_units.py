"""Reduced-unit pins against the values printed in Table 1 (Sec 4.1)."""
import os

import pytest

from oracle import units

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_units.txt")


def load():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        vals[k] = float(v)
    return vals


def test_table1_beta_and_bjerrum_length():
    g = load()
    T, eps = g["temperature_K"], g["eps_r"]
    # the printed beta carries more digits than its k_B: agreement is 1.4e-5
    assert units.beta_per_ev(T) == pytest.approx(g["beta_per_eV"], rel=1e-4)
    assert units.bjerrum_length_nm(T, eps) == pytest.approx(g["bjerrum_length_nm"], rel=1e-4)


def test_bjerrum_length_in_grid_units():
    assert units.bjerrum_length_h(300.0, 16.6, 0.5) == pytest.approx(
        2 * units.bjerrum_length_nm(300.0, 16.6), rel=1e-15)
