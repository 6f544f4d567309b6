"""The synthetic input recipes (workloads/) against their stated definitions:
sizes, seeds, value distributions and solver options of each workload."""
import math

import numpy as np

from workloads import (BATCH_GRIDS, batch_specs, bulk_density, film3, film_gummel, mu_microbench,
                       serving_arrivals, serving_spec)


def packing(spec):
    return sum(r * 4.0 / 3.0 * math.pi * R ** 3 for r, R in zip(spec.rho_b, spec.R))


def smooth235(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_mu_microbench_recipe():
    spec, rho = mu_microbench(32)
    assert (spec.nx, spec.ny, spec.nz) == (32, 32, 32) and spec.R == (1.5, 2.0, 3.0)
    assert spec.bc == ("N", "N", "D")
    assert abs(packing(spec) - 0.3) < 1e-12
    # lognormal(0, 0.1) around the bulk density, seed 2, reproducible
    for i in range(3):
        ratio = rho[i] / spec.rho_b[i]
        assert abs(np.log(ratio).mean()) < 0.01 and abs(np.log(ratio).std() - 0.1) < 0.01
    _, rho2 = mu_microbench(32)
    np.testing.assert_array_equal(rho, rho2)


def test_film_recipe():
    spec = film_gummel(32, 32, 32)
    assert spec.bc == ("P", "P", "D") and spec.q == (1, -1) and spec.R == (2.0, 2.0)
    assert abs(spec.rho_b[0] - bulk_density(0.2, 2.0)) < 1e-15
    assert spec.sites.shape == (64, 3) and spec.depth == (1.0, 0.0)
    assert spec.phi_lo == 0.0 and spec.phi_hi == 0.1 and spec.lambda_phi == 0.3
    assert spec.rho_f.shape == (32, 32, 32) and abs(spec.rho_f.std() - 0.01) < 5e-4


def test_film3_recipe():
    spec = film3(bias=0.5)
    assert (spec.nx, spec.ny, spec.nz) == (128, 128, 256)
    assert spec.q == (1, -1, -1) and spec.R == (2.0, 2.0, 1.0)
    assert abs(spec.rho_b[1] - spec.rho_b[0] / 2) < 1e-15 and abs(spec.rho_b[2] - spec.rho_b[0] / 2) < 1e-15
    assert spec.sites.shape == (4096, 3) and spec.depth[0] == 3.0 and spec.phi_hi == 0.5
    assert spec.screened_poisson and spec.eq_init and spec.rho_mix == 2


def test_batch_recipe():
    specs = batch_specs(64)
    assert len(specs) == 64
    kb = 8.617333262e-5
    for j, s in enumerate(specs):
        assert (s.nx, s.ny, s.nz) in BATCH_GRIDS
        assert 250.0 <= s.temperature_K <= 400.0
        assert abs(s.depth[0] - 0.3 / (kb * s.temperature_K)) < 1e-12
        assert 0.1 <= packing(s) <= 0.35 + 1e-12
        assert s.sites.shape[0] == max(1, s.nx * s.ny * s.nz // 512)
        assert s.screened_poisson and s.rho_mix == 3
    # every grid size appears, deterministic
    assert {(s.nx, s.ny, s.nz) for s in specs} == set(BATCH_GRIDS)
    again = batch_specs(64)
    assert all(a.temperature_K == b.temperature_K for a, b in zip(specs, again))


def test_serving_recipe():
    arr = serving_arrivals(600)
    times = [a[0] for a in arr]
    assert all(t1 > t0 for t0, t1 in zip(times, times[1:]))
    # Poisson arrivals at 20/s: mean gap 0.05 s
    assert abs(np.mean(np.diff([0.0] + times)) - 0.05) < 0.005
    edges = [a[1] for a in arr]
    assert all(32 <= n <= 256 and n % 2 == 0 and smooth235(n) for n in edges)
    assert all(0.0 <= a[2] <= 1.0 and 250.0 <= a[3] <= 400.0 for a in arr)
    spec = serving_spec(48, 0.7, 320.0)
    assert (spec.nx, spec.ny, spec.nz) == (48, 48, 48) and spec.phi_hi == 0.7 and spec.temperature_K == 320.0
    assert spec.depth == (1.0, 0.0) and spec.screened_poisson and spec.rho_mix == 3
