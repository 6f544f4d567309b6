"""The autotuner (PNP_FLAG_AUTOTUNE) picks padded lengths and register-FFT
tiles by timing the pipeline on the device.  Whatever it picks, mu_ex stays
within the FP64 bar against the oracle (other lengths change it only by
rounding), and at equal lengths the tiles do not change a single bit."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle
from workloads import film_gummel, lognormal_density, mu_microbench

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 2e-5


@pytest.fixture(scope="module")
def pnp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp as mod
    build.build()
    return mod


def normwise(a, b):
    return max(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max() for i in range(a.shape[0]))


def smooth235(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def test_autotuned_plan_matches_oracle(pnp):
    shape = (28, 20, 18)                     # minimal lengths 32, 24, 22 -> 24
    spec, rho = mu_microbench(shape=shape)
    spec = dataclasses.replace(spec, autotune=True)
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec) as P:
        info = P.info()
        mu = P.excess_mu(rho)
    assert info["tuned_ms"] > 0
    for c, (n, L) in enumerate(zip(shape, info["fft_len"])):
        assert L >= n + info["stencil_halfwidth"] and smooth235(L)
        assert c != 0 or L % 2 == 0
    assert normwise(mu, ref) <= FP64_TOL

    # the same lengths with the built-in tiles give the same bits
    plain = dataclasses.replace(spec, autotune=False, fft_len=info["fft_len"])
    with pnp.Problem(plain) as Q:
        assert Q.info()["tile"] == (0, 0, 0) and Q.info()["tuned_ms"] == 0
        mu2 = Q.excess_mu(rho)
    np.testing.assert_array_equal(mu, mu2)


def test_autotune_cache_reuses_plan(pnp):
    spec, rho = mu_microbench(shape=(28, 20, 18))
    spec = dataclasses.replace(spec, autotune=True)
    with pnp.Problem(spec) as P:
        a = P.info()
    with pnp.Problem(spec) as P:
        b = P.info()
    assert (a["fft_len"], a["tile"], a["tuned_ms"]) == (b["fft_len"], b["tile"], b["tuned_ms"])


def test_autotune_keeps_explicit_lengths(pnp):
    spec, rho = mu_microbench(shape=(20, 12, 14))
    spec = dataclasses.replace(spec, autotune=True, fft_len=(32, 0, 0))
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec) as P:
        info = P.info()
        mu = P.excess_mu(rho)
    assert info["fft_len"][0] == 32
    assert normwise(mu, ref) <= FP64_TOL


def test_autotuned_fp32_film(pnp):
    """Periodic x, y (lengths fixed), z zero-extended with wells; FP32 plan."""
    spec = dataclasses.replace(film_gummel(16, 16, 16), autotune=True)
    rho = lognormal_density(spec, 3, sigma=0.2)
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec, precision="fp32") as P:
        info = P.info()
        mu = P.excess_mu(rho)
    assert info["fft_len"][:2] == (16, 16)
    assert normwise(mu, ref) <= FP32_TOL
