"""Failure paths on the GPU that fault, trap or hang nothing: each error comes
back as a status the host reads, and the device stays usable afterwards.

- A bounded device wait that nothing completes gives up after its limit and
  reports PNP_ERR_TIMEOUT (the same globally-timed wait the tensor-core
  kernels use on their mbarriers).
- An allocation the device cannot hold (a 2048^3 grid: ~0.7 TB of FFT
  workspace) is refused with PNP_ERR_NOMEM before anything else is built.
- After both, a small mu_ex still matches the oracle.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density, mu_microbench

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pnp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp as mod
    build.build()
    return mod


def small_mu_ex_still_works(pnp):
    spec, rho = mu_microbench(10)
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec) as P:
        mu = P.excess_mu(rho)
    assert max(np.abs(mu[i] - ref[i]).max() / np.abs(ref[i]).max() for i in range(3)) <= 1e-10


def test_bounded_wait_times_out_and_reports(pnp):
    assert pnp.selftest_bounded_wait(5.0) == pnp.ERR_TIMEOUT
    assert pnp.selftest_bounded_wait(0.0) == pnp.ERR_INVALID
    small_mu_ex_still_works(pnp)


def test_allocation_failure_is_nomem_and_clean(pnp):
    rb = bulk_density(0.1, 2.0)
    spec = ProblemSpec(nx=2048, ny=2048, nz=2048, bc=("P", "P", "D"), R=(2.0,), q=(0,), rho_b=(rb,),
                       depth=(0.0,), sites=None, rho_f=None)
    dh = pnp.DescHolder(spec)
    h = ctypes.c_void_p()
    rc = pnp.lib().pnp_create_problem(ctypes.byref(dh.desc), ctypes.byref(h))
    assert rc == pnp.ERR_NOMEM
    assert not h.value
    small_mu_ex_still_works(pnp)
