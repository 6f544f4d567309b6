"""pnp_excess_mu_noalloc: the entry point for callers that cannot allocate
device memory (their GPU memory belongs to another allocator, or their loop
must not call cudaMalloc).  It keeps all of its scratch in a fixed array
inside the library.  Through the C ABI, two calls in a row (different
densities, then a different grid) must agree with the regular entry point
pnp_excess_mu_device within the FP64 tolerance of the other mu_ex tests, and
over-size or well-carrying descriptors must be refused without touching the
device.  Collected last on purpose: it must pass alone and after everything.
"""
import numpy as np
import pytest

from workloads import film_gummel, lognormal_density, mu_microbench

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp
    build.build()
    return torch, pnp


def regular(pnp, torch, spec, rho):
    with pnp.Problem(spec) as P:
        d_rho = torch.from_numpy(rho).cuda()
        d_mu = torch.empty_like(d_rho)
        P.excess_mu_device(d_rho, d_mu)
        assert P.status() == 0
        return d_mu.cpu().numpy()


def normwise(a, b):
    return max(np.abs(a[i] - b[i]).max() / np.abs(b[i]).max() for i in range(a.shape[0]))


def test_matches_regular_entry_two_calls_in_a_row(env):
    torch, pnp = env
    spec, rho1 = mu_microbench(16)
    rho2 = lognormal_density(spec, 77, sigma=0.3)
    stream = torch.cuda.Stream()
    for rho in (rho1, rho2):
        d_rho = torch.from_numpy(rho).cuda()
        d_mu = torch.full_like(d_rho, np.nan)
        torch.cuda.synchronize()
        rc = pnp.excess_mu_noalloc(spec, d_rho, d_mu, stream=stream.cuda_stream)
        assert rc == pnp.OK, pnp.error_string(rc)
        got = d_mu.cpu().numpy()
        ref = regular(pnp, torch, spec, rho)
        assert normwise(got, ref) <= FP64_TOL


def test_different_grid_after_previous_call(env):
    torch, pnp = env
    spec, rho = mu_microbench(shape=(13, 11, 9))
    d_rho = torch.from_numpy(rho).cuda()
    d_mu = torch.empty_like(d_rho)
    assert pnp.excess_mu_noalloc(spec, d_rho, d_mu) == pnp.OK
    assert normwise(d_mu.cpu().numpy(), regular(pnp, torch, spec, rho)) <= FP64_TOL


def test_refuses_what_does_not_fit(env):
    torch, pnp = env
    spec, _ = mu_microbench(128, fft_len=256)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert pnp.excess_mu_noalloc(spec, dummy, dummy) == pnp.ERR_TOO_LARGE
    wells = film_gummel(16, 16, 16)
    assert pnp.excess_mu_noalloc(wells, dummy, dummy) == pnp.ERR_INVALID
    # the MSA term is not part of this entry point's pipeline
    msa, _ = mu_microbench(12)
    msa.msa = True
    assert pnp.excess_mu_noalloc(msa, dummy, dummy) == pnp.ERR_INVALID
