"""GPU parity of the MSA electrostatic-correlation term (Sec 2.3.4,
PNP_FLAG_MSA) against the oracle's direct ball-quadrature sums.

Bars: the whole mu_ex with the term at the mu_ex bars (FP64 and double-float
1e-10, FP32 2e-5, normwise per species), and the term itself -- mu_ex with the
flag minus mu_ex without it, on both sides -- to 1e-8 of its own size in FP64
(it is a small part of mu_ex, so the first bar alone would not see an error in
it).  The oracle's l_B comes from a 10-digit k_B, 1.7e-11 from the library's
SI value, which the term carries linearly.  Cases: periodic, zero-extended and
Dirichlet axes (the pair kernels reach R_i + R_j, beyond the FMT reach, so the
padded lengths grow), square wells, a neutral species, the generic
(non-register) z length, and five Gummel iterations with the term.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, film_gummel, lognormal_density, mu_microbench

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 2e-5
TERM_TOL = 1e-8


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


def four_species(bc, shape):
    nx, ny, nz = shape
    spec = ProblemSpec(nx=nx, ny=ny, nz=nz, bc=bc, R=(1.0, 1.5, 0.7, 1.2), q=(1, -1, 2, 0),
                       rho_b=(0.004, 0.006, 0.001, 0.003), msa=True)
    return spec, lognormal_density(spec, 5, sigma=0.3)


CASES = {
    "periodic_10x8x9": lambda: four_species(("P", "P", "P"), (10, 8, 9)),
    "mixed_9x8x10": lambda: four_species(("N", "P", "D"), (9, 8, 10)),
    "zero_extended_three_species": lambda: (lambda s, r: (dataclasses.replace(s, msa=True), r))(
        *mu_microbench(shape=(13, 11, 9))),
    "film_wells_12": lambda: (lambda s: (s, lognormal_density(s, 3, sigma=0.2)))(
        dataclasses.replace(film_gummel(12, 12, 12, nsites=4), msa=True)),
}


def gpu_mu(pnp, spec, rho, prec):
    with pnp.Problem(spec) as P:
        return P.excess_mu(rho, precision=prec)


@pytest.mark.parametrize("case", sorted(CASES))
def test_mu_ex_with_msa_matches_oracle(pnp, case):
    spec, rho = CASES[case]()
    ref, bad = oracle.excess_mu(spec, rho)
    assert bad == 0
    mu = gpu_mu(pnp, spec, rho, "fp64")
    assert normwise(mu, ref) <= FP64_TOL
    assert normwise(gpu_mu(pnp, spec, rho, "df64"), ref) <= FP64_TOL
    assert normwise(gpu_mu(pnp, spec, rho, "fp32"), ref) <= FP32_TOL
    # the term itself
    plain = dataclasses.replace(spec, msa=False)
    ref0, _ = oracle.excess_mu(plain, rho)
    mu0 = gpu_mu(pnp, plain, rho, "fp64")
    term, term_ref = mu - mu0, ref - ref0
    charged = [i for i in range(spec.s) if spec.q[i] != 0]
    assert charged
    for i in charged:
        scale = np.abs(term_ref[i]).max()
        assert scale > 1e-6 * np.abs(ref[i]).max()      # the term is really there
        assert np.abs(term[i] - term_ref[i]).max() <= TERM_TOL * scale
    for i in range(spec.s):
        if spec.q[i] == 0:
            assert np.abs(term[i]).max() <= 1e-12 * np.abs(mu[i]).max()


@pytest.mark.parametrize("s", [2, 3])
def test_msa_z_length_256(pnp, s):
    """Lz = 256: the radix-4 z-back kernels apply the term in double-float,
    the two-factor ones in FP64 and FP32."""
    spec, rho = four_species(("N", "P", "D"), (9, 8, 30))
    keep = slice(0, s)
    spec = dataclasses.replace(spec, R=spec.R[keep], q=spec.q[keep], rho_b=spec.rho_b[keep], fft_len=(32, 8, 256))
    rho = np.ascontiguousarray(rho[keep])
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec) as P:
        assert P.info()["fft_len"] == (32, 8, 256)
        mu = P.excess_mu(rho, precision="fp64")
        mudd = P.excess_mu(rho, precision="df64")
        mu32 = P.excess_mu(rho, precision="fp32")
    assert normwise(mu, ref) <= FP64_TOL
    assert normwise(mudd, ref) <= FP64_TOL
    assert normwise(mu32, ref) <= FP32_TOL


def test_msa_generic_z_length(pnp):
    """Lz = 30 has no register FFT: the shared-memory Stockham z-back kernel
    applies the term."""
    spec, rho = mu_microbench(shape=(12, 9, 10))
    spec = dataclasses.replace(spec, msa=True, fft_len=(32, 16, 30))
    ref, _ = oracle.excess_mu(spec, rho)
    with pnp.Problem(spec) as P:
        assert P.info()["fft_len"] == (32, 16, 30)
        mu = P.excess_mu(rho, precision="fp64")
        mudd = P.excess_mu(rho, precision="df64")
    assert normwise(mu, ref) <= FP64_TOL
    assert normwise(mudd, ref) <= FP64_TOL


def test_msa_gummel_trajectory_matches_oracle(pnp):
    """Five Gummel iterations of a dilute biased film with the term, iterate
    by iterate against the oracle at 1e-8."""
    rng = np.random.default_rng(0)
    nz, ny, nx = 10, 8, 8
    from workloads import bulk_density
    rb = bulk_density(0.05, 1.0)
    spec = ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(1.0, 0.0), well_inner=2.0, well_outer=3.0,
                       sites=rng.uniform(0, 1, (3, 3)) * np.array([nx, ny, nz]),
                       rho_f=rng.normal(0, 0.01, (nz, ny, nx)), phi_lo=0.0, phi_hi=0.5,
                       lambda_phi=0.3, lambda_rho=0.3, tol=1e-30, max_iter=5, lin_tol=1e-13, msa=True)
    ref = oracle.gummel(spec)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["iterations"] == ref["iters"] == 5
    assert np.abs(phi - ref["phi"]).max() / max(np.abs(ref["phi"]).max(), 1.0) <= 1e-8
    for i in range(2):
        assert np.abs(rho[i] - ref["rho"][i]).max() / np.abs(ref["rho"][i]).max() <= 1e-8
    # and the term changed the trajectory
    plain = oracle.gummel(dataclasses.replace(spec, msa=False))
    assert np.abs(plain["rho"][0] - ref["rho"][0]).max() > 1e-6 * np.abs(ref["rho"][0]).max()

