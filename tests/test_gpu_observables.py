"""GPU checks of the observables computed from a solution: the conductivity
(device plane currents, then the host-only pnp_conductivity) and the
square-well free energy F_sh (the device well field summed against the
densities), each against the oracle."""
import numpy as np
import pytest

from oracle import oracle
from test_gpu_gummel import dilute
from workloads import film_gummel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pnp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp as mod
    build.build()
    return mod


def test_conductivity_of_converged_state(pnp):
    """Problem.conductivity (device plane currents, then the host-only
    pnp_conductivity) on a converged biased state against the oracle's
    conductivity of the oracle's discrete currents, reduced and in S/cm."""
    spec = dilute(0.0, 0.5, mix=1)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        sig = P.conductivity(phi, rho, D_m2_per_s=1e-10)
    assert st["status"] == 0
    mu, _ = oracle.excess_mu(spec, rho)
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    flux = [oracle.np_flux(spec, i, phi, mu[i], mub[i], rho[i] * np.exp(spec.q[i] * phi + mu[i]))
            for i in range(spec.s)]
    ref = oracle.conductivity(spec, flux, D_m2_per_s=1e-10)
    assert sig[0] > 0
    assert sig[0] == pytest.approx(ref[0], rel=1e-8)
    assert sig[1] == pytest.approx(ref[1], rel=1e-8)


@pytest.mark.parametrize("depth2,shape", [(0.0, (16, 12, 10)), (0.7, (16, 12, 10)), (0.7, (48, 40, 36))])
def test_square_well_energy_matches_oracle(pnp, depth2, shape):
    """pnp_square_well_energy (the device well field, summed against rho by a
    fixed-shape device reduction; the largest grid spans 270 blocks) against
    the oracle's direct-quadrature F_sh, the same bits on a repeat call; a
    film without wells gives exactly zero."""
    nx, ny, nz = shape
    spec = film_gummel(nx, ny, nz, nsites=6)
    spec.depth = (1.0, depth2)
    rng = np.random.default_rng(12)
    rho = np.stack([spec.rho_b[i] * rng.lognormal(0.0, 0.3, spec.shape) for i in range(spec.s)])
    with pnp.Problem(spec) as P:
        F = P.square_well_energy(rho)
        assert P.square_well_energy(rho) == F
    ref = oracle.square_well_energy(spec, rho)
    assert ref < 0
    assert F == pytest.approx(ref, rel=1e-10)
    spec.depth = (0.0, 0.0)
    with pnp.Problem(spec) as P:
        assert P.square_well_energy(rho) == 0.0
