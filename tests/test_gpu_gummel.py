"""GPU parity of the relaxed Gummel solve (pnp_gummel_solve through the C ABI)
against the oracle, plus properties of the converged state.

Bar: converged potentials and densities agree with the oracle to 1e-8
(normwise relative, phi relative to max(|phi|, phi scale)); fixed-iteration
trajectories likewise.  Both sides solve their linear systems to a relative
residual of 1e-13.
"""
import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density, film_gummel

pytestmark = pytest.mark.gpu
TOL = 1e-8


@pytest.fixture(scope="module")
def pnp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp as mod
    build.build()
    return mod


def dilute(bias_lo, bias_hi, mix=0, tol=1e-11, max_iter=400, shape=(10, 8, 8)):
    rng = np.random.default_rng(0)
    nz, ny, nx = shape
    rb = bulk_density(0.05, 1.0)
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(1.0, 0.0), well_inner=2.0, well_outer=3.0,
                       sites=rng.uniform(0, 1, (3, 3)) * np.array([nx, ny, nz]),
                       rho_f=rng.normal(0, 0.01, shape), phi_lo=bias_lo, phi_hi=bias_hi,
                       lambda_phi=0.3, lambda_rho=0.3, rho_mix=mix, tol=tol, max_iter=max_iter, lin_tol=1e-13)


def rel(a, b, floor=0.0):
    return np.abs(a - b).max() / max(np.abs(b).max(), floor)


def compare(spec, pnp, phi_floor=1.0):
    ref = oracle.gummel(spec)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["iterations"] == ref["iters"], (st, ref["iters"])
    assert rel(phi, ref["phi"], phi_floor) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL
    return phi, rho, st, ref


@pytest.mark.parametrize("mix", [0, 1])
def test_trajectory_matches_oracle(pnp, mix):
    spec = dilute(0.0, 0.5, mix=mix, tol=1e-30, max_iter=6)
    phi, rho, st, ref = compare(spec, pnp)
    assert st["status"] == pnp.ERR_NOT_CONVERGED


def test_df64_trajectory_matches_oracle(pnp):
    spec = dilute(0.0, 0.5, tol=1e-30, max_iter=6)
    ref = oracle.gummel(spec)
    with pnp.Problem(spec, precision="df64") as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["iterations"] == ref["iters"]
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_dense_film_trajectory_matches_oracle(pnp):
    """The film workload's physics (R 2h, packing 0.2 per ion, wells, geometric
    relaxation 0.05) on a 12^3 grid, five iterations."""
    spec = film_gummel(12, 12, 12, tol=1e-30, max_iter=5)
    spec.lin_tol = 1e-13
    compare(spec, pnp)


def test_full_size_film_trajectory_matches_oracle(pnp):
    """The 32^3 film workload itself (2 ions, R 2h, packing 0.2 each, 1 kT
    wells on 64 sites, fixed charge, bias 0.1 kT/e, geometric relaxation
    0.05): its first three Gummel iterates against the oracle's, iterate by
    iterate (the oracle takes about half a minute)."""
    spec = film_gummel(32, 32, 32, tol=1e-30, max_iter=3)
    spec.lin_tol = 1e-13
    phi, rho, st, ref = compare(spec, pnp)
    assert st["iterations"] == 3 and st["status"] == pnp.ERR_NOT_CONVERGED


def test_deep_wells_step_limited_trajectory(pnp):
    """Batch-workload physics at 12^3: wells 12 kT deep, packing 0.3, step-
    limited geometric relaxation; six iterations match the oracle (the step
    limit is active in the first ones)."""
    from workloads import batch_specs
    spec = batch_specs(1, grids=[(12, 12, 12)])[0]
    spec.depth = (12.0, 0.0)
    spec.tol, spec.max_iter, spec.lin_tol = 1e-30, 6, 1e-13
    compare(spec, pnp)


def test_converged_state_matches_oracle(pnp):
    spec = dilute(0.0, 0.5)
    phi, rho, st, ref = compare(spec, pnp)
    assert st["status"] == 0 and ref["status"] == 0


def test_zero_bias_boltzmann(pnp):
    spec = dilute(0.2, 0.2)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        mu = P.excess_mu(rho)
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    for i in range(2):
        q = spec.q[i]
        ref = spec.rho_b[i] * np.exp(mub[i] + q * 0.2 - q * phi - mu[i])
        np.testing.assert_allclose(rho[i], ref, rtol=1e-8)


def test_flux_conserved_full_size_film(pnp):
    """The 32^3 film workload converges to 1e-8; the discrete flux through
    every z plane is then the same for each species."""
    spec = film_gummel(32, 32, 32, tol=1e-8, max_iter=2000)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        mu = P.excess_mu(rho)
    assert st["status"] == 0 and st["residual"] < 1e-8
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    for i in range(2):
        rbar = rho[i] * np.exp(spec.q[i] * phi + mu[i])
        f = oracle.np_flux(spec, i, phi, mu[i], mub[i], rbar)
        assert np.abs(f - f.mean()).max() <= 1e-4 * np.abs(f).max() + 1e-12


def test_warm_start_converges_immediately(pnp):
    spec = dilute(0.0, 0.5)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        phi2, rho2, st2 = P.gummel_solve(phi0=phi, rho0=rho)
    assert st2["iterations"] <= 2
    assert rel(rho2, rho) < 1e-9


def test_not_converged_and_invalid(pnp):
    spec = dilute(0.0, 0.5, max_iter=2)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
        assert st["status"] == pnp.ERR_NOT_CONVERGED and st["iterations"] == 2
        with pytest.raises(pnp.PnpError) as e:
            P.gummel_solve(rho0=-np.ones((2,) + spec.shape))
        assert e.value.code == pnp.ERR_INVALID
        with pytest.raises(pnp.PnpError) as e:
            P.gummel_solve(rho0=np.full((2,) + spec.shape, 0.5))    # packing far above 1
        assert e.value.code == pnp.ERR_PACKING
    bad = dilute(0.0, 0.5)
    bad.bc = ("D", "P", "D")
    with pnp.Problem(bad) as P:
        with pytest.raises(pnp.PnpError) as e:
            P.gummel_solve()
        assert e.value.code == pnp.ERR_INVALID


# ---------------------------------------------------------------------------
# equilibrium cDFT initial guess (PNP_FLAG_EQUILIBRIUM_INIT)

def eq_spec(bias, **kw):
    spec = dilute(0.0, bias, mix=1)
    for k, v in dict(eq_init=True, max_iter=0, lin_tol=1e-13, **kw).items():
        setattr(spec, k, v)
    return spec


def test_equilibrium_trajectory_matches_oracle(pnp):
    """Three equilibrium iterations alone (max_iter 0): Newton steps of the
    Poisson-Boltzmann equation and the Boltzmann relaxation, against the
    oracle's."""
    spec = eq_spec(0.5, eq_tol=1e-30, eq_max_iter=3)
    ref = oracle.equilibrium(spec, tol=1e-30, max_iter=3)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["status"] == pnp.ERR_NOT_CONVERGED and st["iterations"] == 0
    assert st["init_iterations"] == 3 == ref["iters"]
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_equilibrium_converged_matches_oracle(pnp):
    spec = eq_spec(0.5, eq_tol=1e-10, eq_max_iter=2000)
    ref = oracle.equilibrium(spec, tol=1e-10, max_iter=2000)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert ref["status"] == 0 and st["status"] == 0
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_equilibrium_start_reaches_the_same_solution(pnp):
    """A biased solve started from the equilibrium converges to the state the
    default start reaches (one fixed point)."""
    base = dilute(0.0, 0.5, mix=1)
    spec = dilute(0.0, 0.5, mix=1)
    spec.eq_init, spec.eq_tol = True, 1e-8
    with pnp.Problem(base) as P:
        phi0, rho0, st0 = P.gummel_solve()
    with pnp.Problem(spec) as P:
        phi1, rho1, st1 = P.gummel_solve()
    assert st0["status"] == 0 and st1["status"] == 0 and st1["init_iterations"] > 0
    assert rel(phi1, phi0, 1.0) <= 1e-8
    for i in range(spec.s):
        assert rel(rho1[i], rho0[i]) <= 1e-8


def test_equilibrium_skipped_with_warm_start(pnp):
    spec = dilute(0.0, 0.5, mix=1)
    spec.eq_init = True
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        phi2, rho2, st2 = P.gummel_solve(phi0=phi, rho0=rho)
    assert st["init_iterations"] > 0 and st2["init_iterations"] == 0
    assert st2["iterations"] <= 2


# ---------------------------------------------------------------------------
# screened Poisson step (PNP_FLAG_SCREENED_POISSON)

def test_screened_trajectory_matches_oracle(pnp):
    spec = dilute(0.0, 0.5, mix=1, tol=1e-30, max_iter=6)
    spec.screened_poisson = True
    phi, rho, st, ref = compare(spec, pnp)
    assert st["status"] == pnp.ERR_NOT_CONVERGED


def test_screened_long_box_converges_where_plain_does_not(pnp):
    """64 planes, ~20 Debye lengths: the plain relaxed step blows up, the
    screened one converges to the oracle's state."""
    from test_oracle_equilibrium import long_box
    spec = long_box()
    spec.lin_tol = 1e-13
    with pnp.Problem(spec) as P:
        _, _, st0 = P.gummel_solve(raise_on_error=False)
    assert st0["status"] != 0
    spec.screened_poisson = True
    ref = oracle.gummel(spec)
    assert ref["status"] == 0
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["status"] == 0
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_adaptive_relaxation_trajectory(pnp):
    """Per-point adaptive relaxation (PNP_MIX_ADAPTIVE) on the deep-well batch
    physics at 12^3: eight iterations match the oracle's."""
    from workloads import batch_specs
    spec = batch_specs(1, grids=[(12, 12, 12)])[0]
    spec.depth = (12.0, 0.0)
    spec.rho_mix = 3
    spec.tol, spec.max_iter, spec.lin_tol = 1e-30, 8, 1e-13
    compare(spec, pnp)


def test_white_bear_trajectory_matches_oracle(pnp):
    """Gummel iterations with the White Bear functional (its reservoir mu_b
    enters the Dirichlet data of the Nernst-Planck solves)."""
    spec = dilute(0.0, 0.5, mix=1, tol=1e-30, max_iter=5)
    spec.fmt = 1
    compare(spec, pnp)


def test_plane_flux_matches_oracle(pnp):
    """pnp_plane_flux on a converged biased state: each face's current equals
    the oracle's discrete flux (from the oracle's own mu_ex), and at steady
    state every face carries the same current."""
    spec = dilute(0.0, 0.5, mix=1)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
        flux = [P.plane_flux(i, phi, rho) for i in range(spec.s)]
    assert st["status"] == 0
    mu, _ = oracle.excess_mu(spec, rho)
    mub = oracle.bulk_mu(spec.R, spec.rho_b)
    for i in range(spec.s):
        rbar = rho[i] * np.exp(spec.q[i] * phi + mu[i])
        ref = oracle.np_flux(spec, i, phi, mu[i], mub[i], rbar)
        scale = np.abs(ref).max()
        assert scale > 0
        assert np.abs(flux[i] - ref).max() <= 1e-9 * scale
        assert np.abs(flux[i] - flux[i].mean()).max() <= 1e-4 * scale
    # the cation and anion currents run in opposite directions
    assert flux[0].mean() * flux[1].mean() < 0



# ---------------------------------------------------------------------------
# Anderson mixing of the relaxed iteration (anderson_depth > 0): the device
# against the oracle's Anderson iteration (itself pinned to the relaxed
# iteration's fixed point), iterate by iterate and to convergence.

@pytest.mark.parametrize("mix", [0, 2])
def test_anderson_trajectory_matches_oracle(pnp, mix):
    spec = dilute(0.0, 0.5, mix=mix, tol=1e-30, max_iter=8)
    spec.anderson = 3
    ref = oracle.gummel_anderson(spec, m=3)
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve(raise_on_error=False)
    assert st["iterations"] == ref["iters"] == 8
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_anderson_dense_film_converges_like_oracle(pnp):
    """The film physics on 8^3 (geometric relaxation 0.05, where the relaxed
    iteration needs about 390 sweeps): depth-3 Anderson converges in the
    oracle's number of iterations to the oracle's state."""
    spec = film_gummel(8, 8, 8, tol=1e-8, max_iter=600)
    spec.anderson = 3
    spec.lin_tol = 1e-13
    ref = oracle.gummel_anderson(spec, m=3)
    assert ref["status"] == 0
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
    assert st["status"] == 0 and st["iterations"] == ref["iters"] <= 150
    assert rel(phi, ref["phi"], 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= TOL


def test_anderson_full_size_film_same_state_fewer_iterations(pnp):
    """The 32^3 film converged tightly (residual 1e-11) by the relaxed
    iteration and by depth-3 Anderson: the same state to 1e-8, in a fraction
    of the iterations."""
    spec = film_gummel(32, 32, 32, tol=1e-11, max_iter=4000)
    with pnp.Problem(spec) as P:
        phi0, rho0, st0 = P.gummel_solve()
    assert st0["repeated_sweeps"] == 0
    spec.anderson = 3
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
    assert st0["status"] == 0 and st["status"] == 0
    assert st["iterations"] * 3 <= st0["iterations"], (st["iterations"], st0["iterations"])
    assert rel(phi, phi0, 1.0) <= TOL
    for i in range(spec.s):
        assert rel(rho[i], rho0[i]) <= TOL


def test_anderson_backtracking_matches_oracle(pnp):
    """The configs' single relaxation 0.3 on both phi and rho (printed linear
    form) on the 8^3 film physics: the relaxed iteration dies of packing at
    its second sweep; Anderson with the restart and step halving converges to
    the oracle's state.  The path through the repeated, halved sweeps depends
    on rounding (the oracle itself takes 122 iterations on one host and 178 on
    another), so the converged states are compared, at the 1e-6 their stop at
    residual 1e-8 of the 0.3-scaled step allows."""
    spec = film_gummel(8, 8, 8, tol=1e-8, max_iter=300)
    spec.lambda_rho, spec.rho_mix, spec.anderson, spec.lin_tol = 0.3, 0, 3, 1e-13
    ref = oracle.gummel_anderson(spec, m=3)
    assert ref["status"] == 0
    with pnp.Problem(spec) as P:
        phi, rho, st = P.gummel_solve()
    assert st["status"] == 0 and st["iterations"] <= 300
    assert st["repeated_sweeps"] > 0          # the restart / step halving ran
    assert rel(phi, ref["phi"], 1.0) <= 1e-6
    for i in range(spec.s):
        assert rel(rho[i], ref["rho"][i]) <= 1e-6


def test_anderson_refuses_adaptive_relaxation(pnp):
    spec = dilute(0.0, 0.5, mix=3)
    spec.anderson = 3
    with pytest.raises(pnp.PnpError) as e:
        pnp.Problem(spec)
    assert e.value.code == pnp.ERR_INVALID


def test_phase_timing_marks_do_not_change_results(pnp):
    """PNP_FLAG_PHASE_TIMING: every phase of the iteration gets device time,
    the phases sum to no more than the solve's wall time, and the results are
    the same bits as without the marks."""
    import time
    spec = film_gummel(16, 16, 16, tol=1e-30, max_iter=8)
    with pnp.Problem(spec) as P:
        phi0, rho0, st0 = P.gummel_solve(raise_on_error=False)
    spec.phase_timing = True
    with pnp.Problem(spec) as P:
        P.gummel_solve(raise_on_error=False)            # graph build outside the timing
        t0 = time.perf_counter()
        phi, rho, st = P.gummel_solve(raise_on_error=False)
        wall_ms = (time.perf_counter() - t0) * 1e3
        ph = P.gummel_phase_times()
    assert set(ph) == {"mu_ex", "poisson", "nernst_planck", "update"}
    assert all(v > 0 for v in ph.values()), ph
    assert sum(ph.values()) <= wall_ms, (ph, wall_ms)
    assert st["iterations"] == st0["iterations"] == 8
    np.testing.assert_array_equal(phi, phi0)
    np.testing.assert_array_equal(rho, rho0)
