"""Serving (pnp_submit / pnp_poll): independent Gummel solves run
concurrently on one GPU.  Each result must be the same alone and in the mix
(bitwise: the kernels and reductions are deterministic), admission must
respect the device-memory budget, over-budget requests are refused with
PNP_ERR_BUSY, and polls never block."""
import time

import numpy as np
import pytest

from workloads import ProblemSpec, bulk_density

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pnp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build, pnp as mod
    build.build()
    return mod


def small(bias, T=300.0, shape=(10, 8, 8), seed=0, eta=0.05):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    rb = bulk_density(eta, 1.0)
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=(1.0, 1.0), q=(1, -1), rho_b=(rb, rb),
                       depth=(1.0, 0.0), well_inner=2.0, well_outer=3.0,
                       sites=rng.uniform(0, 1, (3, 3)) * np.array([nx, ny, nz]),
                       rho_f=rng.normal(0, 0.01, shape), temperature_K=T, phi_lo=0.0, phi_hi=bias,
                       lambda_phi=0.3, lambda_rho=0.3, tol=1e-10, max_iter=400)


def mix():
    return [small(0.1 * k, T=250 + 20 * k, shape=((10, 8, 8), (12, 8, 8), (8, 16, 16))[k % 3], seed=k)
            for k in range(8)]


def alone(pnp, spec):
    with pnp.Problem(spec) as P:
        return P.gummel_solve()


def drain(server, tickets, timeout=300):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            t1 = time.perf_counter()
            rc, phi, rho, st = server.poll(t)
            assert time.perf_counter() - t1 < 0.05          # poll never blocks
            if rc != 1:
                out[t] = (rc, phi, rho, st)
        assert time.time() - t0 < timeout
        time.sleep(0.005)
    return out


def test_results_same_alone_and_in_the_mix(pnp):
    specs = mix()
    srv = pnp.Server(max_slots=8)
    tickets = []
    for s in specs:
        rc, t = srv.submit(s)
        assert rc == 0
        tickets.append(t)
    assert len(set(tickets)) == len(tickets)
    res = drain(srv, tickets)
    for s, t in zip(specs, tickets):
        rc, phi, rho, st = res[t]
        assert rc == 0 and st["status"] == 0
        phi1, rho1, st1 = alone(pnp, s)
        np.testing.assert_array_equal(phi, phi1)
        np.testing.assert_array_equal(rho, rho1)
        assert st["iterations"] == st1["iterations"]
    stats = srv.stats()
    assert stats["completed"] == len(specs) and stats["failed"] == 0
    srv.close()


def test_served_solves_match_oracle(pnp):
    """Two solves of the eight-solve mix (different grids and temperatures),
    served concurrently with the other six, against the oracle's converged
    states at 1e-8, and bitwise against the same solves run alone."""
    from oracle import oracle
    specs = mix()
    for s in specs:
        s.lin_tol = 1e-13
    srv = pnp.Server(max_slots=8)
    tickets = []
    for s in specs:
        rc, t = srv.submit(s)
        assert rc == 0
        tickets.append(t)
    res = drain(srv, tickets)
    srv.close()
    for k in (0, 2):
        rc, phi, rho, st = res[tickets[k]]
        assert rc == 0 and st["status"] == 0
        ref = oracle.gummel(specs[k])
        assert ref["status"] == 0 and st["iterations"] == ref["iters"]
        assert np.abs(phi - ref["phi"]).max() / max(np.abs(ref["phi"]).max(), 1.0) <= 1e-8
        for i in range(specs[k].s):
            assert np.abs(rho[i] - ref["rho"][i]).max() / np.abs(ref["rho"][i]).max() <= 1e-8
        phi1, rho1, _ = alone(pnp, specs[k])
        np.testing.assert_array_equal(phi, phi1)
        np.testing.assert_array_equal(rho, rho1)


def test_budget_admission_and_busy(pnp):
    specs = mix()[:4]
    # a budget that holds about one of these problems at a time
    from paper_1407_0674_gb300.pnp import DescHolder
    srv = pnp.Server(hbm_budget_bytes=64 << 20, max_slots=4)
    tickets = [srv.submit(s)[1] for s in specs]
    assert all(t is not None for t in tickets)
    res = drain(srv, tickets)
    assert all(r[0] == 0 for r in res.values())
    big = small(0.1, shape=(256, 256, 256))
    rc, t = srv.submit(big)
    assert rc == pnp.ERR_BUSY and t is None
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_tickets_and_invalid(pnp):
    srv = pnp.Server()
    rc, t = srv.submit(small(0.2))
    assert rc == 0
    res = drain(srv, [t])
    assert res[t][0] == 0
    assert srv.poll(t)[0] == pnp.ERR_UNKNOWN_TICKET          # already taken
    assert srv.poll(987654321)[0] == pnp.ERR_UNKNOWN_TICKET
    bad = small(0.2)
    bad.bc = ("D", "P", "D")
    assert srv.submit(bad)[0] == pnp.ERR_INVALID
    bad2 = small(0.2)
    bad2.lambda_rho = 0.0
    assert srv.submit(bad2)[0] == pnp.ERR_INVALID
    srv.close()


def test_warm_start_through_server(pnp):
    s = small(0.3)
    phi, rho, st = alone(pnp, s)
    srv = pnp.Server()
    rc, t = srv.submit(s, phi0=phi, rho0=rho)
    assert rc == 0
    r = drain(srv, [t])[t]
    assert r[0] == 0 and r[3]["iterations"] <= 2
    srv.close()


def completion_order(pnp, policy, specs):
    """Submit `specs` in order to a one-slot server; return the tickets in the
    order their results became ready."""
    srv = pnp.Server(max_slots=1, policy=policy)
    tickets = []
    for s in specs:
        rc, t = srv.submit(s)
        assert rc == 0
        tickets.append(t)
    order, res = [], {}
    t0 = time.time()
    while len(order) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            r = srv.poll(t)
            if r[0] != 1:
                res[t] = r
                order.append(t)
        assert time.time() - t0 < 300
        time.sleep(0.002)
    srv.close()
    return tickets, order, res


def test_smallest_first_lets_a_small_request_overtake(pnp):
    """One slot, three 32^3 solves submitted ahead of an 8x8x10 one: first in,
    first out the small one finishes last; smallest first it finishes right
    after the solve that was already running, with the same bits."""
    big = [small(0.1 * k, shape=(32, 32, 32), seed=10 + k) for k in range(3)]
    for b in big:
        b.screened_poisson = True      # the plain step is unstable on a 32-plane box
    little = small(0.3, seed=3)
    specs = big + [little]
    tk, order, res = completion_order(pnp, "fifo", specs)
    assert order[-1] == tk[3]
    tk2, order2, res2 = completion_order(pnp, "smallest_first", specs)
    assert order2.index(tk2[3]) <= 1, order2
    for a, b in zip(tk, tk2):
        assert res[a][0] == 0 and res2[b][0] == 0
        np.testing.assert_array_equal(res[a][2], res2[b][2])


def test_priority_streams_keep_results_bitwise(pnp):
    """Smallest first with every request admitted at once (priority streams
    only): each result is the same bits as the solve run alone."""
    specs = mix()
    srv = pnp.Server(max_slots=8, policy="smallest_first")
    tickets = [srv.submit(s)[1] for s in specs]
    res = drain(srv, tickets)
    srv.close()
    for s, t in zip(specs, tickets):
        rc, phi, rho, st = res[t]
        assert rc == 0
        phi1, rho1, _ = alone(pnp, s)
        np.testing.assert_array_equal(rho, rho1)
