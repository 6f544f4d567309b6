"""Pin of the oracle's relaxed Gummel sweep (Sec 3.2) against an independent
composition on tiny grids, started from arbitrary states:

- mu_ex,i = mu_hs,i + mu_sh,i (Sec 2.3) from the dense weighted-density
  operators of tests/brute.py, a complex-step derivative of Phi (Rosenfeld or
  White Bear), the transposed operators for the back-convolution, and the
  square-well term from an explicit Gaussian image sum of the site density;
- the Poisson step (Sec 2.1, 3.3) as a dense LU solve of the Kronecker-sum
  Laplacian, plain or as one screened Newton step about the current phi;
- the Slotboom Nernst-Planck solves (Sec 2.1, 3.1) as dense LU solves of the
  harmonic-mean system assembled point by point (tests/test_oracle_linear.py);
- then the phi relaxation and the density relaxation of each mode (linear,
  geometric, step-limited, per-point adaptive), and the sweep residual.

mu_ex and the Poisson right-hand side take the densities the sweep starts
from; the NP solves take the relaxed phi.  The oracle's iteration applies this
sweep repeatedly, so pinning it from arbitrary states pins every iterate of
its trajectory up to the linear-solver tolerance.  The equilibrium stage's
steps (Newton step of Poisson-Boltzmann, clamp, density relaxation) are
pinned the same way.
"""
import math

import numpy as np
import pytest

import brute
from oracle import oracle, units
from test_oracle_linear import lap1d, np_dense
from workloads import ProblemSpec, bulk_density

SHAPE = (7, 6, 6)   # (nz, ny, nx)


def make_spec(rho_mix, screened, fmt, sweeps, msa=False):
    nz, ny, nx = SHAPE
    rng = np.random.default_rng(21)
    R = (1.5, 2.0)
    return ProblemSpec(nx=nx, ny=ny, nz=nz, bc=("P", "P", "D"), R=R, q=(1, -1),
                       rho_b=tuple(bulk_density(0.12, r) for r in R),
                       depth=(1.0, 0.4), well_inner=2.0, well_outer=3.0,
                       sites=rng.uniform(0, 1, (4, 3)) * np.array([nx, ny, nz]), site_alpha=0.8,
                       rho_f=rng.normal(0, 0.002, SHAPE), phi_lo=0.0, phi_hi=0.5,
                       lambda_phi=0.4, lambda_rho=0.3, rho_mix=rho_mix, tol=0.0, max_iter=sweeps,
                       screened_poisson=screened, fmt=fmt, msa=msa)


def start_state(spec, seed=5):
    rng = np.random.default_rng(seed)
    z = np.arange(1, spec.nz + 1)[:, None, None]
    phi = spec.phi_lo + (spec.phi_hi - spec.phi_lo) * z / (spec.nz + 1) + rng.normal(0, 0.1, spec.shape)
    rho = np.stack([spec.rho_b[i] * rng.lognormal(0, 0.2, spec.shape) for i in range(spec.s)])
    return phi, rho


class DenseSweep:
    """One relaxed Gummel sweep built from dense, independently assembled parts."""

    def __init__(self, spec):
        self.spec = spec
        nz, ny, nx = spec.shape
        per = tuple(b == "P" for b in spec.bc)
        self.B = brute.BruteFMT(spec.shape, per, spec.R)
        reach = int(math.ceil(spec.well_outer)) + 1
        p, w, u = brute.nodes("thick", spec.well_outer, r_in=spec.well_inner)
        Mw = brute.dense_operator(brute.kernel_table(p, w, u, reach), reach, spec.shape, per)
        # site density: Gaussians with explicit periodic images on x and y
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        rs = np.zeros(spec.shape)
        for s in spec.sites:
            for ix in range(-3, 4):
                for iy in range(-3, 4):
                    d2 = (x - s[0] - nx * ix) ** 2 + (y - s[1] - ny * iy) ** 2 + (z - s[2]) ** 2
                    rs += np.exp(-spec.site_alpha * d2)
        rs *= (spec.site_alpha / np.pi) ** 1.5
        well = Mw @ rs.reshape(-1)
        self.mu_sh = [0.5 * (-spec.depth[i]) * well for i in range(spec.s)]
        self.A = (np.kron(np.eye(nz), np.kron(np.eye(ny), lap1d(nx, spec.bc[0])))
                  + np.kron(np.eye(nz), np.kron(lap1d(ny, spec.bc[1]), np.eye(nx)))
                  + np.kron(lap1d(nz, "D"), np.eye(ny * nx)))
        self.lB = units.bjerrum_length_h(spec.temperature_K, spec.eps_r, spec.h_nm)
        self.mu_b = oracle.bulk_mu(spec.R, spec.rho_b, fmt=spec.fmt)
        # MSA pair operators (Sec 2.3.4), B from the textbook screening parameter
        self.msa = None
        if getattr(spec, "msa", False):
            kap = math.sqrt(4 * math.pi * self.lB * sum(r * q * q for r, q in zip(spec.rho_b, spec.q)))
            self.msa = [[None] * spec.s for _ in range(spec.s)]
            for i in range(spec.s):
                for j in range(spec.s):
                    qq = spec.q[i] * spec.q[j]
                    if qq == 0:
                        continue
                    sg = spec.R[i] + spec.R[j]
                    gs = 0.5 * (math.sqrt(1 + 2 * kap * sg) - 1)
                    B = gs / (1 + gs)
                    pb, wb, ub = brute.nodes("ball", sg)
                    r = np.linalg.norm(pb, axis=1)
                    C = -qq * self.lB * (2 * B / sg - (B / sg) ** 2 * r - 1 / r)
                    rch = int(math.ceil(sg)) + 1
                    self.msa[i][j] = brute.dense_operator(brute.kernel_table(pb, wb * C, ub, rch), rch, spec.shape, per)
        self.lam = np.full((spec.s,) + spec.shape, spec.lambda_rho)
        self.prev = np.zeros((spec.s,) + spec.shape)

    def mu_ex(self, rho):
        spec = self.spec
        n = self.B.weighted(rho)
        Phi = brute.phi_white_bear if spec.fmt == 1 else brute.phi_rosenfeld
        h = 1e-30
        psi = np.empty_like(n)
        for a in range(10):
            nc = n.astype(complex)
            nc[a] += 1j * h
            psi[a] = Phi(nc).imag / h
        N = int(np.prod(spec.shape))
        P = psi.reshape(10, N)
        out = []
        for i, (M2, M3, Mv) in enumerate(self.B.ops):
            R = spec.R[i]
            c0, c1 = 1 / (4 * np.pi * R * R), 1 / (4 * np.pi * R)
            m = M2.T @ (c0 * P[0] + c1 * P[1] + P[2]) + M3.T @ P[3]
            for c in range(3):
                m += Mv[:, :, c].T @ (c1 * P[4 + c] + P[7 + c])
            if self.msa is not None:
                for j in range(spec.s):
                    if self.msa[i][j] is not None:
                        m = m - self.msa[i][j] @ (rho[j] - spec.rho_b[j]).reshape(-1)
            out.append((m + self.mu_sh[i]).reshape(spec.shape))
        return np.stack(out)

    def poisson(self, phi, rho):
        spec = self.spec
        charge = spec.rho_f + sum(spec.q[i] * rho[i] for i in range(spec.s))
        b = 4 * np.pi * self.lB * charge
        b[0] += spec.phi_lo
        b[-1] += spec.phi_hi
        b = b.reshape(-1)
        if not spec.screened_poisson:
            return np.linalg.solve(self.A, b).reshape(spec.shape)
        shift = 4 * np.pi * self.lB * sum(spec.q[i] ** 2 * rho[i] for i in range(spec.s))
        d = np.linalg.solve(self.A + np.diag(shift.reshape(-1)), b - self.A @ phi.reshape(-1))
        return phi + d.reshape(spec.shape)

    def __call__(self, phi, rho):
        spec = self.spec
        mu = self.mu_ex(rho)
        phi_new = spec.lambda_phi * self.poisson(phi, rho) + (1 - spec.lambda_phi) * phi
        res = np.abs(phi_new - phi).max()
        rho_new = np.empty_like(rho)
        for i in range(spec.s):
            rb = np_dense(spec, i, phi_new, mu[i], self.mu_b[i])
            target = rb * np.exp(-(spec.q[i] * phi_new + mu[i]))
            old = rho[i]
            if spec.rho_mix == 0:
                v = spec.lambda_rho * target + (1 - spec.lambda_rho) * old
            elif spec.rho_mix in (1, 2):
                step = spec.lambda_rho * np.log(target / old)
                if spec.rho_mix == 2:
                    step = np.clip(step, -0.2, 0.2)
                v = old * np.exp(step)
            else:
                d = np.log(target / old)
                flip = d * self.prev[i] < 0
                self.lam[i] = np.where(flip, np.maximum(0.5 * self.lam[i], spec.lambda_rho / 1024),
                                       np.minimum(1.1 * self.lam[i], spec.lambda_rho))
                step = np.clip(self.lam[i] * d, -0.2, 0.2)
                self.prev[i] = step
                v = old * np.exp(step)
            res = max(res, np.abs(v - old).max() / spec.rho_b[i])
            rho_new[i] = v
        return phi_new, rho_new, res


@pytest.mark.parametrize("rho_mix,screened,fmt,sweeps,msa", [
    (0, False, 0, 1, False),      # linear density relaxation, plain Poisson step
    (1, False, 0, 2, False),      # geometric
    (2, True, 0, 2, False),       # step-limited geometric, screened Newton step
    (3, True, 0, 4, False),       # per-point adaptive: factors carried across sweeps
    (1, False, 1, 2, False),      # White Bear functional
    (2, True, 0, 2, True),        # with the MSA electrostatic correlations
])
def test_sweeps_match_dense_composition(rho_mix, screened, fmt, sweeps, msa):
    spec = make_spec(rho_mix, screened, fmt, sweeps, msa)
    phi0, rho0 = start_state(spec)
    r = oracle.gummel(spec, phi0=phi0, rho0=rho0)
    assert r["status"] == 1 and r["iters"] == sweeps
    G = DenseSweep(spec)
    phi, rho = phi0, rho0
    hist = []
    for _ in range(sweeps):
        phi, rho, res = G(phi, rho)
        hist.append(res)
    np.testing.assert_allclose(r["phi"], phi, rtol=0, atol=1e-11 * np.abs(phi).max())
    for i in range(spec.s):
        np.testing.assert_allclose(r["rho"][i], rho[i], rtol=1e-11, atol=0)
    np.testing.assert_allclose(r["hist"], hist, rtol=1e-9)


def test_adaptive_factors_halve_where_the_step_flips():
    """The adaptive mode's factor state matters: on this start the per-point
    factors halve somewhere within four sweeps (a step changed sign), so the
    comparison above exercises both branches of the update."""
    spec = make_spec(3, True, 0, 4)
    phi, rho = start_state(spec)
    G = DenseSweep(spec)
    for _ in range(4):
        phi, rho, _ = G(phi, rho)
    assert (G.lam < spec.lambda_rho * 0.99).any() and (G.lam == spec.lambda_rho).any()


def dense_equilibrium(spec, steps, lam):
    """The equilibrium stage (Sec 3.2, choice of initial guess) by the dense
    parts: from the linear phi profile and the bulk densities, each step takes
    c_i = rho_b,i exp(mu_b,i - mu_ex,i[rho]), one Newton step of the
    Poisson-Boltzmann equation with Boltzmann densities c_i exp(-q_i phi)
    (update clamped to +-1 kT/e), then the step-limited geometric relaxation
    of rho towards c_i exp(-q_i phi).  Returns phi, rho, residual, clamped."""
    G = DenseSweep(spec)
    z = np.arange(1, spec.nz + 1)[:, None, None]
    phi = np.broadcast_to(spec.phi_lo + (spec.phi_hi - spec.phi_lo) * z / (spec.nz + 1), spec.shape).copy()
    rho = np.stack([np.full(spec.shape, spec.rho_b[i]) for i in range(spec.s)])
    res, clamped = 0.0, False
    for _ in range(steps):
        mu = G.mu_ex(rho)
        c = np.stack([spec.rho_b[i] * np.exp(G.mu_b[i] - mu[i]) for i in range(spec.s)])
        r = np.stack([c[i] * np.exp(-spec.q[i] * phi) for i in range(spec.s)])
        b = 4 * np.pi * G.lB * (spec.rho_f + sum(spec.q[i] * r[i] for i in range(spec.s)))
        b[0] += spec.phi_lo
        b[-1] += spec.phi_hi
        shift = 4 * np.pi * G.lB * sum(spec.q[i] ** 2 * r[i] for i in range(spec.s))
        d = np.linalg.solve(G.A + np.diag(shift.reshape(-1)), b.reshape(-1) - G.A @ phi.reshape(-1))
        clamped |= bool((np.abs(d) > 1).any())
        d = np.clip(d, -1.0, 1.0).reshape(spec.shape)
        phi = phi + d
        res = np.abs(d).max()
        for i in range(spec.s):
            step = np.clip(lam * np.log(c[i] * np.exp(-spec.q[i] * phi) / rho[i]), -0.2, 0.2)
            v = rho[i] * np.exp(step)
            res = max(res, np.abs(v - rho[i]).max() / spec.rho_b[i])
            rho[i] = v
    return phi, rho, res, clamped


@pytest.mark.parametrize("bias,steps,clamps", [(0.5, 3, False), (6.0, 2, True)])
def test_equilibrium_steps_match_dense_composition(bias, steps, clamps):
    spec = make_spec(0, False, 0, 1)
    spec.phi_hi = bias
    r = oracle.equilibrium(spec, lam=0.5, tol=0.0, max_iter=steps)
    assert r["status"] == 1 and r["iters"] == steps
    phi, rho, res, clamped = dense_equilibrium(spec, steps, 0.5)
    assert clamped == clamps
    np.testing.assert_allclose(r["phi"], phi, rtol=0, atol=1e-11 * np.abs(phi).max())
    np.testing.assert_allclose(r["rho"], rho, rtol=1e-11, atol=0)
    assert r["residual"] == pytest.approx(res, rel=1e-9)
