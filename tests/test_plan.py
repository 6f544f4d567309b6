"""The library's host-side planning, tested without a GPU through
pnp_plan_problem: the reservoir chemical potentials it feeds to the
Nernst-Planck boundary data (against the oracle, both functionals), the
padded-length rule (Sec 3.4: L >= n + S on zero-extended axes, L = n on
periodic ones; the smallest 2^a 3^b 5^c length, even on x, or a register-FFT
length within 30 % above it) and descriptor rejection."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle
from workloads import ProblemSpec, bulk_density, film_gummel, mu_microbench

REG = (16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 256)


@pytest.fixture(scope="module")
def pnp():
    from paper_1407_0674_gb300 import build, pnp as mod
    import os
    if not os.path.exists(mod.LIB_PATH):
        build.build()
    return mod


def smooth235(n):
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def expected_length(n, need, periodic, even):
    if periodic:
        return n
    m = n + need
    L = m
    while not (smooth235(L) and (not even or L % 2 == 0)):
        L += 1
    for f in REG:
        if f >= L and f <= L + (3 * L) // 10:
            return f
    return L


@pytest.mark.parametrize("fmt", [0, 1])
@pytest.mark.parametrize("R,eta", [((2.0,), (0.3,)), ((1.5, 2.0, 3.0), (0.1, 0.1, 0.1)), ((1.0, 2.5), (0.05, 0.3))])
def test_reservoir_mu_matches_oracle(pnp, fmt, R, eta):
    rb = tuple(bulk_density(e, r) for e, r in zip(eta, R))
    spec = ProblemSpec(nx=8, ny=8, nz=8, bc=("P", "P", "D"), R=R, q=(0,) * len(R), rho_b=rb, fmt=fmt)
    _, mu = pnp.plan(spec)
    np.testing.assert_allclose(mu, oracle.bulk_mu(R, rb, fmt=fmt), rtol=1e-13)


@pytest.mark.parametrize("shape,bc", [((128, 128, 128), ("N", "N", "D")), ((20, 10, 12), ("N", "N", "D")),
                                      ((32, 32, 32), ("P", "P", "D")), ((86, 20, 5), ("N", "N", "D")),
                                      ((96, 96, 96), ("P", "P", "D")), ((13, 11, 9), ("N", "N", "D"))])
def test_padded_lengths_follow_the_rule(pnp, shape, bc):
    spec, _ = mu_microbench(shape=(8, 8, 8))
    spec = dataclasses.replace(spec, nx=shape[0], ny=shape[1], nz=shape[2], bc=bc)
    info, _ = pnp.plan(spec)
    need = int(np.ceil(max(spec.R))) + 1
    for c in range(3):
        assert info["fft_len"][c] == expected_length(shape[c], need, bc[c] == "P", c == 0), (c, info)
    assert info["stencil_halfwidth"] == need and info["device_bytes"] > 0


def test_wells_widen_the_padding(pnp):
    spec = film_gummel(32, 32, 32)
    info, _ = pnp.plan(spec)
    assert info["well_halfwidth"] == int(np.ceil(spec.well_outer)) + 1
    need = max(info["stencil_halfwidth"], info["well_halfwidth"])
    assert info["fft_len"] == (32, 32, expected_length(32, need, False, False))


def test_rejected_descriptors(pnp):
    spec, _ = mu_microbench(shape=(12, 10, 10))
    bad = [
        dataclasses.replace(spec, bc=("P", "N", "D"), nx=13),        # periodic x must be even
        dataclasses.replace(spec, fft_len=(14, 0, 0)),              # shorter than n + S
        dataclasses.replace(spec, fft_len=(34, 0, 0)),              # 34 = 2 x 17 is not 2^a 3^b 5^c
        dataclasses.replace(spec, fmt=2),
        dataclasses.replace(spec, rho_mix=5),
        dataclasses.replace(spec, eq_tol=-1.0),
        dataclasses.replace(spec, rho_b=(0.2, 0.2, 0.2)),            # bulk packing above 1
    ]
    for s in bad:
        with pytest.raises(pnp.PnpError) as e:
            pnp.plan(s)
        assert e.value.code == pnp.ERR_INVALID


def test_bjerrum_length_reproduces_table1(pnp):
    """The library's unit conversion (SI constants) against the values the
    paper prints in Table 1: l_B = 4.514 nm at 223 K with eps_r = 16.6."""
    import os
    g = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_units.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                g[k] = float(v)
    spec, _ = mu_microbench(shape=(8, 8, 8))
    spec = dataclasses.replace(spec, temperature_K=g["temperature_K"], eps_r=g["eps_r"], h_nm=1.0)
    info, _ = pnp.plan(spec)
    assert info["bjerrum_h"] == pytest.approx(g["bjerrum_length_nm"], rel=1e-4)
    # in grid units h = 0.5 nm the same length is twice as many h
    info2, _ = pnp.plan(dataclasses.replace(spec, h_nm=0.5))
    assert info2["bjerrum_h"] == pytest.approx(2 * info["bjerrum_h"], rel=1e-14)


@pytest.mark.parametrize("R", [1.0, 1.5, 2.0, 3.0, 2.37])
def test_weight_stencils_match_independent_tables(pnp, R):
    """The library's set-up stencils (row a1: quadrature of Sec 3.5, trilinear
    deposit) against the brute-force module's tables, built independently from
    numpy's Gauss-Legendre nodes and hat functions."""
    import brute
    S = int(np.ceil(R)) + 1
    ps, ws, us = brute.nodes("shell", R)
    pb, wb, ub = brute.nodes("ball", R)
    shell = brute.kernel_table(ps, ws, us, S)
    ball = brute.kernel_table(pb, wb, ub, S)
    vec = brute.kernel_table(ps, ws, us, S, vector=True)
    np.testing.assert_allclose(pnp.weight_stencil(0, R), shell, rtol=0, atol=1e-13 * shell.max())
    np.testing.assert_allclose(pnp.weight_stencil(1, R), ball, rtol=0, atol=1e-13 * ball.max())
    for c in range(3):
        np.testing.assert_allclose(pnp.weight_stencil(2 + c, R), vec[..., c], rtol=0, atol=1e-13 * shell.max())
    # exact moments of the quadrature: surface 4 pi R^2, volume 4/3 pi R^3
    assert pnp.weight_stencil(0, R).sum() == pytest.approx(4 * np.pi * R * R, rel=1e-13)
    assert pnp.weight_stencil(1, R).sum() == pytest.approx(4 / 3 * np.pi * R ** 3, rel=1e-13)


def test_well_stencil_matches_independent_table(pnp):
    import brute
    r_in, r_out = 4.0, 5.0
    S = int(np.ceil(r_out)) + 1
    p, w, u = brute.nodes("thick", r_out, r_in)
    ref = brute.kernel_table(p, w, u, S)
    got = pnp.weight_stencil(5, r_out, r_in=r_in)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * ref.max())
    assert got.sum() == pytest.approx(4 / 3 * np.pi * (r_out ** 3 - r_in ** 3), rel=1e-13)


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5])
def test_weight_spectra_match_numpy_fft(pnp, kind):
    """The set-up spectra (a separable real transform over the stored octant)
    against numpy's FFT of the stencil embedded periodically in the grid: the
    DFT is the octant (even kernels) or -i times it (vector components)."""
    R, r_in = (5.0, 4.0) if kind == 5 else (2.0, 0.0)
    S = int(np.ceil(R)) + 1
    L = (16, 14, 18)
    K = pnp.weight_stencil(kind, R, r_in=r_in, S=S)
    grid = np.zeros((L[2], L[1], L[0]))
    m = np.arange(-S, S + 1)
    zz, yy, xx = np.meshgrid(m % L[2], m % L[1], m % L[0], indexing="ij")
    np.add.at(grid, (zz, yy, xx), K)
    F = np.fft.fftn(grid)[: L[2] // 2 + 1, : L[1] // 2 + 1, : L[0] // 2 + 1]
    oct_ = pnp.weight_spectrum(kind, R, L, r_in=r_in, S=S)
    scale = np.abs(F).max()
    if kind in (2, 3, 4):
        np.testing.assert_allclose(F.imag, -oct_, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(F.real, 0.0, rtol=0, atol=1e-12 * scale)
    else:
        np.testing.assert_allclose(F.real, oct_, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(F.imag, 0.0, rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("bias,T,h", [(0.5, 300.0, 1.0), (-1.3, 223.0, 0.5), (1e-3, 400.0, 0.25)])
def test_conductivity_matches_oracle(pnp, bias, T, h):
    """pnp_conductivity (host-only arithmetic on plane currents) against the
    oracle's conductivity, on arbitrary currents: reduced and S/cm."""
    spec = film_gummel(6, 5, 9)
    spec.phi_hi, spec.temperature_K, spec.h_nm = bias, T, h
    rng = np.random.default_rng(3)
    flux = rng.normal(0.0, 1.0, (spec.s, spec.nz + 1))
    got = pnp.conductivity(spec, flux, D_m2_per_s=1e-10)
    ref = oracle.conductivity(spec, flux, D_m2_per_s=1e-10)
    assert got[0] == pytest.approx(ref[0], rel=1e-13)
    # the oracle's k_B in eV/K carries 10 digits (1.7e-11 from k_B/e)
    assert got[1] == pytest.approx(ref[1], rel=1e-10)


def test_conductivity_rejections(pnp):
    spec = film_gummel(6, 5, 9)
    flux = np.ones((spec.s, spec.nz + 1))
    for s, f, D in [(dataclasses.replace(spec, phi_hi=spec.phi_lo), flux, 0.0),    # no applied field
                    (spec, np.where(np.arange(flux.size).reshape(flux.shape) == 4, np.nan, flux), 0.0),
                    (spec, flux, -1.0)]:
        with pytest.raises(pnp.PnpError) as e:
            pnp.conductivity(s, f, D)
        assert e.value.code == pnp.ERR_INVALID


def _msa_spec():
    return ProblemSpec(nx=8, ny=6, nz=5, bc=("P", "P", "P"), R=(1.0, 1.5, 0.7), q=(1, -1, 2),
                       rho_b=(0.004, 0.006, 0.001))


@pytest.mark.parametrize("i,j", [(0, 0), (0, 1), (1, 2), (2, 2)])
def test_msa_stencil_matches_independent_table(pnp, i, j):
    """pnp_msa_stencil (row a1's set-up for the MSA term) against the brute
    module's table from numpy's ball nodes, and its sum against the exact
    ball integral of C_ij."""
    import math
    import brute
    spec = _msa_spec()
    lB = pnp.plan(spec)[0]["bjerrum_h"]          # the library's l_B (pinned to Table 1 above)
    kap = math.sqrt(4 * math.pi * lB * sum(r * q * q for r, q in zip(spec.rho_b, spec.q)))
    s = spec.R[i] + spec.R[j]
    gs = 0.5 * (math.sqrt(1 + 2 * kap * s) - 1)
    B = gs / (1 + gs)
    qq = spec.q[i] * spec.q[j]
    p, w, u = brute.nodes("ball", s)
    r = np.linalg.norm(p, axis=1)
    C = -qq * lB * (2 * B / s - (B / s) ** 2 * r - 1 / r)
    S = int(np.ceil(s)) + 1
    ref = brute.kernel_table(p, w * C, u, S)
    got = pnp.msa_stencil(spec, i, j)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    exact = -4 * math.pi * qq * lB * s * s * (2 * B / 3 - B * B / 4 - 0.5)
    assert got.sum() == pytest.approx(exact, rel=1e-12)


def test_msa_stencil_convolution_equals_oracle(pnp):
    """The library's stencils, applied as periodic correlations to rho - rho_b,
    give the oracle's mu_el: both sides compute the same discrete operator."""
    spec = _msa_spec()
    rng = np.random.default_rng(6)
    rho = np.stack([rb * rng.lognormal(0, 0.3, spec.shape) for rb in spec.rho_b])
    ref = oracle.mu_el(spec, rho)
    for i in range(spec.s):
        got = np.zeros(spec.shape)
        for j in range(spec.s):
            K = pnp.msa_stencil(spec, i, j)
            S = (K.shape[0] - 1) // 2
            d = rho[j] - spec.rho_b[j]
            for mz in range(-S, S + 1):
                for my in range(-S, S + 1):
                    for mx in range(-S, S + 1):
                        k = K[mz + S, my + S, mx + S]
                        if k != 0.0:
                            got -= k * np.roll(d, (-mz, -my, -mx), axis=(0, 1, 2))
        # the oracle's l_B comes from a 10-digit k_B in eV/K: 1.7e-11 from the SI value
        np.testing.assert_allclose(got, ref[i], rtol=0, atol=1e-10 * np.abs(ref[i]).max())


def test_msa_plan_covers_the_pair_reach(pnp):
    """With the MSA term the padded lengths of the zero-extended axes cover the
    pair kernels' reach ceil(R_i + R_j) + 1 (> the FMT reach), so the circular
    convolution never wraps into the domain; periodic axes keep their length."""
    base = dataclasses.replace(_msa_spec(), nx=9, ny=8, nz=7, bc=("N", "P", "D"))
    plain, _ = pnp.plan(base)
    msa, _ = pnp.plan(dataclasses.replace(base, msa=True))
    reach = int(np.ceil(2 * max(base.R))) + 1
    assert msa["fft_len"][0] >= base.nx + reach and msa["fft_len"][2] >= base.nz + reach
    assert msa["fft_len"][1] == base.ny
    assert plain["fft_len"][0] < base.nx + reach          # the FMT reach alone is shorter
    assert msa["device_bytes"] > plain["device_bytes"]


def test_msa_spectral_plan_on_zero_extended_axes(pnp):
    """A numpy prototype of the planned device MSA term: zero-padded FFT
    products of the library's stencils with rho_j, minus nothing for the bulk,
    plus the fixed bulk field sum_j rho_b,j (C_ij conv 1_Omega), equals the
    oracle's mu_el on a grid zero-extended on every axis."""
    spec = dataclasses.replace(_msa_spec(), nx=9, ny=7, nz=6, bc=("N", "N", "D"))
    rng = np.random.default_rng(11)
    rho = np.stack([rb * rng.lognormal(0, 0.3, spec.shape) for rb in spec.rho_b])
    ref = oracle.mu_el(spec, rho)
    n = np.array(spec.shape)
    Smax = max(int(np.ceil(spec.R[i] + spec.R[j])) + 1 for i in range(spec.s) for j in range(spec.s))
    L = tuple(int(v) for v in n + Smax)

    def embed(K):
        S = (K.shape[0] - 1) // 2
        g = np.zeros(L)
        m = np.arange(-S, S + 1)
        zz, yy, xx = np.meshgrid(m % L[0], m % L[1], m % L[2], indexing="ij")
        np.add.at(g, (zz, yy, xx), K)
        return np.fft.rfftn(g)

    def pad(f):
        g = np.zeros(L)
        g[:n[0], :n[1], :n[2]] = f
        return np.fft.rfftn(g)

    one = pad(np.ones(spec.shape))
    for i in range(spec.s):
        acc = np.zeros(L[:2] + (L[2] // 2 + 1,), dtype=complex)
        bulk = np.zeros_like(acc)
        for j in range(spec.s):
            Ck = embed(pnp.msa_stencil(spec, i, j))
            acc += Ck * pad(rho[j])
            bulk += spec.rho_b[j] * Ck * one
        got = np.fft.irfftn(-acc + bulk, s=L, axes=(0, 1, 2))[:n[0], :n[1], :n[2]]
        np.testing.assert_allclose(got, ref[i], rtol=0, atol=1e-10 * np.abs(ref[i]).max())
