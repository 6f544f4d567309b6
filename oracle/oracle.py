"""Python front end of the FP64 CPU oracle (``pnp_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import this module; the product library never does.
It shares no code with the CUDA path.  Every function names the passage of
Meng, Zheng, Lin & Sushko (arXiv:1407.0674) it follows; the C file's header
states the quadrature reading.

A problem is any object with the attributes of ``workloads.ProblemSpec``
(grid, boundary types, radii, valences, bulk densities, square-well data,
fixed charge, temperature, relaxation, quadrature counts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import units

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pnp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC = {"P": 0, "D": 1, "N": 2, 0: 0, 1: 1, 2: 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, IEEE semantics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("s", ctypes.c_int),
        ("R", _dp), ("q", _ip), ("rho_b", _dp), ("D", _dp), ("depth", _dp),
        ("well_inner", ctypes.c_double), ("well_outer", ctypes.c_double),
        ("nsites", ctypes.c_int), ("sites", _dp), ("site_alpha", ctypes.c_double),
        ("rho_f", _dp),
        ("lB", ctypes.c_double),
        ("phi_lo", ctypes.c_double), ("phi_hi", ctypes.c_double),
        ("lambda_phi", ctypes.c_double), ("lambda_rho", ctypes.c_double), ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("nmu", ctypes.c_int), ("ntheta", ctypes.c_int), ("nr", ctypes.c_int),
        ("w_nmu", ctypes.c_int), ("w_ntheta", ctypes.c_int), ("w_nr", ctypes.c_int),
        ("sw_half", ctypes.c_int),
        ("lin_tol", ctypes.c_double),
        ("lin_max_iter", ctypes.c_int),
        ("rho_mix", ctypes.c_int),
        ("screened", ctypes.c_int),
        ("fmt", ctypes.c_int),
        ("msa", ctypes.c_int),
    ]


def _declare(L):
    P = ctypes.POINTER(_Problem)
    L.oracle_nodeset.restype = ctypes.c_int
    L.oracle_nodeset.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int] + [_dp] * 7
    L.oracle_weighted_densities.argtypes = [P, _dp, _dp, _dp, ctypes.c_double, _dp]
    L.oracle_dphi.restype = ctypes.c_long
    L.oracle_dphi.argtypes = [ctypes.c_long, _dp, _dp]
    L.oracle_fhs.restype = ctypes.c_double
    L.oracle_fhs.argtypes = [ctypes.c_long, _dp]
    L.oracle_mu_hs.argtypes = [P, _dp, _dp]
    L.oracle_site_density.argtypes = [P, _dp]
    L.oracle_mu_sh.argtypes = [P, _dp, _dp]
    L.oracle_mu_el.argtypes = [P, _dp, _dp, _dp, ctypes.c_double, _dp]
    L.oracle_excess_mu.restype = ctypes.c_long
    L.oracle_excess_mu.argtypes = [P, _dp, _dp]
    L.oracle_bulk_mu.argtypes = [ctypes.c_int, _dp, _dp, _dp]
    L.oracle_excess_mu_sampled.argtypes = [P, _dp, ctypes.c_int, ctypes.POINTER(ctypes.c_long), _dp]
    L.oracle_poisson.restype = ctypes.c_int
    L.oracle_poisson.argtypes = [P, _dp, _dp, _dp]
    L.oracle_np.restype = ctypes.c_int
    L.oracle_np.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
    L.oracle_np_flux.argtypes = [P, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
    L.oracle_gummel.restype = ctypes.c_int
    L.oracle_gummel.argtypes = [P, _dp, _dp, _dp, _dp, _ip, _dp, ctypes.POINTER(ctypes.c_long)]
    L.oracle_dphi_fmt.restype = ctypes.c_long
    L.oracle_dphi_fmt.argtypes = [ctypes.c_int, ctypes.c_long, _dp, _dp]
    L.oracle_fhs_fmt.restype = ctypes.c_double
    L.oracle_fhs_fmt.argtypes = [ctypes.c_int, ctypes.c_long, _dp]
    L.oracle_bulk_mu_fmt.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    L.oracle_gummel_anderson.restype = ctypes.c_int
    L.oracle_gummel_anderson.argtypes = [P, ctypes.c_int, _dp, _dp, _ip, _dp]
    L.oracle_equilibrium.restype = ctypes.c_int
    L.oracle_equilibrium.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp, _ip,
                                     ctypes.POINTER(ctypes.c_double)]
    L.oracle_num_threads.restype = ctypes.c_int
    L.oracle_set_num_threads.argtypes = [ctypes.c_int]


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Problem:
    """Marshals a problem description into the oracle's C struct and keeps
    the backing arrays alive for the struct's lifetime."""

    def __init__(self, spec, lin_tol: float = 1e-13, lin_max_iter: int = 20000):
        s = len(spec.R)
        self.spec = spec
        self.s = s
        self.shape = (spec.nz, spec.ny, spec.nx)
        self.N = spec.nx * spec.ny * spec.nz
        self._R = _f64(spec.R)
        self._q = np.ascontiguousarray(np.asarray(spec.q, dtype=np.int32))
        self._rho_b = _f64(spec.rho_b)
        self._D = _f64(spec.D if spec.D is not None else np.ones(s))
        self._depth = _f64(spec.depth if spec.depth is not None else np.zeros(s))
        sites = np.zeros((0, 3)) if spec.sites is None else spec.sites
        self._sites = _f64(np.asarray(sites).reshape(-1, 3))
        self._rho_f = None if spec.rho_f is None else _f64(spec.rho_f).reshape(-1)
        st = _Problem()
        st.nx, st.ny, st.nz = spec.nx, spec.ny, spec.nz
        for d in range(3):
            st.bc[d] = BC[spec.bc[d]]
        st.s = s
        st.R = _ptr(self._R)
        st.q = self._q.ctypes.data_as(_ip)
        st.rho_b = _ptr(self._rho_b)
        st.D = _ptr(self._D)
        st.depth = _ptr(self._depth)
        st.well_inner, st.well_outer = spec.well_inner, spec.well_outer
        st.nsites = self._sites.shape[0]
        st.sites = _ptr(self._sites) if st.nsites else None
        st.site_alpha = spec.site_alpha
        st.rho_f = _ptr(self._rho_f)
        st.lB = units.bjerrum_length_h(spec.temperature_K, spec.eps_r, spec.h_nm)
        st.phi_lo, st.phi_hi = spec.phi_lo, spec.phi_hi
        st.lambda_phi, st.lambda_rho, st.tol = spec.lambda_phi, spec.lambda_rho, spec.tol
        st.max_iter = spec.max_iter
        st.nmu, st.ntheta, st.nr = spec.quad_nmu, spec.quad_ntheta, spec.quad_nr
        st.w_nmu, st.w_ntheta, st.w_nr = spec.well_nmu, spec.well_ntheta, spec.well_nr
        st.sw_half = 1 if spec.sw_half else 0
        st.lin_tol = lin_tol
        st.lin_max_iter = lin_max_iter
        st.rho_mix = int(getattr(spec, "rho_mix", 0))
        st.screened = 1 if getattr(spec, "screened_poisson", False) else 0
        st.fmt = int(getattr(spec, "fmt", 0))
        st.msa = 1 if getattr(spec, "msa", False) else 0
        self.st = st

    @property
    def ref(self):
        return ctypes.byref(self.st)

    @property
    def lB(self):
        return self.st.lB


def nodeset(kind: int, r_in: float, r_out: float, nmu: int = 0, ntheta: int = 0, nr: int = 0):
    """Quadrature nodes of Sec 3.5: kind 0 shell |r| = r_out, 1 ball, 2 thick
    shell [r_in, r_out].  Returns (p[n,3], w[n], u[n,3])."""
    L = lib()
    n = L.oracle_nodeset(kind, r_in, r_out, nmu, ntheta, nr, *([None] * 7))
    a = [np.zeros(n) for _ in range(7)]
    L.oracle_nodeset(kind, r_in, r_out, nmu, ntheta, nr, *[_ptr(x) for x in a])
    return np.stack(a[0:3], 1), a[3], np.stack(a[4:7], 1)


def weighted_densities(spec, rho=None, wave=None):
    """n_alpha of Sec 2.3.1 by direct quadrature sums.  Returns [10, nz, ny, nx]
    in the order n0, n1, n2, n3, n1x, n1y, n1z, n2x, n2y, n2z.  ``wave`` =
    (k[3], phase, amp[s]) evaluates rho_i = amp_i cos(k.r + phase) exactly at
    the nodes instead of interpolating a grid field."""
    P = Problem(spec)
    out = np.zeros((10,) + P.shape)
    if wave is None:
        r = _f64(rho).reshape(P.s, -1)
        lib().oracle_weighted_densities(P.ref, _ptr(r), _ptr(out), None, 0.0, None)
    else:
        k, ph, amp = wave
        k = _f64(k)
        amp = _f64(amp)
        lib().oracle_weighted_densities(P.ref, None, _ptr(out), _ptr(k), float(ph), _ptr(amp))
    return out


def dphi(n, fmt=0):
    """The ten FMT derivatives of Sec 2.3.1 (fmt 0 Rosenfeld, 1 White Bear).
    Returns (psi, bad)."""
    n = _f64(n)
    N = n.size // 10
    psi = np.zeros_like(n)
    bad = lib().oracle_dphi_fmt(int(fmt), N, _ptr(n), _ptr(psi))
    return psi, int(bad)


def fhs(n, fmt=0):
    """sum over the grid of Phi (h = 1), Sec 2.3.1 (fmt 0 Rosenfeld, 1 White Bear)."""
    n = _f64(n)
    return lib().oracle_fhs_fmt(int(fmt), n.size // 10, _ptr(n))


def mu_hs(spec, psi):
    """Back-convolution of Sec 2.3.1.  Returns [s, nz, ny, nx]."""
    P = Problem(spec)
    psi = _f64(psi)
    out = np.zeros((P.s,) + P.shape)
    lib().oracle_mu_hs(P.ref, _ptr(psi), _ptr(out))
    return out


def site_density(spec):
    """rho_s of Sec 2.3.2 at the grid nodes."""
    P = Problem(spec)
    out = np.zeros(P.shape)
    lib().oracle_site_density(P.ref, _ptr(out))
    return out


def mu_sh(spec, rho_s):
    """Square-well mean-field potential of Sec 2.3.2.  Returns [s, nz, ny, nx]."""
    P = Problem(spec)
    rs = _f64(rho_s)
    out = np.zeros((P.s,) + P.shape)
    lib().oracle_mu_sh(P.ref, _ptr(rs), _ptr(out))
    return out


def mu_el(spec, rho=None, wave=None):
    """Electrostatic-correlation chemical potential of Sec 2.3.4 (MSA), the
    integral term: -sum_j int C_ij(|r - r'|) (rho_j(r') - rho_b,j) dr' over
    Omega.  Returns [s, nz, ny, nx].  ``wave`` = (k[3], phase, amp[s]) replaces
    rho_j - rho_b,j by amp_j cos(k.r + phase) evaluated at the nodes."""
    P = Problem(spec)
    out = np.zeros((P.s,) + P.shape)
    if wave is None:
        r = _f64(rho).reshape(P.s, -1)
        lib().oracle_mu_el(P.ref, _ptr(r), _ptr(out), None, 0.0, None)
    else:
        k, ph, amp = wave
        lib().oracle_mu_el(P.ref, None, _ptr(out), _ptr(_f64(k)), float(ph), _ptr(_f64(amp)))
    return out


def square_well_energy(spec, rho):
    """Square-well free energy F_sh of Sec 2.3.2 (kT), the mobile-site part:
    the printed double sum over pairs (alpha, beta) with the factor 1/2 counts
    the pair (i, s) and (s, i), so with the site density held fixed
    F_sh = sum_i int rho_i(r) int rho_s(r') Phi_is(|r - r'|) dr' dr
    (h^3 = 1).  Site-site pairs are a constant and mobile-mobile wells are
    absent (Sec 2.3.2), so neither is included.  The inner integral is the
    oracle's square-well sum without the 1/2 of mu_sh."""
    import dataclasses
    full = dataclasses.replace(spec, sw_half=False)
    w = mu_sh(full, site_density(full))
    r = _f64(rho).reshape(w.shape)
    return float(sum((r[i] * w[i]).sum() for i in range(w.shape[0])))


def excess_mu(spec, rho):
    """mu_ex = mu_hs + mu_sh (Sec 2.3).  Returns (mu[s, nz, ny, nx], bad)."""
    P = Problem(spec)
    r = _f64(rho)
    out = np.zeros((P.s,) + P.shape)
    bad = lib().oracle_excess_mu(P.ref, _ptr(r), _ptr(out))
    return out, int(bad)


def excess_mu_sampled(spec, rho, flat_idx):
    """mu_ex at the given flat grid indices only (same sums as excess_mu).
    Returns [s, nsamp]."""
    if getattr(spec, "msa", False):
        raise NotImplementedError("excess_mu_sampled evaluates mu_hs + mu_sh only")
    P = Problem(spec)
    r = _f64(rho)
    idx = np.ascontiguousarray(np.asarray(flat_idx, dtype=np.int64))
    out = np.zeros((P.s, len(idx)))
    lib().oracle_excess_mu_sampled(P.ref, _ptr(r), len(idx), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                   _ptr(out))
    return out


def bulk_mu(R, rho_b, fmt=0):
    """Reservoir mu_ex: dPhi/dn at bulk n times the weight integrals."""
    R = _f64(R)
    rb = _f64(rho_b)
    out = np.zeros(len(R))
    lib().oracle_bulk_mu_fmt(int(fmt), len(R), _ptr(R), _ptr(rb), _ptr(out))
    return out


def poisson(spec, rho, phi0=None, lin_tol=1e-13):
    """Discrete Poisson solve of Sec 2.1/3.1 (reduced units)."""
    P = Problem(spec, lin_tol=lin_tol)
    r = _f64(rho)
    phi = np.zeros(P.shape) if phi0 is None else _f64(phi0).copy()
    rel = ctypes.c_double()
    it = lib().oracle_poisson(P.ref, _ptr(r), _ptr(phi), ctypes.byref(rel))
    return phi, it, rel.value


def np_solve(spec, i, phi, mu, mu_b, rhobar0=None, lin_tol=1e-13):
    """Slotboom Nernst-Planck solve for species i (Sec 2.1, 3.1)."""
    P = Problem(spec, lin_tol=lin_tol)
    phi = _f64(phi)
    mu = _f64(mu)
    rb = np.ones(P.shape) * spec.rho_b[i] if rhobar0 is None else _f64(rhobar0).copy()
    rel = ctypes.c_double()
    it = lib().oracle_np(P.ref, i, _ptr(phi), _ptr(mu), float(mu_b), _ptr(rb), ctypes.byref(rel))
    return rb, it, rel.value


def np_flux(spec, i, phi, mu, mu_b, rhobar):
    """Discrete z-flux through every z face plane (nz+1 values)."""
    P = Problem(spec)
    out = np.zeros(spec.nz + 1)
    lib().oracle_np_flux(P.ref, i, _ptr(_f64(phi)), _ptr(_f64(mu)), float(mu_b), _ptr(_f64(rhobar)),
                         _ptr(out))
    return out


def conductivity(spec, flux, D_m2_per_s=0.0):
    """Ionic conductivity (Sec 4.2.1, size dependency of the conductivity): the
    current density along the transport axis averaged over its length, over
    the applied field.  flux [s][nz+1] are the species' currents through the
    z faces (np_flux: reduced units, h = 1, each summed over the nx*ny faces of
    a plane).  The charge current density is sum_i q_i flux_i / (nx ny); its
    mean over the nz+1 faces stands for (1/L) int J dz; the field is the applied
    one, E = -(phi_hi - phi_lo) / (nz+1) in kT/e per h.  Returns (sigma in units
    of e^2 D / (kT h^3), sigma in S/cm for the diffusion scale D_m2_per_s and the
    spec's T and h; 0 when D_m2_per_s is 0)."""
    flux = np.asarray(flux, dtype=np.float64).reshape(spec.s, spec.nz + 1)
    current = sum(spec.q[i] * flux[i] for i in range(spec.s)) / (spec.nx * spec.ny)
    field = -(spec.phi_hi - spec.phi_lo) / (spec.nz + 1)
    sigma = current.mean() / field
    # e^2 D / (kT h^3) = e [C] * beta [1/V] * D [m^2/s] / h^3 [m^3]  (S/m), /100 for S/cm
    h_m = spec.h_nm * 1e-9
    si = sigma * units.E_CHARGE_C * units.beta_per_ev(spec.temperature_K) * D_m2_per_s / h_m ** 3 / 100.0
    return float(sigma), float(si)


def gummel(spec, phi0=None, rho0=None, lin_tol=1e-13):
    """Relaxed Gummel iteration of Sec 3.2.  Returns a dict with phi, rho,
    status (0 converged, 1 not converged, 2 packing), iters, hist."""
    P = Problem(spec, lin_tol=lin_tol)
    phi = np.zeros(P.shape)
    rho = np.zeros((P.s,) + P.shape)
    it = ctypes.c_int()
    lin = ctypes.c_long()
    hist = np.zeros(max(spec.max_iter, 1))
    st = lib().oracle_gummel(P.ref, _ptr(None if phi0 is None else _f64(phi0)),
                             _ptr(None if rho0 is None else _f64(rho0)), _ptr(phi), _ptr(rho),
                             ctypes.byref(it), _ptr(hist), ctypes.byref(lin))
    return {"phi": phi, "rho": rho, "status": st, "iters": it.value, "hist": hist[:it.value],
            "lin_iters": lin.value, "lB": P.lB}


def equilibrium(spec, lam=None, tol=1e-10, max_iter=1000, lin_tol=1e-13):
    """Equilibrium cDFT initial guess (Sec 3.2): Boltzmann densities about
    the reservoirs with the Poisson-Boltzmann potential.  lam defaults to the
    problem's lambda_rho.  Returns a dict with phi, rho, status (0 converged,
    1 not converged, 2 packing/overflow), iters, residual."""
    P = Problem(spec, lin_tol=lin_tol)
    phi = np.zeros(P.shape)
    rho = np.zeros((P.s,) + P.shape)
    it = ctypes.c_int()
    res = ctypes.c_double()
    lam = spec.lambda_rho if lam is None else lam
    st = lib().oracle_equilibrium(P.ref, ctypes.c_double(lam), ctypes.c_double(tol), ctypes.c_int(max_iter),
                                  _ptr(phi), _ptr(rho), ctypes.byref(it), ctypes.byref(res))
    return {"phi": phi, "rho": rho, "status": st, "iters": it.value, "residual": res.value, "lB": P.lB}


def gummel_anderson(spec, m=3, lin_tol=1e-13):
    """The relaxed Gummel iteration accelerated by Anderson mixing of depth m
    on (phi, ln rho).  Returns a dict with phi, rho, status, iters, hist."""
    P = Problem(spec, lin_tol=lin_tol)
    phi = np.zeros(P.shape)
    rho = np.zeros((P.s,) + P.shape)
    it = ctypes.c_int()
    hist = np.zeros(max(spec.max_iter, 1))
    st = lib().oracle_gummel_anderson(P.ref, int(m), _ptr(phi), _ptr(rho), ctypes.byref(it), _ptr(hist))
    return {"phi": phi, "rho": rho, "status": st, "iters": it.value, "hist": hist[:it.value]}


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (n <= 0: one per processor)."""
    lib().oracle_set_num_threads(int(n))


def num_threads() -> int:
    return lib().oracle_num_threads()
