"""Thin ctypes binding of libpnp_gb300 (include/pnp.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The library must have been built (``paper_1407_0674_gb300.build``);
a missing library raises instead of falling back to anything else.

A problem description is any object with the attributes of
``workloads.ProblemSpec``.  Host calls take and return numpy arrays; the
``*_device`` calls take objects exposing ``data_ptr()`` (e.g. CUDA tensors)
and an optional stream handle (int).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpnp_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "pnp.h")

OK = 0
PENDING = 1
ERR_INVALID = -1
ERR_NOMEM = -2
ERR_CUDA = -3
ERR_NOT_CONVERGED = -4
ERR_PACKING = -5
ERR_OVERFLOW = -6
ERR_BUSY = -7
ERR_TIMEOUT = -8
ERR_UNKNOWN_TICKET = -9
ERR_TOO_LARGE = -10

BC = {"P": 0, "D": 1, "N": 2, 0: 0, 1: 1, 2: 2}
FLAG_AUTOTUNE = 1
FLAG_EQUILIBRIUM_INIT = 2
FLAG_SCREENED_POISSON = 4
FLAG_MSA = 8
FLAG_PHASE_TIMING = 16
PHASES = ("mu_ex", "poisson", "nernst_planck", "update")
SERVE = {"fifo": 0, "smallest_first": 1}
PREC = {"fp64": 0, "fp32": 1, "df64": 2, "tf32split": 3, None: -1, -1: -1, 0: 0, 1: 1, 2: 2, 3: 3}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class Desc(ctypes.Structure):
    """Mirror of pnp_problem_desc."""
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("nspecies", ctypes.c_int),
        ("valence", _ip), ("radius", _dp), ("rho_bulk", _dp), ("diffusivity", _dp), ("well_depth", _dp),
        ("well_inner", ctypes.c_double), ("well_outer", ctypes.c_double),
        ("nsites", ctypes.c_int), ("site_xyz", _dp), ("site_alpha", ctypes.c_double),
        ("rho_fixed", _dp),
        ("temperature_K", ctypes.c_double), ("eps_r", ctypes.c_double), ("h_nm", ctypes.c_double),
        ("phi_lo", ctypes.c_double), ("phi_hi", ctypes.c_double),
        ("lambda_phi", ctypes.c_double), ("lambda_rho", ctypes.c_double),
        ("rho_mix", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("quad_nmu", ctypes.c_int), ("quad_ntheta", ctypes.c_int), ("quad_nr", ctypes.c_int),
        ("well_nmu", ctypes.c_int), ("well_ntheta", ctypes.c_int), ("well_nr", ctypes.c_int),
        ("sw_half", ctypes.c_int),
        ("fft_len", ctypes.c_int * 3),
        ("precision", ctypes.c_int),
        ("lin_tol", ctypes.c_double),
        ("flags", ctypes.c_uint),
        ("eq_tol", ctypes.c_double),
        ("eq_max_iter", ctypes.c_int),
        ("fmt", ctypes.c_int),
        ("anderson_depth", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("residual", ctypes.c_double),
                ("linear_iterations", ctypes.c_longlong), ("seconds", ctypes.c_double),
                ("init_iterations", ctypes.c_int), ("init_residual", ctypes.c_double),
                ("repeated_sweeps", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("fft_len", ctypes.c_int * 3), ("stencil_halfwidth", ctypes.c_int),
                ("well_halfwidth", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("mg_levels", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("tuned_ms", ctypes.c_double), ("bjerrum_h", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("policy", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("active", ctypes.c_int), ("queued", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t)]


class PnpError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} ({code})")


_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpnp_gb300.so not built ({LIB_PATH}); run paper_1407_0674_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.pnp_desc_init.argtypes = [ctypes.POINTER(Desc)]
        L.pnp_create_problem.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(vp)]
        L.pnp_destroy_problem.argtypes = [vp]
        L.pnp_destroy_problem.restype = None
        L.pnp_get_problem_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.pnp_excess_mu.argtypes = [vp, _dp, _dp, ctypes.c_int]
        L.pnp_excess_mu_device.argtypes = [vp, vp, vp, ctypes.c_int, vp]
        L.pnp_status.argtypes = [vp]
        L.pnp_gummel_solve.argtypes = [vp, _dp, _dp, _dp, _dp, ctypes.POINTER(Stats)]
        L.pnp_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
        L.pnp_server_destroy.argtypes = [vp]
        L.pnp_server_destroy.restype = None
        L.pnp_submit.argtypes = [vp, ctypes.POINTER(Desc), _dp, _dp, ctypes.POINTER(ctypes.c_uint64)]
        L.pnp_poll.argtypes = [vp, ctypes.c_uint64, _dp, _dp, ctypes.POINTER(Stats)]
        L.pnp_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.pnp_excess_mu_noalloc.argtypes = [ctypes.POINTER(Desc), vp, vp, vp]
        L.pnp_selftest_bounded_wait.argtypes = [ctypes.c_double]
        L.pnp_test_fail_alloc_at.argtypes = [ctypes.c_long]
        L.pnp_gummel_phase_times.argtypes = [vp, _dp, ctypes.c_int]
        L.pnp_plane_flux.argtypes = [vp, ctypes.c_int, _dp, _dp, _dp]
        L.pnp_plan_problem.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(Info), _dp]
        L.pnp_conductivity.argtypes = [ctypes.POINTER(Desc), _dp, ctypes.c_double, _dp]
        L.pnp_square_well_energy.argtypes = [vp, _dp, _dp]
        L.pnp_msa_stencil.argtypes = [ctypes.POINTER(Desc), ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.pnp_weight_stencil.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _dp]
        L.pnp_weight_spectrum.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.pnp_stage_timing.argtypes = [vp, ctypes.c_int]
        L.pnp_stage_times.argtypes = [vp, _dp, _ip, ctypes.c_int]
        L.pnp_stage_name.argtypes = [ctypes.c_int]
        L.pnp_stage_name.restype = ctypes.c_char_p
        L.pnp_error_string.argtypes = [ctypes.c_int]
        L.pnp_error_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/pnp.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pnp_[a-z_]+)\s*\(", txt)))


def error_string(code: int) -> str:
    return lib().pnp_error_string(int(code)).decode()


def _check(rc, where):
    if rc != OK:
        raise PnpError(rc, where)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


class DescHolder:
    """pnp_problem_desc filled from a problem description, with the arrays it
    points to kept alive."""

    def __init__(self, spec, precision="fp64"):
        d = Desc()
        lib().pnp_desc_init(ctypes.byref(d))
        s = len(spec.R)
        d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
        for c in range(3):
            d.bc[c] = BC.get(spec.bc[c], spec.bc[c]) if isinstance(spec.bc[c], int) else BC[spec.bc[c]]
        d.nspecies = s
        self._q = np.ascontiguousarray(np.asarray(spec.q, dtype=np.int32))
        self._R = _f64(spec.R)
        self._rb = _f64(spec.rho_b)
        self._D = None if spec.D is None else _f64(spec.D)
        self._dep = None if spec.depth is None else _f64(spec.depth)
        sites = None if spec.sites is None else _f64(np.asarray(spec.sites).reshape(-1, 3))
        self._sites = sites
        self._rf = None if spec.rho_f is None else _f64(spec.rho_f).reshape(-1)
        d.valence = self._q.ctypes.data_as(_ip)
        d.radius = _ptr(self._R)
        d.rho_bulk = _ptr(self._rb)
        d.diffusivity = _ptr(self._D)
        d.well_depth = _ptr(self._dep)
        d.well_inner, d.well_outer = spec.well_inner, spec.well_outer
        d.nsites = 0 if sites is None else sites.shape[0]
        d.site_xyz = _ptr(sites) if d.nsites else None
        d.site_alpha = spec.site_alpha
        d.rho_fixed = _ptr(self._rf)
        d.temperature_K, d.eps_r, d.h_nm = spec.temperature_K, spec.eps_r, spec.h_nm
        d.phi_lo, d.phi_hi = spec.phi_lo, spec.phi_hi
        d.lambda_phi, d.lambda_rho = spec.lambda_phi, spec.lambda_rho
        d.rho_mix = int(getattr(spec, "rho_mix", 0))
        d.tol, d.max_iter = spec.tol, spec.max_iter
        d.quad_nmu, d.quad_ntheta, d.quad_nr = spec.quad_nmu, spec.quad_ntheta, spec.quad_nr
        d.well_nmu, d.well_ntheta, d.well_nr = spec.well_nmu, spec.well_ntheta, spec.well_nr
        d.sw_half = 1 if spec.sw_half else 0
        for c in range(3):
            d.fft_len[c] = int(spec.fft_len[c])
        d.precision = PREC[precision]
        d.lin_tol = float(getattr(spec, "lin_tol", 0.0))
        d.flags = (FLAG_AUTOTUNE if getattr(spec, "autotune", False) else 0) | \
            (FLAG_EQUILIBRIUM_INIT if getattr(spec, "eq_init", False) else 0) | \
            (FLAG_SCREENED_POISSON if getattr(spec, "screened_poisson", False) else 0) | \
            (FLAG_MSA if getattr(spec, "msa", False) else 0) | \
            (FLAG_PHASE_TIMING if getattr(spec, "phase_timing", False) else 0)
        d.eq_tol = float(getattr(spec, "eq_tol", 0.0))
        d.eq_max_iter = int(getattr(spec, "eq_max_iter", 0))
        d.fmt = int(getattr(spec, "fmt", 0))
        d.anderson_depth = int(getattr(spec, "anderson", 0))
        self.desc = d


def plan(spec, precision="fp64"):
    """pnp_plan_problem: host-only validation and plan of a problem.  Returns
    (info dict, reservoir mu_b per species)."""
    dh = DescHolder(spec, precision)
    i = Info()
    mu = np.zeros(len(spec.R))
    _check(lib().pnp_plan_problem(ctypes.byref(dh.desc), ctypes.byref(i), _ptr(mu)), "pnp_plan_problem")
    return ({"fft_len": tuple(i.fft_len), "stencil_halfwidth": i.stencil_halfwidth,
             "well_halfwidth": i.well_halfwidth, "device_bytes": i.device_bytes, "bjerrum_h": i.bjerrum_h}, mu)


def conductivity(spec, flux, D_m2_per_s=0.0):
    """pnp_conductivity (host-only): (reduced sigma, sigma in S/cm) from the
    species' plane currents flux [s][nz+1]."""
    dh = DescHolder(spec)
    f = _f64(flux)
    assert f.shape == (len(spec.R), spec.nz + 1)
    out = np.zeros(2)
    _check(lib().pnp_conductivity(ctypes.byref(dh.desc), _ptr(f), float(D_m2_per_s), _ptr(out)), "pnp_conductivity")
    return float(out[0]), float(out[1])


def weight_stencil(kind, r_out, r_in=0.0, nmu=0, ntheta=0, nr=0, S=None):
    """pnp_weight_stencil: the library's discrete weight stencil, [mz][my][mx]."""
    if S is None:
        S = int(np.ceil(r_out)) + 1
    out = np.zeros((2 * S + 1,) * 3)
    _check(lib().pnp_weight_stencil(int(kind), float(r_in), float(r_out), int(nmu), int(ntheta), int(nr), int(S),
                                    _ptr(out)), "pnp_weight_stencil")
    return out


def msa_stencil(spec, i, j, S=None):
    """pnp_msa_stencil: the MSA pair kernel C_ij on the grid, [mz][my][mx]."""
    if S is None:
        S = int(np.ceil(spec.R[i] + spec.R[j])) + 1
    dh = DescHolder(spec)
    out = np.zeros((2 * S + 1,) * 3)
    _check(lib().pnp_msa_stencil(ctypes.byref(dh.desc), int(i), int(j), int(S), _ptr(out)), "pnp_msa_stencil")
    return out


def weight_spectrum(kind, r_out, L, r_in=0.0, S=None):
    """pnp_weight_spectrum: the stored real octant of a stencil's DFT on an L grid."""
    if S is None:
        S = int(np.ceil(r_out)) + 1
    Lx, Ly, Lz = L
    out = np.zeros((Lz // 2 + 1, Ly // 2 + 1, Lx // 2 + 1))
    _check(lib().pnp_weight_spectrum(int(kind), float(r_in), float(r_out), 0, 0, 0, int(S), Lx, Ly, Lz, _ptr(out)),
           "pnp_weight_spectrum")
    return out


def selftest_bounded_wait(limit_ms):
    """pnp_selftest_bounded_wait: a device wait nothing completes, limited to
    limit_ms; returns the code (ERR_TIMEOUT expected)."""
    return lib().pnp_selftest_bounded_wait(float(limit_ms))


def excess_mu_noalloc(spec, d_rho, d_mu, stream=None):
    """pnp_excess_mu_noalloc: FP64 mu_ex into caller-owned device buffers
    (objects with data_ptr()) with no device allocation; returns the code."""
    dh = DescHolder(spec)
    return lib().pnp_excess_mu_noalloc(ctypes.byref(dh.desc), ctypes.c_void_p(d_rho.data_ptr()),
                                       ctypes.c_void_p(d_mu.data_ptr()),
                                       None if stream is None else ctypes.c_void_p(stream))


class Problem:
    """Owns a pnp_problem handle."""

    def __init__(self, spec, precision="fp64"):
        self.spec = spec
        self.s = len(spec.R)
        self.shape = (spec.nz, spec.ny, spec.nx)
        self._dh = DescHolder(spec, precision)
        h = ctypes.c_void_p()
        _check(lib().pnp_create_problem(ctypes.byref(self._dh.desc), ctypes.byref(h)), "pnp_create_problem")
        self.h = h

    def close(self):
        if self.h:
            lib().pnp_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        i = Info()
        _check(lib().pnp_get_problem_info(self.h, ctypes.byref(i)), "pnp_get_problem_info")
        return {"fft_len": tuple(i.fft_len), "stencil_halfwidth": i.stencil_halfwidth,
                "well_halfwidth": i.well_halfwidth, "device_bytes": i.device_bytes, "mg_levels": i.mg_levels,
                "tile": tuple(i.tile), "tuned_ms": i.tuned_ms, "bjerrum_h": i.bjerrum_h}

    def excess_mu(self, rho, precision=None):
        """pnp_excess_mu on host arrays; returns mu_ex [s, nz, ny, nx]."""
        r = _f64(rho)
        assert r.shape == (self.s,) + self.shape
        out = np.empty_like(r)
        _check(lib().pnp_excess_mu(self.h, _ptr(r), _ptr(out), PREC[precision]), "pnp_excess_mu")
        return out

    def excess_mu_device(self, d_rho, d_mu, precision=None, stream=None):
        """pnp_excess_mu_device on device buffers (objects with data_ptr())."""
        rc = lib().pnp_excess_mu_device(self.h, ctypes.c_void_p(d_rho.data_ptr()), ctypes.c_void_p(d_mu.data_ptr()),
                                        PREC[precision], None if stream is None else ctypes.c_void_p(stream))
        _check(rc, "pnp_excess_mu_device")

    def status(self):
        return lib().pnp_status(self.h)

    def stage_timing(self, enable=True):
        _check(lib().pnp_stage_timing(self.h, 1 if enable else 0), "pnp_stage_timing")

    def stage_times(self):
        """{stage name: (total ms, launches)} since the last read."""
        ms = np.zeros(16)
        n = np.zeros(16, dtype=np.int32)
        k = lib().pnp_stage_times(self.h, _ptr(ms), n.ctypes.data_as(_ip), 16)
        if k < 0:
            raise PnpError(k, "pnp_stage_times")
        return {lib().pnp_stage_name(j).decode(): (float(ms[j]), int(n[j])) for j in range(k)}

    def plane_flux(self, species, phi, rho):
        """pnp_plane_flux: current of one species through the nz + 1 z faces."""
        p = _f64(phi)
        r = _f64(rho)
        assert p.shape == self.shape and r.shape == (self.s,) + self.shape
        out = np.empty(self.shape[0] + 1)
        _check(lib().pnp_plane_flux(self.h, int(species), _ptr(p), _ptr(r), _ptr(out)), "pnp_plane_flux")
        return out

    def gummel_phase_times(self):
        """pnp_gummel_phase_times: ms per phase of the last solve (needs
        spec.phase_timing)."""
        out = np.zeros(len(PHASES))
        n = lib().pnp_gummel_phase_times(self.h, _ptr(out), len(PHASES))
        if n < 0:
            raise PnpError(n, "pnp_gummel_phase_times")
        return dict(zip(PHASES, out.tolist()))

    def square_well_energy(self, rho):
        """pnp_square_well_energy: F_sh (kT) of the densities rho [s][nz][ny][nx]."""
        r = _f64(rho)
        assert r.shape == (self.s,) + self.shape
        out = np.zeros(1)
        _check(lib().pnp_square_well_energy(self.h, _ptr(r), _ptr(out)), "pnp_square_well_energy")
        return float(out[0])

    def conductivity(self, phi, rho, D_m2_per_s=0.0):
        """Plane currents of every species (pnp_plane_flux), then
        pnp_conductivity: (reduced sigma, sigma in S/cm)."""
        flux = np.stack([self.plane_flux(i, phi, rho) for i in range(self.s)])
        return conductivity(self.spec, flux, D_m2_per_s)

    def gummel_solve(self, phi0=None, rho0=None, raise_on_error=True):
        """pnp_gummel_solve; returns (phi, rho, stats dict)."""
        phi = np.empty(self.shape)
        rho = np.empty((self.s,) + self.shape)
        st = Stats()
        p0 = None if phi0 is None else _f64(phi0)
        r0 = None if rho0 is None else _f64(rho0)
        rc = lib().pnp_gummel_solve(self.h, _ptr(p0), _ptr(r0), _ptr(phi), _ptr(rho), ctypes.byref(st))
        stats = {"status": st.status, "iterations": st.iterations, "residual": st.residual,
                 "linear_iterations": st.linear_iterations, "seconds": st.seconds,
                 "init_iterations": st.init_iterations, "init_residual": st.init_residual,
                 "repeated_sweeps": st.repeated_sweeps}
        if raise_on_error and rc not in (OK,):
            raise PnpError(rc, "pnp_gummel_solve")
        return phi, rho, stats


class Server:
    """Owns a pnp_server handle."""

    def __init__(self, hbm_budget_bytes=0, max_slots=0, max_queue=0, policy="fifo"):
        o = ServerOpts(hbm_budget_bytes, max_slots, max_queue, SERVE[policy])
        h = ctypes.c_void_p()
        _check(lib().pnp_server_create(ctypes.byref(o), ctypes.byref(h)), "pnp_server_create")
        self.h = h
        self._shapes = {}

    def close(self):
        if self.h:
            lib().pnp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, spec, phi0=None, rho0=None, precision="fp64"):
        dh = DescHolder(spec, precision)
        t = ctypes.c_uint64()
        p0 = None if phi0 is None else _f64(phi0)
        r0 = None if rho0 is None else _f64(rho0)
        rc = lib().pnp_submit(self.h, ctypes.byref(dh.desc), _ptr(p0), _ptr(r0), ctypes.byref(t))
        if rc != OK:
            return rc, None
        self._shapes[t.value] = (len(spec.R), (spec.nz, spec.ny, spec.nx))
        return OK, t.value

    def poll(self, ticket):
        """Returns (code, phi, rho, stats); phi/rho are None while pending."""
        s, shape = self._shapes.get(ticket, (1, (1, 1, 1)))
        phi = np.empty(shape)
        rho = np.empty((s,) + shape)
        st = Stats()
        rc = lib().pnp_poll(self.h, ctypes.c_uint64(ticket), _ptr(phi), _ptr(rho), ctypes.byref(st))
        if rc == PENDING:
            return rc, None, None, None
        self._shapes.pop(ticket, None)
        stats = {"status": st.status, "iterations": st.iterations, "residual": st.residual,
                 "linear_iterations": st.linear_iterations, "seconds": st.seconds,
                 "init_iterations": st.init_iterations, "init_residual": st.init_residual,
                 "repeated_sweeps": st.repeated_sweeps}
        return rc, phi, rho, stats

    def stats(self):
        st = ServerStats()
        _check(lib().pnp_server_get_stats(self.h, ctypes.byref(st)), "pnp_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}
