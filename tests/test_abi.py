"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/pnp.h declares, its descriptor layout matches the
header (checked with the C compiler), and descriptor validation rejects bad
input before touching the device."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1407_0674_gb300 import build, pnp
from workloads import ProblemSpec, mu_microbench, film_gummel

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return pnp.lib()


def test_exports_every_declared_function(L):
    names = pnp.header_functions()
    assert "pnp_create_problem" in names and "pnp_excess_mu" in names and "pnp_gummel_solve" in names
    assert "pnp_submit" in names and "pnp_poll" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared but not exported"


def test_descriptor_layout_matches_header(L):
    fields = [f for f, _ in pnp.Desc._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"pnp.h\"\nint main(void){\n"
    prog += 'printf("%zu\\n", sizeof(pnp_problem_desc));\n'
    for f in fields:
        prog += f'printf("%zu\\n", offsetof(pnp_problem_desc, {f}));\n'
    for t in ("pnp_stats", "pnp_problem_info", "pnp_server_opts", "pnp_server_stats"):
        prog += f'printf("%zu\\n", sizeof({t}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    assert out[0] == ctypes.sizeof(pnp.Desc)
    for f, off in zip(fields, out[1:1 + len(fields)]):
        assert getattr(pnp.Desc, f).offset == off, f
    rest = out[1 + len(fields):]
    assert rest == [ctypes.sizeof(pnp.Stats), ctypes.sizeof(pnp.Info), ctypes.sizeof(pnp.ServerOpts),
                    ctypes.sizeof(pnp.ServerStats)]


def test_error_strings(L):
    for code in range(-9, 2):
        assert pnp.error_string(code) != "unknown error"
    assert pnp.error_string(-42) == "unknown error"


def _create(spec):
    dh = pnp.DescHolder(spec)
    h = ctypes.c_void_p()
    return pnp.lib().pnp_create_problem(ctypes.byref(dh.desc), ctypes.byref(h)), dh


@pytest.mark.parametrize("mutate", [
    lambda s: setattr(s, "nx", 0),
    lambda s: setattr(s, "R", (0.0, 2.0)),
    lambda s: setattr(s, "rho_b", (-1.0, 0.01)),
    lambda s: setattr(s, "lambda_phi", 0.0),
    lambda s: setattr(s, "lambda_rho", 1.5),
    lambda s: setattr(s, "tol", 0.0),
    lambda s: setattr(s, "bc", ("P", "P", 7)),
    lambda s: setattr(s, "fft_len", (0, 0, 33)),          # below n + S on a zero-extended axis
    lambda s: setattr(s, "fft_len", (48, 0, 0)),          # periodic axis must use L = n
    lambda s: setattr(s, "nx", 14),                        # periodic length must be 2^a 3^b 5^c
    lambda s: setattr(s, "rho_b", (0.05, 0.05)),           # bulk packing above 1
    lambda s: (setattr(s, "well_inner", 5.0), setattr(s, "well_outer", 4.0)),
])
def test_invalid_descriptors_rejected_on_host(L, mutate):
    spec = film_gummel(32, 32, 32)
    mutate(spec)
    rc, _ = _create(spec)
    assert rc == pnp.ERR_INVALID


def test_desc_init_defaults(L):
    d = pnp.Desc()
    assert L.pnp_desc_init(ctypes.byref(d)) == 0
    assert d.lambda_phi == 0.3 and d.max_iter == 500 and d.sw_half == 1 and d.eps_r == 16.6
    assert L.pnp_desc_init(None) == pnp.ERR_INVALID


@pytest.mark.parametrize("ctype,cname", [(pnp.Stats, "pnp_stats"), (pnp.Info, "pnp_problem_info"),
                                          (pnp.ServerOpts, "pnp_server_opts"),
                                          (pnp.ServerStats, "pnp_server_stats")])
def test_struct_field_offsets_match_header(L, ctype, cname):
    fields = [f for f, _ in ctype._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"pnp.h\"\nint main(void){\n"
    for f in fields:
        prog += f'printf("%zu\\n", offsetof({cname}, {f}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    for f, off in zip(fields, out):
        assert getattr(ctype, f).offset == off, (cname, f)


def test_binding_declares_every_header_function(L):
    """Every function of include/pnp.h has ctypes argument types in the
    binding (without them ctypes would pass doubles as ints)."""
    missing = [f for f in pnp.header_functions() if getattr(L, f).argtypes is None]
    assert missing == []


C_CLIENT = r"""
#include <stdio.h>
#include "pnp.h"
int main(void) {
    pnp_problem_desc d;
    if (pnp_desc_init(&d) != PNP_OK) return 1;
    int q[2] = {1, -1};
    double R[2] = {2.0, 2.0}, rb[2] = {0.006, 0.006}, mu[2];
    d.nx = 32; d.ny = 32; d.nz = 30;
    d.bc[0] = PNP_BC_PERIODIC; d.bc[1] = PNP_BC_PERIODIC; d.bc[2] = PNP_BC_DIRICHLET;
    d.nspecies = 2; d.valence = q; d.radius = R; d.rho_bulk = rb;
    d.phi_lo = 0.0; d.phi_hi = 0.5;
    pnp_problem_info info;
    if (pnp_plan_problem(&d, &info, mu) != PNP_OK) return 2;
    printf("%d %d %d %d %.17g %.17g %.17g\n", info.fft_len[0], info.fft_len[1], info.fft_len[2],
           info.stencil_halfwidth, mu[0], mu[1], info.bjerrum_h);
    double flux[2 * 31];
    for (int k = 0; k < 31; ++k) { flux[k] = -1.0; flux[31 + k] = 1.0; }
    double sigma[2];
    if (pnp_conductivity(&d, flux, 1e-10, sigma) != PNP_OK) return 3;
    printf("%.17g %.17g\n", sigma[0], sigma[1]);
    d.nspecies = 0;
    printf("%d %s\n", pnp_plan_problem(&d, &info, NULL), pnp_error_string(PNP_ERR_INVALID));
    return 0;
}
"""


def test_plain_c_client_links_and_calls_host_entry_points(L):
    """A C program built against include/pnp.h and linked to the shared
    library calls the host-only entry points (no device needed): the plan
    and reservoir mu match the Python binding's, the conductivity of unit
    currents is the closed form, and a bad descriptor is refused."""
    from workloads import ProblemSpec
    lib_dir = os.path.dirname(pnp.LIB_PATH)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "client.c")
        open(c, "w").write(C_CLIENT)
        exe = os.path.join(d, "client")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe, "-L", lib_dir,
                               "-lpnp_gb300", "-Wl,-rpath," + lib_dir])
        lines = subprocess.check_output([exe], text=True).splitlines()
    a = lines[0].split()
    spec = ProblemSpec(nx=32, ny=32, nz=30, bc=("P", "P", "D"), R=(2.0, 2.0), q=(1, -1), rho_b=(0.006, 0.006),
                       phi_hi=0.5)
    info, mu = pnp.plan(spec)
    assert tuple(int(x) for x in a[:3]) == info["fft_len"] and int(a[3]) == info["stencil_halfwidth"]
    assert float(a[4]) == mu[0] and float(a[5]) == mu[1] and float(a[6]) == info["bjerrum_h"]
    sig = [float(x) for x in lines[1].split()]
    # charge current -2 per face over 32*32 faces, field -0.5/31
    assert sig[0] == pytest.approx((-2.0 / 1024) / (-0.5 / 31), rel=1e-14)
    assert sig == list(pnp.conductivity(spec, np.stack([-np.ones(31), np.ones(31)]), 1e-10))
    assert lines[2].startswith(f"{pnp.ERR_INVALID} ")
