"""Allocation failures injected on the host (pnp_test_fail_alloc_at(k) makes
the k-th device allocation after it report out-of-memory without calling
CUDA): for every k the failing call returns PNP_ERR_NOMEM, leaves nothing
half-built behind, the same call then succeeds, and the results are bit for
bit those of a run without the fault.  Covers problem creation (workspace,
twiddles, spectra, square-well field), the host-buffer staging, lazy
preparation of another precision and the Gummel solver's set-up and graph.
No GPU fault, trap or hang is involved: the GPU never sees the failure.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_1407_0674_gb300 import pnp
from workloads import film_gummel, lognormal_density

pnp.lib().pnp_test_fail_alloc_at(int(sys.argv[3]))
spec = film_gummel(8, 8, 8, max_iter=3, tol=1e-30)
spec.lin_tol = 1e-13
rho = lognormal_density(spec, 3, sigma=0.2)
events = []

def retry(fn):
    try:
        return fn()
    except pnp.PnpError as e:
        events.append(e.code)
        return fn()

P = retry(lambda: pnp.Problem(spec))
mu = retry(lambda: P.excess_mu(rho, precision="fp64"))
mudd = retry(lambda: P.excess_mu(rho, precision="df64"))
phi, r, st = P.gummel_solve(raise_on_error=False)
if st["status"] == pnp.ERR_NOMEM:
    events.append(st["status"])
    phi, r, st = P.gummel_solve(raise_on_error=False)
P.close()
np.savez(sys.argv[2], mu=mu, mudd=mudd, phi=phi, r=r)
print(json.dumps({"events": events, "status": st["status"], "iterations": st["iterations"]}))
"""


@pytest.fixture(scope="module")
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1407_0674_gb300 import build
    build.build()
    return True


def run_child(k, out, tmp_path):
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(out), str(k)], capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, (k, r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_every_allocation_failure_is_clean(built, tmp_path):
    ref_file = tmp_path / "ref.npz"
    ref = run_child(0, ref_file, tmp_path)
    assert ref["events"] == [] and ref["iterations"] == 3
    want = np.load(ref_file)
    injected = 0
    for k in range(1, 400):
        f = tmp_path / f"k{k}.npz"
        res = run_child(k, f, tmp_path)
        if not res["events"]:
            break                               # past the last allocation of the run
        injected += 1
        assert res["events"] == [-2], (k, res)  # exactly one PNP_ERR_NOMEM, then success
        assert res["iterations"] == 3
        got = np.load(f)
        for name in ("mu", "mudd", "phi", "r"):
            np.testing.assert_array_equal(got[name], want[name], err_msg=f"k={k} {name}")
    assert injected >= 10
