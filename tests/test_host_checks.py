"""Host-side argument checks of the library (no GPU needed): the scan that
validates caller arrays (densities >= 0 or > 0 and finite, potentials
finite) against numpy, on small arrays and on arrays large enough to be split
over threads, with the offending value in every position class."""
import ctypes
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_1407_0674_gb300", "_build", "libpnp_gb300.so")


@pytest.fixture(scope="module")
def check():
    if not os.path.exists(LIB):
        from paper_1407_0674_gb300 import build
        build.build()
    L = ctypes.CDLL(LIB)
    f = getattr(L, "_ZN3pnp14host_values_okEPKdmi")
    f.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_size_t, ctypes.c_int]
    f.restype = ctypes.c_bool

    def run(a, kind):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return bool(f(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.size, kind))
    return run


def expect(a, kind):
    fin = np.isfinite(a)
    if kind == 0:
        return bool(fin.all())
    if kind == 1:
        return bool((fin & (a >= 0)).all())
    return bool((fin & (a > 0)).all())


@pytest.mark.parametrize("n", [1, 7, 1000, (1 << 19) * 3 + 17])
def test_matches_numpy(check, n):
    rng = np.random.default_rng(n)
    base = rng.uniform(0.1, 2.0, n)
    for kind in (0, 1, 2):
        assert check(base, kind) is True
    bads = [np.nan, np.inf, -np.inf, -1e-300, 0.0, -0.0, -5.0]
    positions = sorted({0, n // 3, n // 2, n - 1})
    for v in bads:
        for pos in positions:
            a = base.copy()
            a[pos] = v
            for kind in (0, 1, 2):
                assert check(a, kind) == expect(a, kind), (n, v, pos, kind)


def test_empty_is_valid(check):
    assert check(np.zeros(0), 1) is True


def test_tf32_split_dft16_matrices():
    """The operands of the tensor-core y pass: the real form of the 16-point
    DFT (forward and inverse) split into TF32 hi and lo parts.  Each part must
    be exactly representable in TF32 (low 13 mantissa bits zero), and hi + lo
    must be the matrix to 2^-22 relative -- the accuracy the 3-term product
    relies on."""
    L = ctypes.CDLL(LIB)
    f = getattr(L, "_ZN3pnp17ypass_tc_matricesEPf")
    f.argtypes = [ctypes.POINTER(ctypes.c_float)]
    f.restype = None
    out = np.zeros(4 * 32 * 32, dtype=np.float32)
    f(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    M = out.reshape(2, 2, 32, 32)               # [direction][hi, lo][j][k]
    bits = M.view(np.uint32)
    assert not np.any(bits & np.uint32(0x1FFF))
    n = np.arange(16)
    for d, sign in ((0, -1.0), (1, 1.0)):
        W = np.exp(sign * 2j * np.pi * np.outer(n, n) / 16)   # W[k_out, n_in]
        ref = np.zeros((32, 32))
        ref[0::2, 0::2] = W.real      # out re <- in re
        ref[0::2, 1::2] = -W.imag     # out re <- in im
        ref[1::2, 0::2] = W.imag      # out im <- in re
        ref[1::2, 1::2] = W.real      # out im <- in im
        total = M[d, 0].astype(np.float64) + M[d, 1].astype(np.float64)
        assert np.abs(total - ref).max() <= 2.0 ** -22
        assert np.abs(M[d, 0] - ref).max() <= 2.0 ** -10
