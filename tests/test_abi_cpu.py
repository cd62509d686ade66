"""CPU checks of the C ABI: the library loads, exports every symbol include/*.h
declares, sizes its workspace and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_05424_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.load()


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    text = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dot_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_expected_calls():
    names = declared_symbols()
    for want in ("dot_create", "dot_solve", "dot_get", "dot_destroy", "dot_workspace_bytes"):
        assert want in names
    assert set(names) == set(N.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_workspace_bytes(lib):
    g = N.DotGrid(2, 64, (ctypes.c_int * 3)(256, 256, 1))
    b64 = lib.dot_workspace_bytes(ctypes.byref(g), N.DOT_FP64)
    # FP64 path: 4 node fields + q, alpha (1 + 2 padded planes sets) + beta, z (10 planes each)
    P, n0, nn = 256 * 256, 64 * 256 * 256, 65 * 256 * 256
    lower = 8 * (4 * nn + 2 * (n0 + 2 * nn) + 2 * 10 * n0)
    assert lower <= b64 <= lower * 1.02 + (1 << 22)
    bad = N.DotGrid(4, 8, (ctypes.c_int * 3)(8, 8, 8))
    assert lib.dot_workspace_bytes(ctypes.byref(bad), N.DOT_FP64) == 0
    bad = N.DotGrid(2, 0, (ctypes.c_int * 3)(8, 8, 1))
    assert lib.dot_workspace_bytes(ctypes.byref(bad), N.DOT_FP64) == 0


def _create(lib, grid, r0, r1, opt=None, mask=None):
    dp = ctypes.POINTER(ctypes.c_double)
    ctx = ctypes.c_void_p()
    rc = lib.dot_create(ctypes.byref(grid), r0.ctypes.data_as(dp), r1.ctypes.data_as(dp),
                        None if mask is None else mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        None if opt is None else ctypes.byref(opt), None, 0, None, ctypes.byref(ctx))
    return rc, ctx


def test_create_rejects_bad_arguments_before_any_device_call(lib):
    g = N.DotGrid(2, 4, (ctypes.c_int * 3)(4, 4, 1))
    ok = np.ones(16)
    rc, ctx = _create(lib, N.DotGrid(1, 4, (ctypes.c_int * 3)(4, 1, 1)), ok, ok)
    assert rc == N.DOT_EINVAL and not ctx.value
    assert b"D must be" in lib.dot_last_error(None)
    neg = ok.copy(); neg[3] = -1.0
    rc, _ = _create(lib, g, neg, ok)
    assert rc == N.DOT_EINVAL and b"non-negative" in lib.dot_last_error(None)
    nan = ok.copy(); nan[0] = np.nan
    assert _create(lib, g, ok, nan)[0] == N.DOT_EINVAL
    assert _create(lib, g, np.zeros(16), ok)[0] == N.DOT_EINVAL
    o = N.DotOptions(); lib.dot_default_options(ctypes.byref(o))
    # the defaults are the paper's parameters (fixture with citations)
    golden = os.path.join(os.path.dirname(__file__), "golden", "algorithm_parameters.txt")
    rows = [l.split() for l in open(golden) if l.strip() and not l.startswith("#")]
    for name, value in rows:
        assert getattr(o, name) == float(value), name
    assert o.check_every == 10 and o.use_graphs == 1
    # the mixed path's switch to the ALG2 step below its FP32 floor (Sec. 5.2's tau = 1)
    assert o.tau_switch_below == 3e-7
    o.tau_switch_below = -1.0
    assert _create(lib, g, ok, ok, o)[0] == N.DOT_EINVAL and b"tau_switch_below" in lib.dot_last_error(None)
    o.tau_switch_below = 3e-7
    o.tau = 2.0
    assert _create(lib, g, ok, ok, o)[0] == N.DOT_EINVAL
    o.tau = 1.9; o.s_r = 1.0
    assert _create(lib, g, ok, ok, o)[0] == N.DOT_EINVAL


def test_null_context_calls_fail_cleanly(lib):
    assert lib.dot_solve(None, 1e-6, 10) == N.DOT_EINVAL
    assert lib.dot_kkt(None, None) == N.DOT_EINVAL
    lib.dot_destroy(None)
    assert lib.dot_launch_count(None) == 0


def test_size_limits(lib):
    """Every field's element index, cone components stacked, stays below 2^31 (the
    kernels index with 32-bit integers): a grid at the limit is accepted, one beyond
    it is refused without touching a device."""
    ok = N.DotGrid(2, 31, (ctypes.c_int * 3)(2048, 2048, 1))      # 32 x 2048^2 x 10 < 2^31
    assert lib.dot_workspace_bytes(ctypes.byref(ok), N.DOT_MIXED) > 0
    big = N.DotGrid(2, 63, (ctypes.c_int * 3)(2048, 2048, 1))     # 64 x 2048^2 x 10 >= 2^31
    assert lib.dot_workspace_bytes(ctypes.byref(big), N.DOT_MIXED) == 0
    r = np.ones(2048 * 2048)
    rc, ctx = _create(lib, big, r, r)
    assert rc == N.DOT_EINVAL and not ctx.value and b"too large" in lib.dot_last_error(None)
    for D, T, Ns in ((2, 65536, (8, 8, 1)), (2, 4, (65537, 2, 1)), (2, 4, (1, 8, 1))):
        g = N.DotGrid(D, T, (ctypes.c_int * 3)(*Ns))
        assert lib.dot_workspace_bytes(ctypes.byref(g), N.DOT_FP64) == 0
