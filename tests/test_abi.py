"""Host-only checks of the C ABI: the library builds, loads, exports every
function include/*.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(ffsrqr_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def ff():
    from paper_1803_01982_gb300 import build
    build.build()
    from paper_1803_01982_gb300 import ffsrqr
    return ffsrqr


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["ffsrqr_plan", "ffsrqr_run", "ffsrqr_destroy", "ffsrqr_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(ff):
    lib = ctypes.CDLL(ff._build.LIB)
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_status_strings(ff):
    assert ff.ffsrqr_status_string(0) == b"ok"
    assert b"swap" in ff.ffsrqr_status_string(2)
    assert ff.ffsrqr_status_string(-3) == b"invalid argument"


@pytest.mark.parametrize("args,code", [
    ((0, 10, 2, 1, 0), -2),        # m
    ((10, 0, 2, 1, 0), -3),        # n
    ((10, 8, 0, 1, 0), -4),        # k = 0
    ((10, 8, 9, 0, 0), -4),        # k > n
    ((10, 8, 4, -1, 0), -5),       # p < 0
    ((10, 8, 4, 7, 0), -5),        # k + p > m
    ((10, 8, 4, 2, 5), -6),        # mode (0 plain, 1 TF32x3, 2 BF16x3, 3 FP64 are valid)
])
def test_plan_argument_errors(ff, args, code):
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    rc = ff.ffsrqr_plan(ctypes.byref(h), *args, None, ctypes.byref(ws))
    assert rc == code
    assert not h.value


def test_plan_bad_opts(ff):
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    opts = ff.Opts(1.0, 10, 0)   # g must exceed 1
    assert ff.ffsrqr_plan(ctypes.byref(h), 10, 8, 3, 2, 0, ctypes.byref(opts), ctypes.byref(ws)) == -7
    assert ff.ffsrqr_plan(None, 10, 8, 3, 2, 0, None, ctypes.byref(ws)) == -1
    assert ff.ffsrqr_plan(ctypes.byref(h), 10, 8, 3, 2, 0, None, None) == -8


def test_run_and_destroy_null_plan(ff):
    assert ff.ffsrqr_run(None, None, 0, 0, None, 0, None, None, 0, None, None, None, None) == -1
    assert ff.ffsrqr_destroy(None) == -1
    assert ff.ffsrqr_philox4x32_10(None, None, 1, None) == -1


def test_plan_l_argument_errors(ff):
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    assert ff.ffsrqr_plan_l(ctypes.byref(h), 100, 80, 0, 5, 4, 0, None, ctypes.byref(ws)) == -4
    assert ff.ffsrqr_plan_l(ctypes.byref(h), 100, 80, 6, 5, 4, 0, None, ctypes.byref(ws)) == -5
    assert ff.ffsrqr_plan_l(ctypes.byref(h), 100, 80, 2, 5, -1, 0, None, ctypes.byref(ws)) == -6
    assert ff.ffsrqr_plan_l(ctypes.byref(h), 100, 80, 2, 5, 4, 9, None, ctypes.byref(ws)) == -7
    assert ff.ffsrqr_plan_l(ctypes.byref(h), 100, 80, 2, 5, 4, 0, None, None) == -9
    assert ff.ffsrqr_plan_depth(None) == -1


def test_tucker_plan_argument_errors(ff):
    """Argument checks of ffsrqr_tucker_plan, all before any device call."""
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    dims = (ctypes.c_int64 * 3)(10, 9, 8)
    ranks = (ctypes.c_int32 * 3)(2, 2, 2)
    plan = ff.ffsrqr_tucker_plan
    assert plan(None, 0, 3, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -1
    assert plan(ctypes.byref(h), 2, 3, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -2
    assert plan(ctypes.byref(h), 0, 1, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -3
    assert plan(ctypes.byref(h), 0, 9, dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -3
    bad_dims = (ctypes.c_int64 * 3)(10, 0, 8)
    assert plan(ctypes.byref(h), 0, 3, bad_dims, ranks, None, 2, 0, None, ctypes.byref(ws)) == -4
    big = (ctypes.c_int32 * 3)(2, 10, 2)
    assert plan(ctypes.byref(h), 0, 3, dims, big, None, 2, 0, None, ctypes.byref(ws)) == -5
    bad_order = (ctypes.c_int32 * 3)(0, 0, 1)
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, bad_order, 2, 0, None, ctypes.byref(ws)) == -6
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, None, -1, 0, None, ctypes.byref(ws)) == -7
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, None, 2, 5, None, ctypes.byref(ws)) == -8
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, None, 2, 0, None, None) == -10
    # k_r + p > m_j: the first step's ffsrqr_plan rejects it before any device call
    assert plan(ctypes.byref(h), 0, 3, dims, ranks, None, 9, 0, None, ctypes.byref(ws)) == -11
    assert plan(ctypes.byref(h), 1, 3, dims, ranks, None, 9, 0, None, ctypes.byref(ws)) == -11
    assert ff.ffsrqr_tucker_run(None, None, 0, None, None, None, None, None, None) == -1
    assert ff.ffsrqr_tucker_destroy(None) == -1
    assert ff.ffsrqr_tucker_launch_count(None) == -1


def test_rpca_argument_errors(ff):
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    create = ff.ffsrqr_rpca_create
    assert create(None, 10, 10, None, ctypes.byref(ws)) == -1
    assert create(ctypes.byref(h), 1, 10, None, ctypes.byref(ws)) == -2
    assert create(ctypes.byref(h), 10, 1, None, ctypes.byref(ws)) == -3
    assert create(ctypes.byref(h), 10, 10, None, None) == -5
    bad_mode = ff.RpcaOpts(2, 0, 0, 0, 0, 0, 0.0, 0.0, 0.0, 0.0)
    assert create(ctypes.byref(h), 10, 10, ctypes.byref(bad_mode), ctypes.byref(ws)) == -4
    neg = ff.RpcaOpts(0, 0, 0, 0, 0, 0, 0.0, 0.0, 0.0, -1.0)
    assert create(ctypes.byref(h), 10, 10, ctypes.byref(neg), ctypes.byref(ws)) == -4
    assert ff.ffsrqr_rpca_run(None, None, 0, None, 0, None, 0, 0, None, None, None) == -1
    assert ff.ffsrqr_rpca_destroy(None) == -1
    assert ff.ffsrqr_rpca_launch_count(None) == -1


def test_plan_rsi_argument_errors(ff):
    import ctypes
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    f = ff.ffsrqr_plan_rsi
    assert f(None, 100, 80, 5, 5, 1, 0, None, ctypes.byref(ws)) == -1
    assert f(ctypes.byref(h), 0, 80, 5, 5, 1, 0, None, ctypes.byref(ws)) == -2
    assert f(ctypes.byref(h), 100, 0, 5, 5, 1, 0, None, ctypes.byref(ws)) == -3
    assert f(ctypes.byref(h), 100, 80, 0, 5, 1, 0, None, ctypes.byref(ws)) == -4
    assert f(ctypes.byref(h), 100, 80, 10, 75, 1, 0, None, ctypes.byref(ws)) == -5
    assert f(ctypes.byref(h), 100, 80, 10, 5, -1, 0, None, ctypes.byref(ws)) == -6
    assert f(ctypes.byref(h), 100, 80, 10, 5, 1, 9, None, ctypes.byref(ws)) == -7
    assert f(ctypes.byref(h), 100, 80, 10, 5, 1, 0, None, None) == -9
