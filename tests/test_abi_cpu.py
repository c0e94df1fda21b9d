"""The C-ABI library without a GPU: it builds, loads, exports every function
include/sag.h declares, and rejects bad arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1905_09071_gb300 import sag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sag.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(sag_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return sag.load()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(sag.EXPORTS)


def _struct_fields(name):
    """(type, field) pairs of a typedef struct in include/sag.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    return [(" ".join(t.split()), f) for t, f in re.findall(r"([\w\s\*]+?)\s*\b(\w+)\s*;", body)]


CTYPE = {"int32_t": ctypes.c_int32, "const int32_t*": ctypes.POINTER(ctypes.c_int32),
         "const double*": ctypes.c_void_p}


@pytest.mark.parametrize("name,cls", [("sag_options", sag._Options), ("sag_system", sag._System)])
def test_structs_match_the_header(name, cls):
    # field names, order and types of the ctypes mirrors follow include/sag.h
    fields = _struct_fields(name)
    assert [f for _, f in fields] == [f for f, _ in cls._fields_]
    for (ctype, f), (g, ty) in zip(fields, cls._fields_):
        assert ty == CTYPE[ctype.replace(" *", "*")], (f, ctype, ty)


def test_library_exports_every_declared_function(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_defaults(lib):
    assert b"sm_103a" in lib.sag_version()
    assert sag.default_options() == {"prec": sag.SAG_FP32_SPLIT, "rk": sag.SAG_HEUN,
                                     "symmetrize_q": 1, "autotune": 0, "max_m2": 0, "m2": None,
                                     "keep_repeats": 0}


def _plan_status(N=8, D=3, ranks=(2, 2), fmt=sag.SAG_CP, B=1, opt=None, factors=True, out=True):
    lib = sag.load()
    r = np.array(ranks, dtype=np.int32)
    f = np.ones(1024)
    s = sag._System(N, D, fmt, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    f.ctypes.data if factors else None, 0)
    o = sag._Options(*(opt or (sag.SAG_FP32_SPLIT, sag.SAG_HEUN, 1, 0)))
    h = ctypes.c_void_p()
    st = lib.sag_plan(ctypes.byref(s), B, ctypes.byref(o), ctypes.byref(h) if out else None)
    return st, lib.sag_last_error().decode()


@pytest.mark.parametrize("kw,status", [
    (dict(N=0), sag.SAG_EINVAL),
    (dict(D=1, ranks=()), sag.SAG_EINVAL),
    (dict(D=9, ranks=(1,) * 7), sag.SAG_EINVAL),
    (dict(ranks=(2, -1)), sag.SAG_EINVAL),
    (dict(ranks=(0, 0)), sag.SAG_EINVAL),  # rank 0 leaves an order out, but one must remain
    (dict(fmt=7), sag.SAG_EINVAL),
    (dict(B=0), sag.SAG_EINVAL),
    (dict(factors=False), sag.SAG_EINVAL),
    (dict(out=False), sag.SAG_EINVAL),
    (dict(opt=(9, 0, 1, 0)), sag.SAG_EINVAL),
    (dict(opt=(3, 0, 1, 0)), sag.SAG_EINVAL),  # precisions are 0, 1 and 2
    (dict(opt=(0, 4, 1, 0)), sag.SAG_EINVAL),
    (dict(opt=(0, 0, 2, 0)), sag.SAG_EINVAL),
    (dict(opt=(1, 0, 1, 2)), sag.SAG_EINVAL),  # autotune is 0 or 1
    (dict(opt=(1, 0, 1, 0, 2)), sag.SAG_EINVAL),  # max_m2: 0 or a power of two in [4, 512]
    (dict(opt=(1, 0, 1, 0, 96)), sag.SAG_EINVAL),
    (dict(opt=(1, 0, 1, 0, 1024)), sag.SAG_EINVAL),
    (dict(opt=(1, 0, 1, 0, -4)), sag.SAG_EINVAL),
    (dict(opt=(1, 0, 1, 0, 0, None, 2)), sag.SAG_EINVAL),  # n_m2 without m2
    (dict(opt=(1, 0, 1, 0, 0, None, 0, 2)), sag.SAG_EINVAL),  # keep_repeats is 0 or 1
])
def test_plan_rejects_bad_arguments(kw, status):
    st, msg = _plan_status(**kw)
    assert st == status
    assert msg


@pytest.mark.parametrize("m2,n", [([256, 96], 2), ([2, 0], 2), ([0, 1024], 2), ([256], 0)])
def test_plan_rejects_bad_m2(m2, n):
    arr = np.array(m2, dtype=np.int32)
    opt = (sag.SAG_FP32_SPLIT, sag.SAG_HEUN, 1, 0, 0, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n)
    st, msg = _plan_status(opt=opt)
    assert st == sag.SAG_EINVAL
    assert "m2" in msg


def test_batched_plan_rejects_mixed_formats_and_bad_tt_ranks(lib):
    f = np.ones(4096)
    cp_r = np.array([1, 1], dtype=np.int32)
    tt_r = np.array([1, 2, 1, 1, 2, 2, 1], dtype=np.int32)  # d = 2: (1,2,1); d = 3: (1,2,2,1)
    bad_tt = np.array([1, 17, 1, 1, 2, 2, 1], dtype=np.int32)
    P = ctypes.POINTER(ctypes.c_int32)
    h = ctypes.c_void_p()
    o = sag._Options(sag.SAG_FP32_SPLIT, sag.SAG_HEUN, 1, 0)
    arr = (sag._System * 2)(sag._System(8, 3, sag.SAG_CP, cp_r.ctypes.data_as(P), f.ctypes.data, 0),
                            sag._System(8, 3, sag.SAG_TT, tt_r.ctypes.data_as(P), f.ctypes.data, 0))
    assert lib.sag_plan(arr, 2, ctypes.byref(o), ctypes.byref(h)) == sag.SAG_EUNSUPPORTED
    assert b"one format" in lib.sag_last_error()
    one = (sag._System * 1)(sag._System(8, 3, sag.SAG_TT, bad_tt.ctypes.data_as(P), f.ctypes.data, 0))
    assert lib.sag_plan(one, 1, ctypes.byref(o), ctypes.byref(h)) == sag.SAG_EINVAL


def test_null_plan_calls_are_rejected(lib):
    x = np.zeros(4)
    assert lib.sag_rhs(None, x.ctypes.data, x.ctypes.data, None) == sag.SAG_EINVAL
    assert lib.sag_rk2_step(None, x.ctypes.data, 0.1, None) == sag.SAG_EINVAL
    assert lib.sag_integrate(None, x.ctypes.data, 0.1, 1, None, None) == sag.SAG_EINVAL
    assert lib.sag_rhs_parts(None, x.ctypes.data, None, None, None, None) == sag.SAG_EINVAL
    assert lib.sag_sync_status(None, None) == sag.SAG_EINVAL
    lib.sag_plan_destroy(None)


def test_binding_raises_typed_error():
    with pytest.raises(sag.SagError) as ei:
        sag.Plan(0, 3, [1, 1], np.ones(10))
    assert ei.value.status == sag.SAG_EINVAL
