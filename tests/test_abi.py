"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/pbit.h declares, and its host-side argument logic."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def so():
    from paper_cs_0511020_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared():
    txt = open(os.path.join(ROOT, "include", "pbit.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pbit_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(so):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(so, n), f"{n} declared in pbit.h but not exported"


def test_binding_knows_every_export():
    from paper_cs_0511020_gb300 import pbit
    assert set(pbit.EXPORTS) == set(declared())


def test_status_strings(so):
    so.pbit_status_string.restype = ctypes.c_char_p
    for st in range(8):
        assert so.pbit_status_string(st)
    assert b"unknown" in so.pbit_status_string(99)


def test_workspace_size_host_logic(so):
    f = so.pbit_workspace_size
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    out = ctypes.c_size_t(0)
    sizes = []
    for n in (0, 1, 1000, 1 << 20, 1 << 24):
        assert f(n, 1, 4, None, ctypes.byref(out)) == 0
        sizes.append(out.value)
    assert sizes == sorted(sizes) and sizes[-1] > (1 << 24) * 16
    assert f(1 << 20, 1, 3, None, ctypes.byref(out)) == 1        # bad key width
    assert f(-1, 1, 4, None, ctypes.byref(out)) == 1             # bad size
    assert f(1 << 31, 1, 4, None, ctypes.byref(out)) == 1        # >= 2^31 nodes
    assert f(100, 0, 4, None, ctypes.byref(out)) == 1            # no list
    # more lists need more workspace
    a = ctypes.c_size_t(0)
    b = ctypes.c_size_t(0)
    f(1 << 20, 1, 4, None, ctypes.byref(a))
    f(1 << 20, 4096, 4, None, ctypes.byref(b))
    assert b.value > a.value


def test_tune_validation(so):
    from paper_cs_0511020_gb300 import pbit
    f = so.pbit_workspace_size
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    out = ctypes.c_size_t(0)
    for tune, ok in (((4, 0, 0, 0), True), ((8, 0, 0, 0), False), ((0, 512, 0, 0), True), ((0, 513, 0, 0), False),
                     ((0, 0, 64, 0), True), ((0, 0, 48, 0), False), ((0, 0, 1 << 13, 0), False)):
        t = pbit.Tune(*tune)
        assert (f(1 << 20, 1, 4, ctypes.addressof(t), ctypes.byref(out)) == 0) == ok, tune


def test_sort_rejects_bad_arguments_without_touching_the_device(so):
    from paper_cs_0511020_gb300 import pbit
    f = so.pbit_sort_list
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                  ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    nr = ctypes.c_int32(0)
    pool = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, 10, 0, 0)
    assert f(ctypes.addressof(pool), 0, 10, 32, 5, ctypes.byref(nr), None, None, 0, None) == 1   # K does not divide M
    assert f(ctypes.addressof(pool), 0, 10, 33, 1, ctypes.byref(nr), None, None, 0, None) == 1   # M > key bits
    assert f(ctypes.addressof(pool), 0, 9, 32, 4, ctypes.byref(nr), None, None, 0, None) == 1    # n != pool size
    assert f(ctypes.addressof(pool), 12, 10, 32, 4, ctypes.byref(nr), None, None, 0, None) == 3  # root out of range
    empty = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, 0, 0, 0)
    assert f(ctypes.addressof(empty), -1, 0, 32, 4, ctypes.byref(nr), None, None, 0, None) == 0
    assert nr.value == -1
    signed_m = pbit.Pool(0x1000, 4, 0x2000, 4, 4, pbit.SIGNED, 10, 0, 0)
    assert f(ctypes.addressof(signed_m), 0, 10, 16, 4, ctypes.byref(nr), None, None, 0, None) == 1
