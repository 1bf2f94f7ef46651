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
    for tune, ok in (((4, 0, 0, 0), True), ((8, 0, 0, 0), True), ((1, 0, 0, 0), True), ((9, 0, 0, 0), False),
                     ((0, 512, 0, 0), True), ((0, 513, 0, 0), False),
                     ((0, 0, 64, 0), True), ((0, 0, 48, 0), False), ((0, 0, 1 << 13, 0), False),
                     ((0, 0, 0, 2), True), ((0, 0, 0, 3), False), ((0, 0, 0, -1), False)):
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


def test_autotune_workspace_covers_every_candidate(so):
    from paper_cs_0511020_gb300 import pbit
    n, L = 1 << 22, 64
    big = pbit.autotune_workspace_size(n, L, 4)
    for d in (4, 8):
        for c in (128, 256, 512):
            for r in (16, 32, 64, 128):
                assert big >= pbit.workspace_size(n, L, 4, {"digit_bits": d, "smem_cutoff": c, "ruler_stride": r})
    assert big >= pbit.workspace_size(n, L, 4)


def test_workspace_without_a_digit_width_covers_every_width(so):
    """A workspace sized with no tune must do for any K the call brings
    (the digit width follows K): it is at least the size of every width."""
    from paper_cs_0511020_gb300 import pbit
    for n, L, kb in ((1 << 20, 1, 4), (1 << 16, 300, 8), (5000, 1, 1)):
        free = pbit.workspace_size(n, L, kb)
        for d in range(1, 9):
            assert free >= pbit.workspace_size(n, L, kb, {"digit_bits": d})


_TUNE_PROBE = """
import json
from paper_cs_0511020_gb300 import pbit
n = 1 << 20
print(json.dumps([pbit.workspace_size(n, 1, 4), pbit.workspace_size(n, 1, 4, {"smem_cutoff": 128, "ruler_stride": 4}),
                  pbit.workspace_size(n, 1, 4, {"smem_cutoff": 512, "ruler_stride": 8}),
                  pbit.workspace_size(1 << 24, 1, 4),
                  pbit.workspace_size(1 << 24, 1, 4, {"smem_cutoff": 512, "ruler_stride": 16})]))
"""


def test_tune_file_is_read_for_its_size_class(so, tmp_path):
    """A tuned choice stored in PBIT_TUNE_FILE is taken (tune = NULL) for its
    size class only: the workspace size then leaves room for it.  Host logic
    only: without a device the library keys entries by its fallback SM count
    148 and compute capability 0."""
    import json
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("device present: the entry below is keyed for the no-device fallback")
    f = tmp_path / "tune.txt"
    f.write_text("garbage line\npbit-tune sms=148 cc=0 kb=4 lg_n=20 lg_l=0 cutoff=128 stride=4 ms=1.5\n")
    env = dict(os.environ, PBIT_TUNE_FILE=str(f))
    out = subprocess.run([sys.executable, "-c", _TUNE_PROBE], env=env, cwd=ROOT, capture_output=True, text=True,
                         check=True).stdout
    none_20, tuned_20, default_20, none_24, default_24 = json.loads(out.strip().splitlines()[-1])
    assert tuned_20 > default_20        # (the built-in default at 2^20 nodes: cutoff 512, stride 8)
    assert none_20 == tuned_20          # room for the stored choice
    assert none_24 == default_24        # another size class: built-in default (stride 16)


def test_more_argument_checks_without_a_device(so):
    """Host-side validation that returns before any CUDA call."""
    from paper_cs_0511020_gb300 import pbit
    L = pbit.lib()
    nr = ctypes.c_int32(7)
    empty = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, 0, 0, 0)
    assert L.pbit_sort_list(ctypes.addressof(empty), 3, 0, 32, 4, ctypes.byref(nr), None, None, 0, None) == pbit.EBADLIST
    big = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, pbit.NOALLOC_MAX_NODES + 1, 0, 0)
    assert L.pbit_sort_list_noalloc(ctypes.addressof(big), 0, pbit.NOALLOC_MAX_NODES + 1, 32, 4, ctypes.byref(nr),
                                    None) == pbit.ENOMEM
    pool = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, 100, 0, 0)
    h = ctypes.c_void_p()
    assert L.pbit_graph_create_single(ctypes.addressof(pool), 0, 100, 32, 5, None, None, 0, ctypes.byref(h)) == pbit.EINVAL
    assert L.pbit_graph_create_single(ctypes.addressof(pool), 100, 100, 32, 4, None, None, 0, ctypes.byref(h)) == pbit.EBADLIST
    assert L.pbit_graph_create_batched(ctypes.addressof(pool), 0, None, None, 32, 4, None, None, None, 0,
                                       ctypes.byref(h)) == pbit.EINVAL
    best = pbit.Tune()
    assert L.pbit_autotune_batched(ctypes.addressof(pool), 1, 0x10, 0x20, 32, 4, 0x30, None, 0, 0, None,
                                   ctypes.addressof(best), None) == pbit.EINVAL  # reps = 0
    assert L.pbit_graph_launch(None, None) == pbit.EINVAL
    assert L.pbit_graph_result(None, None, None) == pbit.EINVAL
    assert L.pbit_graph_node_count(None) == 0
    out = ctypes.c_void_p(0x4000)
    for stage in (0, 3):
        assert L.pbit_debug_stage(ctypes.addressof(pool), 0, 100, 32, 4, stage, None, 0, out, out, None) == pbit.EINVAL
    # stage 2 needs two nodes or more to split
    one = pbit.Pool(0x1000, 4, 0x2000, 4, 4, 0, 1, 0, 0)
    assert L.pbit_debug_stage(ctypes.addressof(one), 0, 1, 32, 4, 2, None, 0, out, out, None) == pbit.EINVAL
    assert L.pbit_debug_stage(ctypes.addressof(pool), 0, 100, 32, 4, 1, None, 0, None, out, None) == pbit.EINVAL
    assert L.pbit_debug_stage(ctypes.addressof(pool), 100, 100, 32, 4, 1, None, 0, out, out, None) == pbit.EBADLIST
    assert L.pbit_selftest_bounded_wait(0, None) == pbit.EINVAL
    assert L.pbit_selftest_bounded_wait((1 << 24) + 1, None) == pbit.EINVAL
