"""The entry point that allocates nothing (pbit_sort_list_noalloc).

Some callers cannot allocate device memory when they sort: their process's
allocator has handed the device's memory to a framework pool, or they sort
inside a loop that cannot afford an allocation and its synchronization, or
their own API has no room for a workspace.  This entry point keeps its
scratch in a fixed array inside the library.  Through the C ABI its result
must equal the oracle's and pbit_sort_list's bit for bit, on two calls in a
row (the array keeps the previous call's contents, which must not leak into
the next result), and once warmed up a call must take no device memory.
Collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_cs_0511020_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu
_VIEW = {1: np.uint8, 2: np.int16, 4: np.int32, 8: np.int64}


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0511020_gb300 import pbit
    pbit.lib()
    return pbit


def _case(n, kb, seed):
    nxt, root = I.random_list(n, seed)
    key = I.uniform_keys(n, kb, seed + 1)
    key[::5] = key[2]
    return nxt, key, root


def _with_workspace(pb, nxt, key, root, M):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(np.ascontiguousarray(key).view(_VIEW[key.itemsize])).cuda()
    st, r = pb.sort_pool_list(pb.make_pool(d_next, d_key), root, nxt.size, M, 4, check=False)
    assert st == pb.OK
    return d_next.cpu().numpy(), r


def _call(pb, pool, root, n, M):
    nr = ctypes.c_int32(-7)
    st = pb.lib().pbit_sort_list_noalloc(ctypes.addressof(pool), int(root), int(n), int(M), 4,
                                         ctypes.byref(nr), int(torch.cuda.current_stream().cuda_stream))
    return st, int(nr.value)


def _no_alloc(pb, nxt, key, root, M):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(np.ascontiguousarray(key).view(_VIEW[key.itemsize])).cuda()
    pool = pb.make_pool(d_next, d_key)
    torch.cuda.synchronize()
    st, r = _call(pb, pool, root, nxt.size, M)
    return st, d_next.cpu().numpy(), r


# (65536, 8): the largest list with the widest key, whose workspace sets the
# size of the array
@pytest.mark.parametrize("n,kb", [(65536, 8), (65536, 4), (50000, 8), (4097, 2), (300, 1)])
def test_no_alloc_equals_oracle_and_workspace_call_twice(pb, n, kb):
    for seed in (901, 902):  # two calls in a row on different lists
        nxt, key, root = _case(n, kb, seed + n + kb)
        want, wr, _ = O.pbit_sort(nxt, key, root, 8 * kb, 4)
        st, got, r = _no_alloc(pb, nxt, key, root, 8 * kb)
        assert st == pb.OK, pb.status_string(st)
        assert r == wr and (got == want).all(), "differs from the oracle"
        ws_next, ws_root = _with_workspace(pb, nxt, key, root, 8 * kb)
        assert ws_root == r and (ws_next == got).all(), "differs from pbit_sort_list"


def test_no_alloc_aos_pool_twice(pb):
    n = 30000
    for seed in (911, 912):
        nxt, key, root = _case(n, 4, seed)
        want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
        nodes = torch.from_numpy(I.aos_pack(nxt, key)).cuda()
        pool = pb.make_pool_aos(nodes)
        torch.cuda.synchronize()
        st, r = _call(pb, pool, root, n, 32)
        assert st == pb.OK, pb.status_string(st)
        got = nodes.cpu().numpy().reshape(-1, 2)[:, 0].copy()
        assert r == wr and (got == want).all()


def test_no_alloc_takes_no_device_memory_after_warm_up(pb):
    n = 40000
    nxt, key, root = _case(n, 4, 921)
    st, _, _ = _no_alloc(pb, nxt, key, root, 32)  # warm-up: kernels and the array are loaded
    assert st == pb.OK
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    pool = pb.make_pool(d_next, d_key)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st, r = _call(pb, pool, root, n, 32)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert st == pb.OK
    assert free1 == free0, f"device memory changed by {free0 - free1} bytes"
    want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
    assert r == wr and (d_next.cpu().numpy() == want).all()


def test_no_alloc_rejects_longer_lists(pb):
    n = pb.NOALLOC_MAX_NODES + 1
    nxt, key, root = _case(n, 4, 77)
    st, got, _ = _no_alloc(pb, nxt, key, root, 32)
    assert st == pb.ENOMEM
    assert (got == nxt).all()
