"""The entry point that allocates nothing (pbit_sort_list_noalloc), for
callers that cannot allocate device memory: through the C ABI its result
must equal pbit_sort_list's bit for bit, on two calls in a row (the scratch
array keeps the previous call's contents, which must not leak into the next
result).  Collected last so that a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _no_alloc(pb, nxt, key, root, M):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(np.ascontiguousarray(key).view(_VIEW[key.itemsize])).cuda()
    pool = pb.make_pool(d_next, d_key)
    nr = ctypes.c_int32(-7)
    torch.cuda.synchronize()
    st = pb.lib().pbit_sort_list_noalloc(ctypes.addressof(pool), int(root), int(nxt.size), int(M), 4,
                                         ctypes.byref(nr), int(torch.cuda.current_stream().cuda_stream))
    return st, d_next.cpu().numpy(), int(nr.value)


@pytest.mark.parametrize("n,kb", [(65536, 4), (50000, 8), (4097, 2), (300, 1)])
def test_no_alloc_equals_workspace_call_twice(pb, n, kb):
    for seed in (901, 902):  # two calls in a row on different lists
        nxt, key, root = _case(n, kb, seed + n + kb)
        want, wr = _with_workspace(pb, nxt, key, root, 8 * kb)
        st, got, r = _no_alloc(pb, nxt, key, root, 8 * kb)
        assert st == pb.OK, pb.status_string(st)
        assert r == wr and (got == want).all()


def test_no_alloc_rejects_longer_lists(pb):
    n = pb.NOALLOC_MAX_NODES + 1
    nxt, key, root = _case(n, 4, 77)
    st, got, _ = _no_alloc(pb, nxt, key, root, 32)
    assert st == pb.ENOMEM
    assert (got == nxt).all()
