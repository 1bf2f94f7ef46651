"""The host-buffer call (pbit_sort_list_host): the pool lives in host memory,
the call copies it to the device, sorts, and copies next[] back (window by
window, each as soon as its relink kernel has run).  Results are compared
with the oracle node for node."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_cs_0511020_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0511020_gb300 import pbit
    pbit.lib()
    return pbit


def _host_sort(pb, nxt, key, root, M, pinned=True, tune=None):
    h_next = torch.from_numpy(nxt.copy())
    h_key = torch.from_numpy(np.ascontiguousarray(key).view(np.int32))
    if pinned:
        h_next, h_key = h_next.pin_memory(), h_key.pin_memory()
    pool = pb.host_pool(h_next, h_key)
    st, r = pb.sort_pool_list_host(pool, root, nxt.size, M, 4, tune=tune, check=False)
    torch.cuda.synchronize()
    return st, h_next.numpy(), r


@pytest.mark.parametrize("n", [3000, 300_001, (1 << 23) + 7])
@pytest.mark.parametrize("tune", [None, {"digit_bits": 8}])
def test_host_call_matches_oracle(pb, n, tune):
    """3000 nodes: the one-kernel short-list path (no relink windows);
    300 001: one window; 2^23 + 7: three windows of 2^22 nodes."""
    nxt, root = I.random_list(n, 300 + n)
    key = I.uniform_keys(n, 4, 301 + n)
    st, got, r = _host_sort(pb, nxt, key, root, 32, tune=tune)
    assert st == pb.OK, pb.status_string(st)
    if n <= 300_001:
        want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
    else:
        want, wr = O.stable_sort_definition(nxt, key, root, 32)
    assert r == wr
    assert (got == want).all(), f"{(got != want).sum()} next[] entries differ"


def test_host_call_pageable(pb):
    """Pageable (not pinned) host arrays give the same result."""
    n = 200_003
    nxt, root = I.random_list(n, 310)
    key = I.uniform_keys(n, 4, 311)
    st, got, r = _host_sort(pb, nxt, key, root, 32, pinned=False)
    want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
    assert st == pb.OK and r == wr and (got == want).all()


def test_host_call_aos(pb):
    """An AoS host pool {int32 next; uint32 key}: next[] is sorted, the keys
    between the links come back unchanged."""
    n = 300_007
    nxt, root = I.random_list(n, 320)
    key = I.uniform_keys(n, 4, 321)
    nodes = torch.from_numpy(np.stack([nxt, key.view(np.int32)], axis=1).copy()).pin_memory()
    base = nodes.data_ptr()
    pool = pb.Pool(base, 8, base + 4, 8, 4, 0, n, 0, 0)
    st, r = pb.sort_pool_list_host(pool, root, n, 32, 4, check=False)
    torch.cuda.synchronize()
    want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
    got = nodes.numpy()
    assert st == pb.OK and r == wr
    assert (got[:, 0] == want).all()
    assert (got[:, 1].view(np.uint32) == key).all()


def test_host_call_bad_list_leaves_next(pb):
    """A cycle is reported and the host next[] is left as it was."""
    n = 300_001
    nxt, root = I.random_list(n, 330)
    order = [root]
    for _ in range(1000):
        order.append(int(nxt[order[-1]]))
    bad = nxt.copy()
    bad[order[-1]] = order[10]  # the walk from the root meets node order[10] again
    st, got, _ = _host_sort(pb, bad, I.uniform_keys(n, 4, 331), root, 32)
    assert st == pb.EBADLIST
    assert (got == bad).all()
