"""Parity at the workloads' full sizes, in the launch configuration bench.py
times.  The oracle's literal Pbit is too slow for 10^8 nodes, so the full
outputs are checked with the oracle's property check (a permutation of the
input list, keys non-decreasing, equal keys in input order: together these
determine a stable sort uniquely), and sampled lists are compared with the
literal oracle node for node."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(_VIEW[a.itemsize])).cuda()


def _sort_and_check(pb, nxt, key, root, M):
    d_next = torch.from_numpy(nxt).cuda()
    d_key = _dev(key)
    st, r = pb.sort_pool_list(pb.make_pool(d_next, d_key), root, nxt.size, M, 4, check=False)
    assert st == pb.OK, pb.status_string(st)
    got = d_next.cpu().numpy()
    del d_next, d_key
    torch.cuda.empty_cache()
    O.check_sorted_list(nxt, root, got, r, key, M)
    return got, r


@pytest.mark.parametrize("order", ["random", "push_built"])
def test_2p27_u32_soa(pb, order):
    n = 1 << 27
    nxt, root = I.random_list(n, I.SEED_BASE + 2) if order == "random" else I.push_built_list(n)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 3)
    _sort_and_check(pb, nxt, key, root, 32)


def test_2p26_u64_zipf_and_u8(pb):
    n = 1 << 26
    nxt, root = I.random_list(n, I.SEED_BASE + 30)
    _sort_and_check(pb, nxt, I.zipf_u64_keys(n, I.SEED_BASE + 31), root, 64)
    nxt, root = I.random_list(n, I.SEED_BASE + 32)
    _sort_and_check(pb, nxt, I.uniform_keys(n, 1, I.SEED_BASE + 33), root, 8)


def test_aos_pool_many_relink_windows(pb):
    """An AoS pool {int32 next; uint32 key} of 2^26 + 3 nodes: the relink
    windows of an 8-byte stride hold 2^21 nodes, so this list has 33 of them
    and a last one of 3 nodes; the keys between the links are left as they
    were."""
    n = (1 << 26) + 3
    nxt, root = I.random_list(n, I.SEED_BASE + 50)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 51)
    nodes = torch.from_numpy(np.stack([nxt, key.view(np.int32)], axis=1)).cuda()
    st, r = pb.sort_pool_list(pb.make_pool_aos(nodes), root, n, 32, 4, check=False)
    assert st == pb.OK, pb.status_string(st)
    got = nodes.cpu().numpy()
    del nodes
    torch.cuda.empty_cache()
    assert (got[:, 1].view(np.uint32) == key).all()
    O.check_sorted_list(nxt, root, np.ascontiguousarray(got[:, 0]), r, key, 32)


def test_batched_4096_lists(pb):
    lens = I.config4_lengths(I.SEED_BASE + 4)
    nxt, key, roots, off = I.batched_pool(lens, 4, I.SEED_BASE + 40)
    d_next = torch.from_numpy(nxt).cuda()
    d_key = _dev(key)
    nr = pb.sort_lists_batched(d_next, d_key, torch.from_numpy(roots).cuda(), torch.from_numpy(off).cuda(),
                               M=32, K=4)
    got = d_next.cpu().numpy()
    nr = nr.cpu().numpy()
    del d_next, d_key
    torch.cuda.empty_cache()
    g = I.rng(41)
    sample = np.unique(np.concatenate([g.choice(lens.size, 48, replace=False), [int(np.argmax(lens))]]))
    for i in sample:
        a, b = int(off[i]), int(off[i + 1])
        sub = np.where(nxt[a:b] >= 0, nxt[a:b] - a, -1).astype(np.int32)
        want, wr, _ = O.pbit_sort(sub, key[a:b], int(roots[i]) - a, 32, 4)
        assert nr[i] == wr + a, f"list {i}"
        assert (got[a:b] == np.where(want >= 0, want + a, -1)).all(), f"list {i}"


def test_served_request_stream_sample(pb):
    _, lengths, kb = I.config5_requests(40, I.SEED_BASE + 5)
    srv = pb.Server(mem_budget_bytes=16 << 30, streams=4, max_batch=64)
    items = []
    try:
        for i, (n, w) in enumerate(zip(lengths, kb)):
            n, w = int(n), int(w)
            nxt, root = I.random_list(n, I.SEED_BASE + 500 + i)
            key = I.uniform_keys(n, w, I.SEED_BASE + 600 + i)
            d_next, d_key = torch.from_numpy(nxt.copy()).cuda(), _dev(key)
            torch.cuda.synchronize()
            t = srv.submit(pb.make_pool(d_next, d_key), root, n, 8 * w, 4, keep=(d_next, d_key))
            items.append((t, nxt, key, root, d_next, 8 * w))
        for t, nxt, key, root, d_next, M in items:
            st, r = srv.wait(t, 300000)
            assert st == pb.OK, pb.status_string(st)
            O.check_sorted_list(nxt, root, d_next.cpu().numpy(), r, key, M)
    finally:
        srv.close()
