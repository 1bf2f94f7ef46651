"""Request server on the GPU: every result equals the oracle's and the
one-list-at-a-time call's (alone vs in the mix); a malformed request fails
alone; the memory budget is enforced."""
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


def _alone(pb, nxt, key, root, M):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    r = pb.sort_list(d_next, _dev(key), root, M=M, K=4)
    return d_next.cpu().numpy(), r


def test_serve_mix_equals_alone_and_oracle(pb):
    g = I.rng(301)
    srv = pb.Server(mem_budget_bytes=3 << 30, streams=3, max_batch=16)
    reqs = []
    try:
        for i in range(48):
            kb = int(g.choice([2, 4, 4, 8]))
            n = int(np.clip(np.floor(2.0 ** (4 + 14 * g.random())), 16, 1 << 18))
            nxt, root = I.random_list(n, 400 + i)
            key = I.uniform_keys(n, kb, 500 + i)
            if i % 5 == 0:
                key[::3] = key[0]
            d_next, d_key = torch.from_numpy(nxt.copy()).cuda(), _dev(key)
            torch.cuda.synchronize()
            t = srv.submit(pb.make_pool(d_next, d_key), root, n, 8 * kb, 4, keep=(d_next, d_key))
            reqs.append((t, nxt, key, root, d_next, kb))
        for t, nxt, key, root, d_next, kb in reqs:
            st, r = srv.wait(t, 120000)
            assert st == pb.OK, pb.status_string(st)
            got = d_next.cpu().numpy()
            alone, ra = _alone(pb, nxt, key, root, 8 * kb)
            assert r == ra and (got == alone).all()
            want, wr, _ = O.pbit_sort(nxt, key, root, 8 * kb, 4)
            assert r == wr and (got == want).all()
        stats = srv.stats()
        assert stats["completed"] == len(reqs)
        assert stats["batches"] <= len(reqs)
    finally:
        srv.close()


def test_serve_bad_request_fails_alone(pb):
    srv = pb.Server(mem_budget_bytes=1 << 30, streams=1, max_batch=8)
    try:
        items = []
        for i in range(6):
            n = 3000 + 17 * i
            nxt, root = I.random_list(n, 600 + i)
            key = I.uniform_keys(n, 4, 700 + i)
            bad = nxt.copy()
            if i == 3:
                order = O.list_order(nxt, root)
                bad[order[-1]] = order[10]   # cycle
            d_next, d_key = torch.from_numpy(bad.copy()).cuda(), _dev(key)
            items.append((nxt, bad, key, root, d_next, d_key))
        torch.cuda.synchronize()
        tickets = [srv.submit(pb.make_pool(d_next, d_key), root, bad.size, 32, 4, keep=(d_next, d_key))
                   for nxt, bad, key, root, d_next, d_key in items]
        for i, (t, (nxt, bad, key, root, d_next, d_key)) in enumerate(zip(tickets, items)):
            st, r = srv.wait(t, 60000)
            if i == 3:
                assert st == pb.EBADLIST
                assert (d_next.cpu().numpy() == bad).all()
            else:
                assert st == pb.OK
                want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
                assert r == wr and (d_next.cpu().numpy() == want).all()
    finally:
        srv.close()


def test_serve_budget_and_empty(pb):
    srv = pb.Server(mem_budget_bytes=64 << 20, streams=1, max_batch=4)
    try:
        n = 1 << 22
        d_next = torch.zeros(n, dtype=torch.int32, device="cuda")
        d_key = torch.zeros(n, dtype=torch.int32, device="cuda")
        with pytest.raises(pb.PbitError) as ei:
            srv.submit(pb.make_pool(d_next, d_key), 0, n, 32, 4)
        assert ei.value.status == pb.EAGAIN
        e_next = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
        e_key = torch.zeros(1, dtype=torch.int32, device="cuda")[:0]
        t = srv.submit(pb.make_pool(e_next, e_key), -1, 0, 32, 4)
        assert srv.wait(t, 1000) == (pb.OK, -1)
    finally:
        srv.close()


def test_serve_times_and_release(pb):
    srv = pb.Server(mem_budget_bytes=1 << 30, streams=2, max_batch=8)
    try:
        items = []
        for i in range(5):
            n = 5000 + i
            nxt, root = I.random_list(n, 800 + i)
            d_next, d_key = torch.from_numpy(nxt.copy()).cuda(), _dev(I.uniform_keys(n, 4, 810 + i))
            torch.cuda.synchronize()
            items.append(srv.submit(pb.make_pool(d_next, d_key), root, n, 32, 4, keep=(d_next, d_key)))
        for t in items:
            assert srv.wait(t, 60000)[0] == pb.OK
            sub, done = srv.times(t)
            assert 0 < sub <= done
            assert srv.release(t) == pb.OK
            assert srv.poll(t)[0] == pb.EINVAL
            assert srv.release(t) == pb.EINVAL
    finally:
        srv.close()
