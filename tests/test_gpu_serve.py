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


def _submit_many(pb, srv, specs, seed):
    """Submit lists of the given (n, key bytes) back to back; returns the
    requests with their inputs for checking."""
    reqs = []
    for i, (n, kb) in enumerate(specs):
        nxt, root = I.random_list(n, seed + i)
        key = I.uniform_keys(n, kb, seed + 1000 + i)
        d_next, d_key = torch.from_numpy(nxt.copy()).cuda(), _dev(key)
        reqs.append((nxt, key, root, d_next, d_key, kb))
    torch.cuda.synchronize()
    out = []
    for nxt, key, root, d_next, d_key, kb in reqs:
        t = srv.submit(pb.make_pool(d_next, d_key), root, nxt.size, 8 * kb, 4, keep=(d_next, d_key))
        out.append((t, nxt, key, root, d_next, kb))
    return out


def _check_all(pb, srv, reqs, alone=True):
    for t, nxt, key, root, d_next, kb in reqs:
        st, r = srv.wait(t, 300000)
        assert st == pb.OK, pb.status_string(st)
        got = d_next.cpu().numpy()
        want, wr, _ = O.pbit_sort(nxt, key, root, 8 * kb, 4)
        assert r == wr and (got == want).all()
        if alone:
            a, ra = _alone(pb, nxt, key, root, 8 * kb)
            assert ra == r and (a == got).all()


def test_serve_merges_requests_that_arrive_while_the_gpu_is_busy(pb):
    """Continuous batching: while a large request occupies the only stream,
    the short requests that arrive queue up and are launched together, as
    batches of several requests; every result equals the oracle's and the
    same list sorted alone."""
    srv = pb.Server(mem_budget_bytes=4 << 30, streams=1, max_batch=32)
    try:
        g = I.rng(1301)
        specs = [(1 << 22, 4)] + [(int(g.integers(2000, 40000)), 4) for _ in range(120)]
        reqs = _submit_many(pb, srv, specs, 1400)
        _check_all(pb, srv, reqs[:1] + reqs[1::10])
        _check_all(pb, srv, reqs, alone=False)
        stats = srv.stats()
        assert stats["completed"] == len(reqs)
        assert stats["batches"] < len(reqs), stats
        assert stats["max_batch"] > 1, stats
    finally:
        srv.close()


def test_serve_admits_large_requests_as_memory_frees(pb):
    """Admission by the budget: three requests whose workspaces each take
    most of the arena run one after another (never two at once), with short
    requests around them; all finish and the workspace in flight never
    exceeds the budget."""
    n_big = 1 << 21
    ws_big = pb.workspace_size(n_big, 1, 4)
    budget = (ws_big * 3) // 2
    srv = pb.Server(mem_budget_bytes=budget, streams=3, max_batch=8)
    try:
        specs = [(n_big, 4), (3000, 4), (n_big, 4), (9000, 8), (n_big, 4), (700, 2)]
        reqs = _submit_many(pb, srv, specs, 1500)
        _check_all(pb, srv, reqs, alone=False)
        stats = srv.stats()
        assert stats["completed"] == len(reqs)
        assert 0 < stats["peak_bytes"] <= budget
    finally:
        srv.close()


def test_serve_with_a_tune(pb):
    """A server-wide tune (8-bit GPU digits) gives the same results."""
    srv = pb.Server(mem_budget_bytes=2 << 30, streams=2, max_batch=16, tune={"digit_bits": 8})
    try:
        g = I.rng(1601)
        specs = [(int(np.clip(np.floor(2.0 ** (4 + 16 * g.random())), 16, 1 << 20)), int(g.choice([2, 4, 8])))
                 for _ in range(30)]
        reqs = _submit_many(pb, srv, specs, 1700)
        _check_all(pb, srv, reqs, alone=False)
    finally:
        srv.close()
