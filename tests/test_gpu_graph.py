"""CUDA-graph replays and the autotuner, against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_cs_0511020_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0511020_gb300 import pbit
    pbit.lib()
    return pbit


def _check_batch(nxt, key, roots, off, got, nr, M=32):
    for i in range(roots.size):
        a, b = int(off[i]), int(off[i + 1])
        if a == b:
            assert nr[i] == -1
            continue
        sub = np.where(nxt[a:b] >= 0, nxt[a:b] - a, -1).astype(np.int32)
        want, wr, _ = O.pbit_sort(sub, key[a:b], int(roots[i]) - a, M, 4)
        assert nr[i] == wr + a, f"list {i}"
        assert (got[a:b] == np.where(want >= 0, want + a, -1)).all(), f"list {i}"


def test_batched_graph_replays_new_data(pb):
    """One capture sorts different batches laid out in the same pool: new
    list orders, new keys and new list lengths (d_offsets) on every replay."""
    P = 400000
    d_next = torch.empty(P, dtype=torch.int32, device="cuda")
    d_key = torch.empty(P, dtype=torch.int32, device="cuda")
    d_roots = torch.empty(200, dtype=torch.int32, device="cuda")
    d_off = torch.empty(201, dtype=torch.int64, device="cuda")
    pool = pb.make_pool(d_next, d_key)
    g = pb.Graph.batched(pool, d_roots, d_off, M=32, K=4)
    assert g.node_count() > 20
    for rep in range(3):
        lens = I.log_uniform_lengths(200, 0, 15, 900 + rep, 1, 1 << 15)
        lens[rep] = 0
        scale = min(1.0, P / lens.sum())
        lens = np.maximum((lens * scale).astype(np.int64), 0)
        nxt, key, roots, off = I.batched_pool(lens, 4, 910 + rep)
        n = nxt.size
        d_next[:n].copy_(torch.from_numpy(nxt))
        d_next[n:].fill_(-5)                     # beyond the last list: must stay untouched
        d_key[:n].copy_(torch.from_numpy(key.view(np.int32)))
        d_roots.copy_(torch.from_numpy(roots))
        d_off.copy_(torch.from_numpy(off))
        g.launch()
        st, _ = g.result()
        assert st == pb.OK
        got = d_next.cpu().numpy()
        assert (got[n:] == -5).all()
        _check_batch(nxt, key, roots, off, got[:n], g.new_roots.cpu().numpy())
    g.close()


def test_single_graph_repeats(pb):
    n = 250001
    nxt, root = I.random_list(n, 920)
    key = I.uniform_keys(n, 8, 921)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int64)).cuda()
    pool = pb.make_pool(d_next, d_key)
    g = pb.Graph.single_list(pool, root, n, 64, 4)
    want, wr, _ = O.pbit_sort(nxt, key, root, 64, 4)
    for _ in range(2):
        d_next.copy_(torch.from_numpy(nxt))
        g.launch()
        st, r = g.result()
        assert st == pb.OK and r == wr
        assert (d_next.cpu().numpy() == want).all()
    g.close()


def test_graph_rejects_bad_list(pb):
    n = 30000
    nxt, root = I.random_list(n, 930)
    key = I.uniform_keys(n, 4, 931)
    bad = nxt.copy()
    order = O.list_order(nxt, root)
    bad[order[-1]] = order[10]  # cycle
    d_next = torch.from_numpy(bad.copy()).cuda()
    g = pb.Graph.single_list(pb.make_pool(d_next, torch.from_numpy(key.view(np.int32)).cuda()), root, n, 32)
    g.launch()
    assert g.result(check=False)[0] == pb.EBADLIST
    assert (d_next.cpu().numpy() == bad).all()
    g.close()


def test_autotune_leaves_pool_and_tunes(pb):
    lens = I.log_uniform_lengths(64, 4, 14, 940, 16, 1 << 14)
    nxt, key, roots, off = I.batched_pool(lens, 4, 941)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    d_roots, d_off = torch.from_numpy(roots).cuda(), torch.from_numpy(off).cuda()
    pool = pb.make_pool(d_next, d_key)
    best, ms = pb.autotune_batched(pool, d_roots, d_off, 32, 4, reps=2)
    assert best["smem_cutoff"] in (128, 256, 512) and best["ruler_stride"] in (16, 32, 64, 128)
    assert ms > 0
    assert (d_next.cpu().numpy() == nxt).all()  # restored
    # tune=None now takes the tuned choice for this size class
    ws_none = pb.workspace_size(nxt.size, lens.size, 4)
    assert ws_none >= pb.workspace_size(nxt.size, lens.size, 4, best)
    st, nr = pb.sort_pool_batched(pool, d_roots, d_off, 32, 4)
    assert st == pb.OK
    _check_batch(nxt, key, roots, off, d_next.cpu().numpy(), nr.cpu().numpy())


def test_single_graph_short_list(pb):
    """A short list's graph holds the one-kernel path; replays equal the oracle."""
    n = 3000
    nxt, root = I.random_list(n, 950)
    key = I.uniform_keys(n, 2, 951)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int16)).cuda()
    g = pb.Graph.single_list(pb.make_pool(d_next, d_key), root, n, 16, 4)
    want, wr, _ = O.pbit_sort(nxt, key, root, 16, 4)
    for _ in range(3):
        d_next.copy_(torch.from_numpy(nxt))
        g.launch()
        st, r = g.result()
        assert st == pb.OK and r == wr and (d_next.cpu().numpy() == want).all()
    assert g.node_count() < 20
    g.close()
