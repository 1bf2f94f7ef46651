"""The seeded input generators against the recipes they state (CPU): every
list is one list over exactly its pool range, the push-built order is the
one pushing builds, key ranges and the Zipf mix hold, and the batched and
request-stream workloads have their stated shape.  Both the oracle and the
GPU path take their inputs from these generators."""
import numpy as np

from paper_cs_0511020_gb300 import inputs as I


def _walk(nxt, root):
    out = []
    v = root
    while v != -1:
        out.append(v)
        assert len(out) <= nxt.size, "cycle"
        v = int(nxt[v])
    return np.array(out, dtype=np.int64)


def test_random_list_is_one_list_over_the_whole_pool():
    for n in (1, 2, 17, 5000):
        nxt, root = I.random_list(n, I.SEED_BASE + n)
        order = _walk(nxt, root)
        assert order.size == n and np.array_equal(np.sort(order), np.arange(n))
    a, ra = I.random_list(1000, 7)
    b, rb = I.random_list(1000, 7)
    c, _ = I.random_list(1000, 8)
    assert ra == rb and np.array_equal(a, b) and not np.array_equal(a, c)


def test_push_built_order():
    nxt, root = I.push_built_list(6)
    assert root == 5 and nxt.tolist() == [-1, 0, 1, 2, 3, 4]
    assert _walk(nxt, root).tolist() == [5, 4, 3, 2, 1, 0]
    assert I.push_built_list(0)[1] == -1


def test_list_from_order_leaves_other_nodes_off_the_list():
    nxt, root = I.list_from_order(np.array([4, 1, 6]), pool_size=8)
    assert root == 4 and _walk(nxt, root).tolist() == [4, 1, 6]
    assert all(nxt[v] == -1 for v in (0, 2, 3, 5, 7))
    empty, r = I.list_from_order(np.array([], dtype=np.int32))
    assert r == -1 and empty.size == 0


def test_uniform_keys_cover_the_width():
    for kb, dt in ((1, np.uint8), (2, np.uint16), (4, np.uint32), (8, np.uint64)):
        k = I.uniform_keys(200000, kb, 3)
        assert k.dtype == dt
        if kb == 1:  # every value appears
            assert np.unique(k).size == 256
        top = np.iinfo(dt).max
        assert k.max() > top - top // 64 and k.min() < top // 64  # the range's both ends are reached
    assert np.array_equal(I.uniform_keys(100, 4, 5), I.uniform_keys(100, 4, 5))


def test_zipf_keys_constant_top_half_and_top_rank_share():
    n = 1 << 18
    k = I.zipf_u64_keys(n, 11)
    assert k.dtype == np.uint64
    assert np.all((k >> np.uint64(32)) == np.uint64(0xA5A5A5A5))
    vals, counts = np.unique(k, return_counts=True)
    assert vals.size <= 1024
    # the most frequent value carries the Zipf(1.1) mass of rank 1 over 1024 ranks
    p1 = 1.0 / np.sum(1.0 / np.arange(1, 1025, dtype=np.float64) ** 1.1)
    share = counts.max() / n
    assert abs(share - p1) < 4 * np.sqrt(p1 * (1 - p1) / n)
    assert 0.15 < p1 < 0.21  # about a fifth of all nodes hold one value


def test_aos_pack_round_trip():
    nxt, _ = I.random_list(50, 1)
    key = I.uniform_keys(50, 4, 2)
    a = I.aos_pack(nxt, key)
    assert a.shape == (50, 2) and a.dtype == np.int32
    assert np.array_equal(a[:, 0], nxt) and np.array_equal(a[:, 1].view(np.uint32), key)


def test_batched_pool_lists_own_their_ranges():
    lengths = np.array([0, 1, 5, 0, 33, 2])
    nxt, key, roots, off = I.batched_pool(lengths, 4, 21)
    assert off.tolist() == [0, 0, 1, 6, 6, 39, 41] and key.size == 41
    for i, ln in enumerate(lengths):
        if ln == 0:
            assert roots[i] == -1
            continue
        order = _walk(nxt, int(roots[i]))
        assert np.array_equal(np.sort(order), np.arange(off[i], off[i + 1]))


def test_batched_lengths_log_uniform():
    ln = I.config4_lengths(I.SEED_BASE + 4)
    assert ln.size == 4096 and ln.min() >= 16 and ln.max() <= 1 << 20
    e = np.log2(ln)
    assert abs(np.median(e) - 12.0) < 0.5  # log-uniform exponent over [4, 20]
    assert abs(np.mean(e < 8) - 0.25) < 0.04


def test_request_stream_shape():
    t, ln, kb = I.config5_requests(20000, I.SEED_BASE + 5)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.5e-3) < 0.05e-3
    assert ln.min() >= 16 and ln.max() <= 1 << 24
    assert set(np.unique(kb).tolist()) <= {2, 4, 8}
    frac = np.array([np.mean(kb == w) for w in (2, 4, 8)])
    assert np.all(np.abs(frac - np.array([0.25, 0.5, 0.25])) < 0.02)
