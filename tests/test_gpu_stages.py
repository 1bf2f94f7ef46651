"""Stage checks through the C ABI (pbit_debug_stage): the ranking against a
serial walk of the list, the first MSD pass against a stable partition of
the ranked order by the top digit (4 and 8 bits wide), and the first pass of
the paper's worked example against the groups it prints."""
import os

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


_VIEW = {1: np.uint8, 2: np.int16, 4: np.int32, 8: np.int64}
_UVIEW = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def _stage(pb, nxt, key, root, M, stage, K=4):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(_VIEW[key.itemsize])).cuda()
    pool = pb.make_pool(d_next, d_key)
    st, idx, k = pb.debug_stage(pool, root, nxt.size, M, stage, K=K)
    torch.cuda.synchronize()
    assert (d_next.cpu().numpy() == nxt).all(), "a stage check must not touch next[]"
    return st, idx.cpu().numpy(), k.cpu().numpy().view(_UVIEW[key.itemsize])


@pytest.mark.parametrize("n", [1, 2, 37, 4097, 20000, 300001])
def test_ranking_matches_a_serial_walk(pb, n):
    nxt, root = I.random_list(n, I.SEED_BASE + 300 + n % 97)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 400 + n % 89)
    st, idx, k = _stage(pb, nxt, key, root, 32, 1)
    assert st == pb.OK, pb.status_string(st)
    order = O.list_order(nxt, root)
    assert (idx == order).all()
    assert (k == key[order]).all()


def test_ranking_of_the_push_built_order(pb):
    n = 50000
    nxt, root = I.push_built_list(n)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 501)
    st, idx, k = _stage(pb, nxt, key, root, 32, 1)
    assert st == pb.OK
    assert (idx == np.arange(n - 1, -1, -1)).all()
    assert (k == key[::-1]).all()


@pytest.mark.parametrize("K", [4, 8])
@pytest.mark.parametrize("n", [100, 4097, 20000, 262147])
def test_first_pass_is_a_stable_partition_by_the_top_digit(pb, n, K):
    """With K = 4 the first pass splits on bits 28..31 into 16 buckets, with
    K = 8 on bits 24..31 into 256 (the GPU digit width follows K)."""
    nxt, root = I.random_list(n, I.SEED_BASE + 600 + n % 83)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 700 + n % 79)
    st, idx, k = _stage(pb, nxt, key, root, 32, 2, K=K)
    assert st == pb.OK, pb.status_string(st)
    order = O.list_order(nxt, root)
    want = order[np.argsort(key[order] >> (32 - K), kind="stable")]
    assert (idx == want).all()
    assert (k == key[want]).all()


def test_worked_example_first_pass(pb):
    """Sec. "The idea of sorting using Pbit": eight one-byte keys, K = 4.  The
    first GPU pass splits on the top four bits; its buckets, read in order,
    must be the groups the paper prints (tests/golden/worked_example.txt)."""
    g = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            a, b = line.split(":", 1)
            g[a.strip()] = b.strip()
    keys = np.array([int(x) for x in g["keys"].split()], dtype=np.uint8)
    nxt, root = I.list_from_order(np.arange(keys.size))
    st, idx, k = _stage(pb, nxt, keys, root, int(g["M"]), 2, K=int(g["K"]))
    assert st == pb.OK, pb.status_string(st)
    printed = [[int(x) for x in grp.split()] for grp in g["pass1"].split("|")]
    assert [int(x) for x in k] == sum(printed, [])
    assert [int(keys[v]) for v in idx] == sum(printed, [])
    # node identity: the two 3s keep their list order (positions 1 and 6)
    assert [int(v) for v in idx if keys[v] == 3] == [1, 6]


def test_stage_arguments(pb):
    nxt, root = I.random_list(100, I.SEED_BASE + 800)
    key = I.uniform_keys(100, 4, I.SEED_BASE + 801)
    one, r1 = I.list_from_order(np.arange(1))
    assert _stage(pb, one, key[:1], r1, 32, 2)[0] == pb.EINVAL  # a single node has nothing to split
    assert _stage(pb, nxt, key, root, 32, 3)[0] == pb.EINVAL
    bad = nxt.copy()
    bad[bad == -1] = root  # a cycle: caught by the ranking's validation
    st, _, _ = _stage(pb, bad, key, root, 32, 1)
    assert st == pb.EBADLIST
