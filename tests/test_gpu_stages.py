"""Stage checks through the C ABI (pbit_debug_stage): the ranking against a
serial walk of the list, and the first MSD pass against a stable partition
of the ranked order by the top 4-bit digit."""
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


def _stage(pb, nxt, key, root, M, stage):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    pool = pb.make_pool(d_next, d_key)
    st, idx, k = pb.debug_stage(pool, root, nxt.size, M, stage)
    torch.cuda.synchronize()
    assert (d_next.cpu().numpy() == nxt).all(), "a stage check must not touch next[]"
    return st, idx.cpu().numpy(), k.cpu().numpy().view(np.uint32)


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


@pytest.mark.parametrize("n", [4097, 20000, 262147])
def test_first_pass_is_a_stable_partition_by_the_top_digit(pb, n):
    nxt, root = I.random_list(n, I.SEED_BASE + 600 + n % 83)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 700 + n % 79)
    st, idx, k = _stage(pb, nxt, key, root, 32, 2)
    assert st == pb.OK, pb.status_string(st)
    order = O.list_order(nxt, root)
    want = order[np.argsort(key[order] >> 28, kind="stable")]
    assert (idx == want).all()
    assert (k == key[want]).all()


def test_stage_arguments(pb):
    nxt, root = I.random_list(100, I.SEED_BASE + 800)
    key = I.uniform_keys(100, 4, I.SEED_BASE + 801)
    assert _stage(pb, nxt, key, root, 32, 2)[0] == pb.EINVAL  # no global pass for 100 nodes
    assert _stage(pb, nxt, key, root, 32, 3)[0] == pb.EINVAL
    bad = nxt.copy()
    bad[bad == -1] = root  # a cycle: caught by the ranking's validation
    st, _, _ = _stage(pb, bad, key, root, 32, 1)
    assert st == pb.EBADLIST
