"""Failure detection on the GPU without a fault: a bounded device wait that
is made to run out reports PBIT_ETIMEOUT through the status word, and the
CUDA context stays usable (a sort right after it matches the oracle)."""
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


def test_bounded_wait_gives_up_with_timeout_status(pb):
    for iterations in (1, 64, 1 << 12):
        assert pb.selftest_bounded_wait(iterations) == pb.ETIMEOUT
    # the context is still usable: the next sort is correct
    n = 6000
    nxt, root = I.random_list(n, I.SEED_BASE + 41)
    key = I.uniform_keys(n, 4, I.SEED_BASE + 42)
    want, want_root, _ = O.pbit_sort(nxt, key, root, 32, 4)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    assert pb.sort_list(d_next, d_key, root, M=32, K=4) == want_root
    assert (d_next.cpu().numpy() == want).all()
