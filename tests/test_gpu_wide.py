"""Parity of the 256-bucket MSD passes (GPU digit widths 5..8 bits) with the
oracle, bit for bit through the C ABI.  The paper's K = 8 and K = 16 (two
8-bit passes per level) select them (Sec. "The length of bit pattern"), and
so does a tune with digit_bits = 8 whatever K is."""
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


def _gpu_sort(pb, nxt, key, root, M, K, flags=0, tune=None):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(np.ascontiguousarray(key).view(_VIEW[key.itemsize])).cuda()
    pool = pb.make_pool(d_next, d_key, flags)
    st, r = pb.sort_pool_list(pool, root, nxt.size, M, K, tune=tune, check=False)
    torch.cuda.synchronize()
    return st, d_next.cpu().numpy(), r


def _check(pb, nxt, key, root, M, K, tune=None):
    st, got, r = _gpu_sort(pb, nxt, key, root, M, K, tune=tune)
    assert st == pb.OK, pb.status_string(st)
    if (M // K) % 2 == 0:
        want, wr, _ = O.pbit_sort(nxt, key, root, M, K)
    else:  # odd number of levels: the literal code is not stable; use the definition
        want, wr = O.stable_sort_definition(nxt, key, root, M)
    assert r == wr
    assert (got == want).all(), f"{(got != want).sum()} next[] entries differ"


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("n", [1, 2, 33, 257, 4095, 4097, 8193, 65537, 300001])
def test_sizes_u32(pb, n, K):
    nxt, root = I.random_list(n, 5000 + n)
    key = I.uniform_keys(n, 4, 5100 + n)
    key[::3] = key[0]
    _check(pb, nxt, key, root, 32, K)


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("kb", [1, 2, 4, 8])
@pytest.mark.parametrize("n", [5000, 200003, 1 << 20])
def test_key_types(pb, kb, n, K):
    if 8 * kb % K:
        pytest.skip("K must divide M")
    nxt, root = I.random_list(n, 5200 + n + kb)
    key = I.uniform_keys(n, kb, 5300 + n + kb)
    _check(pb, nxt, key, root, 8 * kb, K)


@pytest.mark.parametrize("M,K", [(30, 5), (30, 6), (28, 7), (30, 10), (24, 12), (28, 14), (40, 8), (56, 8)])
def test_window_widths(pb, M, K):
    """Windows of 5, 6 and 7 bits, K above 8 split into two windows, and M
    below the key width (bits above M ignored)."""
    n = 150001
    nxt, root = I.random_list(n, 5400 + M + K)
    key = I.uniform_keys(n, 8, 5500 + M + K)
    key[::7] = key[3]
    _check(pb, nxt, key, root, M, K)


def test_tune_digit_bits_8_with_K_4(pb):
    """The tune may widen the GPU digit: same result as the paper's K = 4."""
    n = 400000
    nxt, root = I.random_list(n, 5600)
    key = I.uniform_keys(n, 4, 5601)
    key[::5] = key[11]
    _check(pb, nxt, key, root, 32, 4, tune={"digit_bits": 8})
    _check(pb, nxt, key, root, 32, 8, tune={"digit_bits": 4})


@pytest.mark.parametrize("pattern", ["low18", "mid_const", "hi_lo_only", "two_values", "u64_sparse", "all_equal",
                                     "decreasing"])
def test_constant_windows_and_special_orders(pb, pattern):
    n = 300000
    g = I.rng(5700 + len(pattern))
    nxt, root = I.random_list(n, 5701)
    if pattern == "low18":
        key = g.integers(0, 1 << 18, n, dtype=np.uint32)
    elif pattern == "mid_const":
        key = (g.integers(0, 1 << 6, n, dtype=np.uint32) << np.uint32(26)) | np.uint32(0x5A5A << 8) | \
            g.integers(0, 256, n, dtype=np.uint32)
    elif pattern == "hi_lo_only":
        key = (g.integers(0, 3, n, dtype=np.uint32) << np.uint32(30)) | g.integers(0, 16, n, dtype=np.uint32)
    elif pattern == "two_values":
        key = np.where(g.random(n) < 0.5, 0x10000, 0x10001).astype(np.uint32)
    elif pattern == "all_equal":
        key = np.full(n, 0xABCDEF01, np.uint32)
    elif pattern == "decreasing":
        order = O.list_order(nxt, root)
        key = np.empty(n, np.uint32)
        key[order] = np.arange(n, 0, -1, dtype=np.uint32)
    else:
        key = (g.integers(0, 5, n, dtype=np.uint64) << np.uint64(50)) | \
            (g.integers(0, 1 << 20, n, dtype=np.uint64) << np.uint64(3))
    _check(pb, nxt, key, root, 8 * key.itemsize, 8)


def test_skewed_u64_and_u8(pb):
    n = 1 << 20
    nxt, root = I.random_list(n, 5800)
    _check(pb, nxt, I.zipf_u64_keys(n, 5801), root, 64, 8)
    _check(pb, nxt, I.zipf_u64_keys(n, 5802), root, 64, 16)
    nxt, root = I.random_list(n, 5803)
    _check(pb, nxt, I.uniform_keys(n, 1, 5804), root, 8, 8)


@pytest.mark.parametrize("flags", ["signed", "descending", "float", "float_desc"])
def test_flags(pb, flags):
    n = 200003
    nxt, root = I.random_list(n, 5900)
    if flags.startswith("float"):
        key = I.rng(5901).standard_normal(n).astype(np.float64).view(np.uint64).copy()
        key[::13] = 0
        key[1::17] = np.uint64(1) << np.uint64(63)
        f = pb.FLOAT | (pb.DESCENDING if flags == "float_desc" else 0)
        st, got, r = _gpu_sort(pb, nxt, key, root, 64, 8, flags=f)
        want, wr = O.stable_sort_definition(nxt, key, root, 64, float_keys=True, descending=flags == "float_desc")
    else:
        key = I.uniform_keys(n, 4, 5902)
        key[::4] = key[1]
        f = pb.SIGNED if flags == "signed" else pb.DESCENDING
        st, got, r = _gpu_sort(pb, nxt, key, root, 32, 8, flags=f)
        want, wr = O.stable_sort_definition(nxt, key, root, 32, signed=flags == "signed",
                                            descending=flags == "descending")
    assert st == pb.OK and r == wr and (got == want).all()


def test_batched_K_8(pb):
    lens = I.log_uniform_lengths(300, 4, 17, 6000, 16, 1 << 17)
    lens[5] = 0
    lens[6] = 1
    nxt, key, roots, off = I.batched_pool(lens, 4, 6001)
    roots[5] = -1
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    nr = pb.sort_lists_batched(d_next, d_key, torch.from_numpy(roots).cuda(), torch.from_numpy(off).cuda(),
                               M=32, K=8)
    got = d_next.cpu().numpy()
    nr = nr.cpu().numpy()
    for i in range(lens.size):
        a, b = off[i], off[i + 1]
        if b == a:
            assert nr[i] == -1
            continue
        sub_next = nxt[a:b] - np.where(nxt[a:b] >= 0, a, 0)
        want, wr, _ = O.pbit_sort(sub_next.astype(np.int32), key[a:b], roots[i] - a, 32, 8)
        want = np.where(want >= 0, want + a, -1)
        assert nr[i] == wr + a
        assert (got[a:b] == want).all(), f"list {i}"
