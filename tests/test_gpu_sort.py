"""GPU parity: the CUDA path (through the C ABI) against the oracle, bit-exact
on next[] and the root, on seeded inputs of the workloads' shapes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_cs_0511020_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

_NP = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}
_TORCH_VIEW = {1: np.uint8, 2: np.int16, 4: np.int32, 8: np.int64}


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_cs_0511020_gb300 import pbit
    pbit.lib()
    return pbit


def _dev_key(key):
    return torch.from_numpy(np.ascontiguousarray(key).view(_TORCH_VIEW[key.itemsize])).cuda()


def _gpu_sort(pb, nxt, key, root, M, K=4, flags=0, tune=None):
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_key = _dev_key(key)
    pool = pb.make_pool(d_next, d_key, flags)
    st, r = pb.sort_pool_list(pool, root, nxt.size, M, K, tune=tune, check=False)
    torch.cuda.synchronize()
    return st, d_next.cpu().numpy(), r


def _check_vs_oracle(pb, nxt, key, root, M, K=4, tune=None):
    st, got, r = _gpu_sort(pb, nxt, key, root, M, K, tune=tune)
    assert st == pb.OK, pb.status_string(st)
    if (M // K) % 2 == 0:
        want, wr, _ = O.pbit_sort(nxt, key, root, M, K)
    else:  # odd number of levels: the literal code is not stable; use the definition
        want, wr = O.stable_sort_definition(nxt, key, root, M)
    assert r == wr
    assert (got == want).all(), f"{(got != want).sum()} next[] entries differ"


def test_worked_example(pb):
    keys = np.array([21, 3, 209, 14, 156, 47, 3, 214], dtype=np.uint8)
    nxt, root = I.list_from_order(np.arange(8))
    st, got, r = _gpu_sort(pb, nxt, keys, root, 8, 4)
    assert st == pb.OK
    order = O.list_order(got, r)
    assert keys[order].tolist() == [3, 3, 14, 21, 47, 156, 209, 214]
    assert [v for v in order if keys[v] == 3] == [1, 6]


@pytest.mark.parametrize("n", [1, 2, 3, 15, 16, 17, 31, 32, 33, 255, 256, 257, 4095, 4096, 4097,
                               8191, 8192, 8193, 65535, 65537, 300001])
def test_sizes_u32(pb, n):
    nxt, root = I.random_list(n, 1000 + n)
    key = I.uniform_keys(n, 4, 2000 + n)
    key[::3] = key[0]
    _check_vs_oracle(pb, nxt, key, root, 32)


@pytest.mark.parametrize("kb", [1, 2, 4, 8])
@pytest.mark.parametrize("n", [5000, 200003])
def test_key_types(pb, kb, n):
    nxt, root = I.random_list(n, 3000 + n + kb)
    key = I.uniform_keys(n, kb, 4000 + n + kb)
    _check_vs_oracle(pb, nxt, key, root, 8 * kb)


@pytest.mark.parametrize("K", [1, 2, 4, 8, 16])
def test_K_independent(pb, K):
    n = 100000
    nxt, root = I.random_list(n, 51)
    key = I.uniform_keys(n, 4, 52) & np.uint32(0xFFF0FFFF)
    _check_vs_oracle(pb, nxt, key, root, 32, K)


def test_M_below_width(pb):
    n = 70000
    nxt, root = I.random_list(n, 61)
    key = I.uniform_keys(n, 8, 62)
    _check_vs_oracle(pb, nxt, key, root, 40, 4)
    _check_vs_oracle(pb, nxt, key, root, 12, 4)


def test_push_built_and_special(pb):
    n = 150000
    nxt, root = I.push_built_list(n)
    key = I.uniform_keys(n, 4, 71)
    _check_vs_oracle(pb, nxt, key, root, 32)
    # all equal: unchanged
    nxt, root = I.random_list(n, 72)
    st, got, r = _gpu_sort(pb, nxt, np.full(n, 7, np.uint32), root, 32)
    assert st == pb.OK and r == root and (got == nxt).all()
    # strictly decreasing along the list: reversed
    order = O.list_order(nxt, root)
    key = np.empty(n, np.uint32)
    key[order] = np.arange(n, 0, -1, dtype=np.uint32)
    st, got, r = _gpu_sort(pb, nxt, key, root, 32)
    assert st == pb.OK and O.list_order(got, r).tolist() == order[::-1].tolist()


def test_skewed_u64_and_u8(pb):
    n = 1 << 20
    nxt, root = I.random_list(n, 81)
    _check_vs_oracle(pb, nxt, I.zipf_u64_keys(n, 82), root, 64)
    nxt, root = I.random_list(n, 83)
    _check_vs_oracle(pb, nxt, I.uniform_keys(n, 1, 84), root, 8)


def test_aos_pool(pb):
    n = 1 << 20
    nxt, root = I.random_list(n, 91)
    key = I.uniform_keys(n, 4, 92)
    nodes = torch.from_numpy(I.aos_pack(nxt, key)).cuda()
    pool = pb.make_pool_aos(nodes)
    st, r = pb.sort_pool_list(pool, root, n, 32, 4, check=False)
    assert st == pb.OK
    got = nodes[:, 0].cpu().numpy()
    want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
    assert r == wr and (got == want).all()
    assert (nodes[:, 1].cpu().numpy().view(np.uint32) == key).all()


def test_batched(pb):
    lens = I.log_uniform_lengths(300, 4, 17, 101, 16, 1 << 17)
    lens[5] = 0
    lens[6] = 1
    nxt, key, roots, off = I.batched_pool(lens, 4, 102)
    roots[5] = -1
    d_next = torch.from_numpy(nxt.copy()).cuda()
    nr = pb.sort_lists_batched(d_next, _dev_key(key), torch.from_numpy(roots).cuda(),
                               torch.from_numpy(off).cuda(), M=32, K=4)
    got = d_next.cpu().numpy()
    nr = nr.cpu().numpy()
    for i in range(lens.size):
        a, b = off[i], off[i + 1]
        if b == a:
            assert nr[i] == -1
            continue
        sub_next = nxt[a:b] - np.where(nxt[a:b] >= 0, a, 0)
        want, wr, _ = O.pbit_sort(sub_next.astype(np.int32), key[a:b], roots[i] - a, 32, 4)
        want = np.where(want >= 0, want + a, -1)
        assert nr[i] == wr + a
        assert (got[a:b] == want).all(), f"list {i}"


@pytest.mark.parametrize("case", ["cycle", "range", "short", "root"])
def test_malformed_untouched(pb, case):
    n = 50000
    nxt, root = I.random_list(n, 111)
    key = I.uniform_keys(n, 4, 112)
    bad = nxt.copy()
    order = O.list_order(nxt, root)
    if case == "cycle":
        bad[order[-1]] = order[n // 2]
    elif case == "range":
        bad[order[100]] = n + 5
    elif case == "short":
        bad[order[n - 10]] = -1
    else:
        root = n + 3
    d_next = torch.from_numpy(bad.copy()).cuda()
    pool = pb.make_pool(d_next, _dev_key(key))
    st, _ = pb.sort_pool_list(pool, root, n, 32, 4, check=False)
    assert st == pb.EBADLIST
    assert (d_next.cpu().numpy() == bad).all()


def test_bad_arguments(pb):
    n = 100
    nxt, root = I.random_list(n, 121)
    d_next = torch.from_numpy(nxt).cuda()
    pool = pb.make_pool(d_next, _dev_key(I.uniform_keys(n, 4, 122)))
    assert pb.sort_pool_list(pool, root, n, 32, 5, check=False)[0] == pb.EINVAL
    assert pb.sort_pool_list(pool, root, n, 33, 1, check=False)[0] == pb.EINVAL
    assert pb.sort_pool_list(pool, root, n - 1, 32, 4, check=False)[0] == pb.EINVAL


@pytest.mark.parametrize("flags", ["signed", "descending", "signed_desc", "float"])
def test_signed_descending_float(pb, flags):
    n = 120000
    nxt, root = I.random_list(n, 131)
    if flags == "float":
        vals = I.rng(132).standard_normal(n).astype(np.float32)
        vals[::11] = 0.0
        vals[1::97] = -0.0
        key = vals.view(np.uint32)
        f = pb.FLOAT
    else:
        key = I.uniform_keys(n, 4, 133)
        key[::4] = key[1]
        f = {"signed": pb.SIGNED, "descending": pb.DESCENDING,
             "signed_desc": pb.SIGNED | pb.DESCENDING}[flags]
    st, got, r = _gpu_sort(pb, nxt, key, root, 32, 4, flags=f)
    assert st == pb.OK
    if flags == "float":
        want, wr = O.stable_sort_definition(nxt, key, root, 32, float_keys=True)
    else:
        want, wr = O.stable_sort_definition(nxt, key, root, 32, signed="signed" in flags,
                                            descending="desc" in flags)
    assert r == wr and (got == want).all()


def test_doubly_linked(pb):
    n = 90000
    nxt, root = I.random_list(n, 141)
    key = I.uniform_keys(n, 2, 142)
    prev = np.full(n, -1, np.int32)
    order = O.list_order(nxt, root)
    prev[order[1:]] = order[:-1]
    d_next = torch.from_numpy(nxt.copy()).cuda()
    d_prev = torch.from_numpy(prev.copy()).cuda()
    r = pb.sort_list(d_next, _dev_key(key), root, M=16, K=4, prev_t=d_prev)
    got = d_next.cpu().numpy()
    want, wr, _ = O.pbit_sort(nxt, key, root, 16, 4)
    assert r == wr and (got == want).all()
    out = O.list_order(got, r)
    gp = d_prev.cpu().numpy()
    assert gp[out[0]] == -1 and (gp[out[1:]] == out[:-1]).all()


def test_tune_variants(pb):
    n = 400000
    nxt, root = I.random_list(n, 151)
    key = I.uniform_keys(n, 4, 152)
    for tune in ({"smem_cutoff": 64}, {"ruler_stride": 8}, {"ruler_stride": 256},
                 {"smem_cutoff": 256, "ruler_stride": 64}, {"smem_cutoff": 1}):
        _check_vs_oracle(pb, nxt, key, root, 32, tune=tune)


@pytest.mark.parametrize("pattern", ["low18", "mid_const", "hi_lo_only", "two_values", "u64_sparse"])
def test_constant_windows(pb, pattern):
    """Keys whose top or middle digit windows never vary: exercises the
    skipping of constant windows (pending segments re-queued one window lower,
    buckets whose next window is constant)."""
    n = 300000
    g = I.rng(161 + len(pattern))
    nxt, root = I.random_list(n, 162)
    if pattern == "low18":
        key = g.integers(0, 1 << 18, n, dtype=np.uint32)
    elif pattern == "mid_const":
        key = (g.integers(0, 1 << 6, n, dtype=np.uint32) << np.uint32(26)) | np.uint32(0x5A5A << 8) | \
            g.integers(0, 256, n, dtype=np.uint32)
    elif pattern == "hi_lo_only":
        key = (g.integers(0, 3, n, dtype=np.uint32) << np.uint32(30)) | g.integers(0, 16, n, dtype=np.uint32)
    elif pattern == "two_values":
        key = np.where(g.random(n) < 0.5, 0x10000, 0x10001).astype(np.uint32)
    else:
        key = (g.integers(0, 5, n, dtype=np.uint64) << np.uint64(50)) | \
            (g.integers(0, 1 << 20, n, dtype=np.uint64) << np.uint64(3))
    _check_vs_oracle(pb, nxt, key, root, 8 * key.itemsize)


@pytest.mark.parametrize("pack", [1, 2])
@pytest.mark.parametrize("case", ["u8", "u16", "u32", "u64", "signed", "float64", "aos"])
def test_gather_pack_on_and_off(pb, case, pack):
    """The ranking walk reads {next, sort key} records packed by a pre-pass
    (gather_pack = 2) or gathers next[] and key[] itself (1): same result."""
    n = 150001
    nxt, root = I.random_list(n, 171)
    tune = {"gather_pack": pack}
    if case == "aos":
        key = I.uniform_keys(n, 4, 172)
        nodes = torch.from_numpy(I.aos_pack(nxt, key)).cuda()
        st, r = pb.sort_pool_list(pb.make_pool_aos(nodes), root, n, 32, 4, tune=tune, check=False)
        want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
        assert st == pb.OK and r == wr and (nodes[:, 0].cpu().numpy() == want).all()
        return
    if case in ("signed", "float64"):
        if case == "signed":
            key = I.uniform_keys(n, 4, 173)
            flags = pb.SIGNED
            want, wr = O.stable_sort_definition(nxt, key, root, 32, signed=True)
        else:
            vals = I.rng(174).standard_normal(n)
            vals[::7] = 0.0
            key = vals.view(np.uint64)
            flags = pb.FLOAT
            want, wr = O.stable_sort_definition(nxt, key, root, 64, float_keys=True)
        st, got, r = _gpu_sort(pb, nxt, key, root, 8 * key.itemsize, 4, flags=flags, tune=tune)
        assert st == pb.OK and r == wr and (got == want).all()
        return
    kb = {"u8": 1, "u16": 2, "u32": 4, "u64": 8}[case]
    _check_vs_oracle(pb, nxt, I.uniform_keys(n, kb, 175 + kb), root, 8 * kb, tune=tune)


@pytest.mark.parametrize("pattern", ["split", "big_sub_bucket", "wide_span", "narrow_span", "u16_direct",
                                     "u8_direct", "u64_mid", "equal_top"])
@pytest.mark.parametrize("n", [600, 2049, 4096])
def test_mid_size_buckets(pb, pattern, n):
    """Buckets of 513..4096 nodes whose keys vary in at most 16 bits are
    finished by one CTA: one split on the top 4 varying bits then register
    networks per sub-bucket, or least-significant windows over the whole
    span when a sub-bucket would exceed 512 nodes or its network key 32
    bits."""
    g = I.rng(200 + n + len(pattern))
    nxt, root = I.random_list(n, 201 + n)
    M = 32
    if pattern == "split":            # 12 varying bits: split + networks
        key = g.integers(0, 1 << 12, n, dtype=np.uint32)
    elif pattern == "big_sub_bucket":  # 70% share their top varying bits: LSD fallback
        key = g.integers(0, 1 << 14, n, dtype=np.uint32)
        key[g.random(n) < 0.7] &= np.uint32(0x3FF)
    elif pattern == "wide_span":       # bits 16..31 vary: network key too wide, LSD windows
        key = g.integers(0, 1 << 16, n, dtype=np.uint32) << np.uint32(16)
    elif pattern == "narrow_span":     # 3 varying bits: one window
        key = (g.integers(0, 8, n, dtype=np.uint32) << np.uint32(9)) | np.uint32(0x40000001)
    elif pattern == "u16_direct":      # M = 16: the list itself goes to the CTA finish
        key = I.uniform_keys(n, 2, 202 + n)
        M = 16
    elif pattern == "u8_direct":
        key = I.uniform_keys(n, 1, 203 + n)
        M = 8
    elif pattern == "u64_mid":         # 64-bit keys, 16 varying bits in the middle
        key = (g.integers(0, 1 << 16, n, dtype=np.uint64) << np.uint64(20)) | np.uint64(0x5 << 60)
        M = 64
    else:                              # all keys equal in the varying window's top, ties in list order
        key = np.full(n, 0x1234, np.uint32)
        key[::5] = 0x1235
    if (M // 4) % 2 == 0:
        _check_vs_oracle(pb, nxt, key, root, M)
    else:
        st, got, r = _gpu_sort(pb, nxt, key, root, M)
        want, wr = O.stable_sort_definition(nxt, key, root, M)
        assert st == pb.OK and r == wr and (got == want).all()


def test_mid_size_buckets_batched(pb):
    """Many mid-size lists in one batch (the CTA finish takes them from the
    initial plan) next to small and large ones."""
    lens = np.array([513, 4096, 700, 12, 5000, 1, 3000, 4097, 2048, 520] * 6, dtype=np.int64)
    nxt, key, roots, off = I.batched_pool(lens, 2, 210)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    nr = pb.sort_lists_batched(d_next, _dev_key(key), torch.from_numpy(roots).cuda(),
                               torch.from_numpy(off).cuda(), M=16, K=4)
    got, nr = d_next.cpu().numpy(), nr.cpu().numpy()
    for i in range(lens.size):
        a, b = off[i], off[i + 1]
        sub_next = np.where(nxt[a:b] >= 0, nxt[a:b] - a, -1).astype(np.int32)
        want, wr, _ = O.pbit_sort(sub_next, key[a:b], roots[i] - a, 16, 4)
        assert nr[i] == wr + a
        assert (got[a:b] == np.where(want >= 0, want + a, -1)).all(), f"list {i}"


@pytest.mark.parametrize("kb", [4, 8])
def test_mid_size_buckets_both_capacities(pb, kb):
    """Keys of 4 and 8 bytes: buckets of up to 2560 nodes are finished by the
    CTA finish sized for them, larger ones (up to 4096) are deferred to the
    one sized for 4096; a batch with lengths on both sides of 2560."""
    lens = np.array([513, 2559, 2560, 2561, 3000, 4095, 4096, 700, 2048, 1] * 4, dtype=np.int64)
    nxt, key, roots, off = I.batched_pool(lens, kb, 212 + kb)
    d_next = torch.from_numpy(nxt.copy()).cuda()
    nr = pb.sort_lists_batched(d_next, _dev_key(key), torch.from_numpy(roots).cuda(),
                               torch.from_numpy(off).cuda(), M=16, K=4)
    got, nr = d_next.cpu().numpy(), nr.cpu().numpy()
    for i in range(lens.size):
        a, b = off[i], off[i + 1]
        sub_next = np.where(nxt[a:b] >= 0, nxt[a:b] - a, -1).astype(np.int32)
        want, wr, _ = O.pbit_sort(sub_next, key[a:b], roots[i] - a, 16, 4)
        assert nr[i] == wr + a
        assert (got[a:b] == np.where(want >= 0, want + a, -1)).all(), f"list {i}"


@pytest.mark.parametrize("kb", [4, 8])
@pytest.mark.parametrize("n", [600_000, 700_000])
def test_mid_buckets_after_a_pass(pb, n, kb):
    """Keys below 2^20: one 8-bit pass leaves 256 buckets of n / 256 nodes with
    12 bits to sort (about 2340 nodes at 600 000: the smaller CTA finish;
    about 2730 at 700 000: deferred to the larger one)."""
    nxt, root = I.random_list(n, 215 + n)
    dt = np.uint32 if kb == 4 else np.uint64
    key = I.uniform_keys(n, kb, 216 + n) & dt((1 << 20) - 1)
    _check_vs_oracle(pb, nxt, key, root, 8 * kb, tune={"digit_bits": 8})


@pytest.mark.parametrize("n", [1, 2, 33, 1000, 4095, 4096])
@pytest.mark.parametrize("kb", [1, 2, 4, 8])
def test_short_list_kernel(pb, n, kb):
    """Lists of at most 4096 nodes are sorted by one kernel (one CTA per list):
    same result as the oracle, for every key width."""
    nxt, root = I.random_list(n, 220 + n + kb)
    key = I.uniform_keys(n, kb, 221 + n + kb)
    if n > 4:
        key[::7] = key[3]
    _check_vs_oracle(pb, nxt, key, root, 8 * kb)


@pytest.mark.parametrize("variant", ["signed", "descending", "float", "aos", "doubly", "M_below", "push"])
def test_short_list_kernel_variants(pb, variant):
    n = 3001
    nxt, root = I.random_list(n, 230)
    key = I.uniform_keys(n, 4, 231)
    key[::5] = key[2]
    if variant in ("signed", "descending"):
        f = pb.SIGNED if variant == "signed" else pb.DESCENDING
        st, got, r = _gpu_sort(pb, nxt, key, root, 32, 4, flags=f)
        want, wr = O.stable_sort_definition(nxt, key, root, 32, signed=variant == "signed",
                                            descending=variant == "descending")
        assert st == pb.OK and r == wr and (got == want).all()
    elif variant == "float":
        vals = I.rng(232).standard_normal(n).astype(np.float32)
        vals[::9] = -0.0
        st, got, r = _gpu_sort(pb, nxt, vals.view(np.uint32), root, 32, 4, flags=pb.FLOAT)
        want, wr = O.stable_sort_definition(nxt, vals.view(np.uint32), root, 32, float_keys=True)
        assert st == pb.OK and r == wr and (got == want).all()
    elif variant == "aos":
        nodes = torch.from_numpy(I.aos_pack(nxt, key)).cuda()
        st, r = pb.sort_pool_list(pb.make_pool_aos(nodes), root, n, 32, 4, check=False)
        want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
        assert st == pb.OK and r == wr and (nodes[:, 0].cpu().numpy() == want).all()
    elif variant == "doubly":
        prev = np.full(n, -1, np.int32)
        order = O.list_order(nxt, root)
        prev[order[1:]] = order[:-1]
        d_next, d_prev = torch.from_numpy(nxt.copy()).cuda(), torch.from_numpy(prev.copy()).cuda()
        r = pb.sort_list(d_next, _dev_key(key), root, M=32, K=4, prev_t=d_prev)
        got, gp = d_next.cpu().numpy(), d_prev.cpu().numpy()
        want, wr, _ = O.pbit_sort(nxt, key, root, 32, 4)
        assert r == wr and (got == want).all()
        out = O.list_order(got, r)
        assert gp[out[0]] == -1 and (gp[out[1:]] == out[:-1]).all()
    elif variant == "M_below":
        _check_vs_oracle(pb, nxt, I.uniform_keys(n, 8, 233), root, 24)
    else:
        nxt, root = I.push_built_list(n)
        _check_vs_oracle(pb, nxt, key, root, 32)


@pytest.mark.parametrize("case", ["cycle", "range", "short", "root", "self"])
def test_short_list_kernel_malformed_untouched(pb, case):
    n = 2500
    nxt, root = I.random_list(n, 240)
    key = I.uniform_keys(n, 4, 241)
    bad = nxt.copy()
    order = O.list_order(nxt, root)
    if case == "cycle":
        bad[order[-1]] = order[7]
    elif case == "range":
        bad[order[100]] = n + 5
    elif case == "short":
        bad[order[n - 10]] = -1
    elif case == "self":
        bad[order[50]] = order[50]
    else:
        root = n + 3
    d_next = torch.from_numpy(bad.copy()).cuda()
    st, _ = pb.sort_pool_list(pb.make_pool(d_next, _dev_key(key)), root, n, 32, 4, check=False)
    assert st == pb.EBADLIST
    assert (d_next.cpu().numpy() == bad).all()


def _float_edge_keys(n, width, seed):
    """Float bit patterns with every class the IEEE order distinguishes:
    NaNs of both signs (quiet and signaling, several payloads), infinities,
    both zeros, subnormals of both signs, normals, and repeated patterns."""
    g = I.rng(seed)
    dt, ft = (np.uint32, np.float32) if width == 4 else (np.uint64, np.float64)
    fbits = 23 if width == 4 else 52
    ebits = 8 if width == 4 else 11
    sign = dt(1) << dt(8 * width - 1)
    exp_all = dt((1 << ebits) - 1) << dt(fbits)
    quiet = dt(1) << dt(fbits - 1)
    key = (g.standard_normal(n) * 10.0 ** g.integers(-20, 20, n)).astype(ft).view(dt).copy()
    payload = g.integers(1, 1 << 20, n).astype(dt)
    key[0::11] = exp_all | quiet | payload[0::11]            # +qNaN
    key[1::13] = sign | exp_all | quiet | payload[1::13]      # -qNaN
    key[2::17] = exp_all | (payload[2::17] & (quiet - dt(1)))  # +sNaN
    key[3::19] = sign | exp_all | (payload[3::19] & (quiet - dt(1)))  # -sNaN
    key[4::23] = exp_all                                      # +inf
    key[5::29] = sign | exp_all                               # -inf
    key[6::31] = 0                                            # +0
    key[7::37] = sign                                         # -0
    key[8::41] = payload[8::41]                               # +subnormal
    key[9::43] = sign | payload[9::43]                        # -subnormal
    key[10::9] = key[12]                                      # repeated pattern
    return key


@pytest.mark.parametrize("descending", [False, True])
@pytest.mark.parametrize("width", [4, 8])
@pytest.mark.parametrize("n", [3001, 120007])
def test_float_edge_cases_vs_oracle(pb, n, width, descending):
    """IEEE keys with NaN payloads of both signs, infinities, signed zeros and
    subnormals against the oracle's totalOrder reading (short-list kernel at
    3001 nodes, the full pipeline at 120007)."""
    nxt, root = I.random_list(n, 251 + width)
    key = _float_edge_keys(n, width, 252 + width)
    flags = pb.FLOAT | (pb.DESCENDING if descending else 0)
    st, got, r = _gpu_sort(pb, nxt, key, root, 8 * width, 4, flags=flags)
    want, wr = O.stable_sort_definition(nxt, key, root, 8 * width, float_keys=True, descending=descending)
    assert st == pb.OK and r == wr and (got == want).all()
