"""Pins of the oracle against facts that do not come from the oracle itself:
the paper's worked example and storage bound (tests/golden/), a library
stable sort (Python's ``sorted``) by brute force on tiny lists, closed-form
special cases, invariants and the paper's linearity counters."""
import itertools
import os
import random

import numpy as np
import pytest

from oracle import oracle as O
from paper_cs_0511020_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(":", 1)
            out[k.strip()] = v.strip()
    return out


def _py_stable(order, key, M, signed=False, descending=False):
    """Independent restatement with Python's stable ``sorted``."""
    width = 8 * key.itemsize

    def val(v):
        x = int(key[v]) & ((1 << width) - 1)
        if signed:
            return x - (1 << width) if x >> (width - 1) else x
        return x & ((1 << M) - 1)

    return sorted(order, key=val, reverse=False) if not descending else \
        [v for _, v in sorted(((-val(v), i), v) for i, v in enumerate(order))]


def _walk(nxt, root):
    out, v = [], root
    while v != -1:
        out.append(v)
        v = int(nxt[v])
        assert len(out) <= len(nxt)
    return out


# ---------------------------------------------------------------- worked example
def test_worked_example_final_order():
    g = _golden("worked_example.txt")
    keys = np.array([int(x) for x in g["keys"].split()], dtype=np.uint8)
    nxt, root = I.list_from_order(np.arange(keys.size))
    out, r, cnt = O.pbit_sort(nxt, keys, root, int(g["M"]), int(g["K"]))
    order = _walk(out, r)
    assert [int(keys[v]) for v in order] == [int(x) for x in g["sorted"].split()]
    # node identity: the two 3s (list positions 1 and 6) stay in list order
    assert [v for v in order if keys[v] == 3] == [1, 6]
    assert cnt["merges"] == keys.size and cnt["splits"] == keys.size * 2


def test_worked_example_split_groups():
    """First split of the example: printed groups {3,14,3}|{21}|{47}|{156}|{209,214}.
    The push-to-front split holds each bucket in reverse list order."""
    g = _golden("worked_example.txt")
    keys = np.array([int(x) for x in g["keys"].split()], dtype=np.uint8)
    nxt, root = I.list_from_order(np.arange(keys.size))
    buckets = O.split_once(nxt, keys, root, 8, 4)
    printed = [[int(x) for x in grp.split()] for grp in g["pass1"].split("|")]
    got = [[int(keys[v]) for v in reversed(b)] for b in buckets if b]
    assert got == printed
    # second split, inside each first-level group, on the low nibble
    printed2 = [[[int(x) for x in sub.split()] for sub in grp.split("|")]
                for grp in g["pass2"].split("||")]
    # Reading: the paper prints the two 3s as {3} | {3}, but both have low
    # nibble 3 and share one bucket; so the flattened order must match and
    # every printed sub-group must lie inside one bucket.
    for grp_nodes, want in zip([list(reversed(b)) for b in buckets if b], printed2):
        sub_keys = keys[grp_nodes]
        snxt, sroot = I.list_from_order(np.arange(len(grp_nodes)))
        sb = O.split_once(snxt, sub_keys, sroot, 4, 4)
        got2 = [[int(sub_keys[v]) for v in reversed(b)] for b in sb if b]
        assert sum(got2, []) == sum(want, [])
        for sub in want:
            assert any(all(x in b for x in sub) for b in got2)


def test_storage_bound_depth():
    """T = (Omega*4 + 3*4) * depth + 8 with depth = M/K recursion levels."""
    for line in open(os.path.join(GOLDEN, "storage_bound.txt")):
        if line.startswith("#") or not line.strip():
            continue
        M, K, T = (int(x) for x in line.split())
        n = 64
        kb = max(1, M // 8)
        keys = I.uniform_keys(n, kb, 7)
        nxt, root = I.random_list(n, 8)
        _, _, cnt = O.pbit_sort(nxt, keys, root, M, K)
        assert cnt["depth"] == M // K
        assert ((1 << K) * 4 + 12) * cnt["depth"] + 8 == T


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("n", [0, 1, 2, 3, 4])
def test_brute_force_all_orders_small_alphabet(n):
    alphabet = [0, 1, 0x7F, 0xFF]
    for perm in itertools.permutations(range(n)):
        nxt, root = I.list_from_order(np.array(perm, dtype=np.int32), n)
        for tup in itertools.product(alphabet, repeat=n):
            keys = np.array(tup, dtype=np.uint8)
            out, r, _ = O.pbit_sort(nxt, keys, root, 8, 4)
            want = _py_stable(list(perm), keys, 8)
            assert _walk(out, r) == want


def test_brute_force_random_tuples():
    rnd = random.Random(11)
    for _ in range(3000):
        n = rnd.randint(5, 12)
        kb = rnd.choice([1, 2, 4, 8])
        K = rnd.choice([k for k in (1, 2, 4, 8) if (8 * kb) % k == 0 and ((8 * kb) // k) % 2 == 0])
        M = 8 * kb
        perm = list(range(n))
        rnd.shuffle(perm)
        keys = np.array([rnd.choice([0, 1, 2, rnd.getrandbits(M)]) for _ in range(n)],
                        dtype=I._UINT[kb])
        nxt, root = I.list_from_order(np.array(perm, dtype=np.int32), n)
        out, r, cnt = O.pbit_sort(nxt, keys, root, M, K)
        assert _walk(out, r) == _py_stable(perm, keys, M)
        assert cnt["merges"] == n and cnt["splits"] == n * (M // K)


# ---------------------------------------------------------------- closed forms
def test_already_sorted_unchanged():
    n = 5000
    keys = np.sort(I.uniform_keys(n, 4, 3))
    order = I.rng(4).permutation(n).astype(np.int32)
    k2 = np.empty_like(keys)
    k2[order] = keys                      # keys ascending along the list
    nxt, root = I.list_from_order(order)
    out, r, _ = O.pbit_sort(nxt, k2, root, 32, 4)
    assert r == root and (out == nxt).all()


def test_all_equal_unchanged():
    n = 3000
    nxt, root = I.random_list(n, 5)
    keys = np.full(n, 0xDEADBEEF, dtype=np.uint32)
    out, r, _ = O.pbit_sort(nxt, keys, root, 32, 4)
    assert r == root and (out == nxt).all()


def test_strictly_decreasing_reversed():
    n = 4096
    nxt, root = I.random_list(n, 6)
    order = _walk(nxt, root)
    keys = np.empty(n, dtype=np.uint32)
    keys[np.array(order)] = np.arange(n - 1, -1, -1, dtype=np.uint32) * 977
    out, r, _ = O.pbit_sort(nxt, keys, root, 32, 4)
    assert _walk(out, r) == order[::-1]


def test_high_bits_ignored_below_M():
    n = 2000
    nxt, root = I.random_list(n, 9)
    keys = I.uniform_keys(n, 4, 10)
    out16, r16, _ = O.pbit_sort(nxt, keys, root, 16, 4)
    low = keys & np.uint32(0xFFFF)
    outl, rl, _ = O.pbit_sort(nxt, low, root, 32, 4)
    assert r16 == rl and (out16 == outl).all()


def test_empty_and_single():
    nxt = np.full(4, -1, dtype=np.int32)
    out, r, cnt = O.pbit_sort(nxt, np.zeros(4, np.uint32), -1, 32, 4)
    assert r == -1 and (out == nxt).all() and cnt["length"] == 0
    out, r, _ = O.pbit_sort(nxt, np.arange(4, dtype=np.uint32), 2, 32, 4)
    assert r == 2 and (out == nxt).all()


# ---------------------------------------------------------------- invariants / counters
@pytest.mark.parametrize("kb,M,K", [(1, 8, 4), (2, 16, 4), (4, 32, 4), (8, 64, 4), (4, 32, 8),
                                    (4, 32, 2), (8, 64, 16), (4, 24, 4)])
def test_invariants_and_counters(kb, M, K):
    n = 20000
    nxt, root = I.random_list(n, 100 + kb + K)
    keys = I.uniform_keys(n, kb, 200 + M)
    keys[::7] = keys[3]                   # plenty of equal keys
    out, r, cnt = O.pbit_sort(nxt, keys, root, M, K)
    O.check_sorted_list(nxt, root, out, r, keys, M)
    assert cnt["merges"] == n                    # Sec. 5.1: count always equals n
    assert cnt["splits"] == n * (M // K)         # Sec. 3: (M/K) n split steps
    d_out, d_r = O.stable_sort_definition(nxt, keys, root, M)
    assert d_r == r and (d_out == out).all()


def test_nodes_off_the_list_untouched():
    n, pool = 1000, 1500
    order = I.rng(21).permutation(pool)[:n].astype(np.int32)
    nxt, root = I.list_from_order(order, pool)
    nxt[np.setdiff1d(np.arange(pool), order)] = 1234
    keys = I.uniform_keys(pool, 4, 22)
    out, r, _ = O.pbit_sort(nxt, keys, root, 32, 4)
    O.check_sorted_list(nxt, root, out, r, keys, 32)


def test_cross_K_identical_when_M_over_K_even():
    n = 10000
    nxt, root = I.random_list(n, 31)
    keys = (I.uniform_keys(n, 4, 32) & np.uint32(0xFF00FF0F))
    ref = O.pbit_sort(nxt, keys, root, 32, 4)[:2]
    for K in (1, 2, 8, 16):
        out, r, _ = O.pbit_sort(nxt, keys, root, 32, K)
        assert r == ref[1] and (out == ref[0]).all()


def test_odd_M_over_K_reverses_equal_keys():
    """Reading of the paper: the push-to-front split reverses equal digits at
    every level, so with an odd number of levels (K = M = 8) equal keys come
    out in reverse list order, while keys themselves are ascending."""
    n = 3000
    nxt, root = I.random_list(n, 41)
    keys = I.uniform_keys(n, 1, 42)
    out, r, _ = O.pbit_sort(nxt, keys, root, 8, 8)
    order_in = _walk(nxt, root)
    rank = {v: i for i, v in enumerate(order_in)}
    order = _walk(out, r)
    ks = [int(keys[v]) for v in order]
    assert ks == sorted(ks)
    for a, b in zip(order, order[1:]):
        if keys[a] == keys[b]:
            assert rank[a] > rank[b]


def test_malformed_lists_rejected():
    nxt = np.array([1, 2, 0, -1], dtype=np.int32)          # cycle 0->1->2->0
    with pytest.raises(O.OracleError):
        O.pbit_sort(nxt, np.zeros(4, np.uint32), 0, 32, 4)
    nxt = np.array([1, 7, -1], dtype=np.int32)              # index out of range
    with pytest.raises(O.OracleError):
        O.pbit_sort(nxt, np.zeros(3, np.uint32), 0, 32, 4)
    with pytest.raises(ValueError):
        O.pbit_sort(np.array([-1], np.int32), np.zeros(1, np.uint32), 0, 32, 5)


# ---------------------------------------------------------------- signed / descending
@pytest.mark.parametrize("signed,descending", [(False, True), (True, False), (True, True)])
def test_signed_and_descending_vs_python_sorted(signed, descending):
    rnd = random.Random(5 + signed * 2 + descending)
    for _ in range(400):
        n = rnd.randint(0, 40)
        kb = rnd.choice([1, 2, 4, 8])
        M = 8 * kb
        perm = list(range(n))
        rnd.shuffle(perm)
        keys = np.array([rnd.choice([0, 1, (1 << M) - 1, 1 << (M - 1), rnd.getrandbits(M)])
                         for _ in range(n)], dtype=I._UINT[kb])
        nxt, root = I.list_from_order(np.array(perm, dtype=np.int32), n)
        d_out, d_r = O.stable_sort_definition(nxt, keys, root, M, signed, descending)
        assert _walk(d_out, d_r) == _py_stable(perm, keys, M, signed, descending)
        out, r, _ = O.pbit_sort(nxt, keys, root, M, 4, signed, descending)
        # the literal code orders keys correctly; equal keys follow the parity
        # of its reversals, so compare key sequences
        assert [int(keys[v]) for v in _walk(out, r)] == \
            [int(keys[v]) for v in _walk(d_out, d_r)]


def test_check_sorted_list_catches_planted_mistakes():
    """The any-size property check must reject a plausible wrong answer."""
    n = 5000
    nxt, root = I.random_list(n, 51)
    keys = I.uniform_keys(n, 2, 52) & np.uint16(0xF0FF)
    good, r = O.stable_sort_definition(nxt, keys, root, 16)
    O.check_sorted_list(nxt, root, good, r, keys, 16)
    order = _walk(good, r)
    # swap two equal-key neighbours (a stability error)
    i = next(i for i in range(n - 1) if keys[order[i]] == keys[order[i + 1]])
    bad_order = order[:i] + [order[i + 1], order[i]] + order[i + 2:]
    bad, br = O.relink(nxt, np.array(bad_order, dtype=np.int32))
    with pytest.raises(AssertionError):
        O.check_sorted_list(nxt, root, bad, br, keys, 16)
    # drop the last node (a length error)
    bad, br = O.relink(nxt, np.array(order[:-1], dtype=np.int32))
    with pytest.raises(AssertionError):
        O.check_sorted_list(nxt, root, bad, br, keys, 16)


# ------------------------------------------------------------- float keys
# Sec. "Floating-point numbers sorting": the paper sorts floats by mantissa and
# then stably by characteristic.  The oracle's reading (IEEE 754 totalOrder,
# written from the decoded fields) is pinned three ways: an example whose
# order is worked out by hand from the IEEE definition, Python's ``sorted``
# on values decoded by ``struct``, and the paper's own two-step recipe, which
# is right for non-negative values.
import struct  # noqa: E402

_F32 = {"+1": 0x3F800000, "-0": 0x80000000, "+qnan": 0x7FC00000, "-inf": 0xFF800000, "+0": 0x00000000,
        "-snan1": 0xFF800001, "+sub": 0x00000001, "-1.5": 0xBFC00000, "+inf": 0x7F800000,
        "-qnan": 0xFFC00000, "+2": 0x40000000, "-sub": 0x80000001, "+snan1": 0x7F800001,
        "+max": 0x7F7FFFFF, "-qnan5": 0xFFC00005}
_F64 = {"+1": 0x3FF0000000000000, "-0": 0x8000000000000000, "+qnan": 0x7FF8000000000000,
        "-inf": 0xFFF0000000000000, "+0": 0, "-snan1": 0xFFF0000000000001, "+sub": 1,
        "-1.5": 0xBFF8000000000000, "+inf": 0x7FF0000000000000, "-qnan": 0xFFF8000000000000,
        "+2": 0x4000000000000000, "-sub": 0x8000000000000001, "+snan1": 0x7FF0000000000001,
        "+max": 0x7FEFFFFFFFFFFFFF, "-qnan5": 0xFFF8000000000005}
# list order of the example (two equal +1 patterns: they must keep this order)
_EXAMPLE = ["+1", "-0", "+qnan", "-inf", "+0", "-snan1", "+sub", "-1.5", "+inf", "-qnan", "+2", "-sub",
            "+snan1", "+1", "+max", "-qnan5"]
# ascending totalOrder worked out by hand: NaNs with the sign set first (a
# quiet NaN, whose top fraction bit is set, before a signaling one; a larger
# payload further out), then -inf, the negative numbers, -0, +0, the positive
# numbers, +inf, and the positive NaNs (signaling before quiet)
_EXAMPLE_SORTED = [15, 9, 5, 3, 7, 11, 1, 4, 6, 0, 13, 10, 14, 8, 12, 2]


@pytest.mark.parametrize("width", [4, 8])
def test_float_order_hand_example(width):
    pat = _F32 if width == 4 else _F64
    dt = np.uint32 if width == 4 else np.uint64
    key = np.array([pat[name] for name in _EXAMPLE], dtype=dt)
    nxt, root = I.list_from_order(np.arange(key.size))
    out, r = O.stable_sort_definition(nxt, key, root, 8 * width, float_keys=True)
    assert _walk(out, r) == _EXAMPLE_SORTED
    out, r = O.stable_sort_definition(nxt, key, root, 8 * width, float_keys=True, descending=True)
    want = list(reversed(_EXAMPLE_SORTED))
    i, j = want.index(13), want.index(0)  # equal patterns keep list order in both directions
    want[i], want[j] = want[j], want[i]
    assert _walk(out, r) == want


def _decode(key, width):
    fmt = "<f" if width == 4 else "<d"
    return [struct.unpack(fmt, int(k).to_bytes(width, "little"))[0] for k in key]


def _finite_and_inf(n, width, seed):
    g = np.random.default_rng(seed)
    dt, ft = (np.uint32, np.float32) if width == 4 else (np.uint64, np.float64)
    vals = (g.standard_normal(n) * 10.0 ** g.integers(-30, 30, n)).astype(ft)
    key = vals.view(dt).copy()
    tiny = g.integers(1, 1000, n).astype(dt)  # subnormal patterns
    sign = dt(1) << dt(8 * width - 1)
    key[::13] = tiny[::13]
    key[1::17] = tiny[1::17] | sign
    key[2::19] = 0
    key[3::23] = sign
    key[4::29] = np.array(_F32["+inf"] if width == 4 else _F64["+inf"], dtype=dt)
    key[5::31] = np.array(_F32["-inf"] if width == 4 else _F64["-inf"], dtype=dt)
    key[6::7] = key[0]  # repeated patterns
    return key


@pytest.mark.parametrize("width", [4, 8])
def test_float_order_vs_python_sorted(width):
    n = 5000
    key = _finite_and_inf(n, width, 701 + width)
    nxt, root = I.random_list(n, 702)
    order = _walk(nxt, root)
    dec = _decode(key, width)
    # numbers by value; of the two zeros, the one with the sign set first;
    # Python's sort is stable, so equal patterns keep list order
    want = sorted(order, key=lambda v: (dec[v], 0 if struct.pack(">d", dec[v])[0] & 0x80 else 1))
    out, r = O.stable_sort_definition(nxt, key, root, 8 * width, float_keys=True)
    assert _walk(out, r) == want


@pytest.mark.parametrize("width", [4, 8])
def test_float_order_matches_paper_recipe_on_non_negative_values(width):
    """The paper's recipe: stable sort by the mantissa (fraction field), then
    stable sort by the characteristic (exponent field).  For values without
    the sign bit (zeros, subnormals, normals, +inf) it orders by value."""
    n = 4000
    key = _finite_and_inf(n, width, 711 + width)
    sign = (1 << (8 * width - 1))
    key = key & key.dtype.type(sign - 1)  # clear the sign bit
    nxt, root = I.random_list(n, 712)
    order = _walk(nxt, root)
    fbits = 23 if width == 4 else 52
    by_mantissa = sorted(order, key=lambda v: int(key[v]) & ((1 << fbits) - 1))
    recipe = sorted(by_mantissa, key=lambda v: int(key[v]) >> fbits)
    out, r = O.stable_sort_definition(nxt, key, root, 8 * width, float_keys=True)
    assert _walk(out, r) == recipe
    # with negative values the recipe (which ignores the sign) is not an order
    # by value, and the oracle's reading departs from it
    key2 = key.copy()
    key2[::3] |= key.dtype.type(sign)
    by_mantissa = sorted(order, key=lambda v: int(key2[v]) & ((1 << fbits) - 1))
    recipe2 = sorted(by_mantissa, key=lambda v: (int(key2[v]) & (sign - 1)) >> fbits)
    out2, r2 = O.stable_sort_definition(nxt, key2, root, 8 * width, float_keys=True)
    assert _walk(out2, r2) != recipe2
