"""Pbit oracle (Python side).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library.

Three pieces, each written from the paper "Pbit and other list sorting
algorithms" (D. S. Planeta):

* ``pbit_sort`` -- calls the literal recursive Pbit of ``pbit_oracle.c``
  (Sec. "Implementation in C++", ascending bucket order of Sec. "Differences
  between sorting in descending and ascending order", sign split of
  Sec. "Negative numbers sorting").
* ``stable_sort_definition`` -- the plain definition the method reaches: a
  stable sort of the list's nodes by ``key mod 2^M`` (ascending), then the
  concatenation of Sec. 5.1 written as ``next[s[i]] = s[i+1]``.  The paper
  claims stability (abstract, Sec. 3); numpy's stable argsort is the library
  primitive used as the sort step.
* ``float_order_keys`` -- the order of IEEE-754 keys (Sec. "Floating-point
  numbers sorting"): the paper sorts by mantissa and then stably by
  characteristic, which orders non-negative values but ignores the sign.  The
  reading taken here extends it to every bit pattern with the totalOrder
  relation of IEEE 754-2008 (Sec. 5.10): -NaN < -inf < negative numbers < -0
  < +0 < positive numbers < +inf < +NaN, NaNs of one sign ordered by their
  payload (a quiet NaN beyond a signaling one).  It is written from the
  decoded sign, exponent and fraction fields.
* ``check_sorted_list`` -- properties that pin the result at any size:
  the output list is a permutation of the input list, keys are
  non-decreasing along it, and equal keys keep their input list order.  These
  three together determine a stable sort uniquely.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbit_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpbit_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        _lib.pbit_oracle_sort.restype = ctypes.c_int
        _lib.pbit_oracle_sort.argtypes = [i64, vp, i64, vp, i64, ctypes.c_int, i32, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.pbit_oracle_list_order.restype = i64
        _lib.pbit_oracle_list_order.argtypes = [i64, vp, i64, i32, vp, i64]
        _lib.pbit_oracle_split_once.restype = i64
        _lib.pbit_oracle_split_once.argtypes = [i64, vp, vp, ctypes.c_int, i32, ctypes.c_int,
                                                ctypes.c_int, vp, vp]
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def list_order(next_idx: np.ndarray, root: int, max_len: int | None = None) -> np.ndarray:
    """Node ids in list order, walking ``next`` from ``root`` (-1 = NULL)."""
    next_idx = np.ascontiguousarray(next_idx, dtype=np.int32)
    n = next_idx.size
    out = np.empty(max(n, 1), dtype=np.int32)
    ln = lib().pbit_oracle_list_order(n, _ptr(next_idx), 4, int(root), _ptr(out),
                                      n if max_len is None else max_len)
    if ln == -1:
        raise OracleError("index out of range")
    if ln == -2:
        raise OracleError("cycle or list longer than the pool")
    return out[:ln].copy()


def pbit_sort(next_idx: np.ndarray, key: np.ndarray, root: int, M: int, K: int,
              signed: bool = False, descending: bool = False):
    """Literal Pbit.  Returns (next_out, new_root, counters) with counters =
    dict(splits, merges, depth, length)."""
    next_idx = np.ascontiguousarray(next_idx, dtype=np.int32)
    key = np.ascontiguousarray(key)
    assert key.size == next_idx.size
    out = np.empty_like(next_idx)
    new_root = ctypes.c_int32(-7)
    cnt = np.zeros(4, dtype=np.uint64)
    rc = lib().pbit_oracle_sort(next_idx.size, _ptr(next_idx), 4, _ptr(key), key.itemsize,
                                key.itemsize, int(root), M, K, int(signed), int(descending),
                                _ptr(out), ctypes.addressof(new_root), _ptr(cnt))
    if rc == -1:
        raise ValueError("bad M/K for this key width")
    if rc != 0:
        raise OracleError(f"oracle error {rc}")
    return out, int(new_root.value), dict(splits=int(cnt[0]), merges=int(cnt[1]),
                                          depth=int(cnt[2]), length=int(cnt[3]))


def split_once(next_idx: np.ndarray, key: np.ndarray, root: int, M: int, K: int):
    """Buckets left by ONE split loop at bits [M-K, M): list of node-id lists,
    bucket 0 first, each in the order the push-to-front split leaves them."""
    next_idx = np.ascontiguousarray(next_idx, dtype=np.int32)
    key = np.ascontiguousarray(key)
    n = next_idx.size
    seq = np.empty(max(n, 1), dtype=np.int32)
    blen = np.zeros(1 << K, dtype=np.int64)
    ln = lib().pbit_oracle_split_once(n, _ptr(next_idx), _ptr(key), key.itemsize, int(root),
                                      M, K, _ptr(seq), _ptr(blen))
    if ln < 0:
        raise OracleError(f"split error {ln}")
    out, w = [], 0
    for c in blen:
        out.append(seq[w:w + c].tolist())
        w += int(c)
    return out


def sort_key(key: np.ndarray, M: int, signed: bool = False) -> np.ndarray:
    """The value the list is ordered by: the low M bits of the key as an
    unsigned number; for signed keys (M = key width) the two's complement
    value, which the sign split of Sec. "Negative numbers sorting" orders
    negatives first."""
    k = np.ascontiguousarray(key)
    if signed:
        assert M == 8 * k.itemsize
        return k.view({1: np.int8, 2: np.int16, 4: np.int32, 8: np.int64}[k.itemsize]).astype(np.int64)
    u = k.view({1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[k.itemsize]).astype(np.uint64)
    if M < 64:
        u = u & np.uint64((1 << M) - 1)
    return u


_FLOAT_FIELDS = {4: (np.uint32, np.float32, 23, 8), 8: (np.uint64, np.float64, 52, 11)}


def float_order_keys(key: np.ndarray):
    """Three arrays (cls, val, zero_rank) whose lexicographic order is the
    IEEE 754 totalOrder of the binary32 / binary64 values whose bit patterns
    are ``key``: cls 0 = NaN with the sign set, 1 = a number or an infinity,
    2 = NaN without the sign; val = the NaN's fraction field (negated for a
    negative NaN: a larger payload lies further out) or the value itself;
    zero_rank orders -0 before +0, the only distinct patterns of equal value."""
    k = np.ascontiguousarray(key)
    utype, ftype, fbits, ebits = _FLOAT_FIELDS[k.itemsize]
    u = k.view(utype)
    sign = (u >> utype(fbits + ebits)) & utype(1)
    expo = (u >> utype(fbits)) & utype((1 << ebits) - 1)
    frac = u & utype((1 << fbits) - 1)
    is_nan = (expo == utype((1 << ebits) - 1)) & (frac != 0)
    with np.errstate(invalid="ignore"):  # NaN patterns are not used as values
        value = k.view(ftype).astype(np.float64)  # exact: binary32 widens without rounding
    frac_f = frac.astype(np.float64)  # exact: at most 52 bits
    neg = sign == 1
    cls = np.where(is_nan, np.where(neg, 0, 2), 1).astype(np.int8)
    val = np.where(is_nan, np.where(neg, -frac_f, frac_f), value)
    zero_rank = np.where(neg, 0, 1).astype(np.int8)
    return cls, val, zero_rank


def relink(next_idx: np.ndarray, sorted_nodes: np.ndarray):
    """Concatenate the sorted fragments: next[s[i]] = s[i+1], last -> -1."""
    out = np.array(next_idx, dtype=np.int32, copy=True)
    if sorted_nodes.size == 0:
        return out, -1
    out[sorted_nodes[:-1]] = sorted_nodes[1:]
    out[sorted_nodes[-1]] = -1
    return out, int(sorted_nodes[0])


def stable_sort_definition(next_idx: np.ndarray, key: np.ndarray, root: int, M: int,
                           signed: bool = False, descending: bool = False, float_keys: bool = False):
    """(next_out, new_root) of a stable sort of the list by its key
    (``float_keys``: by the IEEE order of ``float_order_keys``)."""
    order = list_order(next_idx, root)
    if float_keys:
        assert M == 8 * key.itemsize and key.itemsize in (4, 8)
        cls, val, zr = float_order_keys(key[order])
        pos = np.arange(order.size)
        if descending:  # largest first, equal patterns still in list order
            perm = np.lexsort((pos, -zr.astype(np.int16), -val, -cls.astype(np.int16)))
        else:
            perm = np.lexsort((pos, zr, val, cls))
        return relink(next_idx, order[perm])
    sk = sort_key(key, M, signed)[order]
    if descending:
        # stable descending: reverse a stable ascending sort of the reversed list
        perm = np.argsort(sk[::-1], kind="stable")[::-1]
        perm = (order.size - 1 - perm)
    else:
        perm = np.argsort(sk, kind="stable")
    return relink(next_idx, order[perm])


def check_sorted_list(next_in: np.ndarray, root_in: int, next_out: np.ndarray, root_out: int,
                      key: np.ndarray, M: int, signed: bool = False, descending: bool = False):
    """Raise AssertionError unless (next_out, root_out) is the stable sort of
    the list (next_in, root_in).  Nodes off the list must be untouched."""
    order_in = list_order(next_in, root_in)
    n = order_in.size
    order_out = list_order(next_out, root_out, max_len=n)
    assert order_out.size == n, f"output list has {order_out.size} nodes, input {n}"
    rank_in = np.full(next_in.size, -1, dtype=np.int64)
    rank_in[order_in] = np.arange(n)
    r = rank_in[order_out]
    assert (r >= 0).all(), "output list contains a node that was not on the input list"
    seen = np.zeros(next_in.size, dtype=bool)
    seen[order_out] = True
    assert seen.sum() == n, "output list repeats a node"
    sk = sort_key(key, M, signed)[order_out]
    if descending:
        sk = ~sk  # order-reversing and exact for both int64 and uint64
    if n > 1:
        assert (sk[:-1] <= sk[1:]).all(), "keys out of order"
        eq = sk[:-1] == sk[1:]
        assert (r[:-1][eq] < r[1:][eq]).all(), "equal keys not in input list order"
    off = np.ones(next_in.size, dtype=bool)
    off[order_in] = False
    assert (next_out[off] == next_in[off]).all(), "a node off the list was written"
