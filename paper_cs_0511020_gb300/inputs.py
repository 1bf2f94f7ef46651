"""Seeded synthetic inputs for the Pbit list sort (shared by tests, bench and
smoke; holds none of the sort's arithmetic).

A list lives in a node pool: ``next[v]`` is the pool index of v's successor
(-1 = NULL) and ``key[v]`` its key (paper, Sec. "Structure of data
representing a node").  All generators are numpy PCG64 streams seeded with
``0x0511020 + workload id`` unless a seed is given.

Workloads (sizes as the paper's experiments scale them up to the GPU):
  1  2^20 nodes, AoS {int32 next; uint32 key}, random list order, uniform u32
  2  2^27 nodes, SoA, random order (and the push-built order), uniform u32
  3  2^26 nodes u64 Zipf(1.1) over 1024 values with a constant top half;
     2^26 nodes u8 uniform
  4  4096 lists in one pool, lengths log-uniform in [16, 2^20], uniform u32
  5  request stream: Poisson arrivals, lengths log-uniform in [2^4, 2^24],
     key types u16:u32:u64 = 1:2:1
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 0x0511020
_UINT = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def list_from_order(order: np.ndarray, pool_size: int | None = None):
    """next[] with next[order[i]] = order[i+1] and the last node -> -1."""
    order = np.asarray(order, dtype=np.int32)
    size = order.size if pool_size is None else pool_size
    nxt = np.full(size, -1, dtype=np.int32)
    if order.size:
        nxt[order[:-1]] = order[1:]
    return nxt, (int(order[0]) if order.size else -1)


def random_list(n: int, seed: int):
    """A list over pool indices 0..n-1 in a seeded random order."""
    return list_from_order(rng(seed).permutation(n).astype(np.int32))


def push_built_list(n: int):
    """The list that pushing pool nodes 0..n-1 onto an empty list builds
    (paper, Sec. 2 push): root = n-1, next[v] = v-1, next[0] = -1."""
    nxt = np.arange(-1, n - 1, dtype=np.int32)
    return nxt, (n - 1 if n else -1)


def uniform_keys(n: int, key_bytes: int, seed: int) -> np.ndarray:
    dt = _UINT[key_bytes]
    return rng(seed).integers(0, np.iinfo(dt).max, size=n, dtype=dt, endpoint=True)


def zipf_u64_keys(n: int, seed: int, distinct: int = 1024, s: float = 1.1,
                  top: int = 0xA5A5A5A5) -> np.ndarray:
    """u64 keys: constant top 32 bits, low 32 bits one of ``distinct`` seeded
    values; value ranks drawn Zipf(s) by inverse CDF, rank -> value random."""
    g = rng(seed)
    vals = np.unique(g.integers(0, 1 << 32, size=4 * distinct, dtype=np.uint64))
    vals = g.permutation(vals)[:distinct]
    w = 1.0 / np.arange(1, distinct + 1, dtype=np.float64) ** s
    cdf = np.cumsum(w / w.sum())
    ranks = np.searchsorted(cdf, g.random(n), side="right").clip(0, distinct - 1)
    return (np.uint64(top) << np.uint64(32)) | vals[ranks]


def aos_pack(nxt: np.ndarray, key_u32: np.ndarray) -> np.ndarray:
    """Interleave into the 8-byte AoS node {int32 next; uint32 key}."""
    a = np.empty((nxt.size, 2), dtype=np.int32)
    a[:, 0] = nxt
    a[:, 1] = key_u32.view(np.int32)
    return a


def log_uniform_lengths(count: int, lo_log2: float, hi_log2: float, seed: int,
                        lo: int, hi: int) -> np.ndarray:
    u = rng(seed).random(count)
    return np.clip(np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)), lo, hi).astype(np.int64)


def batched_pool(lengths: np.ndarray, key_bytes: int, seed: int):
    """Lists packed into one pool: list i owns [off[i], off[i+1]) with a
    random order inside it.  Returns (next, key, roots, offsets)."""
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.zeros(lengths.size + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    total = int(off[-1])
    g = rng(seed)
    nxt = np.full(total, -1, dtype=np.int32)
    roots = np.full(lengths.size, -1, dtype=np.int32)
    for i, ln in enumerate(lengths):
        if ln == 0:
            continue
        a = int(off[i])
        order = g.permutation(int(ln)).astype(np.int32) + np.int32(a)
        nxt[order[:-1]] = order[1:]
        roots[i] = order[0]
    key = uniform_keys(total, key_bytes, seed + 1)
    return nxt, key, roots, off


def config4_lengths(seed: int, count: int = 4096) -> np.ndarray:
    """Batched workload: `count` list lengths log-uniform in [16, 2^20]."""
    return log_uniform_lengths(count, 4.0, 20.0, seed, 16, 1 << 20)


def config5_requests(count: int, seed: int):
    """Request stream: exponential gaps of mean 0.5 ms (Poisson, 2000/s),
    lengths log-uniform in [2^4, 2^24], key widths 2:4:8 in 1:2:1."""
    g = rng(seed)
    gaps = g.exponential(0.5e-3, count)
    lengths = np.clip(np.floor(2.0 ** (4.0 + 20.0 * g.random(count))), 16, 1 << 24).astype(np.int64)
    kb = g.choice(np.array([2, 4, 4, 8]), size=count)
    return np.cumsum(gaps), lengths, kb


# ---------------------------------------------------------------------------
# Device-side generators for the benchmark's large workloads (same recipes,
# drawn with torch's CUDA generator instead of numpy: 10^9 nodes are drawn in
# seconds).  The parity tests use the numpy generators above.

_TORCH_KEY = {2: "int16", 4: "int32", 8: "int64"}


def device_keys(n: int, key_bytes: int, gen):
    """Uniform keys over all 8*key_bytes bits, as a signed torch view."""
    import torch
    dt = getattr(torch, _TORCH_KEY.get(key_bytes, "uint8"))
    if key_bytes == 1:
        return torch.randint(0, 256, (n,), dtype=torch.uint8, device=gen.device, generator=gen)
    if key_bytes == 8:
        hi = torch.randint(-2**31, 2**31, (n,), dtype=torch.int64, device=gen.device, generator=gen)
        lo = torch.randint(0, 2**32, (n,), dtype=torch.int64, device=gen.device, generator=gen)
        return (hi << 32) | lo
    lim = 1 << (8 * key_bytes - 1)
    return torch.randint(-lim, lim, (n,), dtype=dt, device=gen.device, generator=gen)


def device_random_list(n: int, gen):
    """next[] (int32, on gen's device) of one list in a random order, and its root."""
    import torch
    perm = torch.randperm(n, dtype=torch.int64, device=gen.device, generator=gen)
    nxt = torch.empty(n, dtype=torch.int32, device=gen.device)
    nxt[perm[:-1]] = perm[1:].to(torch.int32)
    nxt[perm[-1]] = -1
    return nxt, int(perm[0])


def device_batched_pool(lengths, key_bytes: int, gen):
    """Lists packed into one pool (list i owns [off[i], off[i+1])), each in a
    random order of its own range: (next, key, roots, offsets) on gen's device."""
    import torch
    dev = gen.device
    lens = torch.as_tensor(np.asarray(lengths, dtype=np.int64), device=dev)
    L = lens.numel()
    off = torch.zeros(L + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(lens, 0)
    total = int(off[-1])
    lid = torch.repeat_interleave(torch.arange(L, device=dev), lens)
    # a random order inside every range: sort by (list id, random value)
    r = torch.rand(total, dtype=torch.float64, device=dev, generator=gen)
    order = torch.argsort(lid.to(torch.float64) * 2.0 + r)
    nxt = torch.empty(total, dtype=torch.int32, device=dev)
    last = off[1:] - 1                      # position of each list's tail in `order`
    succ = torch.empty(total, dtype=torch.int64, device=dev)
    succ[:-1] = order[1:]
    succ[last[lens > 0]] = -1
    nxt[order] = succ.to(torch.int32)
    roots = torch.full((L,), -1, dtype=torch.int32, device=dev)
    nz = lens > 0
    roots[nz] = order[off[:-1][nz]].to(torch.int32)
    key = device_keys(total, key_bytes, gen)
    return nxt, key, roots, off
