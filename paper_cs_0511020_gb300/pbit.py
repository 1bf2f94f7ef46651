"""ctypes binding of libpbit.so (include/pbit.h) taking torch device tensors.

Argument marshalling only: every step of the sort runs in the library's CUDA
kernels.  If the library is missing this module raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpbit.so")

OK, EINVAL, ENOMEM, EBADLIST, ETIMEOUT, ECUDA, EAGAIN, EPENDING = range(8)
SIGNED, DESCENDING, DOUBLY, FLOAT = 1, 2, 4, 8

EXPORTS = ("pbit_status_string", "pbit_workspace_size", "pbit_sort_list", "pbit_sort_lists_batched",
           "pbit_workspace_size_host", "pbit_sort_list_host", "pbit_sort_list_noalloc", "pbit_last_launch_count",
           "pbit_profile_enable", "pbit_profile_read", "pbit_serve_create", "pbit_serve_submit",
           "pbit_serve_poll", "pbit_serve_wait", "pbit_serve_times", "pbit_serve_release", "pbit_serve_stats",
           "pbit_serve_destroy", "pbit_graph_create_batched", "pbit_graph_create_single", "pbit_graph_launch",
           "pbit_graph_result", "pbit_graph_node_count", "pbit_graph_destroy", "pbit_autotune_workspace_size",
           "pbit_autotune_batched", "pbit_selftest_bounded_wait", "pbit_debug_stage")


class PbitError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: pbit status {status} ({status_string(status)})")


class Pool(ctypes.Structure):
    _fields_ = [("next", ctypes.c_void_p), ("next_stride_bytes", ctypes.c_int64),
                ("key", ctypes.c_void_p), ("key_stride_bytes", ctypes.c_int64),
                ("key_type", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("pool_size", ctypes.c_int64), ("prev", ctypes.c_void_p),
                ("prev_stride_bytes", ctypes.c_int64)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int32), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class Tune(ctypes.Structure):
    _fields_ = [("digit_bits", ctypes.c_int32), ("smem_cutoff", ctypes.c_int32),
                ("ruler_stride", ctypes.c_int32), ("gather_pack", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.pbit_status_string.restype = ctypes.c_char_p
        L.pbit_status_string.argtypes = [ctypes.c_int]
        L.pbit_workspace_size.restype = ctypes.c_int
        L.pbit_workspace_size.argtypes = [i64, i32, i32, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.pbit_sort_list.restype = ctypes.c_int
        L.pbit_sort_list.argtypes = [vp, i32, i64, i32, i32, ctypes.POINTER(i32), vp, vp,
                                     ctypes.c_size_t, vp]
        L.pbit_sort_lists_batched.restype = ctypes.c_int
        L.pbit_sort_lists_batched.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, vp,
                                              ctypes.c_size_t, vp]
        L.pbit_last_launch_count.restype = i64
        L.pbit_last_launch_count.argtypes = []
        L.pbit_workspace_size_host.restype = ctypes.c_int
        L.pbit_workspace_size_host.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
        L.pbit_sort_list_host.restype = ctypes.c_int
        L.pbit_sort_list_host.argtypes = [vp, i32, i64, i32, i32, ctypes.POINTER(i32), vp, vp,
                                          ctypes.c_size_t, vp]
        L.pbit_sort_list_noalloc.restype = ctypes.c_int
        L.pbit_sort_list_noalloc.argtypes = [vp, i32, i64, i32, i32, ctypes.POINTER(i32), vp]
        L.pbit_profile_enable.restype = None
        L.pbit_profile_enable.argtypes = [i32]
        L.pbit_profile_read.restype = i32
        L.pbit_profile_read.argtypes = [vp, i32]
        L.pbit_serve_create.restype = ctypes.c_int
        L.pbit_serve_create.argtypes = [ctypes.POINTER(vp), ctypes.c_size_t, i32, i32, i32, vp]
        L.pbit_serve_submit.restype = ctypes.c_int
        L.pbit_serve_submit.argtypes = [vp, vp, i32, i64, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
        L.pbit_serve_poll.restype = ctypes.c_int
        L.pbit_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32)]
        L.pbit_serve_wait.restype = ctypes.c_int
        L.pbit_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32), i64]
        L.pbit_serve_times.restype = ctypes.c_int
        L.pbit_serve_times.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.pbit_serve_release.restype = ctypes.c_int
        L.pbit_serve_release.argtypes = [vp, ctypes.c_uint64]
        L.pbit_graph_create_batched.restype = ctypes.c_int
        L.pbit_graph_create_batched.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, vp, ctypes.c_size_t,
                                                ctypes.POINTER(vp)]
        L.pbit_graph_create_single.restype = ctypes.c_int
        L.pbit_graph_create_single.argtypes = [vp, i32, i64, i32, i32, vp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.pbit_graph_launch.restype = ctypes.c_int
        L.pbit_graph_launch.argtypes = [vp, vp]
        L.pbit_graph_result.restype = ctypes.c_int
        L.pbit_graph_result.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.pbit_graph_node_count.restype = i64
        L.pbit_graph_node_count.argtypes = [vp]
        L.pbit_graph_destroy.restype = None
        L.pbit_graph_destroy.argtypes = [vp]
        L.pbit_autotune_workspace_size.restype = ctypes.c_int
        L.pbit_autotune_workspace_size.argtypes = [i64, i32, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.pbit_autotune_batched.restype = ctypes.c_int
        L.pbit_autotune_batched.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, ctypes.c_size_t, i32, vp, vp,
                                            ctypes.POINTER(ctypes.c_float)]
        L.pbit_debug_stage.restype = ctypes.c_int
        L.pbit_debug_stage.argtypes = [vp, i32, i64, i32, i32, i32, vp, ctypes.c_size_t, vp, vp, vp]
        L.pbit_selftest_bounded_wait.restype = ctypes.c_int
        L.pbit_selftest_bounded_wait.argtypes = [i64, vp]
        L.pbit_serve_stats.restype = None
        L.pbit_serve_stats.argtypes = [vp, ctypes.POINTER(i64)]
        L.pbit_serve_destroy.restype = None
        L.pbit_serve_destroy.argtypes = [vp]
        _lib = L
    return _lib


def debug_stage(pool: Pool, root: int, n: int, M: int, stage: int, K: int = 4, ws=None, stream=None):
    """(status, idx, key) after the ranking (stage 1) or the first MSD pass
    (stage 2) of the single-list pipeline; idx and key are new device tensors."""
    if ws is None:
        ws = alloc_workspace(workspace_size(n, 1, pool.key_type))
    idx = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    key = torch.empty(max(n, 1) * pool.key_type, dtype=torch.uint8, device="cuda")
    st = lib().pbit_debug_stage(ctypes.addressof(pool), int(root), int(n), int(M), int(K), int(stage),
                                ws.data_ptr(), ws.numel() * ws.element_size(), idx.data_ptr(), key.data_ptr(),
                                _stream_handle(stream))
    return int(st), idx[:n], key[:n * pool.key_type]


def selftest_bounded_wait(iterations: int = 1 << 12, stream=None) -> int:
    """Make a bounded device wait run out on purpose; returns the status the
    library reports (ETIMEOUT when the wait gave up as designed)."""
    return int(lib().pbit_selftest_bounded_wait(int(iterations), _stream_handle(stream)))


def status_string(st: int) -> str:
    return lib().pbit_status_string(int(st)).decode()


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _tune_ptr(tune):
    if tune is None:
        return None, None
    if isinstance(tune, dict):
        tune = Tune(tune.get("digit_bits", 0), tune.get("smem_cutoff", 0), tune.get("ruler_stride", 0),
                    tune.get("gather_pack", 0))
    return tune, ctypes.addressof(tune)


def make_pool(next_t: torch.Tensor, key_t: torch.Tensor, flags: int = 0,
              prev_t: torch.Tensor | None = None) -> Pool:
    """SoA pool: next_t int32[n] and key_t of 1/2/4/8-byte elements, both CUDA."""
    assert next_t.is_cuda and key_t.is_cuda and next_t.dtype == torch.int32
    assert next_t.is_contiguous() and key_t.is_contiguous() and next_t.numel() == key_t.numel()
    kb = key_t.element_size()
    p = Pool(next_t.data_ptr(), 4, key_t.data_ptr(), kb, kb, flags, next_t.numel(), 0, 0)
    if prev_t is not None:
        assert prev_t.dtype == torch.int32 and prev_t.is_contiguous() and prev_t.numel() == next_t.numel()
        p.prev, p.prev_stride_bytes = prev_t.data_ptr(), 4
        p.flags |= DOUBLY
    return p


def make_pool_aos(nodes_t: torch.Tensor, flags: int = 0) -> Pool:
    """AoS pool of 8-byte nodes {int32 next; uint32 key}: an int32 tensor [n, 2]."""
    assert nodes_t.is_cuda and nodes_t.dtype == torch.int32 and nodes_t.dim() == 2 and nodes_t.shape[1] == 2
    assert nodes_t.is_contiguous()
    base = nodes_t.data_ptr()
    return Pool(base, 8, base + 4, 8, 4, flags, nodes_t.shape[0], 0, 0)


def workspace_size(pool_size: int, num_lists: int, key_bytes: int, tune=None) -> int:
    out = ctypes.c_size_t(0)
    tune, tp = _tune_ptr(tune)
    st = lib().pbit_workspace_size(int(pool_size), int(num_lists), int(key_bytes), tp, ctypes.byref(out))
    if st != OK:
        raise PbitError(st, "pbit_workspace_size")
    return int(out.value)


def alloc_workspace(nbytes: int, device=None) -> torch.Tensor:
    """Device workspace (torch's caching allocator returns >= 512-byte alignment)."""
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")
    assert ws.data_ptr() % 256 == 0
    return ws


def sort_pool_list(pool: Pool, root: int, n: int, M: int, K: int = 4, ws: torch.Tensor | None = None,
                   tune=None, stream=None, check: bool = True):
    """pbit_sort_list on a prepared Pool; returns (status, new_root)."""
    if ws is None:
        ws = alloc_workspace(workspace_size(pool.pool_size, 1, pool.key_type, tune))
    tune, tp = _tune_ptr(tune)
    nr = ctypes.c_int32(-7)
    st = lib().pbit_sort_list(ctypes.addressof(pool), int(root), int(n), int(M), int(K), ctypes.byref(nr), tp,
                              ws.data_ptr(), ws.numel(), _stream_handle(stream))
    if check and st != OK:
        raise PbitError(st, "pbit_sort_list")
    return st, int(nr.value)


def sort_list(next_t: torch.Tensor, key_t: torch.Tensor, root: int, M: int | None = None, K: int = 4,
              flags: int = 0, prev_t=None, ws=None, tune=None, stream=None) -> int:
    """Sort the list in place (next_t relinked); returns the new root."""
    pool = make_pool(next_t, key_t, flags, prev_t)
    M = 8 * key_t.element_size() if M is None else M
    return sort_pool_list(pool, root, next_t.numel(), M, K, ws, tune, stream)[1]


def sort_pool_batched(pool: Pool, roots_t: torch.Tensor, offsets_t: torch.Tensor, M: int, K: int = 4,
                      new_roots_t: torch.Tensor | None = None, ws=None, tune=None, stream=None,
                      check: bool = True):
    assert roots_t.dtype == torch.int32 and offsets_t.dtype == torch.int64
    L = roots_t.numel()
    assert offsets_t.numel() == L + 1
    if new_roots_t is None:
        new_roots_t = torch.empty(L, dtype=torch.int32, device=roots_t.device)
    if ws is None:
        ws = alloc_workspace(workspace_size(pool.pool_size, L, pool.key_type, tune))
    tune, tp = _tune_ptr(tune)
    st = lib().pbit_sort_lists_batched(ctypes.addressof(pool), L, roots_t.data_ptr(), offsets_t.data_ptr(),
                                       int(M), int(K), new_roots_t.data_ptr(), tp, ws.data_ptr(), ws.numel(),
                                       _stream_handle(stream))
    if check and st != OK:
        raise PbitError(st, "pbit_sort_lists_batched")
    return st, new_roots_t


def sort_lists_batched(next_t, key_t, roots_t, offsets_t, M=None, K=4, flags=0, ws=None, tune=None,
                       stream=None):
    pool = make_pool(next_t, key_t, flags)
    M = 8 * key_t.element_size() if M is None else M
    return sort_pool_batched(pool, roots_t, offsets_t, M, K, None, ws, tune, stream)[1]


NOALLOC_MAX_NODES = 1 << 16


def sort_pool_list_noalloc(pool: Pool, root: int, n: int, M: int, K: int = 4, stream=None, check: bool = True):
    """pbit_sort_list_noalloc: same as sort_pool_list but with the library's
    static scratch array instead of a workspace (lists up to
    NOALLOC_MAX_NODES nodes; for callers that cannot allocate device
    memory).  Returns (status, new_root)."""
    nr = ctypes.c_int32(-7)
    st = lib().pbit_sort_list_noalloc(ctypes.addressof(pool), int(root), int(n), int(M), int(K), ctypes.byref(nr),
                                      _stream_handle(stream))
    if check and st != OK:
        raise PbitError(st, "pbit_sort_list_noalloc")
    return st, int(nr.value)


def last_launch_count() -> int:
    return int(lib().pbit_last_launch_count())


def profile_enable(on: bool = True) -> None:
    """Per-kernel CUDA-event timing of the following sort calls on this thread."""
    lib().pbit_profile_enable(1 if on else 0)


def profile_read() -> list:
    """[{name, launches, ms, bytes}] for the last sort call on this thread."""
    arr = (KernelStat * 32)()
    n = lib().pbit_profile_read(ctypes.addressof(arr), 32)
    if n < 0:
        raise PbitError(ECUDA, "pbit_profile_read")
    return [dict(name=arr[i].name.decode(), launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes)
            for i in range(n)]


def host_pool(next_h, key_h, flags: int = 0) -> Pool:
    """SoA pool over HOST tensors/arrays (torch CPU tensors, pinned or not)."""
    kb = key_h.element_size()
    return Pool(next_h.data_ptr(), 4, key_h.data_ptr(), kb, kb, flags, next_h.numel(), 0, 0)


def workspace_size_host(pool: Pool, tune=None) -> int:
    out = ctypes.c_size_t(0)
    tune, tp = _tune_ptr(tune)
    st = lib().pbit_workspace_size_host(ctypes.addressof(pool), tp, ctypes.byref(out))
    if st != OK:
        raise PbitError(st, "pbit_workspace_size_host")
    return int(out.value)


def sort_pool_list_host(pool: Pool, root: int, n: int, M: int, K: int = 4, ws=None, tune=None, stream=None,
                        check: bool = True):
    """pbit_sort_list_host: the pool is in host memory; returns (status, new_root)."""
    if ws is None:
        ws = alloc_workspace(workspace_size_host(pool, tune))
    tune, tp = _tune_ptr(tune)
    nr = ctypes.c_int32(-7)
    st = lib().pbit_sort_list_host(ctypes.addressof(pool), int(root), int(n), int(M), int(K), ctypes.byref(nr),
                                   tp, ws.data_ptr(), ws.numel(), _stream_handle(stream))
    if check and st != OK:
        raise PbitError(st, "pbit_sort_list_host")
    return st, int(nr.value)


class Graph:
    """A sort call captured once as a CUDA graph (pbit_graph_*) and replayed.

    Keeps references to every tensor the graph points at (pool arrays,
    roots, offsets, new roots, workspace) so they stay allocated."""

    def __init__(self, handle, keep, single: bool):
        self._h = handle
        self._keep = keep
        self.single = single

    @classmethod
    def batched(cls, pool: Pool, roots_t: torch.Tensor, offsets_t: torch.Tensor, M: int, K: int = 4,
                new_roots_t: torch.Tensor | None = None, ws=None, tune=None, keep=()):
        assert roots_t.dtype == torch.int32 and offsets_t.dtype == torch.int64
        L = roots_t.numel()
        assert offsets_t.numel() == L + 1
        if new_roots_t is None:
            new_roots_t = torch.empty(L, dtype=torch.int32, device=roots_t.device)
        if ws is None:
            ws = alloc_workspace(workspace_size(pool.pool_size, L, pool.key_type, tune))
        tune_s, tp = _tune_ptr(tune)
        h = ctypes.c_void_p()
        st = lib().pbit_graph_create_batched(ctypes.addressof(pool), L, roots_t.data_ptr(), offsets_t.data_ptr(),
                                             int(M), int(K), new_roots_t.data_ptr(), tp, ws.data_ptr(), ws.numel(),
                                             ctypes.byref(h))
        if st != OK:
            raise PbitError(st, "pbit_graph_create_batched")
        g = cls(h, (pool, roots_t, offsets_t, ws, tune_s, keep), False)
        g.new_roots = new_roots_t
        return g

    @classmethod
    def single_list(cls, pool: Pool, root: int, n: int, M: int, K: int = 4, ws=None, tune=None, keep=()):
        if ws is None:
            ws = alloc_workspace(workspace_size(pool.pool_size, 1, pool.key_type, tune))
        tune_s, tp = _tune_ptr(tune)
        h = ctypes.c_void_p()
        st = lib().pbit_graph_create_single(ctypes.addressof(pool), int(root), int(n), int(M), int(K), tp,
                                            ws.data_ptr(), ws.numel(), ctypes.byref(h))
        if st != OK:
            raise PbitError(st, "pbit_graph_create_single")
        return cls(h, (pool, ws, tune_s, keep), True)

    def launch(self, stream=None) -> None:
        st = lib().pbit_graph_launch(self._h, _stream_handle(stream))
        if st != OK:
            raise PbitError(st, "pbit_graph_launch")

    def result(self, stream=None, check: bool = True):
        """(status, new_root) of the last replay; new_root is -1 for a batched graph."""
        nr = ctypes.c_int32(-1)
        st = lib().pbit_graph_result(self._h, _stream_handle(stream), ctypes.byref(nr))
        if check and st != OK:
            raise PbitError(st, "pbit_graph_result")
        return st, int(nr.value)

    def node_count(self) -> int:
        return int(lib().pbit_graph_node_count(self._h))

    def close(self):
        if self._h:
            lib().pbit_graph_destroy(self._h)
            self._h = None
            self._keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_workspace_size(pool_size: int, num_lists: int, key_bytes: int) -> int:
    out = ctypes.c_size_t(0)
    st = lib().pbit_autotune_workspace_size(int(pool_size), int(num_lists), int(key_bytes), ctypes.byref(out))
    if st != OK:
        raise PbitError(st, "pbit_autotune_workspace_size")
    return int(out.value)


def autotune_batched(pool: Pool, roots_t: torch.Tensor, offsets_t: torch.Tensor, M: int, K: int = 4,
                     reps: int = 3, ws=None, stream=None):
    """pbit_autotune_batched: returns ({smem_cutoff, ruler_stride, digit_bits}, median ms).
    The pool is left in its input state."""
    L = roots_t.numel()
    new_roots_t = torch.empty(L, dtype=torch.int32, device=roots_t.device)
    if ws is None:
        ws = alloc_workspace(autotune_workspace_size(pool.pool_size, L, pool.key_type))
    best = Tune()
    ms = ctypes.c_float(0)
    st = lib().pbit_autotune_batched(ctypes.addressof(pool), L, roots_t.data_ptr(), offsets_t.data_ptr(), int(M),
                                     int(K), new_roots_t.data_ptr(), ws.data_ptr(), ws.numel(), int(reps),
                                     _stream_handle(stream), ctypes.addressof(best), ctypes.byref(ms))
    if st != OK:
        raise PbitError(st, "pbit_autotune_batched")
    return dict(digit_bits=best.digit_bits, smem_cutoff=best.smem_cutoff, ruler_stride=best.ruler_stride), ms.value


class Server:
    """Request server (pbit_serve_*): continuous batching of sort requests
    whose pools the caller keeps alive until they finish."""

    def __init__(self, mem_budget_bytes: int = 16 << 30, device: int = 0, streams: int = 4,
                 max_batch: int = 64, tune=None):
        self._h = ctypes.c_void_p()
        tune, tp = _tune_ptr(tune)
        st = lib().pbit_serve_create(ctypes.byref(self._h), int(mem_budget_bytes), int(device), int(streams),
                                     int(max_batch), tp)
        if st != OK:
            raise PbitError(st, "pbit_serve_create")
        self._keep = {}

    def submit(self, pool: Pool, root: int, n: int, M: int, K: int = 4, keep=None) -> int:
        """Queue one request; returns its ticket (raises on refusal)."""
        t = ctypes.c_uint64(0)
        st = lib().pbit_serve_submit(self._h, ctypes.addressof(pool), int(root), int(n), int(M), int(K),
                                     ctypes.byref(t))
        if st != OK:
            raise PbitError(st, "pbit_serve_submit")
        self._keep[t.value] = (pool, keep)
        return int(t.value)

    def poll(self, ticket: int):
        nr = ctypes.c_int32(-7)
        st = lib().pbit_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(nr))
        return st, int(nr.value)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        nr = ctypes.c_int32(-7)
        st = lib().pbit_serve_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(nr), int(timeout_ms))
        return st, int(nr.value)

    def times(self, ticket: int):
        """(submit_ns, done_ns) on the host steady clock; done_ns is 0 while pending."""
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        st = lib().pbit_serve_times(self._h, ctypes.c_uint64(ticket), ctypes.byref(a), ctypes.byref(b))
        if st != OK:
            raise PbitError(st, "pbit_serve_times")
        return int(a.value), int(b.value)

    def release(self, ticket: int) -> int:
        """Forget a finished ticket and drop the references kept for it."""
        st = lib().pbit_serve_release(self._h, ctypes.c_uint64(ticket))
        if st == OK:
            self._keep.pop(ticket, None)
        return st

    def stats(self) -> dict:
        a = (ctypes.c_int64 * 5)()
        lib().pbit_serve_stats(self._h, a)
        return dict(submitted=a[0], completed=a[1], batches=a[2], max_batch=a[3], peak_bytes=a[4])

    def close(self):
        if self._h:
            lib().pbit_serve_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
