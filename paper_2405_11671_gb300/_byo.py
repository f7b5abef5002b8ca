"""ctypes binding of libbyo.so: the same names as ``include/byo.h``.

Argument marshalling only -- every step of every algorithm runs in the CUDA
library.  Device buffers are torch CUDA tensors (``data_ptr()`` is passed), the
stream is torch's current stream unless one is given.  There is no CPU
fallback: if ``libbyo.so`` is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbyo.so")

BYO_OK = 0
BYO_ERR_INVALID_ARG = 1
BYO_ERR_OUT_OF_MEMORY = 2
BYO_ERR_CUDA = 3
BYO_ERR_TIMEOUT = 4
BYO_ERR_UNSUPPORTED = 5
BYO_ERR_NOT_SYMMETRIC = 6
BYO_INF = 0xFFFFFFFF

BYO_CSR = 0x1
BYO_DYNAMIC = 0x2
BYO_SYMMETRIZE = 0x4
BYO_OFFSETS64 = 0x8
BYO_DYN_NO_INLINE = 0x10
BYO_COMPRESSED = 0x20
BYO_DYN_HASH = 0x40

BYO_SCHED_HEURISTIC = 0
BYO_SCHED_LEARNED = 1
BYO_SCHED_PUSH = 2
BYO_SCHED_PULL = 3
BYO_SCHED_FIXED = 4
BYO_NUM_ACTIONS = 5
BYO_SCHED_NO_EARLY_EXIT = 0x1
BYO_SCHED_SEQUENTIAL_MAPS = 0x2


class ByoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"byo status {status}: {msg}")
        self.status = status


class byo_sched(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("thr_thread", ctypes.c_uint32), ("thr_warp", ctypes.c_uint32),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_float), ("mlp", ctypes.c_void_p),
                ("action", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class byo_bfs_iter(ctypes.Structure):
    _fields_ = [("level", ctypes.c_uint32), ("direction", ctypes.c_uint32), ("action", ctypes.c_uint32),
                ("frontier", ctypes.c_uint32), ("frontier_edges", ctypes.c_uint64),
                ("edges_examined", ctypes.c_uint64), ("unvisited_edges", ctypes.c_uint64),
                ("unvisited", ctypes.c_uint32), ("hist", ctypes.c_uint32 * 4), ("reserved", ctypes.c_uint32),
                ("t_ns", ctypes.c_uint64)]


class byo_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_st = ctypes.c_int

# (name, restype, argtypes) of every exported symbol declared in include/byo.h
SIGNATURES = [
    ("byo_last_error", ctypes.c_char_p, []),
    ("byo_graph_build", _st, [_u32, _vp, _vp, _u64, _u32, _vp, ctypes.POINTER(_vp)]),
    ("byo_graph_destroy", _st, [_vp]),
    ("byo_space", _st, [_vp, ctypes.POINTER(_u64), _vp]),
    ("byo_export_codes", _st, [_vp, _vp, _vp, ctypes.POINTER(_u64), _vp]),
    ("byo_num_vertices", _st, [_vp, ctypes.POINTER(_u32)]),
    ("byo_num_edges", _st, [_vp, ctypes.POINTER(_u64)]),
    ("byo_degree", _st, [_vp, _vp, _u64, _vp, _vp]),
    ("byo_graph_export_csr", _st, [_vp, _vp, _vp, _vp]),
    ("byo_insert_batch", _st, [_vp, _vp, _vp, _u64, _vp]),
    ("byo_delete_batch", _st, [_vp, _vp, _vp, _u64, _vp]),
    ("byo_sched_default", byo_sched, []),
    ("byo_bfs", _st, [_vp, ctypes.POINTER(_u32), _u32, _vp, _vp, ctypes.POINTER(byo_sched), _vp]),
    ("byo_bfs_trace", _st, [_vp, ctypes.POINTER(byo_bfs_iter), _u32, ctypes.POINTER(_u32), _vp]),
    ("byo_cc", _st, [_vp, _vp, _vp]),
    ("byo_pagerank", _st, [_vp, ctypes.c_float, _u32, _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    ("byo_tc", _st, [_vp, ctypes.POINTER(_u64), _vp]),
    ("byo_tc_work", _st, [_vp, ctypes.POINTER(_u64), _vp]),
    ("byo_bc", _st, [_vp, _u32, _vp, _vp, _vp, _vp]),
    ("byo_mlp_num_params", _u32, []),
    ("byo_mlp_create", _st, [_u64, ctypes.POINTER(_vp)]),
    ("byo_mlp_destroy", _st, [_vp]),
    ("byo_mlp_get_params", _st, [_vp, _vp]),
    ("byo_mlp_set_params", _st, [_vp, _vp]),
    ("byo_mlp_loss_grad", _st, [_vp, _vp, _vp, _vp, _u32, _vp, ctypes.POINTER(ctypes.c_float), _vp]),
    ("byo_mlp_train", _st, [_vp, _vp, _vp, _vp, _u32, _u32, ctypes.c_float, ctypes.POINTER(ctypes.c_float), _vp]),
    ("byo_mlp_predict", _st, [_vp, _vp, _u32, _vp, _vp]),
    ("byo_batch_build", _st, [_u32, ctypes.POINTER(_u32), ctypes.POINTER(_u64), _vp, _vp, _u32, _vp,
                               ctypes.POINTER(_vp)]),
    ("byo_batch_member_base", _st, [_vp, _u32, ctypes.POINTER(_u32)]),
    ("byo_msbfs", _st, [_vp, ctypes.POINTER(_u32), _u32, _vp, ctypes.POINTER(byo_sched), _vp]),
    ("byo_bfs_noalloc", _st, [_u32, _u64, _vp, _vp, _u32, _vp, _vp, ctypes.POINTER(byo_sched), _vp]),
    ("byo_kernel_launches", _u64, []),
    ("byo_profile_enable", _st, [ctypes.c_int]),
    ("byo_profile_reset", _st, []),
    ("byo_profile_read", _st, [ctypes.POINTER(byo_kernel_stat), _u32, ctypes.POINTER(_u32)]),
]

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libbyo.so (built by ``paper_2405_11671_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing: build it with `python -m paper_2405_11671_gb300.build` "
                                  "(there is no CPU fallback)")
            lib = ctypes.CDLL(p)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != BYO_OK:
        msg = load().byo_last_error()
        raise ByoError(status, msg.decode() if msg else "")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _u32t(t: torch.Tensor, name: str) -> torch.Tensor:
    """A CUDA tensor of 32-bit ids (int32 or uint32; the library reads them as uint32)."""
    ok = (torch.int32,) + ((torch.uint32,) if hasattr(torch, "uint32") else ())
    if not isinstance(t, torch.Tensor) or t.dtype not in ok:
        raise TypeError(f"{name} must be an int32/uint32 CUDA tensor")
    return _dev(t, t.dtype, name)


# ----------------------------------------------------------------------------- graph

def byo_graph_build(n: int, src: torch.Tensor, dst: torch.Tensor, flags: int = BYO_CSR | BYO_SYMMETRIZE,
                    stream=None) -> int:
    """Handle of a new container built from device pair arrays (int32/uint32, same length)."""
    src = _u32t(src, "src")
    dst = _u32t(dst, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    out = _vp()
    _check(load().byo_graph_build(n, src.data_ptr(), dst.data_ptr(), src.numel(), flags, _stream(stream),
                                  ctypes.byref(out)))
    return out.value


def byo_graph_destroy(g: int) -> None:
    _check(load().byo_graph_destroy(g))


def byo_space(g: int, stream=None) -> int:
    """Bytes the container occupies (CSR arrays, or records + held pool blocks)."""
    v = _u64()
    _check(load().byo_space(g, ctypes.byref(v), _stream(stream)))
    return v.value


def byo_export_codes(g: int, stream=None):
    """(boff int64[n+1], bytes uint8[boff[n]]) of a compressed container (device tensors)."""
    n = byo_num_vertices(g)
    boff = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    nb = _u64()
    _check(load().byo_export_codes(g, boff.data_ptr(), None, ctypes.byref(nb), _stream(stream)))
    data = torch.empty(max(nb.value, 1), dtype=torch.uint8, device="cuda")
    _check(load().byo_export_codes(g, boff.data_ptr(), data.data_ptr(), ctypes.byref(nb), _stream(stream)))
    return boff, data[:nb.value]


def byo_num_vertices(g: int) -> int:
    v = _u32()
    _check(load().byo_num_vertices(g, ctypes.byref(v)))
    return v.value


def byo_num_edges(g: int) -> int:
    v = _u64()
    _check(load().byo_num_edges(g, ctypes.byref(v)))
    return v.value


def byo_degree(g: int, vs: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None):
    n = byo_num_vertices(g)
    k = n if vs is None else vs.numel()
    dev = vs.device if vs is not None else torch.device("cuda")
    if out is None:
        out = torch.empty(k, dtype=torch.int32, device=dev)
    vp = 0 if vs is None else _u32t(vs, "vs").data_ptr()
    _check(load().byo_degree(g, vp, k, out.data_ptr(), _stream(stream)))
    return out


def byo_graph_export_csr(g: int, stream=None):
    n, m = byo_num_vertices(g), byo_num_edges(g)
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    _check(load().byo_graph_export_csr(g, off.data_ptr(), col.data_ptr(), _stream(stream)))
    return off, col[:m]


def byo_insert_batch(g: int, src: torch.Tensor, dst: torch.Tensor, stream=None) -> None:
    src, dst = _u32t(src, "src"), _u32t(dst, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    _check(load().byo_insert_batch(g, src.data_ptr(), dst.data_ptr(), src.numel(), _stream(stream)))


def byo_delete_batch(g: int, src: torch.Tensor, dst: torch.Tensor, stream=None) -> None:
    src, dst = _u32t(src, "src"), _u32t(dst, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    _check(load().byo_delete_batch(g, src.data_ptr(), dst.data_ptr(), src.numel(), _stream(stream)))


# ----------------------------------------------------------------------------- algorithms

def byo_sched_default() -> byo_sched:
    return load().byo_sched_default()


def make_sched(mode: int = BYO_SCHED_HEURISTIC, thr_thread: int = 16, thr_warp: int = 1024, alpha: float = 15.0,
               beta: float = 18.0, mlp: int | None = None, action: int = 1, flags: int = 0) -> byo_sched:
    return byo_sched(mode, thr_thread, thr_warp, alpha, beta, mlp, action, flags)


def byo_bfs(g: int, sources, levels: torch.Tensor | None = None, parents: torch.Tensor | None = None,
            sched: byo_sched | None = None, want_parents: bool = True, stream=None):
    """levels[len(sources), n] (int32; INF = -1 as int32) and optionally parents."""
    srcs = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32).reshape(-1))
    n = byo_num_vertices(g)
    ns = len(srcs)
    if levels is None:
        levels = torch.empty((ns, n), dtype=torch.int32, device="cuda")
    if parents is None and want_parents:
        parents = torch.empty((ns, n), dtype=torch.int32, device="cuda")
    sp = ctypes.byref(sched) if sched is not None else None
    _check(load().byo_bfs(g, srcs.ctypes.data_as(ctypes.POINTER(_u32)), ns, levels.data_ptr(),
                          parents.data_ptr() if parents is not None else None, sp, _stream(stream)))
    return levels, parents


def byo_bfs_trace(g: int, cap: int = 1 << 16, stream=None):
    recs = (byo_bfs_iter * cap)()
    cnt = _u32()
    _check(load().byo_bfs_trace(g, recs, cap, ctypes.byref(cnt), _stream(stream)))
    return [recs[i] for i in range(min(cnt.value, cap))]


def byo_cc(g: int, labels: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = byo_num_vertices(g)
    if labels is None:
        labels = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(load().byo_cc(g, labels.data_ptr(), _stream(stream)))
    return labels


def byo_pagerank(g: int, damping: float = 0.85, iters: int = 20, ranks: torch.Tensor | None = None,
                 want_residual: bool = True, stream=None):
    n = byo_num_vertices(g)
    if ranks is None:
        ranks = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    r = ctypes.c_double(0.0)
    _check(load().byo_pagerank(g, damping, iters, ranks.data_ptr(), ctypes.byref(r) if want_residual else None,
                               _stream(stream)))
    return ranks[:n], (r.value if want_residual else None)


def byo_tc(g: int, stream=None) -> int:
    c = _u64()
    _check(load().byo_tc(g, ctypes.byref(c), _stream(stream)))
    return c.value


def byo_tc_work(g: int, stream=None):
    """(sum d+^2, sum d- d+, walked ids) of the triangle-count DAG."""
    w = (_u64 * 3)()
    _check(load().byo_tc_work(g, w, _stream(stream)))
    return int(w[0]), int(w[1]), int(w[2])


def byo_bc(g: int, source: int, levels: torch.Tensor | None = None, stream=None):
    """(levels int32[n], sigma float64[n], delta float64[n]) of single-source betweenness."""
    n = byo_num_vertices(g)
    sigma = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    delta = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    if levels is None:
        levels = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    _check(load().byo_bc(g, source, _u32t(levels, "levels").data_ptr(), sigma.data_ptr(), delta.data_ptr(),
                         _stream(stream)))
    return levels[:n], sigma[:n], delta[:n]


# ----------------------------------------------------------------------------- schedule network

def byo_mlp_num_params() -> int:
    return int(load().byo_mlp_num_params())


def byo_mlp_create(seed: int = 0) -> int:
    out = _vp()
    _check(load().byo_mlp_create(seed, ctypes.byref(out)))
    return out.value


def byo_mlp_destroy(m: int) -> None:
    _check(load().byo_mlp_destroy(m))


def byo_mlp_get_params(m: int) -> np.ndarray:
    out = np.empty(byo_mlp_num_params(), np.float32)
    _check(load().byo_mlp_get_params(m, out.ctypes.data))
    return out


def byo_mlp_set_params(m: int, params) -> None:
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != byo_mlp_num_params():
        raise ValueError("wrong parameter count")
    _check(load().byo_mlp_set_params(m, p.ctypes.data))


def byo_mlp_loss_grad(m: int, X: torch.Tensor, y: torch.Tensor, w: torch.Tensor | None = None, stream=None):
    grad = torch.empty(byo_mlp_num_params(), dtype=torch.float32, device="cuda")
    loss = ctypes.c_float(0.0)
    _check(load().byo_mlp_loss_grad(m, _dev(X, torch.float32, "X").data_ptr(), _dev(y, torch.int32, "y").data_ptr(),
                                    _dev(w, torch.float32, "w").data_ptr() if w is not None else None, y.numel(),
                                    grad.data_ptr(), ctypes.byref(loss), _stream(stream)))
    return loss.value, grad


def byo_mlp_train(m: int, X: torch.Tensor, y: torch.Tensor, w: torch.Tensor | None = None, epochs: int = 200,
                  lr: float = 1e-2, stream=None) -> float:
    loss = ctypes.c_float(0.0)
    _check(load().byo_mlp_train(m, _dev(X, torch.float32, "X").data_ptr(), _dev(y, torch.int32, "y").data_ptr(),
                                _dev(w, torch.float32, "w").data_ptr() if w is not None else None, y.numel(), epochs,
                                lr, ctypes.byref(loss), _stream(stream)))
    return loss.value


def byo_mlp_predict(m: int, X: torch.Tensor, stream=None) -> torch.Tensor:
    X = _dev(X, torch.float32, "X")
    out = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    _check(load().byo_mlp_predict(m, X.data_ptr(), X.shape[0], out.data_ptr(), _stream(stream)))
    return out


def byo_batch_build(ns, ks, src: torch.Tensor, dst: torch.Tensor, flags: int = BYO_CSR | BYO_SYMMETRIZE,
                    stream=None) -> int:
    """One container over the disjoint union of len(ns) graphs (local-id pairs concatenated)."""
    n_arr = np.ascontiguousarray(np.asarray(ns, dtype=np.uint32))
    k_arr = np.ascontiguousarray(np.asarray(ks, dtype=np.uint64))
    src, dst = _u32t(src, "src"), _u32t(dst, "dst")
    if src.numel() != int(k_arr.sum()) or dst.numel() != src.numel():
        raise ValueError("pair arrays do not match the per-member counts")
    out = _vp()
    _check(load().byo_batch_build(len(n_arr), n_arr.ctypes.data_as(ctypes.POINTER(_u32)),
                                  k_arr.ctypes.data_as(ctypes.POINTER(_u64)), src.data_ptr(), dst.data_ptr(), flags,
                                  _stream(stream), ctypes.byref(out)))
    return out.value


def byo_batch_member_base(g: int, i: int) -> int:
    v = _u32()
    _check(load().byo_batch_member_base(g, i, ctypes.byref(v)))
    return v.value


def byo_msbfs(g: int, sources, num_sources: int, levels: torch.Tensor | None = None,
              sched: byo_sched | None = None, stream=None) -> torch.Tensor:
    """levels[num_sources, n]; sources = members x num_sources LOCAL ids (row-major)."""
    srcs = np.ascontiguousarray(np.asarray(sources, dtype=np.uint32).reshape(-1))
    n = byo_num_vertices(g)
    if levels is None:
        levels = torch.empty((num_sources, n), dtype=torch.int32, device="cuda")
    sp = ctypes.byref(sched) if sched is not None else None
    _check(load().byo_msbfs(g, srcs.ctypes.data_as(ctypes.POINTER(_u32)), num_sources, levels.data_ptr(), sp,
                            _stream(stream)))
    return levels


BYO_NOALLOC_MAX_VERTICES = 1 << 20


def byo_bfs_noalloc(n: int, m: int, offsets: torch.Tensor, col: torch.Tensor, source: int, levels: torch.Tensor,
                    parents: torch.Tensor | None = None, sched: byo_sched | None = None, stream=None) -> None:
    """BFS from one source over a caller-owned CSR, using only the library's
    built-in scratch array (no device allocation by the library or here).
    offsets: int64 CUDA tensor [n+1]; col: int32 CUDA tensor, 16-byte aligned,
    with at least m+4 entries; levels/parents: int32 CUDA tensors [n]."""
    _dev(offsets, torch.int64, "offsets")
    _u32t(col, "col")
    _u32t(levels, "levels")
    if parents is not None:
        _u32t(parents, "parents")
    # the kernel trusts these sizes: check them here, before the call
    if offsets.numel() < n + 1:
        raise ValueError(f"offsets has {offsets.numel()} entries, needs n+1 = {n + 1}")
    if col.numel() < m + 4:
        raise ValueError(f"col has {col.numel()} entries, needs m+4 = {m + 4} (16-byte vector reads of the tail)")
    if col.data_ptr() % 16:
        raise ValueError("col must start on a 16-byte boundary")
    if levels.numel() < n or (parents is not None and parents.numel() < n):
        raise ValueError(f"levels/parents need n = {n} entries")
    sp = ctypes.byref(sched) if sched is not None else None
    _check(load().byo_bfs_noalloc(n, m, offsets.data_ptr(), col.data_ptr(), source, levels.data_ptr(),
                                  parents.data_ptr() if parents is not None else None, sp, _stream(stream)))


# ----------------------------------------------------------------------------- tracing

def byo_kernel_launches() -> int:
    return int(load().byo_kernel_launches())


def byo_profile_enable(on: bool = True) -> None:
    _check(load().byo_profile_enable(int(bool(on))))


def byo_profile_reset() -> None:
    _check(load().byo_profile_reset())


def byo_profile_read(cap: int = 64) -> dict:
    """{kernel name: (launches, total device ms)} since the last reset."""
    recs = (byo_kernel_stat * cap)()
    cnt = _u32()
    _check(load().byo_profile_read(recs, cap, ctypes.byref(cnt)))
    return {recs[i].name.decode(): (int(recs[i].launches), float(recs[i].total_ms))
            for i in range(min(cnt.value, cap))}


# ----------------------------------------------------------------------------- convenience

class Graph:
    """Owning wrapper of a byo_graph handle."""

    def __init__(self, n: int, src: torch.Tensor, dst: torch.Tensor, flags: int = BYO_CSR | BYO_SYMMETRIZE,
                 stream=None):
        self.handle = byo_graph_build(n, src, dst, flags, stream)

    def close(self):
        if self.handle:
            byo_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return byo_num_vertices(self.handle)

    @property
    def m(self) -> int:
        return byo_num_edges(self.handle)
