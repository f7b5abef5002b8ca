"""THE ORACLE -- test infrastructure only.

Python handle on ``byo_oracle.c``: a plain, serial CPU restatement of the BYO
paper's definitions (CSR build, BFS, connected components, PageRank, triangle
counting, single-source betweenness, byte-coded neighbour lists, batch updates
of the edge set) plus the FP64 schedule network.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the CUDA library never does, and this module imports
nothing from it.

Pinning: every function here is checked in ``tests/test_oracle.py`` against
closed forms, brute force or an independent library routine (see the header of
that file).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

INF = 0xFFFFFFFF
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "byo_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc -O2, serial)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.ora_csr_build.restype = ctypes.c_uint64
        lib.ora_csr_build.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint64, _u64p, _u32p]
        lib.ora_bfs.restype = None
        lib.ora_bfs.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32, _u32p, _u32p]
        lib.ora_bfs_check_parents.restype = ctypes.c_int64
        lib.ora_bfs_check_parents.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32, _u32p, _u32p]
        lib.ora_cc.restype = None
        lib.ora_cc.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u32p]
        lib.ora_pagerank.restype = None
        lib.ora_pagerank.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_double, ctypes.c_uint32,
                                     _f64p, _f64p]
        lib.ora_bc.restype = None
        lib.ora_bc.argtypes = [ctypes.c_uint32, _u64p, _u32p, ctypes.c_uint32, _u32p, _f64p, _f64p]
        lib.ora_bytecode_encode.restype = ctypes.c_uint64
        lib.ora_bytecode_encode.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u64p, _u8p, ctypes.c_uint64]
        lib.ora_bytecode_decode.restype = None
        lib.ora_bytecode_decode.argtypes = [ctypes.c_uint32, _u64p, _u64p, _u8p, _u32p]
        lib.ora_tc.restype = ctypes.c_uint64
        lib.ora_tc.argtypes = [ctypes.c_uint32, _u64p, _u32p]
        lib.ora_tc_dag_build.restype = None
        lib.ora_tc_dag_build.argtypes = [ctypes.c_uint32, _u64p, _u32p, _u64p, _u32p]
        lib.ora_tc_dag_count.restype = ctypes.c_uint64
        lib.ora_tc_dag_count.argtypes = [_u64p, _u32p, ctypes.c_uint32, ctypes.c_uint32]
        lib.ora_dyn_create.restype = ctypes.c_void_p
        lib.ora_dyn_create.argtypes = [ctypes.c_uint32, _u32p, _u32p, ctypes.c_uint64]
        lib.ora_dyn_destroy.restype = None
        lib.ora_dyn_destroy.argtypes = [ctypes.c_void_p]
        lib.ora_dyn_num_edges.restype = ctypes.c_uint64
        lib.ora_dyn_num_edges.argtypes = [ctypes.c_void_p]
        lib.ora_dyn_update.restype = ctypes.c_int
        lib.ora_dyn_update.argtypes = [ctypes.c_void_p, _u32p, _u32p, ctypes.c_uint64, ctypes.c_int]
        lib.ora_dyn_export.restype = None
        lib.ora_dyn_export.argtypes = [ctypes.c_void_p, _u64p, _u32p]
        lib.ora_mlp_loss.restype = ctypes.c_double
        lib.ora_mlp_loss.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _f64p,
                                     _i32p, _f64p, ctypes.c_int, _f64p, _f64p]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as({np.dtype(np.uint32): _u32p, np.dtype(np.uint64): _u64p,
                             np.dtype(np.float64): _f64p, np.dtype(np.int32): _i32p,
                             np.dtype(np.uint8): _u8p}[a.dtype])


class CSR:
    """Oracle CSR: ``off`` (uint64, n+1) and ``col`` (uint32, m)."""

    def __init__(self, n: int, off: np.ndarray, col: np.ndarray):
        self.n, self.off, self.col = n, off, col

    @property
    def m(self) -> int:
        return int(self.off[-1])

    def degree(self) -> np.ndarray:
        return np.diff(self.off).astype(np.uint64)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.off[v]:self.off[v + 1]]


def csr_build(n: int, src, dst) -> CSR:
    src, dst = _c(src, np.uint32), _c(dst, np.uint32)
    off = np.zeros(n + 1, np.uint64)
    col = np.empty(max(2 * len(src), 1), np.uint32)
    m = int(_load().ora_csr_build(n, _p(src), _p(dst), len(src), _p(off), _p(col)))
    if m == 2**64 - 1:
        raise ValueError("ora_csr_build: vertex id out of range or allocation failure")
    return CSR(n, off, col[:m].copy())


def bfs(g: CSR, s: int):
    level = np.empty(g.n, np.uint32)
    parent = np.empty(g.n, np.uint32)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    _load().ora_bfs(g.n, _p(g.off), _p(col), s, _p(level), _p(parent))
    return level, parent


def bfs_check_parents(g: CSR, s: int, level, parent) -> int:
    """-1 when ``parent`` is a valid BFS tree for ``level``; else the first bad vertex."""
    level, parent = _c(level, np.uint32), _c(parent, np.uint32)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    return int(_load().ora_bfs_check_parents(g.n, _p(g.off), _p(col), s, _p(level), _p(parent)))


def cc(g: CSR) -> np.ndarray:
    label = np.empty(g.n, np.uint32)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    _load().ora_cc(g.n, _p(g.off), _p(col), _p(label))
    return label


def pagerank(g: CSR, damping: float = 0.85, iters: int = 20):
    p = np.empty(max(g.n, 1), np.float64)
    r = np.empty(max(iters, 1), np.float64)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    _load().ora_pagerank(g.n, _p(g.off), _p(col), damping, iters, _p(p), _p(r))
    return p[:g.n], r[:iters]


def bc(g: CSR, s: int):
    """Single-source betweenness from ``s``: (level, sigma = shortest-path
    counts, delta = dependency of s on each vertex), Brandes' accumulation."""
    level = np.empty(max(g.n, 1), np.uint32)
    sigma = np.empty(max(g.n, 1), np.float64)
    delta = np.empty(max(g.n, 1), np.float64)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    _load().ora_bc(g.n, _p(g.off), _p(col), s, _p(level), _p(sigma), _p(delta))
    return level[:g.n], sigma[:g.n], delta[:g.n]


def bytecode_encode(g: CSR):
    """Byte-coded neighbour lists: (boff uint64[n+1], bytes uint8[boff[n]])."""
    boff = np.zeros(g.n + 1, np.uint64)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    lib = _load()
    size = int(lib.ora_bytecode_encode(g.n, _p(g.off), _p(col), _p(boff), None, 0))
    if size == 2**64 - 1:  # sizing pass: no buffer
        size = int(boff[g.n])
    out = np.zeros(max(size, 1), np.uint8)
    got = int(lib.ora_bytecode_encode(g.n, _p(g.off), _p(col), _p(boff), _p(out), len(out)))
    assert got == size
    return boff, out[:size]


def bytecode_decode(n: int, off: np.ndarray, boff: np.ndarray, data: np.ndarray) -> CSR:
    """Inverse of :func:`bytecode_encode`, given the CSR offsets (degrees)."""
    off, boff = _c(off, np.uint64), _c(boff, np.uint64)
    data = _c(data, np.uint8) if len(data) else np.zeros(1, np.uint8)
    col = np.zeros(max(int(off[-1]), 1), np.uint32)
    _load().ora_bytecode_decode(n, _p(off), _p(boff), _p(data), _p(col))
    return CSR(n, off, col[:int(off[-1])].copy())


def tc(g: CSR) -> int:
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    return int(_load().ora_tc(g.n, _p(g.off), _p(col)))


def tc_dag(g: CSR):
    """Out-lists of the (degree, id)-ordered DAG: (dag_off uint64[n+1], dag_col uint32[m/2])."""
    dag_off = np.zeros(g.n + 1, np.uint64)
    dag_col = np.empty(max(g.m // 2, 1), np.uint32)
    col = g.col if len(g.col) else np.zeros(1, np.uint32)
    _load().ora_tc_dag_build(g.n, _p(g.off), _p(col), _p(dag_off), _p(dag_col))
    return dag_off, dag_col


def tc_dag_count(dag_off: np.ndarray, dag_col: np.ndarray, lo: int, hi: int) -> int:
    """Triangles counted at the DAG edges whose centre lies in [lo, hi)."""
    return int(_load().ora_tc_dag_count(_p(dag_off), _p(dag_col), lo, hi))


def tc_ordered(g: CSR, threads: int = 1, chunks: int = 1) -> int:
    """Triangle count through the degree-ordered DAG; the sum over centre
    ranges may be split across host threads (each range runs the serial C
    routine, which releases the GIL), for the full-size reference values."""
    dag_off, dag_col = tc_dag(g)
    if threads <= 1 or g.n < 2:
        return tc_dag_count(dag_off, dag_col, 0, g.n)
    import concurrent.futures as cf
    bounds = [g.n * i // chunks for i in range(chunks + 1)]
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = ex.map(lambda i: tc_dag_count(dag_off, dag_col, bounds[i], bounds[i + 1]), range(chunks))
        return sum(parts)


class DynGraph:
    """Oracle dynamic graph: the edge set under batch insert/delete."""

    def __init__(self, n: int, src, dst):
        src, dst = _c(src, np.uint32), _c(dst, np.uint32)
        self.n = n
        self._h = _load().ora_dyn_create(n, _p(src), _p(dst), len(src))
        if not self._h:
            raise ValueError("ora_dyn_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.ora_dyn_destroy(h)
            self._h = None

    @property
    def m(self) -> int:
        return int(_load().ora_dyn_num_edges(self._h))

    def update(self, src, dst, insert: bool):
        src, dst = _c(src, np.uint32), _c(dst, np.uint32)
        if _load().ora_dyn_update(self._h, _p(src), _p(dst), len(src), int(insert)) != 0:
            raise ValueError("ora_dyn_update failed")

    def insert(self, src, dst):
        self.update(src, dst, True)

    def delete(self, src, dst):
        self.update(src, dst, False)

    def csr(self) -> CSR:
        off = np.zeros(self.n + 1, np.uint64)
        col = np.empty(max(self.m, 1), np.uint32)
        _load().ora_dyn_export(self._h, _p(off), _p(col))
        return CSR(self.n, off, col[:self.m].copy())


def mlp_num_params(F: int, H1: int, H2: int, K: int) -> int:
    return H1 * F + H1 + H2 * H1 + H2 + K * H2 + K


def mlp_loss(params, F, H1, H2, K, X, y, w=None, want_grad=True):
    """FP64 loss, gradient (packed like ``params``) and logits of the schedule network."""
    params = _c(params, np.float64)
    X = _c(X, np.float64)
    y = _c(y, np.int32)
    B = len(y)
    wp = None
    if w is not None:
        w = _c(w, np.float64)
        wp = _p(w)
    grad = np.zeros(len(params), np.float64) if want_grad else None
    logits = np.zeros((B, K), np.float64)
    L = _load().ora_mlp_loss(_p(params), F, H1, H2, K, _p(X), _p(y), wp, B,
                             _p(grad) if grad is not None else None, _p(logits))
    return float(L), grad, logits
