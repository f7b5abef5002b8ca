"""Seeded synthetic graph inputs (no arithmetic of the graph method).

Shared by the oracle tests, the CUDA parity tests and ``bench.py``: each side
receives the same raw edge draws and does its own CSR build.  The C source
(``graphgen.c``) is compiled on first use with gcc; draws are counter-based, so
the output does not depend on the thread count or on the host architecture.

Workload recipes (all undirected, unweighted, as in the paper's evaluation,
Section 6.2; the paper's real graphs are replaced by these synthetic shapes):

=========  ===================================================================
name       recipe
=========  ===================================================================
tiny       ER G(n,m): n=16,384, 131,072 uniform pair draws
rmat22     RMAT scale 22, edge factor 16, a=.57 b=c=.19 d=.05, ids permuted
grid       4096x4096 4-neighbour grid, 10% edges dropped, 0.01% shortcuts
rmat24     RMAT scale 24, edge factor 16 (dynamic-container base graph)
rmat25     RMAT scale 25, edge factor 16
rmat26     RMAT scale 26, edge factor 16
=========  ===================================================================
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

GRAPH500 = (0.57, 0.19, 0.19)  # a, b, c (d = 0.05)
BASE_SEED = 0xB10
SEEDS = {"tiny": BASE_SEED + 1, "rmat22": BASE_SEED + 2, "grid": BASE_SEED + 3,
         "rmat24": BASE_SEED + 4, "batched": BASE_SEED + 5, "rmat26": BASE_SEED + 6,
         "rmat25": BASE_SEED + 7}


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, -O2, pthreads)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.gg_rand.restype = ctypes.c_uint64
        lib.gg_rand.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_stream.restype = ctypes.c_uint64
        lib.gg_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_uniform.restype = ctypes.c_double
        lib.gg_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_er.restype = None
        lib.gg_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p, ctypes.c_int]
        lib.gg_rmat.restype = ctypes.c_int
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int, u32p, u32p, ctypes.c_int]
        lib.gg_permutation.restype = None
        lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
        lib.gg_grid_capacity.restype = ctypes.c_uint64
        lib.gg_grid_capacity.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double]
        lib.gg_grid.restype = ctypes.c_uint64
        lib.gg_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                ctypes.c_uint64, u32p, u32p, ctypes.c_uint64]
        lib.gg_pick_sources.restype = ctypes.c_int64
        lib.gg_pick_sources.argtypes = [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint64, u32p]
        lib.gg_pick_indices.restype = None
        lib.gg_pick_indices.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, u64p]
        _lib = lib
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def rand(seed: int, i: int) -> int:
    """Draw i of the SplitMix64 stream seeded with ``seed``."""
    return int(_load().gg_rand(seed & (2**64 - 1), i))


def stream(seed: int, tag: int) -> int:
    return int(_load().gg_stream(seed & (2**64 - 1), tag))


def uniform(seed: int, i: int) -> float:
    return float(_load().gg_uniform(seed & (2**64 - 1), i))


def er(n: int, k: int, seed: int):
    """k ordered pairs uniform on [0,n)^2 (self-loops and duplicates kept)."""
    src = np.empty(k, np.uint32)
    dst = np.empty(k, np.uint32)
    if k:
        _load().gg_er(n, k, seed, _p32(src), _p32(dst), _threads())
    return src, dst


def rmat(scale: int, k: int, seed: int, abc=GRAPH500, permute: bool = True):
    """k RMAT draws on 2^scale vertices; ids optionally relabelled by a seeded permutation."""
    src = np.empty(k, np.uint32)
    dst = np.empty(k, np.uint32)
    a, b, c = abc
    rc = _load().gg_rmat(scale, k, a, b, c, seed, int(permute), _p32(src), _p32(dst), _threads())
    if rc != 0:
        raise MemoryError("gg_rmat failed")
    return src, dst


def permutation(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.uint32)
    _load().gg_permutation(n, seed, _p32(out))
    return out


def grid(rows: int, cols: int, drop: float, shortcut_frac: float, seed: int):
    cap = int(_load().gg_grid_capacity(rows, cols, shortcut_frac))
    src = np.empty(cap, np.uint32)
    dst = np.empty(cap, np.uint32)
    k = int(_load().gg_grid(rows, cols, drop, shortcut_frac, seed, _p32(src), _p32(dst), cap))
    if cap and k == 0 and rows * cols > 1:
        raise RuntimeError("grid capacity exceeded")
    return src[:k].copy(), dst[:k].copy()


def pick_sources(n: int, src: np.ndarray, dst: np.ndarray, count: int, seed: int) -> np.ndarray:
    """Distinct sources uniform among vertices touched by a non-loop draw."""
    out = np.empty(max(count, 1), np.uint32)
    src = np.ascontiguousarray(src, np.uint32)
    dst = np.ascontiguousarray(dst, np.uint32)
    got = int(_load().gg_pick_sources(n, _p32(src), _p32(dst), len(src), count, seed, _p32(out)))
    if got < 0:
        raise MemoryError("gg_pick_sources failed")
    return out[:got].copy()


def pick_indices(pool: int, count: int, seed: int) -> np.ndarray:
    out = np.empty(count, np.uint64)
    if count:
        _load().gg_pick_indices(pool, count, seed, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return out


# ----------------------------------------------------------------------------
# workload recipes
# ----------------------------------------------------------------------------

def workload(name: str, seed: int | None = None):
    """Return (n, src, dst) raw draws for a named workload."""
    s = SEEDS.get(name, BASE_SEED) if seed is None else seed
    if name == "tiny":
        n = 16384
        src, dst = er(n, 131072, s)
        return n, src, dst
    if name.startswith("rmat"):
        scale = int(name[4:])
        src, dst = rmat(scale, 16 << scale, s)
        return 1 << scale, src, dst
    if name == "grid":
        src, dst = grid(4096, 4096, 0.10, 1e-4, s)
        return 4096 * 4096, src, dst
    raise KeyError(name)


def rmat_small(scale: int, ef: int, seed: int, permute: bool = True):
    """(n, src, dst) for an RMAT graph of any scale (test sizes)."""
    src, dst = rmat(scale, ef << scale, seed, GRAPH500, permute)
    return 1 << scale, src, dst


def grid_small(rows: int, cols: int, drop: float, shortcut_frac: float, seed: int):
    src, dst = grid(rows, cols, drop, shortcut_frac, seed)
    return rows * cols, src, dst


def batched_params(count: int = 256, seed: int | None = None, lo_log2: int = 10, hi_log2: int = 18,
                   deg_lo: float = 4.0, deg_hi: float = 64.0):
    """Per-member (kind, n, draws, seed) for the many-graphs workload.

    Half ER, half RMAT (Graph500 a,b,c).  n is log-uniform in [2^lo, 2^hi]:
    RMAT members draw the scale uniformly from {lo..hi}; ER members draw
    log2(n) uniformly on [lo, hi] and round.  The average degree of the
    symmetrised graph is uniform in [deg_lo, deg_hi], so draws = n*deg/2.
    """
    base = SEEDS["batched"] if seed is None else seed
    ps = stream(base, 40)
    out = []
    for g in range(count):
        kind = "er" if g < count // 2 else "rmat"
        u = uniform(ps, 3 * g)
        deg = deg_lo + (deg_hi - deg_lo) * uniform(ps, 3 * g + 1)
        if kind == "rmat":
            scale = lo_log2 + min(hi_log2 - lo_log2, int(u * (hi_log2 - lo_log2 + 1)))
            n = 1 << scale
        else:
            n = int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))
        k = int(n * deg / 2)
        out.append((kind, n, k, stream(base, 1000 + g)))
    return out


def batched_member(kind: str, n: int, k: int, seed: int):
    if kind == "er":
        return er(n, k, seed)
    return rmat(int(round(math.log2(n))), k, seed)


def batched_workload(count: int = 256, sources: int = 64):
    """The many-graphs workload: per member (n, src, dst) with LOCAL ids and
    ``sources`` BFS sources (distinct non-isolated vertices where the member
    has that many, then 0, 1, 2, ... to fill the row)."""
    members = []
    for kind, n, k, sd in batched_params(count):
        s, d = batched_member(kind, n, k, sd)
        picked = pick_sources(n, s, d, sources, sd + 1).tolist()
        picked += [v % n for v in range(sources - len(picked))]
        members.append((n, s, d, picked[:sources]))
    return members


def dynamic_rounds(n: int, src: np.ndarray, dst: np.ndarray, rounds: int = 10, batch: int = 1_000_000,
                   seed: int | None = None, scale: int = 24):
    """Update batches of the dynamic-container workload, one per round:
    (insert_src, insert_dst, delete_src, delete_dst).  Inserts are ``batch``
    RMAT draws; deletes are ``batch`` pairs drawn uniformly (with repetition)
    from every pair inserted before this round, the base graph included."""
    s = SEEDS["rmat24"] if seed is None else seed
    pool_s, pool_d = [src], [dst]
    for r in range(rounds):
        ins_s, ins_d = rmat(scale, batch, stream(s, 100 + r))
        ps, pd = np.concatenate(pool_s), np.concatenate(pool_d)
        pick = pick_indices(len(ps), batch, stream(s, 200 + r))
        yield ins_s, ins_d, ps[pick], pd[pick]
        pool_s.append(ins_s)
        pool_d.append(ins_d)

