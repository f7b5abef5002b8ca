"""Autotuner for the schedule parameters of BFS and multi-source BFS.

For a given container and workload it times a small grid of candidates on the
device (CUDA events, best of `repeats`) and keeps the fastest:

* BFS: the push bins (thr_thread, thr_warp) under the direction heuristic;
* multi-source BFS: alpha, the top-down / bottom-up switch.

Results are cached in a JSON file keyed by the GPU name, the operation and the
workload's size (``BYO_AUTOTUNE_CACHE``, default ``~/.cache/byo_gb300/autotune.json``),
so later runs of the same workload reuse them without timing.  Tuning never
changes results: every candidate computes the same levels.
"""
from __future__ import annotations

import json
import os

BFS_BINS = ((2, 64), (4, 128), (8, 512), (16, 1024), (32, 2048), (64, 4096))
MSBFS_ALPHAS = (1.0, 4.0, 15.0, 40.0, 120.0)


def _cache_path() -> str:
    return os.environ.get("BYO_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "byo_gb300", "autotune.json"))


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    c = _load_cache()
    c[key] = value
    p = _cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _key(byo, g, op: str, extra: str = "") -> str:
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|{op}|n={byo.byo_num_vertices(g)}|m={byo.byo_num_edges(g)}{extra}"


def _time(fn, repeats: int) -> float:
    import torch
    fn()
    best = float("inf")
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_bfs(byo, g: int, sources, repeats: int = 3, use_cache: bool = True) -> dict:
    """Fastest push bins for the heuristic BFS schedule on this graph."""
    key = _key(byo, g, "bfs", f"|S={len(sources)}")
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit
    table = {}
    for tt, tw in BFS_BINS:
        sp = byo.make_sched(byo.BYO_SCHED_HEURISTIC, tt, tw)
        table[f"{tt},{tw}"] = _time(lambda: byo.byo_bfs(g, sources, sched=sp, want_parents=False), repeats)
    best = min(table, key=table.get)
    tt, tw = (int(x) for x in best.split(","))
    res = {"thr_thread": tt, "thr_warp": tw, "ms": table[best], "table_ms": table}
    _store(key, res)
    return res


def tune_msbfs(byo, g: int, sources, num_sources: int, levels=None, repeats: int = 3, use_cache: bool = True) -> dict:
    """Fastest top-down / bottom-up switch for multi-source BFS on this batch."""
    key = _key(byo, g, "msbfs", f"|S={num_sources}")
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return hit
    table = {}
    for a in MSBFS_ALPHAS:
        sp = byo.make_sched(byo.BYO_SCHED_HEURISTIC, 16, 1024, a)
        table[str(a)] = _time(lambda: byo.byo_msbfs(g, sources, num_sources, levels, sched=sp), repeats)
    best = min(table, key=table.get)
    res = {"alpha": float(best), "ms": table[best], "table_ms": table}
    _store(key, res)
    return res
