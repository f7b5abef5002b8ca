#!/usr/bin/env python3
"""Benchmark of the BYO hot path on GB300: BFS, CC, PageRank and TC on one graph.

One step = one pass of the whole path over a resident graph: BFS from S
seeded non-isolated sources (levels + parents), connected components,
PageRank (d = 0.85, 20 iterations), triangle count.  The metric is traversed
edges per second over the step (GTEPS), with each algorithm's edges counted by
its usual convention:
  BFS  undirected edges in the source's component, per source (Graph500)
  CC   m/2 (every undirected edge once)
  PR   20 * m (every stored entry, every iteration)
  TC   m
``value`` times the step with the graph already in HBM; ``e2e`` times the same
step through the C ABI from host buffers: pinned host -> device copy of the
pair arrays, CSR build, the four algorithms, device -> host copy of levels,
labels and ranks -- as a streaming pipeline in which step i+1's input copy
overlaps step i and step i's output copy overlaps its triangle count.

After the timed region the line also carries the BFS schedules side by side
(learned, heuristic, push, pull; median of repeated 8-source runs) on this
graph and on the high-diameter grid, and the bandwidth of the largest push and
pull levels.  Byte counts are the method's (what the algorithm must move, from
its outputs), never a kernel's own counters.

  python bench.py [--gpus N --steps K --warmup W --workload rmat25 --sources 8]
  python bench.py --workload batched | dynamic | ablation | space
  python bench.py --impl reference ...   # the serial CPU oracle, bounded sample

N > 1 (torchrun, one rank per GPU) runs independent replicas: the path does not
shard (replicas only), so value = edges of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS & % HBM roofline (BFS/PR/CC/TC, RMAT-25); learned vs heuristic schedule"
PR_ITERS = 20
DAMPING = 0.85
INF = 0xFFFFFFFF
SCHEDULES = ("learned", "heuristic", "push", "pull")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="byo", choices=["byo", "reference"])
    ap.add_argument("--workload", default="rmat25")
    ap.add_argument("--sources", type=int, default=8)
    ap.add_argument("--sched", default="heuristic", choices=["heuristic", "push", "pull", "learned", "solo"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-schedules", action="store_true", help="skip the schedule comparison")
    ap.add_argument("--sched-reps", type=int, default=5, help="timed repetitions per schedule")
    ap.add_argument("--sample-scale", type=int, default=18, help="RMAT scale of the oracle's bounded sample")
    ap.add_argument("--rounds", type=int, default=10, help="update rounds of the dynamic workload")
    ap.add_argument("--dyn-scale", type=int, default=24,
                    help="RMAT scale of the dynamic workload's base graph (batches scale with it)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers

def reduce_over_ranks(dist, x: float, op: str, device: str) -> float:
    """MAX or SUM of a per-rank float over the process group (identity alone)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_value(dist, edges_per_step: float, ms_per_step: float, device: str) -> tuple[float, float]:
    """Whole-job GTEPS of independent replicas: edges of all ranks over the
    slowest rank's step time.  Returns (GTEPS, max ms per step)."""
    ms = reduce_over_ranks(dist, ms_per_step, "max", device)
    edges = reduce_over_ranks(dist, edges_per_step, "sum", device)
    return edges / (ms / 1e3) / 1e9, ms


def dev_u32(torch, a):
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def pinned_u32(torch, a):
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).pin_memory()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def sched_struct(byo, name, mlp=None):
    if name == "solo":  # push by one CTA at every level
        return byo.make_sched(byo.BYO_SCHED_FIXED, 16, 1024, 15.0, 18.0, None, 4)
    mode = {"heuristic": byo.BYO_SCHED_HEURISTIC, "push": byo.BYO_SCHED_PUSH, "pull": byo.BYO_SCHED_PULL,
            "learned": byo.BYO_SCHED_LEARNED}[name]
    return byo.make_sched(mode, 16, 1024, 15.0, 18.0, mlp)


def load_mlp(byo):
    import numpy as np
    p = os.path.join(ROOT, "paper_2405_11671_gb300", "sched_mlp.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        prm = np.array(json.load(f)["params"], np.float32)
    m = byo.byo_mlp_create(0)
    byo.byo_mlp_set_params(m, prm)
    return m


def roof_entry(name, bytes_, avg_ms, peak, peak_kind, share=None):
    achieved = bytes_ / (avg_ms / 1e3) / 1e9
    e = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
         "frac": round(achieved / peak, 4), "traffic": None, "algorithmic_bytes_per_launch": bytes_,
         "avg_launch_ms": round(avg_ms, 4), "peak_kind": peak_kind}
    if share is not None:
        e["share"] = round(share, 4)
    return e


# ----------------------------------------------------------------------------- algorithmic bytes

def algo_bytes(kernel: str, n: int, m: int, off: int) -> float | None:
    """Bytes the method must move per launch of `kernel` (a model, not a counter)."""
    if kernel == "pr_iter":
        # offsets of the degree-ordered copy (always 8 bytes) + neighbour ids + one
        # read of every contribution + read/write rank + write next contribution
        return 8.0 * (n + 1) + 4.0 * m + 16.0 * n
    if kernel == "cc_sample":
        # identity labels, two sampling rounds (offsets, one neighbour id and the
        # two endpoints' labels each), one flattening pass (read + write)
        return 4.0 * n + 2 * (off * (n + 1) + 4.0 * n + 8.0 * n) + 8.0 * n
    if kernel == "tc_fill":
        # offsets and ids of the graph, the rank of every vertex and of every
        # neighbour, the DAG rows written (4 B per entry), row starts and records
        return off * (n + 1) + 4.0 * n + 4.0 * m + 4.0 * m + 4.0 * m + 8.0 * (n + 1) + 16.0 * n
    return None


def _vertex_chunks(torch, off, chunk_edges):
    """Vertex ranges [v0, v1) holding about chunk_edges neighbour entries each."""
    n = off.numel() - 1
    v0 = 0
    while v0 < n:
        target = torch.tensor([int(off[v0]) + chunk_edges], dtype=off.dtype, device=off.device)
        v1 = int(torch.searchsorted(off, target, right=True)[0]) - 1
        v1 = min(n, max(v1, v0 + 1))
        yield v0, v1
        v0 = v1


def first_hit_positions(torch, off, col, want_level, lvl, chunk_edges=1 << 26):
    """fp[v] = index, within N(v) in stored (ascending) order, of the first
    neighbour u with lvl[u] == want_level[v]; -1 where there is none or
    want_level[v] is negative.  lvl and want_level are int64."""
    n = off.numel() - 1
    fp = torch.full((n,), -1, dtype=torch.long, device=lvl.device)
    deg = off[1:] - off[:-1]
    for v0, v1 in _vertex_chunks(torch, off, chunk_edges):
        e0, e1 = int(off[v0]), int(off[v1])
        if e1 == e0:
            continue
        rows = torch.repeat_interleave(torch.arange(v0, v1, device=lvl.device), deg[v0:v1])
        nb = col[e0:e1].long() & INF
        w = want_level[rows]
        hit = (w >= 0) & (lvl[nb] == w)
        pos = torch.arange(e0, e1, device=lvl.device) - off[rows]
        fp.scatter_reduce_(0, rows[hit], pos[hit], reduce="amin", include_self=False)
    return fp


def bfs_method_bytes(torch, off, col, lv, trace, off_bytes: int):
    """Bytes one BFS traversal must move, level by level, by the method's
    definition (from its output levels, not from kernel counters):
      push level: sum over u in F of (offset + 4 deg u) + 4|F| (queue) + 12|F'|
                  (queue, level, parent of the next frontier) + n/8 (visited bits)
      pull level: sum over unvisited v of (offset + 4 scanned(v)) + 3n/8 (frontier,
                  visited and next bit arrays) + 8|F'|, where scanned(v) counts
                  v's neighbours in ascending order up to and including the first
                  one in the frontier (all of them when none is); a vertex without
                  neighbours has nothing to scan and is not counted
      plus 8n + n/8 to initialise levels, parents and visited bits.
    The direction of each level is the one the traversal took (trace).
    Returns (total bytes, [(level, direction, bytes, t_ns), ...])."""
    n = lv.numel()
    m = int(off[-1])
    L = lv.long() & INF
    reached = L != INF
    deg = (off[1:] - off[:-1]).long()
    # the first neighbour one level closer, for every reached vertex but the source
    want = torch.where(reached & (L > 0), L - 1, torch.full_like(L, -1))
    fp = first_hit_positions(torch, off, col, want, L)
    Lr = L[reached]
    top = int(Lr.max()) if Lr.numel() else 0
    cnt = torch.bincount(Lr, minlength=top + 2).double()
    degL = torch.bincount(Lr, weights=deg[reached].double(), minlength=top + 2)
    sel = reached & (L > 0)
    fpL = torch.bincount(L[sel], weights=(fp[sel] + 1).double(), minlength=top + 2)
    pos = reached & (deg > 0)
    cum_pos = torch.cumsum(torch.bincount(L[pos], minlength=top + 2).double(), 0)   # reached, with neighbours
    n_pos = int((deg > 0).sum())
    cum_deg = torch.cumsum(degL, 0)
    cnt, degL, fpL, cum_pos, cum_deg = (x.cpu().tolist() for x in (cnt, degL, fpL, cum_pos, cum_deg))
    out = []
    total = 8.0 * n + n / 8.0
    for r in trace:
        lvl_ = int(r.level)
        F = cnt[lvl_] if lvl_ < len(cnt) else 0.0
        Fn = cnt[lvl_ + 1] if lvl_ + 1 < len(cnt) else 0.0
        if r.direction == 1:
            b = off_bytes * F + 4.0 * degL[lvl_] + 4.0 * F + 12.0 * Fn + n / 8.0
        else:
            unvis = n_pos - cum_pos[lvl_]
            deg_beyond = m - (cum_deg[lvl_ + 1] if lvl_ + 1 < len(cum_deg) else cum_deg[-1])
            scanned = (fpL[lvl_ + 1] if lvl_ + 1 < len(fpL) else 0.0) + deg_beyond
            b = off_bytes * unvis + 4.0 * scanned + 3.0 * n / 8.0 + 8.0 * Fn
        total += b
        out.append((lvl_, int(r.direction), b, int(r.t_ns)))
    return total, out


def bc_method_bytes(torch, off, col, lv, off_bytes: int, chunk_edges=1 << 26):
    """Bytes single-source betweenness must move after its BFS: every reached
    vertex reads its list and the levels of its neighbours in both sweeps
    (off + 8 deg each), the forward sweep reads the path counts of the
    neighbours one level closer (8 each) and writes sigma (8), the backward
    sweep reads sigma and delta of the neighbours one level deeper (16 each)
    and writes delta (8); plus sigma/delta initialisation (16n) and the
    grouping of the vertices by level (levels read twice, order written)."""
    n = lv.numel()
    L = lv.long() & INF
    reached = L != INF
    deg = (off[1:] - off[:-1]).long()
    closer = 0
    for v0, v1 in _vertex_chunks(torch, off, chunk_edges):
        e0, e1 = int(off[v0]), int(off[v1])
        if e1 == e0:
            continue
        rows = torch.repeat_interleave(torch.arange(v0, v1, device=L.device), deg[v0:v1])
        nb = col[e0:e1].long() & INF
        lr = L[rows]
        closer += int(((lr != INF) & (lr > 0) & (L[nb] + 1 == lr)).sum())
    r = int(reached.sum())
    dsum = float(deg[reached].sum())
    sweeps = 2.0 * (off_bytes * r + 8.0 * dsum)
    return 16.0 * n + 8.0 * n + 4.0 * r + sweeps + 8.0 * closer + 8.0 * r + 16.0 * closer + 16.0 * r


def level_bandwidth(levels, peak):
    """Bandwidth of the push and pull levels: the largest level of each
    direction (by bytes) and each direction's total bytes over total time."""
    res = {}
    for d, name in ((1, "push"), (0, "pull")):
        lv = [x for x in levels if x[1] == d and x[3] > 0]
        if not lv:
            continue
        big = max(lv, key=lambda x: x[2])
        tb, tt = sum(x[2] for x in lv), sum(x[3] for x in lv)
        res[name] = {"largest_level": big[0], "largest_bytes": big[2], "largest_us": round(big[3] / 1e3, 2),
                     "largest_gbs": round(big[2] / big[3], 1), "largest_frac": round(big[2] / big[3] / peak, 4),
                     "levels": len(lv), "total_bytes": tb, "total_us": round(tt / 1e3, 1),
                     "total_gbs": round(tb / tt, 1), "total_frac": round(tb / tt / peak, 4)}
    return res


def msbfs_method_bytes(torch, off, col, lv, alpha: float, S: int, off_bytes: int = 4):
    """Bytes the 64-source BFS must move (one launch), from its output levels
    lv[S, n].  Per level: top-down reads the frontier words (8n) and, for each
    vertex whose word is non-empty, its offsets, its neighbour ids and their
    seen words (off + 12 per neighbour); bottom-up reads the seen words (8n)
    and, for each vertex with sources still unseen, neighbours in order until
    every missing source is found (all of them when some source cannot reach
    it), 12 bytes each; every level then rewrites the three words (24n) and
    writes 4 bytes per newly reached (vertex, source) pair.  The direction of
    each level follows the launch's own rule (top-down while the frontier's
    edges x alpha < the edges of vertices never in a frontier), applied to the
    same counts.  Plus 24n + 4Sn to initialise."""
    n = lv.shape[1]
    m = int(off[-1])
    L = lv.long() & INF
    deg = (off[1:] - off[:-1]).long()
    big = 1 << 40
    Lx = torch.where(L == INF, torch.full_like(L, big), L)
    first = Lx.min(0).values           # first level any source reaches v
    last = Lx.max(0).values            # level by which every source has reached v
    top = int(Lx[Lx < big].max()) if (Lx < big).any() else 0   # the deepest (vertex, source) level
    # union frontier per level: v is in it at level l iff some source reaches v at l
    counts = torch.zeros(top + 2, dtype=torch.float64, device=L.device)
    degsum = torch.zeros(top + 2, dtype=torch.float64, device=L.device)
    pairs = torch.zeros(top + 2, dtype=torch.float64, device=L.device)
    for j in range(S):
        r = L[j] != INF
        pairs += torch.bincount(L[j][r], minlength=top + 2).double()[:top + 2]
    for lvl_ in range(top + 1):
        inF = (L == lvl_).any(0)
        counts[lvl_] = inF.sum()
        degsum[lvl_] = deg[inF].sum()
    # bottom-up scan length at the level before `last`: first neighbour of each
    # source whose level at v is `last`, the latest of them
    fpmax = torch.full((n,), -1, dtype=torch.long, device=L.device)
    for j in range(S):
        want = torch.where((Lx[j] == last) & (last < big) & (last > 0), last - 1, torch.full_like(last, -1))
        fp = first_hit_positions(torch, off, col, want, L[j])
        fpmax = torch.maximum(fpmax, fp)
    counts, degsum, pairs = (x.cpu().tolist() for x in (counts, degsum, pairs))
    total = 24.0 * n + 4.0 * S * n
    mseen = 0.0
    for lvl_ in range(top + 1):
        nf, mf = counts[lvl_], degsum[lvl_]
        if nf == 0:
            break
        mseen += mf
        top_down = mf * alpha < max(m - mseen, 0) or lvl_ == 0
        if top_down:
            b = 8.0 * n + off_bytes * nf + 12.0 * mf
        else:
            pend = last > lvl_
            exact = pend & (last == lvl_ + 1)
            whole = pend & (last > lvl_ + 1)
            b = (8.0 * n + off_bytes * float(pend.sum()) + 12.0 * float((fpmax[exact] + 1).sum())
                 + 12.0 * float(deg[whole].sum()))
        total += b + 24.0 * n + 4.0 * (pairs[lvl_ + 1] if lvl_ + 1 < len(pairs) else 0.0)
    return total


# ----------------------------------------------------------------------------- oracle samples

def cpu_baseline(sample_scale: int, sources: int):
    """The serial oracle on a bounded sample of the same workload family."""
    import numpy as np

    import graphgen
    import oracle
    n, src, dst = graphgen.rmat_small(sample_scale, 16, graphgen.SEEDS["rmat25"])
    g = oracle.csr_build(n, src, dst)
    srcs = graphgen.pick_sources(n, src, dst, sources, graphgen.SEEDS["rmat25"] + 1)
    deg = np.diff(g.off).astype(np.int64)
    t0 = time.perf_counter()
    bfs_edges = 0
    for s in srcs:
        lv, _ = oracle.bfs(g, int(s))
        bfs_edges += int(deg[lv != oracle.INF].sum()) // 2
    oracle.cc(g)
    oracle.pagerank(g, DAMPING, PR_ITERS)
    oracle.tc(g)
    dt = time.perf_counter() - t0
    edges = bfs_edges + g.m // 2 + PR_ITERS * g.m + g.m
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"RMAT scale {sample_scale} ef16 (same a,b,c,d, ids permuted), {len(srcs)} BFS sources + "
                      f"CC + PR20 + TC, serial oracle, {dt:.2f} s",
            "seconds": dt, "host": platform.machine()}


def cpu_baseline_batched(members, stride: int = 32):
    """The oracle on every `stride`-th member of the batch: 64 BFS + CC each."""
    import numpy as np

    import oracle
    picked = members[::stride]
    t0 = time.perf_counter()
    edges = 0
    for n, s, d, srcs in picked:
        g = oracle.csr_build(n, s, d)
        deg = np.diff(g.off).astype(np.int64)
        for x in srcs:
            lv, _ = oracle.bfs(g, int(x))
            edges += int(deg[lv != oracle.INF].sum()) // 2
        oracle.cc(g)
        edges += g.m // 2
    dt = time.perf_counter() - t0
    return {"value": edges / dt / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"members 0, {stride}, {2 * stride}, ... ({len(picked)} of {len(members)}): 64 BFS + CC each, "
                      f"serial oracle (CSR build untimed), {dt:.2f} s"}


def cpu_baseline_dynamic(scale: int = 16, rounds: int = 3, batch: int = 16384):
    """The oracle's edge set under the same kind of rounds on a smaller base."""
    import graphgen
    import oracle
    n, src, dst = graphgen.rmat_small(scale, 16, graphgen.SEEDS["rmat24"])
    dg = oracle.DynGraph(n, src, dst)
    t0 = time.perf_counter()
    for ins_s, ins_d, del_s, del_d in graphgen.dynamic_rounds(n, src, dst, rounds, batch, scale=scale):
        dg.insert(ins_s, ins_d)
        dg.delete(del_s, del_d)
    dt = time.perf_counter() - t0
    return {"value": 2 * rounds * batch / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
            "sample": f"RMAT-{scale} base, {rounds} rounds x ({batch} inserts + {batch} deletes), serial oracle, "
                      f"{dt:.2f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import graphgen
    import oracle
    graphgen.build()
    oracle.build()
    vals = []
    for _ in range(max(args.warmup, 0)):
        cpu_baseline(max(args.sample_scale - 2, 8), args.sources)
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(args.sample_scale, args.sources)
        vals.append(cb["seconds"])
    v = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(vals),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32",
            "data": "synthetic", "config": {"workload": f"rmat{args.sample_scale} sample of {args.workload}",
                                            "sources": args.sources, "pr_iters": PR_ITERS},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- schedules

def schedule_table(byo, torch, g, srcs, levels, parents, reps: int, stream):
    """Median device time of the S-source BFS under each schedule."""
    out = {}
    for name in SCHEDULES:
        mm = load_mlp(byo) if name == "learned" else None
        if name == "learned" and mm is None:
            continue
        spx = sched_struct(byo, name, mm)
        byo.byo_bfs(g, srcs, levels, parents, spx)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            byo.byo_bfs(g, srcs, levels, parents, spx)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        out[name] = {"median_ms": round(statistics.median(times), 4), "min_ms": round(min(times), 4), "runs": reps}
        if mm:
            byo.byo_mlp_destroy(mm)
    if "learned" in out:
        out["heuristic_over_learned"] = round(out["heuristic"]["median_ms"] / out["learned"]["median_ms"], 4)
    return out


def grid_schedules(byo, torch, reps: int, stream):
    """The schedules on the high-diameter grid (4096 x 4096, 10 % dropped,
    0.01 % shortcuts): the corner vertex plus seven seeded sources."""
    import graphgen
    n, src, dst = graphgen.workload("grid")
    picked = [int(x) for x in graphgen.pick_sources(n, src, dst, 8, graphgen.SEEDS["grid"] + 1) if int(x) != 0]
    srcs = [0] + picked[:7]
    g = byo.Graph(n, dev_u32(torch, src), dev_u32(torch, dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE)
    lv = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
    par = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
    try:
        tab = schedule_table(byo, torch, g.handle, srcs, lv, par, reps, stream)
        corner = schedule_table(byo, torch, g.handle, [0], lv[:1], par[:1], reps, stream)
    finally:
        g.close()
    return {"workload": "grid 4096x4096, 10% dropped, 0.01% shortcuts", "sources": srcs, "all_sources": tab,
            "corner_only": corner}


# ----------------------------------------------------------------------------- batched workload

def run_batched(args, byo, torch):
    """256 graphs (half ER, half RMAT; n log-uniform in [2^10, 2^18], average
    degree uniform in [4, 64]) in one container: one step = 64-source
    multi-source BFS in every member + CC of the whole batch."""
    import numpy as np

    import graphgen
    from paper_2405_11671_gb300 import autotune
    members = graphgen.batched_workload(256, 64)
    ns = [mb[0] for mb in members]
    ks = [len(mb[1]) for mb in members]
    sources = [mb[3] for mb in members]
    src, dst = np.concatenate([mb[1] for mb in members]), np.concatenate([mb[2] for mb in members])
    g = byo.byo_batch_build(ns, ks, dev_u32(torch, src), dev_u32(torch, dst))
    N, m = byo.byo_num_vertices(g), byo.byo_num_edges(g)
    levels = torch.empty((64, N), dtype=torch.int32, device="cuda")
    labels = torch.empty(N, dtype=torch.int32, device="cuda")
    tuned = autotune.tune_msbfs(byo, g, sources, 64, levels)
    sp = byo.make_sched(byo.BYO_SCHED_HEURISTIC, 16, 1024, tuned["alpha"])
    stream = torch.cuda.current_stream()

    def step():
        byo.byo_msbfs(g, sources, 64, levels, sched=sp)
        byo.byo_cc(g, labels)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    byo.byo_profile_enable(True)
    byo.byo_profile_reset()
    l0 = byo.byo_kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    launches = byo.byo_kernel_launches() - l0
    prof = byo.byo_profile_read()
    byo.byo_profile_enable(False)
    clk = clocks.stop()
    ms = a.elapsed_time(b) / args.steps
    deg = byo.byo_degree(g).to(torch.int64)
    ms_edges = int(((levels != -1).to(torch.int64) * deg.unsqueeze(0)).sum().item()) // 2
    edges = {"msbfs": ms_edges, "cc": m // 2}
    step_edges = sum(edges.values())
    tot = sum(v[1] for v in prof.values()) or 1.0
    peak, peak_kind = measured_peaks()
    roof = None
    if "msbfs_persistent" in prof:
        nl, kms = prof["msbfs_persistent"]
        off, col = byo.byo_graph_export_csr(g)
        mb = msbfs_method_bytes(torch, off, col, levels, tuned["alpha"], 64, 8 if m >= 2 ** 32 else 4)
        del off, col
        roof = roof_entry("msbfs_persistent", mb, kms / nl, peak, peak_kind, kms / tot)

    # end to end: pinned host pairs in, batch built, both algorithms, levels and labels out
    e2e = None
    if not args.no_e2e:
        src_h, dst_h = pinned_u32(torch, src), pinned_u32(torch, dst)
        lv_h = torch.empty((64, N), dtype=torch.int32).pin_memory()
        lab_h = torch.empty(N, dtype=torch.int32).pin_memory()
        byo.byo_graph_destroy(g)
        g = None
        torch.cuda.synchronize()
        steps = max(1, args.e2e_steps)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            s_d, d_d = src_h.cuda(non_blocking=True), dst_h.cuda(non_blocking=True)
            ge = byo.byo_batch_build(ns, ks, s_d, d_d)
            byo.byo_msbfs(ge, sources, 64, levels, sched=sp)
            byo.byo_cc(ge, labels)
            lv_h.copy_(levels, non_blocking=True)
            lab_h.copy_(labels, non_blocking=True)
            torch.cuda.synchronize()
            byo.byo_graph_destroy(ge)
            del s_d, d_d
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b) / steps
        e2e = {"value": round(step_edges / (e2e_ms / 1e3) / 1e9, 3), "unit": "GTEPS", "ms_per_step": round(e2e_ms, 3),
               "h2d_bytes_per_step": int(8 * len(src)), "d2h_bytes_per_step": int(4 * (lv_h.numel() + lab_h.numel()))}
    cb = None if args.no_cpu_baseline else cpu_baseline_batched(members)
    line = {"metric": METRIC, "value": round(step_edges / (ms / 1e3) / 1e9, 3), "unit": "GTEPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
            "config": {"workload": "batched256", "graphs": 256, "n": N, "m": m, "sources_per_graph": 64,
                       "msbfs_alpha": tuned["alpha"], "autotune_ms": tuned["table_ms"],
                       "l2": "inputs larger than L2 (1.8 GB of neighbour ids)"},
            "edges_per_step": edges, "roofline": roof,
            "kernels": {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / tot, 4)}
                        for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
            "gpu_launches": int(launches), "clocks": clk, "e2e": e2e, "cpu_baseline": cb}
    print(json.dumps(line), flush=True)
    if g is not None:
        byo.byo_graph_destroy(g)


# ----------------------------------------------------------------------------- dynamic workload

def update_method_bytes(torch, ins_s, ins_d, deg_before, deg_after, lb: int):
    """Bytes a batch update must move: the batch sorted in both directions
    (8-byte keys read and written once per 8-bit radix pass over 2 lb key
    bits) and, for every vertex the batch touches, its old list read, its new
    list written and its 64-byte record rewritten."""
    k = len(ins_s)
    passes = (2 * lb + 7) // 8
    sort_b = 2.0 * k * 8 * 2 * passes
    touched = torch.unique(torch.cat([dev_u32(torch, ins_s), dev_u32(torch, ins_d)]).long())
    merge_b = float(4 * (deg_before[touched] + deg_after[touched]).sum()) + 64.0 * touched.numel()
    return sort_b + merge_b


def hashed_insert_bytes(k: int, new_entries: int, touched: int) -> float:
    """Bytes a batch insert into the hash-indexed container must move: the k
    pairs read (8 B each); the counting semisort over the 2k symmetrised
    entries (the source read to count, 4 B, and the entry read and written
    into its group, 8 + 4 B); one index slot read per entry (4 B); per new
    stored id its key, position and list slot written (12 B); and per touched
    vertex its 64-byte record read and written."""
    return 8.0 * k + 2.0 * k * (4 + 12) + 2.0 * k * 4 + 12.0 * new_entries + 128.0 * touched


def run_dynamic(args, byo, torch, rounds: int = 10, batch: int = 1_000_000, scale: int = 24):
    """RMAT-24 (ef 16) in the dynamic container, then `rounds` rounds of one
    insert batch of RMAT pairs and one delete batch of earlier pairs
    (graphgen.dynamic_rounds), each followed by BFS (one source) + CC +
    PageRank.  Reported: batch update throughput (pairs/s, before
    symmetrisation), the algorithms' time on the dynamic container, and a full
    GPU CSR rebuild of the same edge set."""
    import graphgen
    seed = graphgen.SEEDS["rmat24"]
    if scale == 24:
        n, src, dst = graphgen.workload("rmat24")
    else:  # a smaller base (for counter captures of the update kernels)
        n, src, dst = graphgen.rmat_small(scale, 16, seed)
    g = byo.Graph(n, dev_u32(torch, src), dev_u32(torch, dst), byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE)
    s0 = int(graphgen.pick_sources(n, src, dst, 1, seed + 1)[0])
    levels = torch.empty((1, n), dtype=torch.int32, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    ranks = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ins_ms, del_ms, alg_ms, csr_alg_ms, rebuild_ms, e2e_ms, ins_bytes = [], [], [], [], [], [], []
    m_rounds = []
    lv_h = torch.empty(n, dtype=torch.int32).pin_memory()
    lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
    rk_h = torch.empty(n, dtype=torch.float32).pin_memory()
    lb = max(1, (n - 1).bit_length())
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    l0 = byo.byo_kernel_launches()
    for r, (ins_s, ins_d, del_s, del_d) in enumerate(graphgen.dynamic_rounds(n, src, dst, rounds, batch,
                                                                             scale=scale)):
        # end to end through the C ABI: the round's pairs from pinned host
        # memory, the two updates, the three algorithms, their outputs back
        hs = [pinned_u32(torch, x) for x in (ins_s, ins_d, del_s, del_d)]
        deg_before = byo.byo_degree(g.handle).long()
        torch.cuda.synchronize()
        a, b, c, c2, d = ev(), ev(), ev(), ev(), ev()
        a.record(stream)
        di, dd_, ds, dd = (x.cuda(non_blocking=True) for x in hs)
        b.record(stream)
        byo.byo_insert_batch(g.handle, di, dd_)
        c.record(stream)
        deg_mid = byo.byo_degree(g.handle).long()  # for the byte model only, outside both update timings
        c2.record(stream)
        byo.byo_delete_batch(g.handle, ds, dd)
        d.record(stream)
        x0, x1 = ev(), ev()
        x0.record(stream)
        byo.byo_bfs(g.handle, [s0], levels, None, None, want_parents=False)
        byo.byo_cc(g.handle, labels)
        byo.byo_pagerank(g.handle, DAMPING, PR_ITERS, ranks, want_residual=False)
        x1.record(stream)
        lv_h.copy_(levels[0], non_blocking=True)
        lab_h.copy_(labels, non_blocking=True)
        rk_h.copy_(ranks, non_blocking=True)
        e = ev()
        e.record(stream)
        torch.cuda.synchronize()
        ins_ms.append(b.elapsed_time(c))
        del_ms.append(c2.elapsed_time(d))
        alg_ms.append(x0.elapsed_time(x1))
        e2e_ms.append(a.elapsed_time(e) - c.elapsed_time(c2))
        ins_bytes.append(update_method_bytes(torch, ins_s, ins_d, deg_before, deg_mid, lb))
        # the same edge set rebuilt as a static CSR, and the same algorithms on it
        off, col = byo.byo_graph_export_csr(g.handle)
        rows = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int32), off.diff())
        a, b = ev(), ev()
        a.record(stream)
        gc = byo.Graph(n, rows, col, byo.BYO_CSR)
        b.record(stream)
        torch.cuda.synchronize()
        rebuild_ms.append(a.elapsed_time(b))
        a, b = ev(), ev()
        a.record(stream)
        byo.byo_bfs(gc.handle, [s0], levels, None, None, want_parents=False)
        byo.byo_cc(gc.handle, labels)
        byo.byo_pagerank(gc.handle, DAMPING, PR_ITERS, ranks, want_residual=False)
        b.record(stream)
        torch.cuda.synchronize()
        csr_alg_ms.append(a.elapsed_time(b))
        gc.close()
        del rows, off, col
        m_rounds.append(g.m)
    launches = byo.byo_kernel_launches() - l0
    clk = clocks.stop()
    space_sorted = byo.byo_space(g.handle)
    g.close()
    hashed = run_dynamic_hashed(byo, torch, n, src, dst, s0, rounds, batch, m_rounds, scale)
    med = statistics.median
    peak, peak_kind = measured_peaks()
    round_ms = [i + d + x for i, d, x in zip(ins_ms, del_ms, alg_ms)]
    line = {"metric": "dynamic container: batch updates/s and algorithm time vs CSR", "value":
            round(2 * batch / (med([i + d for i, d in zip(ins_ms, del_ms)]) / 1e3), 1), "unit": "pairs/s",
            "higher_is_better": True, "n_gpus": 1, "steps": rounds, "warmup": 0,
            "ms_per_step": round(med(round_ms), 3), "dtype": "u32+f32", "data": "synthetic", "scaling": "weak",
            "vs_baseline": None,
            "config": {"workload": f"rmat{scale}-dynamic", "n": n, "m_final": m_rounds[-1], "rounds": rounds, "batch_pairs": batch,
                       "l2": f"{4 * m_rounds[-1] / 1e9:.2f} GB of neighbour ids (L2: 129 MB)"},
            "insert_ms_median": round(med(ins_ms), 3), "delete_ms_median": round(med(del_ms), 3),
            "insert_pairs_per_s": round(batch / (med(ins_ms) / 1e3), 1),
            "delete_pairs_per_s": round(batch / (med(del_ms) / 1e3), 1),
            "bfs_cc_pr_ms_dynamic": round(med(alg_ms), 3), "bfs_cc_pr_ms_csr": round(med(csr_alg_ms), 3),
            "dynamic_over_csr": round(med(alg_ms) / med(csr_alg_ms), 3),
            "csr_rebuild_ms_median": round(med(rebuild_ms), 3),
            "update_round_vs_rebuild": round((med(ins_ms) + med(del_ms)) / med(rebuild_ms), 3),
            "roofline": roof_entry("dyn_insert", med(ins_bytes), med(ins_ms), peak, peak_kind),
            "e2e": {"value": round(2 * batch / (med(e2e_ms) / 1e3), 1), "unit": "pairs/s",
                    "ms_per_step": round(med(e2e_ms), 3), "h2d_bytes_per_step": 16 * batch,
                    "d2h_bytes_per_step": 12 * n,
                    "note": "pairs in, both updates, BFS + CC + PageRank, their outputs out"},
            "gpu_launches": int(launches), "clocks": clk, "space_bytes": space_sorted,
            "hashed": {**hashed,
                       "insert_speedup_vs_sorted": round(med(ins_ms) / hashed["insert_ms_median"], 3),
                       "delete_speedup_vs_sorted": round(med(del_ms) / hashed["delete_ms_median"], 3),
                       "bfs_cc_pr_over_sorted": round(hashed["bfs_cc_pr_ms"] / med(alg_ms), 3)},
            "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline_dynamic()}
    print(json.dumps(line), flush=True)


def run_dynamic_hashed(byo, torch, n, src, dst, s0, rounds, batch, m_rounds, scale=24):
    """The same rounds on the hash-indexed container (BYO_DYN_HASH: semisorted
    batches, unsorted lists, per-run hash indexes): insert, delete and BFS + CC
    + PageRank times per round, and the container's bytes.  Its edge count must
    equal the sorted container's after every round."""
    import graphgen
    g = byo.Graph(n, dev_u32(torch, src), dev_u32(torch, dst),
                  byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE | byo.BYO_DYN_HASH)
    levels = torch.empty((1, n), dtype=torch.int32, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    ranks = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ins_ms, del_ms, alg_ms, ins_bytes = [], [], [], []
    for r, (ins_s, ins_d, del_s, del_d) in enumerate(graphgen.dynamic_rounds(n, src, dst, rounds, batch,
                                                                             scale=scale)):
        di, dd_, ds, dd = (dev_u32(torch, x) for x in (ins_s, ins_d, del_s, del_d))
        touched = int(torch.unique(torch.cat([di, dd_]).long()).numel())
        m0 = g.m
        torch.cuda.synchronize()
        a, b, c, x1 = ev(), ev(), ev(), ev()
        a.record(stream)
        byo.byo_insert_batch(g.handle, di, dd_)
        b.record(stream)
        m1 = g.m  # host metadata, updated when the call returns
        byo.byo_delete_batch(g.handle, ds, dd)
        c.record(stream)
        byo.byo_bfs(g.handle, [s0], levels, None, None, want_parents=False)
        byo.byo_cc(g.handle, labels)
        byo.byo_pagerank(g.handle, DAMPING, PR_ITERS, ranks, want_residual=False)
        x1.record(stream)
        torch.cuda.synchronize()
        ins_ms.append(a.elapsed_time(b))
        del_ms.append(b.elapsed_time(c))
        alg_ms.append(c.elapsed_time(x1))
        ins_bytes.append(hashed_insert_bytes(len(ins_s), m1 - m0, touched))
        if g.m != m_rounds[r]:
            raise RuntimeError(f"hashed container: m {g.m} != {m_rounds[r]} after round {r}")
    med = statistics.median
    out = {"insert_ms_median": round(med(ins_ms), 3), "delete_ms_median": round(med(del_ms), 3),
           "insert_pairs_per_s": round(batch / (med(ins_ms) / 1e3), 1),
           "delete_pairs_per_s": round(batch / (med(del_ms) / 1e3), 1),
           "bfs_cc_pr_ms": round(med(alg_ms), 3), "space_bytes": byo.byo_space(g.handle)}
    peak, peak_kind = measured_peaks()
    out["roofline"] = roof_entry("hashed insert batch", med(ins_bytes), med(ins_ms), peak, peak_kind)
    g.close()
    return out


# ----------------------------------------------------------------------------- API ablation

def run_ablation(args, byo, torch):
    """The paper's API-components study (Section 6.3) on the GPU path: BFS
    from the benchmark sources with the full API, without the early-exit map
    (pull iterations read whole lists), without the parallel map (a list is
    only ever walked by one thread) and without both, on RMAT-22 and the grid
    (heuristic schedule).  Results are identical; only the time changes."""
    import graphgen
    stream = torch.cuda.current_stream()
    out = {}
    variants = {"full": 0, "no_early_exit": byo.BYO_SCHED_NO_EARLY_EXIT,
                "sequential_maps": byo.BYO_SCHED_SEQUENTIAL_MAPS,
                "neither": byo.BYO_SCHED_NO_EARLY_EXIT | byo.BYO_SCHED_SEQUENTIAL_MAPS}
    for name in ("rmat22", "grid"):
        n, src, dst = graphgen.workload(name)
        srcs = graphgen.pick_sources(n, src, dst, args.sources, graphgen.SEEDS[name] + 1)
        flags = byo.BYO_CSR | byo.BYO_SYMMETRIZE | (byo.BYO_OFFSETS64 if name.startswith("rmat") else 0)
        g = byo.Graph(n, dev_u32(torch, src), dev_u32(torch, dst), flags)
        lv = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        par = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        ref = None
        res = {}
        for vname, fl in variants.items():
            sp = byo.make_sched(byo.BYO_SCHED_HEURISTIC, flags=fl)
            byo.byo_bfs(g.handle, srcs, lv, par, sp)
            torch.cuda.synchronize()
            if ref is None:
                ref = lv.clone()
            same = bool(torch.equal(lv, ref))
            times = []
            for _ in range(max(1, args.sched_reps)):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                byo.byo_bfs(g.handle, srcs, lv, par, sp)
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b))
            res[vname] = {"median_ms": round(statistics.median(times), 3), "levels_identical": same}
        for vname in variants:
            res[vname]["slowdown"] = round(res[vname]["median_ms"] / res["full"]["median_ms"], 3)
        out[name] = res
        g.close()
    print(json.dumps({"metric": "BFS time without API components (Section 6.3 ablation)", "unit": "ms",
                      "sources": args.sources, "sched": "heuristic", "results": out}), flush=True)


# ----------------------------------------------------------------------------- containers: space and time

def run_space(args, byo, torch):
    """The container comparison of Section 6.5 on the GPU path: bytes per
    stored edge of the CSR, the dynamic container with and without its inline
    head, and the compressed CSR (byte codes), beside the paper's 4.1 / 5.1 /
    10.6 bytes per edge (its CSR, min / mean / max over its graphs); BFS from
    the benchmark sources on each, and BFS + CC + PageRank on the dynamic
    container with and without the inline head.  Heuristic schedule."""
    import graphgen
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return round(statistics.median(ts), 3)

    out = {}
    for name in ("rmat22", "rmat25"):
        n, src, dst = graphgen.workload(name)
        srcs = graphgen.pick_sources(n, src, dst, args.sources, graphgen.SEEDS[name] + 1)
        s_d, d_d = dev_u32(torch, src), dev_u32(torch, dst)
        sym = byo.BYO_SYMMETRIZE | byo.BYO_OFFSETS64
        kinds = {"csr": byo.BYO_CSR | sym, "compressed": byo.BYO_CSR | sym | byo.BYO_COMPRESSED,
                 "dynamic_inline": byo.BYO_DYNAMIC | sym, "dynamic_no_inline": byo.BYO_DYNAMIC | sym | byo.BYO_DYN_NO_INLINE}
        lv = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        par = torch.empty((len(srcs), n), dtype=torch.int32, device="cuda")
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        rk = torch.empty(n, dtype=torch.float32, device="cuda")
        res = {}
        ref = None
        for kind, fl in kinds.items():
            g = byo.Graph(n, s_d, d_d, fl)
            m = g.m
            e = {"bytes_per_edge": round(byo.byo_space(g.handle) / m, 3)}
            e["bfs_ms"] = timed(lambda: byo.byo_bfs(g.handle, srcs, lv, par), args.sched_reps)
            if ref is None:
                ref = lv.clone()
            e["levels_identical"] = bool(torch.equal(lv, ref))
            if kind.startswith("dynamic") or kind == "csr":
                def three():
                    byo.byo_bfs(g.handle, srcs, lv, par)
                    byo.byo_cc(g.handle, lab)
                    byo.byo_pagerank(g.handle, DAMPING, PR_ITERS, rk, want_residual=False)
                e["bfs_cc_pr_ms"] = timed(three, max(1, args.sched_reps // 2))
            res[kind] = e
            g.close()
        res["m"] = m
        out[name] = res
        del s_d, d_d, lv, par
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "container space (bytes per stored edge) and time (Section 6.5 comparison)",
                      "paper_csr_bytes_per_edge": {"min": 4.1, "mean": 5.1, "max": 10.6},
                      "sources": args.sources, "sched": "heuristic", "results": out}), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch

    import graphgen
    from paper_2405_11671_gb300 import build as lib_build

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        lib_build.build()
    if dist:
        dist.barrier()
    import paper_2405_11671_gb300 as byo
    byo.load()
    # all work on one non-default stream (PageRank's iterations then run as a
    # captured CUDA graph)
    work_stream = torch.cuda.Stream()
    torch.cuda.set_stream(work_stream)
    if args.workload == "batched":
        run_batched(args, byo, torch)
        return
    if args.workload == "dynamic":
        scale = args.dyn_scale
        run_dynamic(args, byo, torch, rounds=args.rounds, batch=max(1, 1_000_000 >> max(0, 24 - scale)), scale=scale)
        return
    if args.workload == "ablation":
        run_ablation(args, byo, torch)
        return
    if args.workload == "space":
        run_space(args, byo, torch)
        return

    def barrier():
        if dist:
            dist.barrier()

    # ---- inputs (seeded, synthetic; replicas use the same graph)
    n, src, dst = graphgen.workload(args.workload)
    srcs = graphgen.pick_sources(n, src, dst, args.sources, graphgen.SEEDS.get(args.workload, 0) + 1)
    S = len(srcs)
    src_d, dst_d = dev_u32(torch, src), dev_u32(torch, dst)
    flags = byo.BYO_CSR | byo.BYO_SYMMETRIZE | (byo.BYO_OFFSETS64 if args.workload.startswith("rmat") else 0)
    torch.cuda.synchronize()
    tb0 = time.perf_counter()
    g = byo.Graph(n, src_d, dst_d, flags)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - tb0
    m = g.m
    off_bytes = 8 if (flags & byo.BYO_OFFSETS64) or m >= 2 ** 32 else 4
    levels = torch.empty((S, n), dtype=torch.int32, device="cuda")
    parents = torch.empty((S, n), dtype=torch.int32, device="cuda")
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    ranks = torch.empty(n, dtype=torch.float32, device="cuda")
    mlp = load_mlp(byo) if args.sched == "learned" else None
    if args.sched == "learned" and mlp is None:
        raise SystemExit("--sched learned needs paper_2405_11671_gb300/sched_mlp.json (train it first)")
    sp = sched_struct(byo, args.sched, mlp)
    stream = torch.cuda.current_stream()
    algos = ["bfs", "cc", "pr", "tc"]
    ev = {a: [] for a in algos}
    tri = {"count": None}

    def step(record: bool):
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if record else None
        if record:
            marks[0].record(stream)
        byo.byo_bfs(g.handle, srcs, levels, parents, sp)
        if record:
            marks[1].record(stream)
        byo.byo_cc(g.handle, labels)
        if record:
            marks[2].record(stream)
        byo.byo_pagerank(g.handle, DAMPING, PR_ITERS, ranks, want_residual=False)
        if record:
            marks[3].record(stream)
        tri["count"] = byo.byo_tc(g.handle)
        if record:
            marks[4].record(stream)
            for i, a in enumerate(algos):
                ev[a].append((marks[i], marks[i + 1]))

    for _ in range(max(args.warmup, 0)):
        step(False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    byo.byo_profile_enable(True)
    byo.byo_profile_reset()
    launches0 = byo.byo_kernel_launches()
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = byo.byo_kernel_launches() - launches0
    prof = byo.byo_profile_read()
    byo.byo_profile_enable(False)
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    local_ms = total_ms / args.steps
    algo_ms = {a: statistics.mean(x.elapsed_time(y) for x, y in ev[a]) for a in algos}

    # ---- edges per step (from the parity-checked outputs)
    deg = byo.byo_degree(g.handle).to(torch.int64)
    reached = levels != -1
    bfs_edges = int((reached.to(torch.int64) * deg.unsqueeze(0)).sum().item()) // 2
    edges = {"bfs": bfs_edges, "cc": m // 2, "pr": PR_ITERS * m, "tc": m}
    step_edges = sum(edges.values())
    value, step_ms = replica_value(dist, step_edges, local_ms, "cuda")
    per_algo = {a: {"ms": round(algo_ms[a], 4), "gteps": round(edges[a] / (algo_ms[a] / 1e3) / 1e9, 3)}
                for a in algos}

    # ---- roofline of the dominant kernel (method bytes / CUDA-event time)
    peak, peak_kind = measured_peaks()
    off_d, col_d = byo.byo_graph_export_csr(g.handle)
    bfs_bytes, bfs_lv = [], []
    examined = [0.0, 0.0]
    for s_ in srcs:  # one trace per source: the BFS launch processes one source
        byo.byo_bfs(g.handle, [int(s_)], levels[:1], parents[:1], sp)
        tr = byo.byo_bfs_trace(g.handle)
        b, per_level = bfs_method_bytes(torch, off_d, col_d, levels[0], tr, off_bytes)
        bfs_bytes.append(b)
        bfs_lv += per_level
        examined[0] += sum(4.0 * r.edges_examined for r in tr)
        examined[1] += sum(x[2] for x in per_level)
    # single-source betweenness from the first source (not part of the step):
    # BFS + forward and backward sweeps, median of three calls
    bc = None
    if rank == 0:
        s0 = int(srcs[0])
        byo.byo_bc(g.handle, s0, levels[0])
        torch.cuda.synchronize()
        bt = []
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            byo.byo_bc(g.handle, s0, levels[0])
            b.record(stream)
            torch.cuda.synchronize()
            bt.append(a.elapsed_time(b))
        bc_ms = statistics.median(bt)
        byo.byo_bfs(g.handle, [s0], levels[:1], parents[:1], byo.make_sched(byo.BYO_SCHED_HEURISTIC))
        tr0 = byo.byo_bfs_trace(g.handle)
        bfs_b, _ = bfs_method_bytes(torch, off_d, col_d, levels[0], tr0, off_bytes)
        bc_b = bfs_b + bc_method_bytes(torch, off_d, col_d, levels[0], off_bytes)
        deg_all = (off_d[1:] - off_d[:-1]).long()
        comp_edges = int(deg_all[(levels[0].long() & INF) != INF].sum()) // 2
        bc = {"source": s0, "ms": round(bc_ms, 3), "gteps": round(comp_edges / (bc_ms / 1e3) / 1e9, 3),
              "roofline": roof_entry("bc (BFS + both sweeps)", bc_b, bc_ms, peak, peak_kind)}
        del deg_all
    del off_d, col_d
    tot = sum(v[1] for v in prof.values()) or 1.0
    # the two intersection kernels of one triangle count are one unit of work
    merged = dict(prof)
    if "tc_light" in merged or "tc_heavy" in merged:
        nl = max(merged.get("tc_light", (0, 0.0))[0], merged.get("tc_heavy", (0, 0.0))[0])
        merged["tc_count"] = (nl, merged.pop("tc_light", (0, 0.0))[1] + merged.pop("tc_heavy", (0, 0.0))[1])
    ranked = sorted(merged.items(), key=lambda kv: -kv[1][1])
    roof = None
    rooflines = {}
    tc_work = None
    for name, (nl, ms) in ranked:
        if name == "tc_count":
            tc_work = byo.byo_tc_work(g.handle)
            # what this intersection must read: the ids it walks (per DAG edge
            # the shorter out-list, an in-neighbour's sorted list only above the
            # centre: byo_tc_work[2]), every partner's id and out-list bounds
            # (each DAG edge is a partner once from each end: m ids, 2 x 8-byte
            # offsets each), every centre's out-list once (m/2 ids)
            b = 4.0 * tc_work[2] + 20.0 * m + 2.0 * m
        elif name == "bfs_persistent":
            b = statistics.mean(bfs_bytes)
        else:
            b = algo_bytes(name, n, m, off_bytes)
        if b is None or nl == 0:
            continue
        entry = roof_entry(name, b, ms / nl, peak, peak_kind, ms / tot)
        if name == "tc_count":
            merge_b = 4.0 * (tc_work[0] + tc_work[1])
            entry["tc_ids_walked"] = tc_work[2]
            entry["merge_model_bytes"] = merge_b
            entry["merge_model_frac"] = round(merge_b / (ms / nl / 1e3) / 1e9 / peak, 4)
            entry["note"] = ("bytes = shorter out-list of each DAG edge + partner ids and bounds + centre lists "
                             "(the walk-shorter/probe-set method, in-neighbour walks trimmed to the ids above the "
                             "centre). merge_model_* = both out-lists of every DAG edge (a sorted merge's reads)")
        if name == "bfs_persistent":
            entry["ids_read_by_kernel_over_method"] = round(examined[0] / max(examined[1], 1.0), 4)
        if roof is None:
            roof = entry
        else:
            rooflines[name] = {k: entry[k] for k in ("achieved", "frac", "avg_launch_ms", "algorithmic_bytes_per_launch",
                                                     "traffic", "share")}
    kernel_share = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / tot, 4)}
                    for k, v in ranked}
    bfs_levels = level_bandwidth(bfs_lv, peak)

    # ---- schedules side by side (BFS only), here and on the high-diameter grid
    sched_cmp = grid_cmp = None
    if not args.no_schedules and rank == 0:
        sched_cmp = schedule_table(byo, torch, g.handle, srcs, levels, parents, args.sched_reps, stream)
        if args.workload != "grid":
            grid_cmp = grid_schedules(byo, torch, args.sched_reps, stream)

    # ---- end to end through the C ABI from host buffers
    e2e = None
    if not args.no_e2e:
        src_h, dst_h = pinned_u32(torch, src), pinned_u32(torch, dst)
        lv_h = torch.empty((S, n), dtype=torch.int32).pin_memory()
        lab_h = torch.empty(n, dtype=torch.int32).pin_memory()
        rk_h = torch.empty(n, dtype=torch.float32).pin_memory()
        g.close()
        del src_d, dst_d
        torch.cuda.synchronize()
        e2e_steps = max(1, args.e2e_steps)
        # A streaming pipeline: the edge list of step i+1 is copied in (second
        # device buffer, own stream) while step i runs, and step i's results are
        # copied out while its triangle count runs.  Every step's copies are
        # inside the timed region.
        copy_s = torch.cuda.Stream()
        bufs = [(torch.empty_like(src_h, device="cuda"), torch.empty_like(dst_h, device="cuda")) for _ in range(2)]
        in_ev = [torch.cuda.Event() for _ in range(2)]
        out_ev = torch.cuda.Event()
        barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        copy_s.wait_event(a)

        def load(slot):
            with torch.cuda.stream(copy_s):
                bufs[slot][0].copy_(src_h, non_blocking=True)
                bufs[slot][1].copy_(dst_h, non_blocking=True)
                in_ev[slot].record(copy_s)

        load(0)
        for i in range(e2e_steps):
            stream.wait_event(in_ev[i % 2])
            ge = byo.Graph(n, bufs[i % 2][0], bufs[i % 2][1], flags)
            if i + 1 < e2e_steps:
                load((i + 1) % 2)
            byo.byo_bfs(ge.handle, srcs, levels, parents, sp)
            byo.byo_cc(ge.handle, labels)
            byo.byo_pagerank(ge.handle, DAMPING, PR_ITERS, ranks, want_residual=False)
            out_ev.record(stream)
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(out_ev)
                lv_h.copy_(levels, non_blocking=True)
                lab_h.copy_(labels, non_blocking=True)
                rk_h.copy_(ranks, non_blocking=True)
            byo.byo_tc(ge.handle)
            torch.cuda.synchronize()
            ge.close()
        b.record(stream)
        torch.cuda.synchronize()
        del bufs
        e2e_v, e2e_ms = replica_value(dist, step_edges, a.elapsed_time(b) / e2e_steps, "cuda")
        e2e = {"value": round(e2e_v, 3), "unit": "GTEPS",
               "ms_per_step": round(e2e_ms, 3), "h2d_bytes_per_step": int(src_h.numel() * 8),
               "d2h_bytes_per_step": int(lv_h.numel() * 4 + lab_h.numel() * 4 + rk_h.numel() * 4 + 8)}
    else:
        g.close()

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(args.sample_scale, args.sources)
        cb.pop("seconds", None)
        cb.pop("host", None)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32+f32", "data": "synthetic",
                "config": {"workload": args.workload, "n": n, "m": m, "draws": int(len(src)),
                           "offsets": f"u{8 * off_bytes}", "sources": S, "pr_iters": PR_ITERS,
                           "sched": args.sched, "parallelism": "replicas" if world > 1 else "single",
                           "l2": "inputs larger than L2 (graph >> 129 MB)", "build_s": round(build_s, 3),
                           "triangles": tri["count"]},
                "algos": per_algo, "edges_per_step": edges, "roofline": roof, "other_rooflines": rooflines,
                "bfs_levels": bfs_levels, "kernels": kernel_share,
                "gpu_launches": int(launches), "clocks": clk, "e2e": e2e, "cpu_baseline": cb}
        if sched_cmp is not None:
            line["schedules"] = sched_cmp
        if grid_cmp is not None:
            line["schedules_grid"] = grid_cmp
        if bc is not None:
            line["betweenness"] = bc
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
