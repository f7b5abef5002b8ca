"""Learned edgeMap schedule: training data, training and evaluation.

The schedule network (``csrc/mlp.cu``, ``csrc/sched.cuh``) picks, for every BFS
iteration, one of five result-identical actions from 12 frontier features:

====== =========================================================
action meaning
====== =========================================================
0      dense edgeMap (pull) over the frontier bit array
1      sparse edgeMap (push), bins thread < 16, warp < 1024
2      push, bins thread < 4, warp < 128
3      push, bins thread < 64, warp < 4096
4      push by one CTA alone, no grid barrier between such levels
====== =========================================================

The network chooses among the actions a level allows: any push variant; pull
only where a Beamer test would pull (frontier edges > unvisited edges / alpha,
or |F| >= n / beta), so that a misprediction never pulls a small frontier; the
single-CTA push only for small frontiers.  Training data are timings the engine
records itself: every training graph is traversed once per action with that
action forced at every level, and the per-iteration device times
(``byo_bfs_trace``) give, for each level, the time of each action on the same
frontier (BFS frontiers do not depend on the schedule).  Every level is a
sample; its label is the fastest allowed action and its weight the log of the
slowest over the fastest allowed action's time.  The network is trained by the
library's own forward/backward/Adam kernels.

``python -m paper_2405_11671_gb300.schedule train --out sched_mlp.json`` builds
the training set from generated graphs (ER, RMAT, grids) and writes the FP32
parameters that ``--sched learned`` loads.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

NUM_ACTIONS = 5
NUM_FEATURES = 12
DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sched_mlp.json")


def feature_vector(nf, mf, nu, mu, n, m, hist) -> np.ndarray:
    """The 12 network inputs of one iteration; the same formula as the device
    function that feeds the network inside the BFS loop (which evaluates it
    with the hardware's approximate logarithm and division, a few ulp apart)."""
    x = np.zeros(NUM_FEATURES, np.float32)
    f = np.float32
    x[0] = math.log2(1.0 + nf) / 32.0
    x[1] = math.log2(1.0 + mf) / 40.0
    x[2] = math.log2(1.0 + nu) / 32.0
    x[3] = math.log2(1.0 + mu) / 40.0
    x[4] = math.log2(1.0 + n) / 32.0
    x[5] = math.log2(1.0 + m) / 40.0
    x[6] = f(nf) / f(n if n else 1)
    x[7] = mf / (mf + mu + 1.0)
    inv = 1.0 / (nf if nf else 1)
    for k in range(4):
        x[8 + k] = hist[k] * inv
    return x


def trace_features(trace, n: int, m: int) -> np.ndarray:
    return np.stack([feature_vector(r.frontier, r.frontier_edges, r.unvisited, r.unvisited_edges, n, m, list(r.hist))
                     for r in trace]) if trace else np.zeros((0, NUM_FEATURES), np.float32)


ALPHA, BETA = 15.0, 18.0  # the default Beamer constants of a schedule
SOLO_MAX_EDGES = 16384  # the device only lets the network pick action 4 below this
SOLO_MAX_VERTICES = 1024


def forced_sched(byo, action: int):
    return byo.make_sched(byo.BYO_SCHED_FIXED, 16, 1024, action=action)


def time_actions(byo, g, sources, repeats: int = 3):
    """Per-iteration device times of every forced action for each source: the
    median over `repeats` traversals (after one untimed warm-up traversal), so
    that the labels depend as little as possible on timing noise.

    Returns a list of (features [L, 12], times [L, NUM_ACTIONS] in ns,
    frontier edges [L], (|F|, frontier edges, unvisited edges, n) per level)."""
    n, m = byo.byo_num_vertices(g), byo.byo_num_edges(g)
    out = []
    for s in sources:
        feats, times, mf, stats = None, [], None, None
        for a in range(NUM_ACTIONS):
            sp = forced_sched(byo, a)
            byo.byo_bfs(g, [int(s)], sched=sp, want_parents=False)
            runs = []
            for _ in range(repeats):
                byo.byo_bfs(g, [int(s)], sched=sp, want_parents=False)
                tr = byo.byo_bfs_trace(g)
                runs.append(np.array([r.t_ns for r in tr], np.float64))
                if feats is None:
                    feats = trace_features(tr, n, m)
                    mf = np.array([r.frontier_edges for r in tr], np.float64)
                    stats = [(r.frontier, r.frontier_edges, r.unvisited_edges, n) for r in tr]
            times.append(np.median(np.stack(runs), axis=0))
        out.append((feats, np.stack(times, axis=1), mf, stats))
    return out


def allowed(t_row, stats_row, alpha: float = ALPHA, beta: float = BETA):
    """Per-level times with the actions the device would not let the network
    take masked: pull unless a Beamer test would pull (frontier edges >
    unvisited edges / alpha, or |F| >= n / beta), the single-CTA push unless
    the frontier is small.  stats_row: (|F|, frontier edges, unvisited edges, n)."""
    nf, mf, mu, n = stats_row
    t = np.array(t_row, np.float64)
    if mf > SOLO_MAX_EDGES or nf > SOLO_MAX_VERTICES:
        t[4] = np.inf
    if not (mf * alpha > mu or nf * beta >= n):  # the device's form of the two tests
        t[0] = np.inf
    return t


def samples_from_timings(tables):
    """Samples = every level; label = fastest allowed action; weight = log of
    the worst / best allowed action's time on that level (scale-free, so the
    many short levels of a deep traversal count as much as the few long levels
    of a shallow one), clipped to [0.01, 3]."""
    X, y, w = [], [], []
    for feats, t, mf, stats in tables:
        if len(t) == 0:
            continue
        t = np.stack([allowed(t[i], stats[i]) for i in range(len(t))])
        for i in range(len(t)):
            X.append(feats[i])
            y.append(int(np.argmin(t[i])))
            fin = t[i][np.isfinite(t[i])]
            w.append(float(np.clip(np.log(fin.max() / max(fin.min(), 1.0)), 0.01, 3.0)))
    return (np.array(X, np.float32).reshape(-1, NUM_FEATURES), np.array(y, np.int32), np.array(w, np.float32))


def regret(t, choices) -> float:
    """Extra device time (ns) of per-iteration choices over the per-iteration best."""
    t = np.asarray(t)
    return float(sum(t[i, c] - t[i].min() for i, c in enumerate(choices)))




def training_graphs(seed: int = 0xB10 + 50):
    """Generated graphs of the three shapes at sizes up to those of the
    benchmark configurations (RMAT up to scale 24, ER up to 2^21 vertices,
    grids up to 4096 x 4096), drawn from their own seeds: never the benchmark
    graphs themselves.  The network's size features must have seen sizes like
    the ones it is used on."""
    import graphgen
    out = []
    for sc in (14, 16, 18, 20, 22, 23, 24):
        out.append(("rmat%d" % sc, *graphgen.rmat_small(sc, 16, graphgen.stream(seed, sc))))
    for sc, deg in ((15, 8), (17, 16), (19, 32), (21, 16)):
        n = 1 << sc
        out.append(("er%d" % sc, n, *graphgen.er(n, n * deg // 2, graphgen.stream(seed, 100 + sc))))
    for side in (256, 512, 1024, 2048, 4096):
        out.append(("grid%d" % side, *graphgen.grid_small(side, side, 0.1, 1e-4, graphgen.stream(seed, side))))
    return out


def build_training_set(byo, graphs, sources_per_graph: int = 3):
    import torch

    import graphgen
    tables = []
    for name, n, src, dst in graphs:
        sd = torch.from_numpy(np.ascontiguousarray(src, np.uint32).view(np.int32)).cuda()
        dd = torch.from_numpy(np.ascontiguousarray(dst, np.uint32).view(np.int32)).cuda()
        with byo.Graph(n, sd, dd) as g:
            srcs = graphgen.pick_sources(n, src, dst, sources_per_graph, 17)
            tables += time_actions(byo, g.handle, srcs)
    return tables


def train(byo, X, y, w, seed: int = 1, epochs: int = 6000, lr: float = 3e-3):
    import torch
    m = byo.byo_mlp_create(seed)
    loss = byo.byo_mlp_train(m, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(w).cuda(),
                             epochs=epochs, lr=lr)
    return m, loss


def save(byo, m, path: str, meta: dict | None = None):
    params = byo.byo_mlp_get_params(m)
    with open(path, "w") as f:
        json.dump({"features": NUM_FEATURES, "hidden": [32, 32], "actions": NUM_ACTIONS,
                   "params": [float(v) for v in params], "meta": meta or {}}, f)


def load(byo, path: str = DEFAULT_PATH):
    with open(path) as f:
        d = json.load(f)
    m = byo.byo_mlp_create(0)
    byo.byo_mlp_set_params(m, np.array(d["params"], np.float32))
    return m


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", default=DEFAULT_PATH)
    ap.add_argument("--epochs", type=int, default=6000)
    args = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import paper_2405_11671_gb300 as byo
    from paper_2405_11671_gb300 import build
    build.build()
    byo.load()
    tables = build_training_set(byo, training_graphs())
    X, y, w = samples_from_timings(tables)
    m, loss = train(byo, X, y, w, epochs=args.epochs)
    import torch
    pred = byo.byo_mlp_predict(m, torch.from_numpy(X).cuda()).cpu().numpy()
    acc = float(np.mean(pred == y)) if len(y) else 0.0
    save(byo, m, args.out, {"samples": int(len(y)), "loss": loss, "train_accuracy": acc,
                             "label_counts": np.bincount(y, minlength=NUM_ACTIONS).tolist()})
    print(json.dumps({"samples": int(len(y)), "loss": loss, "train_accuracy": acc,
                      "label_counts": np.bincount(y, minlength=NUM_ACTIONS).tolist(), "out": args.out}))


if __name__ == "__main__":
    main()
