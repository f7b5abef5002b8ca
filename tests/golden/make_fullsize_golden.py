"""Writes the full-size reference values in this folder, from the oracle only.

Usage (CPU; each workload takes minutes to about an hour of host time):

    python tests/golden/make_fullsize_golden.py rmat25 rmat26 dynamic batched rmat22 grid

Each workload's raw pairs come from ``graphgen`` (the same seeded draws the GPU
tests and the benchmark use); every value below is computed by ``oracle``:

* ``csr_sha256``: SHA-256 of the CSR (offsets as little-endian uint64, then the
  neighbour ids as little-endian uint32);
* ``bfs``: for each benchmark source, SHA-256 of the level array (uint32, INF =
  0xFFFFFFFF), the number of reached vertices and the deepest level;
* ``cc_sha256``: SHA-256 of the labels (minimum vertex id of each component)
  and the number of components;
* ``pagerank``: FP64 values (d = 0.85, 20 iterations) at seeded uniformly drawn
  vertices and at the highest-degree vertices (ties by id);
* ``triangles``: the count, through the degree-ordered DAG (the serial C
  routine run over ranges of centres on several host threads).

``dynamic``: the RMAT-24 base in the oracle's edge set, then ten rounds of one
insert batch and one delete batch (``graphgen.dynamic_rounds``), with the CSR,
BFS, CC and PageRank values after every round.  ``batched``: for each of the
256 members, SHA-256 of its 64-source level block (64 x n uint32, source-major)
and of its labels in local ids.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
import oracle  # noqa: E402

INF = 0xFFFFFFFF
THREADS = max(1, min(8, os.cpu_count() or 1))


def sha_u32(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<u4").tobytes()).hexdigest()


def sha_csr(off, col) -> str:
    h = hashlib.sha256(np.ascontiguousarray(off, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(col, dtype="<u4").tobytes())
    return h.hexdigest()


def pr_sample_ids(n: int, deg: np.ndarray, seed: int, uniform: int, top: int) -> np.ndarray:
    """Seeded uniform vertex draws plus the `top` highest-degree vertices."""
    drawn = graphgen.pick_indices(n, uniform, graphgen.stream(seed, 300)).astype(np.int64)
    order = np.lexsort((np.arange(n), -deg.astype(np.int64)))[:top]
    return np.unique(np.concatenate([drawn, order]))


def bfs_record(g, s: int) -> dict:
    lv, _ = oracle.bfs(g, int(s))
    reached = lv != INF
    return {"source": int(s), "levels_sha256": sha_u32(lv), "reached": int(reached.sum()),
            "depth": int(lv[reached].max())}


def cc_record(g) -> dict:
    lab = oracle.cc(g)
    return {"cc_sha256": sha_u32(lab), "components": int((lab == np.arange(g.n, dtype=np.uint32)).sum())}


def pr_record(g, ids: np.ndarray) -> dict:
    p, _ = oracle.pagerank(g, 0.85, 20)
    return {"ids": ids.tolist(), "values": [float(x) for x in p[ids]], "mass": float(p.sum())}


def static_workload(name: str) -> dict:
    t0 = time.time()
    n, src, dst = graphgen.workload(name)
    seed = graphgen.SEEDS[name]
    srcs = graphgen.pick_sources(n, src, dst, 8, seed + 1)
    draws = len(src)
    g = oracle.csr_build(n, src, dst)
    del src, dst
    deg = np.diff(g.off.astype(np.int64))
    rec = {"workload": name, "n": n, "m": g.m, "draws": draws, "csr_sha256": sha_csr(g.off, g.col)}
    with cf.ThreadPoolExecutor(max_workers=THREADS) as ex:
        bfs_f = [ex.submit(bfs_record, g, s) for s in srcs]
        cc_f = ex.submit(cc_record, g)
        pr_f = ex.submit(pr_record, g, pr_sample_ids(n, deg, seed, 4096, 1024))
        rec["bfs"] = [f.result() for f in bfs_f]
        rec.update(cc_f.result())
        rec["pagerank"] = pr_f.result()
    rec["triangles"] = oracle.tc_ordered(g, threads=THREADS, chunks=4096)
    rec["oracle_seconds"] = round(time.time() - t0, 1)
    return rec


def dynamic_workload() -> dict:
    t0 = time.time()
    n, src, dst = graphgen.workload("rmat24")
    seed = graphgen.SEEDS["rmat24"]
    s0 = int(graphgen.pick_sources(n, src, dst, 1, seed + 1)[0])
    dg = oracle.DynGraph(n, src, dst)
    rounds = []
    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        pending = []
        for r, (ins_s, ins_d, del_s, del_d) in enumerate(graphgen.dynamic_rounds(n, src, dst)):
            dg.insert(ins_s, ins_d)
            dg.delete(del_s, del_d)
            g = dg.csr()
            deg = np.diff(g.off.astype(np.int64))
            ids = pr_sample_ids(n, deg, seed + 1000 + r, 512, 128)
            pending.append((r, g.m, sha_csr(g.off, g.col), ex.submit(bfs_record, g, s0), ex.submit(cc_record, g),
                            ex.submit(pr_record, g, ids)))
        for r, m, h, bf, cf_, pf in pending:
            rec = {"round": r, "m": m, "csr_sha256": h, "bfs": bf.result(), "pagerank": pf.result()}
            rec.update(cf_.result())
            rounds.append(rec)
    return {"workload": "dynamic", "base": "rmat24", "n": n, "source": s0, "rounds": rounds,
            "oracle_seconds": round(time.time() - t0, 1)}


def batched_member_record(i, n, s, d, sources) -> dict:
    g = oracle.csr_build(n, s, d)
    lv = np.stack([oracle.bfs(g, int(x))[0] for x in sources])
    return {"member": i, "n": n, "m": g.m, "levels_sha256": sha_u32(lv), "cc_sha256": sha_u32(oracle.cc(g))}


def batched_workload() -> dict:
    t0 = time.time()
    members = graphgen.batched_workload(256, 64)
    with cf.ThreadPoolExecutor(max_workers=THREADS) as ex:
        recs = list(ex.map(lambda a: batched_member_record(a[0], *a[1]), enumerate(members)))
    return {"workload": "batched", "graphs": len(members), "sources_per_graph": 64, "members": recs,
            "oracle_seconds": round(time.time() - t0, 1)}


def main(names):
    for name in names:
        if name == "dynamic":
            rec = dynamic_workload()
        elif name == "batched":
            rec = batched_workload()
        else:
            rec = static_workload(name)
        path = os.path.join(HERE, f"fullsize_{name}.json")
        with open(path + ".tmp", "w") as f:
            json.dump(rec, f, separators=(",", ":"))
        os.replace(path + ".tmp", path)
        print(f"{name}: {rec.get('oracle_seconds')} s -> {path}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["rmat25"])
