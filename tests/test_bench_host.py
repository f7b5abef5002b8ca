"""Host logic of bench.py's roofline: the algorithmic byte models, computed
from a traversal's outputs (levels) by the method's definition."""
import numpy as np
import torch

import bench
import graphgen
import oracle


class R:
    def __init__(self, level, direction, t_ns=1000):
        self.level, self.direction, self.t_ns = level, direction, t_ns


def _csr(n, pairs):
    src = np.array([p[0] for p in pairs], np.uint32)
    dst = np.array([p[1] for p in pairs], np.uint32)
    g = oracle.csr_build(n, src, dst)
    return g, torch.from_numpy(g.off.astype(np.int64)), torch.from_numpy(g.col.view(np.int32))


def test_pagerank_bytes_per_iteration():
    # 8-byte offsets of the degree-ordered copy, 4-byte ids, 16 bytes of
    # contributions and ranks per vertex
    n, m = 1000, 30000
    assert bench.algo_bytes("pr_iter", n, m, 4) == 8 * (n + 1) + 4 * m + 16 * n


def test_cc_sampling_bytes():
    n = 1 << 20
    got = bench.algo_bytes("cc_sample", n, 0, 8)
    assert got == 4 * n + 2 * (8 * (n + 1) + 12 * n) + 8 * n


def test_bfs_bytes_square_push_then_pull():
    # square 0-1, 0-2, 1-3, 2-3 from 0: levels 0,1,1,2; level 0 push, level 1 pull
    g, off, col = _csr(4, [(0, 1), (0, 2), (1, 3), (2, 3)])
    lv = torch.tensor([0, 1, 1, 2], dtype=torch.int32)
    total, per = bench.bfs_method_bytes(torch, off, col, lv, [R(0, 1), R(1, 0)], 8)
    push = 8 * 1 + 4 * 2 + 4 * 1 + 12 * 2 + 4 / 8          # F = {0}, F' = {1, 2}
    pull = 8 * 1 + 4 * (1 + 0) + 3 * 4 / 8 + 8 * 1          # unvisited {3}: scans 1 id (its first neighbour 1)
    assert per == [(0, 1, push, 1000), (1, 0, pull, 1000)]
    assert total == 8 * 4 + 4 / 8 + push + pull


def test_bfs_pull_scan_stops_at_first_frontier_neighbour():
    # path 0-1-2-3 from 0, one pull at level 0: vertex 1 stops at its first
    # neighbour (0); 2 and 3 have no frontier neighbour and read whole lists
    g, off, col = _csr(4, [(0, 1), (1, 2), (2, 3)])
    lv = torch.tensor([0, 1, 2, 3], dtype=torch.int32)
    _, per = bench.bfs_method_bytes(torch, off, col, lv, [R(0, 0)], 4)
    assert per[0][2] == 4 * 3 + 4 * (1 + 2 + 1) + 3 * 4 / 8 + 8 * 1


def test_bfs_pull_scan_matches_a_direct_walk():
    # scanned(v) by the definition, walked vertex by vertex with the oracle's
    # CSR and levels, against the vectorised count
    n, src, dst = graphgen.rmat_small(10, 8, 3)
    g = oracle.csr_build(n, src, dst)
    s = int(graphgen.pick_sources(n, src, dst, 1, 4)[0])
    lv, _ = oracle.bfs(g, s)
    off = torch.from_numpy(g.off.astype(np.int64))
    col = torch.from_numpy(g.col.view(np.int32))
    depth = int(lv[lv != oracle.INF].max())
    trace = [R(l, 0) for l in range(depth)]
    _, per = bench.bfs_method_bytes(torch, off, col, torch.from_numpy(lv.view(np.int32)), trace, 8)
    for lvl, _, b, _ in per:
        scanned = 0
        for v in range(n):
            if lv[v] != oracle.INF and lv[v] <= lvl:
                continue
            nb = g.neighbors(v)
            hit = np.nonzero(lv[nb] == lvl)[0]
            scanned += int(hit[0]) + 1 if len(hit) else len(nb)
        deg = np.diff(g.off.astype(np.int64))
        unvis = int(np.sum(((lv == oracle.INF) | (lv > lvl)) & (deg > 0)))
        fnext = int(np.sum(lv == lvl + 1))
        assert b == 8 * unvis + 4 * scanned + 3 * n / 8 + 8 * fnext, lvl


def test_level_bandwidth_picks_largest_levels():
    levels = [(0, 1, 100.0, 10), (1, 1, 900.0, 30), (2, 0, 5000.0, 50), (3, 1, 10.0, 10)]
    bw = bench.level_bandwidth(levels, 100.0)
    assert bw["push"]["largest_level"] == 1 and bw["push"]["largest_gbs"] == 30.0
    assert bw["push"]["total_bytes"] == 1010.0 and bw["pull"]["largest_gbs"] == 100.0
    assert bw["pull"]["largest_frac"] == 1.0


def test_msbfs_bytes_two_sources():
    # path 0-1-2 with sources 0 and 2 (n = 3, m = 4, 4-byte offsets)
    g, off, col = _csr(3, [(0, 1), (1, 2)])
    lv = torch.tensor([[0, 1, 2], [2, 1, 0]], dtype=torch.int32)
    got = bench.msbfs_method_bytes(torch, off, col, lv, 1.0, 2, 4)
    n = 3
    want = 24 * n + 4 * 2 * n                          # three words and both level rows initialised
    # level 0, top-down: F = {0, 2} (degree 1 each); (1, s0), (1, s1) found
    want += 8 * n + 4 * 2 + 12 * 2 + 24 * n + 4 * 2
    # level 1: its 2 frontier edges * alpha are not below the 0 edges never in
    # a frontier, so bottom-up: 0 and 2 each miss one source, found at their
    # first neighbour (1); (2, s0), (0, s1) found
    want += 8 * n + 4 * 2 + 12 * 2 + 24 * n + 4 * 2
    # level 2, bottom-up: every vertex has both sources; nothing found
    want += 8 * n + 24 * n
    assert got == want


def test_bc_bytes_path():
    # path 0-1-2 from 0: three reached vertices, degree sum 4, two edges to a
    # vertex one level closer (1 -> 0, 2 -> 1); 8-byte offsets
    g, off, col = _csr(3, [(0, 1), (1, 2)])
    lv = torch.tensor([0, 1, 2], dtype=torch.int32)
    n, r, dsum, closer = 3, 3, 4, 2
    want = 16 * n + 8 * n + 4 * r + 2 * (8 * r + 8 * dsum) + 8 * closer + 8 * r + 16 * closer + 16 * r
    assert bench.bc_method_bytes(torch, off, col, lv, 8) == want


def test_hashed_insert_bytes():
    # 10 pairs -> 20 entries: 8 B per pair read, 16 B of semisort and 4 B of
    # probe per entry; 6 new stored ids at 12 B; 7 touched records at 128 B
    assert bench.hashed_insert_bytes(10, 6, 7) == 8 * 10 + 20 * 16 + 20 * 4 + 12 * 6 + 128 * 7
