"""Pins for the oracle (CPU only).

The oracle is trusted only after it agrees with something other than itself:
hand-derived fixtures (``tests/golden/``), closed forms (Manhattan distances on a
grid, C(n,3) triangles in K_n, PageRank 1/n on regular graphs, the wheel and
complete-bipartite counts, binomial path counts and cycle/path/star
dependencies for betweenness, hand-derived byte codes and 7-bit group
boundaries), brute force on tiny inputs (Floyd-Warshall,
transitive closure, the O(n^3) triangle loop, trace(A^3)/6, betweenness from
all-pairs path counts), independent library
routines (scipy.sparse CSR construction, csgraph shortest paths and components,
the Google-matrix power and eigenvector in numpy), invariants (sum of PageRank,
relabelling, disjoint unions, insert-then-delete, byte-code round trips) and
central finite
differences for the network gradient.  Each group is chosen so that a plausible
slip (a dropped term, a wrong index or sign, a transposed operand) fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import graphgen
import oracle

INF = oracle.INF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


def _edges_from_adj(A):
    iu, ju = np.nonzero(np.triu(A, 1))
    return iu.astype(np.uint32), ju.astype(np.uint32)


def _dense(g):
    A = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        A[v, g.neighbors(v)] = 1
    return A


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.random((n, n)) < p, 1)
    return _edges_from_adj(A | A.T)


def _path(n):
    return np.arange(n - 1, dtype=np.uint32), np.arange(1, n, dtype=np.uint32)


def _complete(n):
    A = np.ones((n, n), dtype=bool)
    np.fill_diagonal(A, False)
    return _edges_from_adj(A)


def _grid_full(r, c):
    src, dst = [], []
    for i in range(r):
        for j in range(c):
            v = i * c + j
            if j + 1 < c:
                src.append(v); dst.append(v + 1)
            if i + 1 < r:
                src.append(v); dst.append(v + c)
    return np.array(src, np.uint32), np.array(dst, np.uint32)


# ----------------------------------------------------------------------------- CSR

def test_csr_golden_fixture():
    gd = _golden("small_graph.txt")
    n = gd["n"][0]
    pairs = np.array(gd["pairs"], np.uint32).reshape(-1, 2)
    g = oracle.csr_build(n, pairs[:, 0], pairs[:, 1])
    assert g.off.tolist() == gd["off"]
    assert g.col.tolist() == gd["col"]


def test_csr_matches_scipy_on_random_draws():
    n = 3000
    src, dst = graphgen.er(n, 20000, 123)
    g = oracle.csr_build(n, src, dst)
    A = sp.coo_matrix((np.ones(len(src)), (src, dst)), shape=(n, n)).tocsr()
    A = A + A.T
    A.setdiag(0)
    A.eliminate_zeros()
    A.sort_indices()
    assert np.array_equal(g.off, A.indptr.astype(np.uint64))
    assert np.array_equal(g.col, A.indices.astype(np.uint32))


def test_csr_invariants_rmat():
    n, src, dst = graphgen.rmat_small(12, 16, 7)
    g = oracle.csr_build(n, src, dst)
    deg = np.diff(g.off).astype(np.int64)
    assert int(deg.sum()) == g.m and g.m % 2 == 0
    rows = np.repeat(np.arange(n), deg)
    assert not np.any(rows == g.col)                       # no loops
    for v in range(0, n, 97):                              # sorted, unique
        nb = g.neighbors(v)
        assert np.all(np.diff(nb.astype(np.int64)) > 0)
    fwd = set(zip(rows.tolist(), g.col.tolist()))
    assert all((b, a) in fwd for a, b in list(fwd)[:5000])  # symmetric


def test_csr_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.csr_build(4, np.array([0, 4], np.uint32), np.array([1, 2], np.uint32))


# ----------------------------------------------------------------------------- BFS

def test_bfs_golden_fixture():
    gd = _golden("small_graph.txt")
    pairs = np.array(gd["pairs"], np.uint32).reshape(-1, 2)
    g = oracle.csr_build(gd["n"][0], pairs[:, 0], pairs[:, 1])
    assert oracle.bfs(g, 0)[0].tolist() == gd["bfs0"]
    assert oracle.bfs(g, 3)[0].tolist() == gd["bfs3"]


@pytest.mark.parametrize("r,c,s", [(7, 11, 0), (13, 5, 37), (1, 9, 4)])
def test_bfs_grid_is_manhattan(r, c, s):
    src, dst = _grid_full(r, c)
    g = oracle.csr_build(r * c, src, dst)
    level, parent = oracle.bfs(g, s)
    ii, jj = np.divmod(np.arange(r * c), c)
    si, sj = divmod(s, c)
    assert np.array_equal(level, (np.abs(ii - si) + np.abs(jj - sj)).astype(np.uint32))
    assert oracle.bfs_check_parents(g, s, level, parent) == -1


def test_bfs_path_complete_star():
    g = oracle.csr_build(50, *_path(50))
    assert oracle.bfs(g, 0)[0].tolist() == list(range(50))
    assert oracle.bfs(g, 49)[0].tolist() == list(range(49, -1, -1))
    g = oracle.csr_build(20, *_complete(20))
    lv = oracle.bfs(g, 5)[0]
    assert lv[5] == 0 and all(lv[v] == 1 for v in range(20) if v != 5)
    leaves = np.arange(1, 30, dtype=np.uint32)
    g = oracle.csr_build(30, np.zeros(29, np.uint32), leaves)
    assert oracle.bfs(g, 0)[0].tolist() == [0] + [1] * 29
    lv = oracle.bfs(g, 7)[0]
    assert lv[7] == 0 and lv[0] == 1 and all(lv[v] == 2 for v in range(1, 30) if v != 7)


@pytest.mark.parametrize("seed", range(6))
def test_bfs_floyd_warshall(seed):
    n = 48
    src, dst = _random_graph(n, 0.06, seed)
    g = oracle.csr_build(n, src, dst)
    D = np.full((n, n), np.inf)
    np.fill_diagonal(D, 0)
    D[src, dst] = 1
    D[dst, src] = 1
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    for s in range(0, n, 5):
        level, parent = oracle.bfs(g, s)
        want = np.where(np.isinf(D[s]), INF, D[s]).astype(np.uint32)
        assert np.array_equal(level, want)
        assert oracle.bfs_check_parents(g, s, level, parent) == -1


def test_bfs_matches_csgraph():
    n, src, dst = graphgen.rmat_small(11, 8, 3)
    g = oracle.csr_build(n, src, dst)
    A = sp.csr_matrix((np.ones(g.m), g.col, g.off.astype(np.int64)), shape=(n, n))
    for s in (0, 17, 1023):
        d = csgraph.shortest_path(A, unweighted=True, indices=s)
        want = np.where(np.isinf(d), INF, d).astype(np.uint32)
        level, parent = oracle.bfs(g, s)
        assert np.array_equal(level, want)
        assert oracle.bfs_check_parents(g, s, level, parent) == -1


def test_parent_checker_catches_bad_trees():
    src, dst = _grid_full(6, 6)
    g = oracle.csr_build(36, src, dst)
    level, parent = oracle.bfs(g, 0)
    assert oracle.bfs_check_parents(g, 0, level, parent) == -1
    bad = parent.copy(); bad[14] = 35                      # not a neighbour
    assert oracle.bfs_check_parents(g, 0, level, bad) == 14
    bad = parent.copy(); bad[14] = 15                      # neighbour, same level
    assert oracle.bfs_check_parents(g, 0, level, bad) == 14
    bad = parent.copy(); bad[0] = 1                        # source must be its own parent
    assert oracle.bfs_check_parents(g, 0, level, bad) == 0


# ----------------------------------------------------------------------------- CC

def test_cc_golden_fixture():
    gd = _golden("small_graph.txt")
    pairs = np.array(gd["pairs"], np.uint32).reshape(-1, 2)
    g = oracle.csr_build(gd["n"][0], pairs[:, 0], pairs[:, 1])
    assert oracle.cc(g).tolist() == gd["cc"]


def test_cc_disjoint_union_and_min_label():
    parts = [(_path(7), 7), (_complete(5), 5), ((np.zeros(0, np.uint32), np.zeros(0, np.uint32)), 3),
             (_grid_full(3, 4), 12)]
    src, dst, base = [], [], 0
    for (s, d), n in parts:
        src.append(s + base); dst.append(d + base); base += n
    g = oracle.csr_build(base, np.concatenate(src), np.concatenate(dst))
    lab = oracle.cc(g)
    # 1 (path) + 1 (K5) + 3 isolated + 1 (grid) components
    assert len(set(lab.tolist())) == 6
    assert lab.tolist() == [0] * 7 + [7] * 5 + [12, 13, 14] + [15] * 12


@pytest.mark.parametrize("seed", range(4))
def test_cc_transitive_closure(seed):
    n = 40
    src, dst = _random_graph(n, 0.035, seed)
    g = oracle.csr_build(n, src, dst)
    R = (_dense(g) + np.eye(n, dtype=np.int64)) > 0
    for _ in range(7):                                     # 2^7 > n hops
        R = (R.astype(np.int64) @ R.astype(np.int64)) > 0
    want = np.array([np.flatnonzero(R[v]).min() for v in range(n)], np.uint32)
    assert np.array_equal(oracle.cc(g), want)


def test_cc_matches_csgraph_and_relabelling():
    n, src, dst = graphgen.rmat_small(12, 2, 11)
    g = oracle.csr_build(n, src, dst)
    lab = oracle.cc(g)
    A = sp.csr_matrix((np.ones(g.m), g.col, g.off.astype(np.int64)), shape=(n, n))
    k, comp = csgraph.connected_components(A, directed=False)
    assert len(np.unique(lab)) == k
    # same partition, and each label is the component minimum
    mins = {}
    for v in range(n):
        mins.setdefault(comp[v], v)
    assert all(lab[v] == mins[comp[v]] for v in range(n))
    # relabel ids by a permutation: the partition must be carried along
    perm = graphgen.permutation(n, 99)
    g2 = oracle.csr_build(n, perm[src], perm[dst])
    lab2 = oracle.cc(g2)
    back = lab2[perm]                                       # label of the image of v
    # u, v share a component before iff their images share one after: the map
    # lab[v] -> back[v] is a bijection between the two label sets
    pairs = set(zip(lab.tolist(), back.tolist()))
    assert len(pairs) == k == len(set(back.tolist()))


# ----------------------------------------------------------------------------- TC

def test_tc_closed_forms():
    for n in range(1, 26):
        g = oracle.csr_build(n, *_complete(n)) if n > 1 else oracle.csr_build(1, [], [])
        assert oracle.tc(g) == math.comb(n, 3)
    g = oracle.csr_build(64, *_grid_full(8, 8))
    assert oracle.tc(g) == 0
    for n in range(4, 30):                                   # wheel: hub 0 + n-cycle
        rim = np.arange(1, n + 1, dtype=np.uint32)
        src = np.concatenate([np.zeros(n, np.uint32), rim])
        dst = np.concatenate([rim, np.roll(rim, -1)])
        assert oracle.tc(oracle.csr_build(n + 1, src, dst)) == n
    a, b = 9, 13                                              # K_{a,b}
    src = np.repeat(np.arange(a, dtype=np.uint32), b)
    dst = np.tile(np.arange(a, a + b, dtype=np.uint32), a)
    assert oracle.tc(oracle.csr_build(a + b, src, dst)) == 0


def test_tc_golden_fixture():
    gd = _golden("small_graph.txt")
    pairs = np.array(gd["pairs"], np.uint32).reshape(-1, 2)
    g = oracle.csr_build(gd["n"][0], pairs[:, 0], pairs[:, 1])
    assert oracle.tc(g) == gd["tc"][0]


@pytest.mark.parametrize("seed", range(4))
def test_tc_brute_force_triple_loop(seed):
    n = 60
    src, dst = _random_graph(n, 0.15, seed)
    g = oracle.csr_build(n, src, dst)
    A = _dense(g).astype(bool)
    cnt = 0
    for i in range(n):
        for j in range(i + 1, n):
            if A[i, j]:
                cnt += int(np.count_nonzero(A[i, j + 1:] & A[j, j + 1:]))
    assert oracle.tc(g) == cnt


def test_tc_trace_a3():
    n, src, dst = graphgen.rmat_small(9, 8, 5)
    g = oracle.csr_build(n, src, dst)
    A = _dense(g)
    assert oracle.tc(g) * 6 == int(np.trace(A @ A @ A))


def test_tc_ordered_closed_forms_and_brute_force():
    # the degree-ordered DAG count (used for the full-size reference values)
    # against the same closed forms and brute force as the plain count
    for n in (3, 4, 9, 25):
        assert oracle.tc_ordered(oracle.csr_build(n, *_complete(n))) == math.comb(n, 3)
    assert oracle.tc_ordered(oracle.csr_build(64, *_grid_full(8, 8))) == 0
    for n in (4, 7, 30):                                      # wheel: a hub of higher degree
        rim = np.arange(1, n + 1, dtype=np.uint32)
        src = np.concatenate([np.zeros(n, np.uint32), rim])
        dst = np.concatenate([rim, np.roll(rim, -1)])
        assert oracle.tc_ordered(oracle.csr_build(n + 1, src, dst)) == n
    for seed in range(3):
        n = 60
        src, dst = _random_graph(n, 0.2, seed)
        g = oracle.csr_build(n, src, dst)
        A = _dense(g).astype(bool)
        cnt = sum(int(np.count_nonzero(A[i, j + 1:] & A[j, j + 1:]))
                  for i in range(n) for j in range(i + 1, n) if A[i, j])
        assert oracle.tc_ordered(g) == cnt


def test_tc_ordered_dag_and_split_sum():
    n, src, dst = graphgen.rmat_small(11, 16, 21)               # hubs and many equal degrees
    g = oracle.csr_build(n, src, dst)
    dag_off, dag_col = oracle.tc_dag(g)
    deg = np.diff(g.off.astype(np.int64))
    assert int(dag_off[-1]) * 2 == g.m                          # every edge kept once
    rows = np.repeat(np.arange(n), np.diff(dag_off.astype(np.int64)))
    d = dag_col[:int(dag_off[-1])].astype(np.int64)
    assert np.all((deg[rows] < deg[d]) | ((deg[rows] == deg[d]) & (rows < d)))   # (degree, id) order
    A = _dense(g).astype(np.float64)                            # exact: counts stay far below 2^53
    want = int(round(np.trace(A @ A @ A))) // 6
    assert oracle.tc_ordered(g) == want == oracle.tc(g)
    assert oracle.tc_ordered(g, threads=3, chunks=17) == want   # centre ranges sum to the whole


# ----------------------------------------------------------------------------- betweenness

def test_bc_path_star_complete():
    # path from an end: one shortest path to each vertex, v lies on the paths to
    # the n-1-v vertices beyond it
    n = 9
    level, sigma, delta = oracle.bc(oracle.csr_build(n, *_path(n)), 0)
    assert list(level) == list(range(n)) and (sigma == 1).all()
    assert list(delta) == [0] + [n - 1 - v for v in range(1, n)]
    # from the middle of the path: each side on its own
    level, sigma, delta = oracle.bc(oracle.csr_build(n, *_path(n)), 4)
    assert list(delta) == [0, 1, 2, 3, 0, 3, 2, 1, 0]
    # star, source a leaf: the centre is between the source and the n-2 other leaves
    n = 12
    g = oracle.csr_build(n, np.zeros(n - 1, np.uint32), np.arange(1, n, dtype=np.uint32))
    level, sigma, delta = oracle.bc(g, 5)
    assert (sigma[level != INF] == 1).all() and delta[0] == n - 2 and (np.delete(delta, 0) == 0).all()
    # complete graph: every target is a neighbour of the source
    level, sigma, delta = oracle.bc(oracle.csr_build(10, *_complete(10)), 3)
    assert (delta == 0).all() and (sigma == 1).all()


@pytest.mark.parametrize("k", [3, 5, 8])
def test_bc_even_cycle_closed_form(k):
    # cycle of 2k from 0: the antipode k has two shortest paths; the vertex at
    # distance d < k on either side carries the k-1-d vertices beyond it and half
    # of the antipode
    n = 2 * k
    src = np.arange(n, dtype=np.uint32)
    level, sigma, delta = oracle.bc(oracle.csr_build(n, src, (src + 1) % n), 0)
    assert sigma[k] == 2 and (np.delete(sigma, k) == 1).all()
    for v in range(1, n):
        d = min(v, n - v)
        assert delta[v] == (0.0 if d == k else (k - 1 - d) + 0.5)


@pytest.mark.parametrize("r,c", [(4, 6), (7, 5)])
def test_bc_grid_path_counts_are_binomial(r, c):
    # full grid from a corner: the shortest paths to (i, j) are the monotone
    # lattice paths, C(i+j, i) of them
    level, sigma, delta = oracle.bc(oracle.csr_build(r * c, *_grid_full(r, c)), 0)
    for i in range(r):
        for j in range(c):
            assert level[i * c + j] == i + j and sigma[i * c + j] == math.comb(i + j, i)


def _bfs_counts(A, s):
    """Distances and shortest-path counts from s on a dense adjacency matrix."""
    n = len(A)
    dist = [-1] * n
    cnt = [0] * n
    dist[s], cnt[s] = 0, 1
    frontier = [s]
    while frontier:
        nxt = []
        for u in frontier:
            for v in np.nonzero(A[u])[0]:
                if dist[v] == -1:
                    dist[v] = dist[u] + 1
                    nxt.append(v)
                if dist[v] == dist[u] + 1:
                    cnt[v] += cnt[u]
        frontier = nxt
    return dist, cnt


@pytest.mark.parametrize("seed", range(4))
def test_bc_brute_force_definition(seed):
    # delta(v) = sum over t of sigma_st(v) / sigma_st with sigma_st(v) =
    # sigma_sv * sigma_vt when v is on a shortest s-t path, from all-pairs
    # path counts (exact rationals)
    n = 40
    g = oracle.csr_build(n, *_random_graph(n, 0.08, 300 + seed))
    A = _dense(g)
    s = seed % n
    D, C = zip(*[_bfs_counts(A, v) for v in range(n)])
    level, sigma, delta = oracle.bc(g, s)
    for v in range(n):
        want = Fraction(0)
        if v != s and D[s][v] >= 0:
            for t in range(n):
                if t in (s, v) or D[s][t] < 0:
                    continue
                if D[s][v] + D[v][t] == D[s][t]:
                    want += Fraction(C[s][v] * C[v][t], C[s][t])
        assert sigma[v] == C[s][v]
        assert abs(delta[v] - float(want)) <= 1e-12 * max(1.0, float(want))


def test_bc_unreached_and_source():
    # two components: the other one is unreached (level INF, sigma 0, delta 0)
    src = np.array([0, 1, 3], np.uint32)
    dst = np.array([1, 2, 4], np.uint32)
    level, sigma, delta = oracle.bc(oracle.csr_build(5, src, dst), 0)
    assert list(level[:3]) == [0, 1, 2] and level[3] == INF and level[4] == INF
    assert list(sigma) == [1, 1, 1, 0, 0] and list(delta) == [0, 1, 0, 0, 0]


# ----------------------------------------------------------------------------- byte-coded lists

def test_bytecode_golden_fixture():
    fx = _golden("bytecode_small.txt")
    n = fx["n"][0]
    pr = np.array(fx["pairs"], np.uint32).reshape(-1, 2)
    g = oracle.csr_build(n, pr[:, 0], pr[:, 1])
    boff, data = oracle.bytecode_encode(g)
    assert int(boff[-1]) == fx["total"][0] == len(data)
    for v in range(n):
        want = fx.get(f"v{v}", [])
        assert list(data[boff[v]:boff[v + 1]]) == want, v


def _code_len(w):
    return max(1, (int(w).bit_length() + 6) // 7)


def test_bytecode_group_boundaries():
    # gaps of 127 / 128 / 16383 / 16384 take 1 / 2 / 2 / 3 bytes; a first
    # difference of -(2^21 + 1) is stored as 2^22 + 3 and takes 4
    nb = [1, 128, 256, 16639, 33023]  # 1 after the source 0, then gaps 127, 128, 16383, 16384
    n = 2**21 + 2
    off = np.zeros(n + 1, np.uint64)
    off[1:] = len(nb)
    col = np.array(nb, np.uint32)
    boff, data = oracle.bytecode_encode(oracle.CSR(n, off, col))
    assert [b - a for a, b in zip(nb[:-1], nb[1:])] == [127, 128, 16383, 16384]
    assert int(boff[1]) == 1 + 1 + 2 + 2 + 3
    assert list(data) == [2, 127, 128, 1, 255, 127, 128, 128, 1]
    assert oracle.bytecode_decode(n, off, boff, data).col.tolist() == nb
    # the last vertex's only neighbour is 0: first difference -(n - 1)
    off2 = np.zeros(n + 1, np.uint64)
    off2[n] = 1
    b2, d2 = oracle.bytecode_encode(oracle.CSR(n, off2, np.zeros(1, np.uint32)))
    z = 2 * (n - 1) + 1
    assert z == 2**22 + 3 and list(d2) == [3 | 128, 128, 128, 2]
    assert oracle.bytecode_decode(n, off2, b2, d2).col.tolist() == [0]


@pytest.mark.parametrize("seed", range(3))
def test_bytecode_round_trip_and_size(seed):
    # decoding gives the CSR back; the size is the sum of the 7-bit group
    # counts of the values, computed here from the CSR directly
    n, src, dst = graphgen.rmat_small(12, 8, 900 + seed)
    g = oracle.csr_build(n, src, dst)
    boff, data = oracle.bytecode_encode(g)
    back = oracle.bytecode_decode(n, g.off, boff, data)
    assert np.array_equal(back.col, g.col)
    total = 0
    for v in range(n):
        nb = g.neighbors(v).astype(np.int64)
        if len(nb):
            total += _code_len(2 * abs(nb[0] - v) + (nb[0] < v))
            total += sum(_code_len(w) for w in np.diff(nb))
        assert int(boff[v + 1] - boff[v]) <= 5 * len(nb)
    assert total == int(boff[-1]) == len(data)
    assert len(data) < 4 * g.m  # sorted lists compress below 4-byte ids


# ----------------------------------------------------------------------------- PageRank

def _google(g, d):
    n = g.n
    A = _dense(g).astype(np.float64)
    deg = A.sum(axis=1)
    P = np.zeros((n, n))
    for u in range(n):
        if deg[u] > 0:
            P[:, u] = A[u] / deg[u]                          # column u spreads p(u)/deg(u)
        else:
            P[:, u] = 1.0 / n                                # dangling: uniform
    return d * P + (1.0 - d) / n * np.ones((n, n))


@pytest.mark.parametrize("seed", range(3))
def test_pagerank_matches_google_matrix_power(seed):
    n = 40
    src, dst = _random_graph(n, 0.08, seed)
    keep = dst != 3                                           # make sure vertex 3 is isolated
    src, dst = src[keep & (src != 3)], dst[keep & (src != 3)]
    g = oracle.csr_build(n, src, dst)
    assert g.off[4] == g.off[3]
    G = _google(g, 0.85)
    p, resid = oracle.pagerank(g, 0.85, 20)
    want = np.linalg.matrix_power(G, 20) @ np.full(n, 1.0 / n)
    assert np.max(np.abs(p - want)) < 1e-14
    prev = np.linalg.matrix_power(G, 19) @ np.full(n, 1.0 / n)
    assert abs(resid[-1] - np.abs(want - prev).sum()) < 1e-13


def test_pagerank_converges_to_eigenvector():
    n = 30
    src, dst = _random_graph(n, 0.1, 42)
    g = oracle.csr_build(n, src, dst)
    G = _google(g, 0.85)
    w, V = np.linalg.eig(G)
    v = np.real(V[:, np.argmax(np.real(w))])
    v = v / v.sum()
    p, _ = oracle.pagerank(g, 0.85, 300)
    assert np.max(np.abs(p - v)) < 1e-12


def test_pagerank_regular_graphs_are_uniform():
    for src, dst, n in [(*_complete(17), 17),
                        (np.arange(40, dtype=np.uint32), (np.arange(40, dtype=np.uint32) + 1) % 40, 40)]:
        g = oracle.csr_build(n, src, dst)
        for t in (1, 5, 20):
            p, resid = oracle.pagerank(g, 0.85, t)
            assert np.all(p == 1.0 / n) or np.max(np.abs(p - 1.0 / n)) < 1e-17
            assert np.all(resid < 1e-15)


def test_pagerank_mass_is_one():
    n, src, dst = graphgen.rmat_small(12, 4, 8)
    g = oracle.csr_build(n, src, dst)
    assert np.any(np.diff(g.off) == 0)                        # has dangling vertices
    for t in (1, 7, 20):
        p, _ = oracle.pagerank(g, 0.85, t)
        assert abs(p.sum() - 1.0) < 1e-12


def test_pagerank_exact_rational():
    # 20 iterations in exact arithmetic on a 9-vertex graph with 2 dangling vertices
    pairs = [(0, 1), (1, 2), (2, 0), (2, 3), (3, 4), (5, 6), (4, 1)]
    n = 9
    g = oracle.csr_build(n, np.array([a for a, _ in pairs], np.uint32), np.array([b for _, b in pairs], np.uint32))
    nb = [g.neighbors(v).tolist() for v in range(n)]
    d = Fraction(85, 100)
    p = [Fraction(1, n)] * n
    for _ in range(20):
        D = sum((p[u] for u in range(n) if not nb[u]), Fraction(0))
        q = []
        for v in range(n):
            s = sum((p[u] / len(nb[u]) for u in nb[v]), Fraction(0))
            q.append((1 - d) / n + d * (s + D / n))
        p = q
    got, _ = oracle.pagerank(g, 0.85, 20)
    assert np.max(np.abs(got - np.array([float(x) for x in p]))) < 1e-15


# ----------------------------------------------------------------------------- dynamic edge set

def test_dyn_insert_only_equals_rebuild():
    n, src, dst = graphgen.rmat_small(10, 8, 21)
    bs, bd = graphgen.rmat(10, 3000, 77)
    dg = oracle.DynGraph(n, src, dst)
    dg.insert(bs, bd)
    want = oracle.csr_build(n, np.concatenate([src, bs]), np.concatenate([dst, bd]))
    got = dg.csr()
    assert np.array_equal(got.off, want.off) and np.array_equal(got.col, want.col)


def test_dyn_delete_matches_set_difference():
    n, src, dst = graphgen.rmat_small(10, 8, 22)
    dg = oracle.DynGraph(n, src, dst)
    idx = graphgen.pick_indices(len(src), 2000, 5)
    ds, dd = src[idx], dst[idx]
    dg.delete(ds, dd)
    E = {(int(a), int(b)) for a, b in zip(src, dst) if a != b}
    E |= {(b, a) for a, b in E}
    gone = {(int(a), int(b)) for a, b in zip(ds, dd)}
    gone |= {(b, a) for a, b in gone}
    keep = sorted(E - gone)
    want = oracle.csr_build(n, np.array([a for a, _ in keep], np.uint32), np.array([b for _, b in keep], np.uint32))
    got = dg.csr()
    assert got.m == len(keep)
    assert np.array_equal(got.off, want.off) and np.array_equal(got.col, want.col)


def test_dyn_insert_then_delete_restores():
    n, src, dst = graphgen.rmat_small(9, 8, 23)
    dg = oracle.DynGraph(n, src, dst)
    before = dg.csr()
    # a batch of pairs that are certainly absent: (v, v+1) pairs not yet present
    present = set(zip(before.col.tolist(), np.repeat(np.arange(n), np.diff(before.off).astype(np.int64)).tolist()))
    new = [(v, (v + 1) % n) for v in range(n) if (v, (v + 1) % n) not in present][:300]
    bs = np.array([a for a, _ in new] + [5], np.uint32)
    bd = np.array([b for _, b in new] + [5], np.uint32)   # plus a self-loop, ignored
    dg.insert(bs, bd)
    assert dg.m == before.m + 2 * len(new)
    dg.insert(bs, bd)                                      # re-insert: no change
    assert dg.m == before.m + 2 * len(new)
    dg.delete(bd, bs)                                      # reversed pairs delete the same edges
    after = dg.csr()
    assert np.array_equal(after.off, before.off) and np.array_equal(after.col, before.col)


# ----------------------------------------------------------------------------- schedule network

def _mlp_case(F=12, H1=8, H2=7, K=5, B=9, seed=0):
    rng = np.random.default_rng(seed)
    P = oracle.mlp_num_params(F, H1, H2, K)
    prm = rng.normal(0, 0.5, P)
    X = rng.normal(0, 1, (B, F))
    y = rng.integers(0, K, B).astype(np.int32)
    w = rng.uniform(0.1, 2.0, B)
    return prm, X, y, w, (F, H1, H2, K)


def test_mlp_gradient_finite_differences():
    prm, X, y, w, (F, H1, H2, K) = _mlp_case()
    L, g, _ = oracle.mlp_loss(prm, F, H1, H2, K, X, y, w)
    h = 1e-6
    num = np.empty_like(prm)
    for i in range(len(prm)):
        a = prm.copy(); a[i] += h
        b = prm.copy(); b[i] -= h
        num[i] = (oracle.mlp_loss(a, F, H1, H2, K, X, y, w, False)[0] -
                  oracle.mlp_loss(b, F, H1, H2, K, X, y, w, False)[0]) / (2 * h)
    assert np.linalg.norm(num - g) <= 1e-6 * max(1.0, np.linalg.norm(g))


def test_mlp_one_hidden_unit_closed_form():
    # F=H1=H2=1, K=2: h1=relu(a x+b), h2=relu(c h1+e), z=(p h2+q, r h2+s)
    a, b, c, e, p, q, r, s = 0.7, 0.1, -1.3, 2.0, 0.5, -0.2, 1.5, 0.3
    x = 2.0
    prm = np.array([a, b, c, e, p, r, q, s])
    h1 = max(a * x + b, 0.0)            # 1.5
    h2 = max(c * h1 + e, 0.0)           # 0.05
    z0, z1 = p * h2 + q, r * h2 + s
    L_true = math.log(math.exp(z0) + math.exp(z1)) - z1   # label 1
    L, g, logits = oracle.mlp_loss(prm, 1, 1, 1, 2, np.array([[x]]), np.array([1]), None)
    assert abs(L - L_true) < 1e-15
    assert np.allclose(logits[0], [z0, z1], atol=1e-15)
    sm1 = math.exp(z1) / (math.exp(z0) + math.exp(z1))
    dz0, dz1 = 1 - sm1, sm1 - 1
    dh2 = p * dz0 + r * dz1
    dh1 = c * dh2
    want = [dh1 * x, dh1, dh2 * h1, dh2, dz0 * h2, dz1 * h2, dz0, dz1]
    assert np.allclose(g, want, atol=1e-14)


def test_mlp_softmax_shift_invariance():
    prm, X, y, w, (F, H1, H2, K) = _mlp_case(seed=3)
    L, g, _ = oracle.mlp_loss(prm, F, H1, H2, K, X, y, w)
    shifted = prm.copy(); shifted[-K:] += 3.0
    assert abs(oracle.mlp_loss(shifted, F, H1, H2, K, X, y, w, False)[0] - L) < 1e-12
    assert abs(g[-K:].sum()) < 1e-12                           # dL/db3 sums to zero


# ----------------------------------------------------------------------------- generators

def test_generators_deterministic_and_in_range():
    a = graphgen.er(1000, 5000, 1)
    b = graphgen.er(1000, 5000, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[0].max() < 1000 and a[1].max() < 1000
    c = graphgen.er(1000, 5000, 2)
    assert not np.array_equal(a[0], c[0])


def test_rmat_quadrant_frequencies():
    k = 10_000_000
    src, dst = graphgen.rmat(1, k, 5, permute=False)
    q = (src.astype(np.int64) << 1) | dst
    cnt = np.bincount(q, minlength=4)
    for c, p in zip(cnt, (0.57, 0.19, 0.19, 0.05)):
        assert abs(c - p * k) <= 3 * math.sqrt(k * p * (1 - p))


def test_rmat_permutation_is_bijection():
    perm = graphgen.permutation(1 << 12, 3)
    assert np.array_equal(np.sort(perm), np.arange(1 << 12, dtype=np.uint32))
    assert not np.array_equal(perm, np.arange(1 << 12))


def test_grid_generator_counts():
    src, dst = graphgen.grid(20, 30, 0.0, 0.0, 1)
    assert len(src) == 20 * 29 + 19 * 30
    src, dst = graphgen.grid(200, 200, 0.10, 1e-2, 1)
    total = 200 * 199 * 2
    S = len(src) - np.count_nonzero((np.abs(src.astype(np.int64) - dst) == 1) | (np.abs(src.astype(np.int64) - dst) == 200))
    kept = len(src) - S
    assert abs(kept - 0.9 * total) <= 5 * math.sqrt(total * 0.09)
    assert abs(S - round(0.01 * kept)) <= 3            # a few shortcuts may look like grid steps


def test_pick_sources_distinct_non_isolated():
    n = 500
    src = np.array([1, 2, 3, 7, 7], np.uint32)
    dst = np.array([2, 3, 3, 9, 7], np.uint32)
    s = graphgen.pick_sources(n, src, dst, 10, 4)
    assert sorted(s.tolist()) == [1, 2, 3, 7, 9]
