"""Parity at the workloads' full sizes, in the configuration bench.py times.

RMAT-22 (67,108,864 draws, uint64 offsets) and the 4096x4096 grid: BFS from
the benchmark's seeded sources, CC and PageRank are compared with the oracle
element by element; triangle counts are checked exactly on the grid and, on
RMAT-22, through properties that hold at any size (invariance under relabelling
the vertices, and equality between the static and the dynamic container).
RMAT-25 (the benchmark workload) is certified without the oracle by properties
of the outputs checked against the raw generated pairs: level[s] = 0, every
input pair spans at most one level (and is either reached on both ends or on
neither), every reached vertex has a parent one level up joined to it by an
input pair, CC labels agree across every input pair and every BFS-reached set
is exactly its source's component, and PageRank has total mass 1.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu
INF = 0xFFFFFFFF


@pytest.fixture(scope="module")
def byo():
    from paper_2405_11671_gb300 import build
    build.build()
    import paper_2405_11671_gb300 as b
    b.load()
    return b


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def bench_sources(name, n, src, dst, k=8):
    return graphgen.pick_sources(n, src, dst, k, graphgen.SEEDS[name] + 1).tolist()


@pytest.mark.parametrize("name", ["rmat22", "grid"])
def test_full_size_against_oracle(byo, name):
    n, src, dst = graphgen.workload(name)
    flags = byo.BYO_CSR | byo.BYO_SYMMETRIZE | (byo.BYO_OFFSETS64 if name.startswith("rmat") else 0)
    g = byo.Graph(n, dev(src), dev(dst), flags)
    ref = oracle.csr_build(n, src, dst)
    assert g.m == ref.m
    try:
        srcs = bench_sources(name, n, src, dst)
        lv, par = byo.byo_bfs(g.handle, srcs)
        for i, s in enumerate(srcs):
            want, _ = oracle.bfs(ref, s)
            got = host(lv[i])
            assert np.array_equal(got, want), (name, s)
            assert oracle.bfs_check_parents(ref, s, got, host(par[i])) == -1
        assert np.array_equal(host(byo.byo_cc(g.handle)), oracle.cc(ref))
        p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        w, _ = oracle.pagerank(ref, 0.85, 20)
        got = p.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - w) / w) <= 1e-5 and np.sum(np.abs(got - w)) <= 1e-6
        count = byo.byo_tc(g.handle)
        if name == "grid":
            assert count == oracle.tc(ref)
        else:
            # relabelled copy and dynamic container give the same count
            perm = graphgen.permutation(n, 31337)
            g2 = byo.Graph(n, dev(perm[src]), dev(perm[dst]), flags)
            assert byo.byo_tc(g2.handle) == count
            g2.close()
            g3 = byo.Graph(n, dev(src), dev(dst), byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE)
            assert byo.byo_tc(g3.handle) == count
            g3.close()
    finally:
        g.close()


def test_rmat25_properties(byo):
    n, src, dst = graphgen.workload("rmat25")
    g = byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE | byo.BYO_OFFSETS64)
    try:
        srcs = bench_sources("rmat25", n, src, dst, 2)
        lv, par = byo.byo_bfs(g.handle, srcs)
        lab = byo.byo_cc(g.handle)
        s_t, d_t = dev(src).long() & 0xFFFFFFFF, dev(dst).long() & 0xFFFFFFFF
        keys = torch.sort(torch.cat([s_t * (1 << 32) + d_t, d_t * (1 << 32) + s_t])).values
        for i, s in enumerate(srcs):
            L = lv[i].long() & 0xFFFFFFFF
            P = par[i].long() & 0xFFFFFFFF
            assert int(L[s]) == 0 and int(P[s]) == s
            lu, lw = L[s_t], L[d_t]
            reached_u, reached_w = lu != INF, lw != INF
            assert torch.equal(reached_u, reached_w)                       # closed under edges
            assert int((lu[reached_u] - lw[reached_u]).abs().max()) <= 1   # no edge skips a level
            v = torch.nonzero((L != INF) & (torch.arange(n, device="cuda") != s)).squeeze(1)
            pv = P[v]
            assert int((L[pv] + 1 - L[v]).abs().max()) == 0              # parent one level up
            q = pv * (1 << 32) + v
            pos = torch.searchsorted(keys, q).clamp(max=len(keys) - 1)
            assert torch.equal(keys[pos], q)                              # parent joined by an input pair
            comp = (lab.long() & 0xFFFFFFFF) == (int(lab[s]) & 0xFFFFFFFF)
            assert torch.equal(comp, L != INF)                            # reached set = component
        la = lab.long() & 0xFFFFFFFF
        assert torch.equal(la[s_t], la[d_t])                              # labels agree across pairs
        assert int((la > torch.arange(n, device="cuda")).sum()) == 0      # label = a smaller-or-equal id
        assert torch.equal(la[la], la)                                    # labels are roots
        p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        assert abs(float(p.double().sum()) - 1.0) < 1e-5
        assert float(p.min()) >= 0.15 / n * (1 - 1e-5)
    finally:
        g.close()
