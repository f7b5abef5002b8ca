"""Many graphs in one container and multi-source BFS, against the oracle run on
each member separately (levels bit-exact per member and source, CC labels
canonical per member)."""
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


def members(count, lo, hi, seed):
    out = []
    for kind, n, k, s in graphgen.batched_params(count, seed=seed, lo_log2=lo, hi_log2=hi, deg_lo=4, deg_hi=16):
        src, dst = graphgen.batched_member(kind, n, k, s)
        out.append((n, src, dst))
    return out


def sources_for(n, src, dst, S, seed):
    s = graphgen.pick_sources(n, src, dst, S, seed).tolist()
    s += [v % n for v in range(S - len(s))]  # tiny members: fill with any ids
    return s[:S]


@pytest.mark.parametrize("S", [64, 5])
def test_batch_msbfs_and_cc(byo, S):
    mem = members(12, 8, 12, 1234 + S)
    ns = [n for n, _, _ in mem]
    ks = [len(s) for _, s, _ in mem]
    g = byo.byo_batch_build(ns, ks, dev(np.concatenate([s for _, s, _ in mem])),
                            dev(np.concatenate([d for _, _, d in mem])))
    try:
        srcs = [sources_for(n, s, d, S, i) for i, (n, s, d) in enumerate(mem)]
        lv = host(byo.byo_msbfs(g, srcs, S))
        lab = host(byo.byo_cc(g))
        for i, (n, s, d) in enumerate(mem):
            base = byo.byo_batch_member_base(g, i)
            ref = oracle.csr_build(n, s, d)
            assert np.array_equal(lab[base:base + n] - base, oracle.cc(ref))
            for j in range(S):
                want, _ = oracle.bfs(ref, srcs[i][j])
                assert np.array_equal(lv[j, base:base + n], want), (i, j)
        # a plain BFS on the batch stays inside the source's member
        base3 = byo.byo_batch_member_base(g, 3)
        one, _ = byo.byo_bfs(g, [base3 + srcs[3][0]])
        one = host(one[0])
        outside = np.ones(len(one), bool)
        outside[base3:base3 + ns[3]] = False
        assert np.all(one[outside] == INF)
    finally:
        byo.byo_graph_destroy(g)


def test_msbfs_single_graph_and_errors(byo):
    n, src, dst = graphgen.rmat_small(12, 16, 8)
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev(src), dev(dst))
    srcs = graphgen.pick_sources(n, src, dst, 40, 2).tolist()
    lv = host(byo.byo_msbfs(g.handle, srcs, len(srcs)))
    for j, s in enumerate(srcs):
        assert np.array_equal(lv[j], oracle.bfs(ref, s)[0])
    with pytest.raises(byo.ByoError):
        byo.byo_msbfs(g.handle, [n], 1)
    with pytest.raises(byo.ByoError):
        byo.byo_msbfs(g.handle, list(range(65)), 65)
    g.close()
