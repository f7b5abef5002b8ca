"""The dynamic blocked-adjacency container, sorted and hash-indexed
(BYO_DYN_HASH: unsorted lists, per-run hash indexes, semisorted batches),
against the oracle's edge set.

After every batch the container's contents (exported as CSR), m and the
degrees must equal the oracle's bit for bit; after every round BFS levels
(and parent validity), CC labels, triangle counts and PageRank (stated
tolerance) computed over the dynamic container must match the oracle run on
the oracle's own edge set.  Batches follow the dynamic-container workload:
RMAT-distributed inserts and deletes of uniformly drawn earlier pairs, plus
self-loops, duplicates and absent pairs.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def byo():
    from paper_2405_11671_gb300 import build
    build.build()
    import paper_2405_11671_gb300 as b
    b.load()
    return b


@pytest.fixture(params=["sorted", "hashed"])
def dflags(request, byo):
    """BYO_DYNAMIC, alone or with the hash-indexed variant."""
    return byo.BYO_DYNAMIC | (byo.BYO_DYN_HASH if request.param == "hashed" else 0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def same_contents(byo, g, ref):
    off, col = byo.byo_graph_export_csr(g.handle)
    assert g.m == ref.m
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
    assert np.array_equal(host(col), ref.col)
    assert np.array_equal(host(byo.byo_degree(g.handle)).astype(np.uint64), np.diff(ref.off))


def algorithms_match(byo, g, ref, sources):
    lv, par = byo.byo_bfs(g.handle, sources)
    for i, s in enumerate(sources):
        want, _ = oracle.bfs(ref, s)
        assert np.array_equal(host(lv[i]), want)
        assert oracle.bfs_check_parents(ref, s, host(lv[i]), host(par[i])) == -1
    assert np.array_equal(host(byo.byo_cc(g.handle)), oracle.cc(ref))
    assert byo.byo_tc(g.handle) == oracle.tc(ref)
    p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
    w, _ = oracle.pagerank(ref, 0.85, 20)
    got = p.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - w) / w) <= 1e-5 and np.sum(np.abs(got - w)) <= 1e-6


@pytest.mark.parametrize("name", ["tiny", "rmat12", "grid"])
def test_dynamic_build_equals_csr(byo, dflags, name):
    if name == "tiny":
        n, src, dst = graphgen.workload("tiny")
    elif name == "rmat12":
        n, src, dst = graphgen.rmat_small(12, 16, 5)
    else:
        n, src, dst = graphgen.grid_small(50, 60, 0.1, 1e-3, 3)
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev(src), dev(dst), dflags | byo.BYO_SYMMETRIZE)
    same_contents(byo, g, ref)
    algorithms_match(byo, g, ref, [0] + graphgen.pick_sources(n, src, dst, 1, 3).tolist())
    g.close()


def test_dynamic_rounds_match_oracle(byo, dflags):
    scale, seed = 13, 0xB14
    n, src, dst = graphgen.rmat_small(scale, 8, seed)
    g = byo.Graph(n, dev(src), dev(dst), dflags | byo.BYO_SYMMETRIZE)
    dg = oracle.DynGraph(n, src, dst)
    pool_s, pool_d = [src], [dst]
    for r in range(5):
        ins_s, ins_d = graphgen.rmat(scale, 4000, graphgen.stream(seed, 100 + r))
        # add self-loops and duplicates on purpose
        ins_s = np.concatenate([ins_s, ins_s[:50], np.arange(10, dtype=np.uint32)])
        ins_d = np.concatenate([ins_d, ins_d[:50], np.arange(10, dtype=np.uint32)])
        byo.byo_insert_batch(g.handle, dev(ins_s), dev(ins_d))
        dg.insert(ins_s, ins_d)
        same_contents(byo, g, dg.csr())
        pool_s.append(ins_s)
        pool_d.append(ins_d)
        ps, pd = np.concatenate(pool_s), np.concatenate(pool_d)
        pick = graphgen.pick_indices(len(ps), 4000, graphgen.stream(seed, 200 + r))
        del_s, del_d = ps[pick], pd[pick]
        # absent pairs and reversed pairs too
        del_s = np.concatenate([del_s, np.array([1, 2, 3], np.uint32), del_d[:20]])
        del_d = np.concatenate([del_d, np.array([1, 5, 7], np.uint32), del_s[:20]])
        byo.byo_delete_batch(g.handle, dev(del_s), dev(del_d))
        dg.delete(del_s, del_d)
        ref = dg.csr()
        same_contents(byo, g, ref)
        algorithms_match(byo, g, ref, graphgen.pick_sources(n, ps, pd, 2, r).tolist())
    g.close()


def test_hub_grows_through_classes_and_shrinks(byo, dflags):
    n = 20000
    g = byo.Graph(n, dev([1]), dev([2]), dflags | byo.BYO_SYMMETRIZE)
    dg = oracle.DynGraph(n, [1], [2])
    for hi in (5, 11, 12, 13, 40, 700, 5000, 19999):  # inline -> runs of growing class
        leaves = np.arange(3, hi + 3, dtype=np.uint32) % n
        hub = np.zeros(len(leaves), np.uint32)
        byo.byo_insert_batch(g.handle, dev(hub), dev(leaves))
        dg.insert(hub, leaves)
        same_contents(byo, g, dg.csr())
    for hi in (19999, 3000, 12, 2):  # and back down to inline
        leaves = np.arange(hi + 3, n, dtype=np.uint32)
        hub = np.zeros(len(leaves), np.uint32)
        byo.byo_delete_batch(g.handle, dev(leaves), dev(hub))
        dg.delete(leaves, hub)
        same_contents(byo, g, dg.csr())
    algorithms_match(byo, g, dg.csr(), [0, 1])
    g.close()


def test_insert_then_delete_restores(byo, dflags):
    n, src, dst = graphgen.rmat_small(12, 8, 77)
    g = byo.Graph(n, dev(src), dev(dst), dflags | byo.BYO_SYMMETRIZE)
    before = byo.byo_graph_export_csr(g.handle)
    b_s, b_d = graphgen.er(n, 5000, 99)
    base = oracle.csr_build(n, src, dst)
    present = set(zip(np.repeat(np.arange(n), np.diff(base.off).astype(np.int64)).tolist(), base.col.tolist()))
    keep = np.array([(a, b) not in present for a, b in zip(b_s.tolist(), b_d.tolist())])
    b_s, b_d = b_s[keep], b_d[keep]
    byo.byo_insert_batch(g.handle, dev(b_s), dev(b_d))
    byo.byo_delete_batch(g.handle, dev(b_s), dev(b_d))
    after = byo.byo_graph_export_csr(g.handle)
    assert torch.equal(before[0], after[0]) and torch.equal(before[1], after[1])
    g.close()


def test_batch_errors(byo, dflags):
    n, src, dst = graphgen.rmat_small(10, 4, 1)
    g = byo.Graph(n, dev(src), dev(dst))
    with pytest.raises(byo.ByoError) as e:
        byo.byo_insert_batch(g.handle, dev([1]), dev([2]))
    assert e.value.status == byo.BYO_ERR_UNSUPPORTED
    g.close()
    g = byo.Graph(n, dev(src), dev(dst), dflags | byo.BYO_SYMMETRIZE)
    with pytest.raises(byo.ByoError) as e:
        byo.byo_insert_batch(g.handle, dev([1]), dev([n]))
    assert e.value.status == byo.BYO_ERR_INVALID_ARG
    byo.byo_insert_batch(g.handle, dev([]), dev([]))  # empty batch is a no-op
    g.close()


def test_inline_head_ablation_and_space(byo):
    """The dynamic container without its inline head (every list in pool
    blocks) holds the same lists and gives the same results; byo_space counts
    the CSR arrays exactly, and for a freshly built dynamic container the
    vertex records plus the power-of-two runs of 32-id blocks of the lists
    longer than the inline capacity."""
    n, src, dst = graphgen.rmat_small(13, 8, 77)
    ref = oracle.csr_build(n, src, dst)
    deg = np.diff(ref.off.astype(np.int64))

    def runs(icap):
        d = deg[deg > icap]
        blocks = (d + 31) // 32
        return int(np.sum(1 << np.ceil(np.log2(blocks)).astype(np.int64)))

    with byo.Graph(n, dev(src), dev(dst)) as gc:
        assert byo.byo_space(gc.handle) == (n + 1) * 4 + 4 * ref.m
    got = {}
    for flags, icap in ((byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE, 12),
                        (byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE | byo.BYO_DYN_NO_INLINE, 0)):
        with byo.Graph(n, dev(src), dev(dst), flags) as g:
            assert byo.byo_space(g.handle) == 64 * (n + 1) + 128 * runs(icap)
            off, col = byo.byo_graph_export_csr(g.handle)
            assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
            assert np.array_equal(host(col), ref.col)
            lv, _ = byo.byo_bfs(g.handle, [3])
            assert np.array_equal(host(lv[0]), oracle.bfs(ref, 3)[0])
            assert byo.byo_tc(g.handle) == oracle.tc(ref)
            ins_s, ins_d = graphgen.rmat(13, 2000, 78)
            byo.byo_insert_batch(g.handle, dev(ins_s), dev(ins_d))
            got[icap] = byo.byo_graph_export_csr(g.handle)
    assert torch.equal(got[12][0], got[0][0]) and torch.equal(got[12][1], got[0][1])
    with pytest.raises(byo.ByoError):
        byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_DYN_NO_INLINE)


def test_hashed_index_rebuilds_and_space(byo):
    """The hash-indexed container: a hub whose list is emptied and refilled
    again and again (tombstones pile up in its index until an insert rebuilds
    it in place), a small graph flooded with duplicate pairs (an inline list
    planned into a run that stays within the inline capacity, so it goes back
    inline), and byo_space: 64-byte records plus, per block of the runs, 128
    bytes of ids and 512 of index slots."""
    n = 6000
    flags = byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE | byo.BYO_DYN_HASH
    with byo.Graph(n, dev([1]), dev([2]), flags) as g:
        dg = oracle.DynGraph(n, [1], [2])
        rng = np.random.default_rng(41)
        for r in range(8):
            leaves = rng.choice(np.arange(3, n, dtype=np.uint32), size=900, replace=False)
            hub = np.zeros(len(leaves), np.uint32)
            byo.byo_insert_batch(g.handle, dev(hub), dev(leaves))
            dg.insert(hub, leaves)
            same_contents(byo, g, dg.csr())
            gone = leaves[rng.random(len(leaves)) < 0.9]
            byo.byo_delete_batch(g.handle, dev(gone), dev(np.zeros(len(gone), np.uint32)))
            dg.delete(gone, np.zeros(len(gone), np.uint32))
            same_contents(byo, g, dg.csr())
        algorithms_match(byo, g, dg.csr(), [0, 1])
    n = 10
    base_s, base_d = np.zeros(4, np.uint32), np.arange(1, 5, dtype=np.uint32)
    with byo.Graph(n, dev(base_s), dev(base_d), flags) as g:
        dg = oracle.DynGraph(n, base_s, base_d)
        ins_s = np.zeros(80, np.uint32)
        ins_d = np.array([5, 1] * 40, np.uint32)
        byo.byo_insert_batch(g.handle, dev(ins_s), dev(ins_d))
        dg.insert(ins_s, ins_d)
        same_contents(byo, g, dg.csr())
        assert byo.byo_space(g.handle) == 64 * (n + 1)  # every list inline again
        algorithms_match(byo, g, dg.csr(), [0, 5])
    n, src, dst = graphgen.rmat_small(13, 8, 77)
    ref = oracle.csr_build(n, src, dst)
    deg = np.diff(ref.off.astype(np.int64))
    d = deg[deg > 12]
    blocks = int(np.sum(1 << np.ceil(np.log2((d + 31) // 32)).astype(np.int64)))
    with byo.Graph(n, dev(src), dev(dst), flags) as g:
        assert byo.byo_space(g.handle) == 64 * (n + 1) + (128 + 512) * blocks
        same_contents(byo, g, ref)
    with pytest.raises(byo.ByoError) as e:
        byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_DYN_HASH)
    assert e.value.status == byo.BYO_ERR_INVALID_ARG


@pytest.mark.parametrize("no_inline", [False, True], ids=["inline", "no_inline"])
def test_hashed_pool_growth_duplicates_and_no_inline(byo, no_inline):
    """The hash-indexed container outgrowing its pool (the index arrays grow
    and are copied with it), with and without the inline head; a hub whose
    group is thousands of copies of a few pairs (the CTA path must admit each
    id once); and most of the inserted pairs deleted again."""
    n = 30000
    rng = np.random.default_rng(5)
    base_s = rng.integers(0, n, 2000, dtype=np.uint32)
    base_d = rng.integers(0, n, 2000, dtype=np.uint32)
    flags = byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE | byo.BYO_DYN_HASH | (byo.BYO_DYN_NO_INLINE if no_inline else 0)
    with byo.Graph(n, dev(base_s), dev(base_d), flags) as g:
        dg = oracle.DynGraph(n, base_s, base_d)
        space0 = byo.byo_space(g.handle)
        # 6,000 vertices gain about 40 neighbours each: far more runs than the pool's spare blocks
        hubs = np.repeat(np.arange(6000, dtype=np.uint32), 40)
        leaves = rng.integers(0, n, len(hubs), dtype=np.uint32)
        byo.byo_insert_batch(g.handle, dev(hubs), dev(leaves))
        dg.insert(hubs, leaves)
        same_contents(byo, g, dg.csr())
        assert byo.byo_space(g.handle) > space0
        # vertex 29999: 3,000 copies of 10 pairs
        dup_d = np.tile(np.arange(100, 110, dtype=np.uint32), 300)
        dup_s = np.full(len(dup_d), 29999, np.uint32)
        byo.byo_insert_batch(g.handle, dev(dup_s), dev(dup_d))
        dg.insert(dup_s, dup_d)
        same_contents(byo, g, dg.csr())
        gone = rng.random(len(hubs)) < 0.8
        byo.byo_delete_batch(g.handle, dev(leaves[gone]), dev(hubs[gone]))
        dg.delete(leaves[gone], hubs[gone])
        byo.byo_delete_batch(g.handle, dev(dup_s), dev(dup_d))
        dg.delete(dup_s, dup_d)
        ref = dg.csr()
        same_contents(byo, g, ref)
        algorithms_match(byo, g, ref, [0, 7000])
