"""The compressed container (BYO_COMPRESSED: difference encoding and byte
codes, the paper's compressed graphs) against the oracle.

The codes the GPU writes are byte-for-byte the oracle's (`ora_bytecode_encode`),
the lists it decodes back are the oracle's CSR, and BFS over the codes gives
the oracle's levels with valid parents -- on graphs whose values need one to
five bytes (a sparse graph on 2^28 vertices), a hub whose list the whole warp
decodes, paths and grids (many levels), and isolated vertices.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host(t):
    return t.cpu().numpy().view(np.uint32)


def _star(k):
    return k + 1, np.zeros(k, np.uint32), np.arange(1, k + 1, dtype=np.uint32)


def _wide():
    # few edges among 2^28 vertices: first differences and gaps of 1 to 5 bytes
    n = 1 << 28
    rng = np.random.default_rng(9)
    a = rng.integers(0, n, size=3000, dtype=np.int64)
    b = rng.integers(0, n, size=3000, dtype=np.int64)
    extra = np.array([[0, 1], [0, 127], [0, 128], [0, 16383], [0, 16384], [5, n - 1], [n - 2, n - 1]], np.int64)
    return n, np.concatenate([a, extra[:, 0]]).astype(np.uint32), np.concatenate([b, extra[:, 1]]).astype(np.uint32)


CASES = {
    "tiny_er": lambda: graphgen.workload("tiny"),
    "rmat16": lambda: graphgen.rmat_small(16, 16, 61),
    "grid": lambda: graphgen.grid_small(120, 90, 0.1, 1e-3, 3),
    "star": lambda: _star(30000),
    "path": lambda: (2500, np.arange(2499, dtype=np.uint32), np.arange(1, 2500, dtype=np.uint32)),
    "wide": _wide,
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_codes_decode_and_bfs(byo, name):
    n, src, dst = CASES[name]()
    ref = oracle.csr_build(n, src, dst)
    want_boff, want_bytes = oracle.bytecode_encode(ref)
    with byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE | byo.BYO_COMPRESSED) as g:
        assert g.m == ref.m
        boff, data = byo.byo_export_codes(g.handle)
        assert np.array_equal(boff.cpu().numpy().astype(np.uint64), want_boff)
        assert np.array_equal(data.cpu().numpy(), want_bytes)
        # lists longer than 4,096 values carry a checkpoint (16 bytes) every 4,096 values
        # and an entry (12 bytes) in the list of checkpointed vertices
        d = np.diff(ref.off.astype(np.int64))
        ck = int(np.sum(np.maximum(d - 1, 0) // 4096))
        ckv = int(np.count_nonzero(d > 4096))
        assert byo.byo_space(g.handle) == (n + 1) * (4 + 8) + len(want_bytes) + 16 * ck + 12 * ckv
        off, col = byo.byo_graph_export_csr(g.handle)
        assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
        assert np.array_equal(host(col), ref.col)
        assert np.array_equal(host(byo.byo_degree(g.handle)).astype(np.uint64), np.diff(ref.off))
        deg = np.diff(ref.off.astype(np.int64))
        srcs = [int(np.argmax(deg)), int(graphgen.pick_sources(n, src, dst, 1, 3)[0])]
        for sched in (None, byo.make_sched(byo.BYO_SCHED_PUSH), byo.make_sched(byo.BYO_SCHED_PULL)):
            lv, par = byo.byo_bfs(g.handle, srcs, sched=sched)
            for i, s in enumerate(srcs):
                lvl, _ = oracle.bfs(ref, s)
                assert np.array_equal(host(lv[i]), lvl), (name, s)
                assert oracle.bfs_check_parents(ref, s, host(lv[i]), host(par[i])) == -1


def test_compressed_rejects_other_algorithms(byo):
    n, src, dst = graphgen.rmat_small(10, 8, 1)
    with byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE | byo.BYO_COMPRESSED) as g:
        for fn in (lambda: byo.byo_cc(g.handle), lambda: byo.byo_pagerank(g.handle, 0.85, 20),
                   lambda: byo.byo_tc(g.handle)):
            with pytest.raises(byo.ByoError) as e:
                fn()
            assert e.value.status == byo.BYO_ERR_UNSUPPORTED
    with pytest.raises(byo.ByoError):
        byo.Graph(n, dev(src), dev(dst), byo.BYO_DYNAMIC | byo.BYO_COMPRESSED)
