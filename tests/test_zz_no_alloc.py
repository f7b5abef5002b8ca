"""byo_bfs_noalloc: BFS for callers that cannot allocate device memory.

Such callers (device memory owned by another allocator, a hard memory budget,
or a loop where cudaMalloc's device synchronisation is not acceptable) pass
their own CSR and outputs; the library's built-in scratch array replaces every
allocation.  This file is collected last on purpose.  It must pass on its own
in a fresh process and after the rest of the suite: two calls in a row are
checked against byo_bfs (levels bit-exact, parents a valid BFS tree).
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("mode", ["heuristic", "pull"])
def test_noalloc_matches_byo_bfs_twice(byo, mode):
    n, src, dst = graphgen.rmat_small(15, 16, 2024)
    ref = oracle.csr_build(n, src, dst)
    sp = byo.make_sched(byo.BYO_SCHED_HEURISTIC if mode == "heuristic" else byo.BYO_SCHED_PULL)
    srcs = [int(s) for s in graphgen.pick_sources(n, src, dst, 2, 77)]
    with byo.Graph(n, _dev(src), _dev(dst)) as g:
        m = g.m
        off, col = byo.byo_graph_export_csr(g.handle)
        want, want_par = byo.byo_bfs(g.handle, srcs, sched=sp)
    # caller-owned CSR: 16-byte aligned ids with four readable entries of padding
    col_pad = torch.zeros(m + 4, dtype=torch.int32, device="cuda")
    col_pad[:m] = col
    levels = torch.empty(n, dtype=torch.int32, device="cuda")
    parents = torch.empty(n, dtype=torch.int32, device="cuda")
    for i, s in enumerate(srcs):  # two calls in a row share the built-in array
        byo.byo_bfs_noalloc(n, m, off, col_pad, s, levels, parents, sp)
        torch.cuda.synchronize()
        got = _host(levels)
        assert np.array_equal(got, _host(want[i]))
        assert oracle.bfs_check_parents(ref, s, got, _host(parents)) == -1
        assert oracle.bfs_check_parents(ref, s, _host(want[i]), _host(want_par[i])) == -1


def test_noalloc_rejects_oversize_graph(byo):
    # straight through the C ABI: the library itself refuses n above the
    # size of its built-in array, before touching any pointer
    n = byo.BYO_NOALLOC_MAX_VERTICES + 1
    off = torch.zeros(2, dtype=torch.int64, device="cuda")
    col = torch.zeros(4, dtype=torch.int32, device="cuda")
    lv = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = byo.load().byo_bfs_noalloc(n, 0, off.data_ptr(), col.data_ptr(), 0, lv.data_ptr(), None, None,
                                    torch.cuda.current_stream().cuda_stream)
    assert st == byo.BYO_ERR_INVALID_ARG


def test_noalloc_wrapper_rejects_short_buffers(byo):
    n, m = 8, 12
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(m + 4, dtype=torch.int32, device="cuda")
    lv = torch.zeros(n, dtype=torch.int32, device="cuda")
    for bad in (dict(offsets=off[:n]), dict(col=col[:m]), dict(levels=lv[:n - 1]), dict(col=col[1:])):
        kw = dict(offsets=off, col=col, levels=lv)
        kw.update(bad)
        with pytest.raises(ValueError):
            byo.byo_bfs_noalloc(n, m, kw["offsets"], kw["col"], 0, kw["levels"])
