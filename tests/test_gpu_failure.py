"""Failure detection without a GPU fault.

Time limits.  Every device-side wait and every whole traversal is bounded by
BYO_TIMEOUT_MS.  A limit that a long traversal (a 1024 x 1024 grid, over two
thousand levels) cannot meet makes the kernel give up, record BYO_ERR_TIMEOUT
in its status word and return; the call reports that status, and the next call
with the default limit runs normally and is bit-exact against the oracle.

Allocation failures.  BYO_FAULT_INJECT=alloc:K makes the K-th device
allocation of a call report OUT_OF_MEMORY (on the host: no kernel is
involved).  For every K up to the number of allocations the call makes, the
call returns OUT_OF_MEMORY, releases what it had allocated (device memory does
not shrink over repeated failures), and later calls work; a batch update that
fails either leaves the container as it was or applies the whole batch.
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


@pytest.fixture(scope="module")
def long_grid():
    n, src, dst = graphgen.grid_small(1024, 1024, 0.0, 0.0, 5)
    return n, src, dst, oracle.csr_build(n, src, dst)


def test_bfs_timeout_then_clean_call(byo, long_grid, monkeypatch):
    n, src, dst, ref = long_grid
    want0, _ = oracle.bfs(ref, 0)
    want1, _ = oracle.bfs(ref, n - 1)
    with byo.Graph(n, dev(src), dev(dst)) as g:
        monkeypatch.setenv("BYO_TIMEOUT_MS", "1")
        for sp in (None, byo.make_sched(byo.BYO_SCHED_PUSH)):
            with pytest.raises(byo.ByoError) as e:
                byo.byo_bfs(g.handle, [0, n - 1], sched=sp)
            assert e.value.status == byo.BYO_ERR_TIMEOUT
        monkeypatch.delenv("BYO_TIMEOUT_MS")
        lv, par = byo.byo_bfs(g.handle, [0, n - 1])
        assert np.array_equal(host(lv[0]), want0)
        assert np.array_equal(host(lv[1]), want1)
        assert oracle.bfs_check_parents(ref, 0, host(lv[0]), host(par[0])) == -1


def test_noalloc_timeout_then_clean_call(byo, long_grid, monkeypatch):
    n, src, dst, ref = long_grid
    want, _ = oracle.bfs(ref, 0)
    with byo.Graph(n, dev(src), dev(dst)) as g:
        m = g.m
        off, col = byo.byo_graph_export_csr(g.handle)
    col_pad = torch.zeros(m + 4, dtype=torch.int32, device="cuda")
    col_pad[:m] = col
    levels = torch.empty(n, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("BYO_TIMEOUT_MS", "1")
    with pytest.raises(byo.ByoError) as e:
        byo.byo_bfs_noalloc(n, m, off, col_pad, 0, levels)
    assert e.value.status == byo.BYO_ERR_TIMEOUT
    monkeypatch.delenv("BYO_TIMEOUT_MS")
    byo.byo_bfs_noalloc(n, m, off, col_pad, 0, levels)
    assert np.array_equal(host(levels), want)


def test_msbfs_timeout_then_clean_call(byo, long_grid, monkeypatch):
    n, src, dst, ref = long_grid
    srcs = [0, n - 1, 512 * 1024 + 3]
    with byo.Graph(n, dev(src), dev(dst)) as g:
        monkeypatch.setenv("BYO_TIMEOUT_MS", "1")
        with pytest.raises(byo.ByoError) as e:
            byo.byo_msbfs(g.handle, srcs, len(srcs))
        assert e.value.status == byo.BYO_ERR_TIMEOUT
        monkeypatch.delenv("BYO_TIMEOUT_MS")
        lv = byo.byo_msbfs(g.handle, srcs, len(srcs))
        for j, s in enumerate(srcs):
            want, _ = oracle.bfs(ref, s)
            assert np.array_equal(host(lv[j]), want)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _fail_every_allocation(byo, monkeypatch, call, max_k=2000):
    """Run call() with its K-th allocation failing, K = 1, 2, ... until it
    succeeds; every failing run must report OUT_OF_MEMORY.  Returns how many
    allocations the call makes."""
    for k in range(1, max_k + 1):
        monkeypatch.setenv("BYO_FAULT_INJECT", f"alloc:{k}")
        try:
            call()
        except byo.ByoError as e:
            assert e.status == byo.BYO_ERR_OUT_OF_MEMORY, (k, str(e))
            assert "injected" in str(e)
            continue
        finally:
            monkeypatch.delenv("BYO_FAULT_INJECT")
        return k - 1
    raise AssertionError("the call never succeeded")


def test_build_allocation_failures_release_memory(byo, monkeypatch):
    n, src, dst = graphgen.rmat_small(16, 16, 4242)
    ref = oracle.csr_build(n, src, dst)
    s_d, d_d = dev(src), dev(dst)
    for flags in (byo.BYO_CSR | byo.BYO_SYMMETRIZE, byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE):
        byo.Graph(n, s_d, d_d, flags).close()  # warm the scratch pool
        before = _free_bytes()
        for _ in range(2):
            made = []
            allocs = _fail_every_allocation(byo, monkeypatch, lambda: made.append(byo.Graph(n, s_d, d_d, flags)))
            assert allocs >= 3
            for g in made:
                g.close()
        # the failed builds leaked nothing (each failed build held up to ~17 MB of CSR)
        assert before - _free_bytes() < (8 << 20)
        with byo.Graph(n, s_d, d_d, flags) as g:
            off, col = byo.byo_graph_export_csr(g.handle)
            assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
            assert np.array_equal(host(col), ref.col)


def test_algorithm_allocation_failures_then_exact(byo, monkeypatch):
    n, src, dst = graphgen.rmat_small(14, 16, 99)
    ref = oracle.csr_build(n, src, dst)
    for k in range(1, 12):
        # a fresh graph each time, so that every first-use allocation happens
        with byo.Graph(n, dev(src), dev(dst)) as g:
            monkeypatch.setenv("BYO_FAULT_INJECT", f"alloc:{k}")
            outcomes = []
            for fn in (lambda: byo.byo_bfs(g.handle, [1]), lambda: byo.byo_cc(g.handle),
                       lambda: byo.byo_pagerank(g.handle, 0.85, 20), lambda: byo.byo_tc(g.handle)):
                try:
                    fn()
                    outcomes.append("ok")
                except byo.ByoError as e:
                    assert e.status == byo.BYO_ERR_OUT_OF_MEMORY, str(e)
                    outcomes.append("oom")
            monkeypatch.delenv("BYO_FAULT_INJECT")
            lv, _ = byo.byo_bfs(g.handle, [1])
            assert np.array_equal(host(lv[0]), oracle.bfs(ref, 1)[0])
            assert np.array_equal(host(byo.byo_cc(g.handle)), oracle.cc(ref))
            p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
            w, _ = oracle.pagerank(ref, 0.85, 20)
            assert np.max(np.abs(p.cpu().numpy() - w) / w) <= 1e-5
            assert byo.byo_tc(g.handle) == oracle.tc(ref)


def test_batch_update_allocation_failures(byo, monkeypatch):
    n, src, dst = graphgen.rmat_small(13, 8, 5)
    ins_s, ins_d = graphgen.rmat(13, 3000, 6)
    base = oracle.DynGraph(n, src, dst)
    after = oracle.DynGraph(n, src, dst)
    after.insert(ins_s, ins_d)
    b0, b1 = base.csr(), after.csr()
    k = 1
    while True:
        with byo.Graph(n, dev(src), dev(dst), byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE) as g:
            monkeypatch.setenv("BYO_FAULT_INJECT", f"alloc:{k}")
            try:
                byo.byo_insert_batch(g.handle, dev(ins_s), dev(ins_d))
                failed = False
            except byo.ByoError as e:
                assert e.status == byo.BYO_ERR_OUT_OF_MEMORY, str(e)
                failed = True
            monkeypatch.delenv("BYO_FAULT_INJECT")
            off, col = byo.byo_graph_export_csr(g.handle)
            got_off, got_col = off.cpu().numpy().astype(np.uint64), host(col)
            whole = np.array_equal(got_off, b1.off) and np.array_equal(got_col, b1.col)
            none = np.array_equal(got_off, b0.off) and np.array_equal(got_col, b0.col)
            assert whole or (failed and none), k
            ref = b1 if whole else b0
            lv, _ = byo.byo_bfs(g.handle, [0])
            assert np.array_equal(host(lv[0]), oracle.bfs(ref, 0)[0]), k
            if not failed:
                break
        k += 1
        assert k < 2000
