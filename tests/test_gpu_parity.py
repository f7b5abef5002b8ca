"""Parity of the CUDA path (through the C ABI) with the oracle, element by element.

Integer results are bit-exact (CSR contents, degrees, BFS levels, CC labels,
triangle counts); BFS parents are checked for validity (a BFS tree is not
unique); PageRank meets the stated FP64 tolerance: max relative error per
vertex <= 1e-5 and L1 error <= 1e-6.  Inputs come from ``graphgen`` only.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

INF = 0xFFFFFFFF
PR_MAX_REL = 1e-5
PR_L1 = 1e-6


@pytest.fixture(scope="module")
def byo():
    from paper_2405_11671_gb300 import build
    build.build()
    import paper_2405_11671_gb300 as b
    b.load()
    return b


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host_u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def _star(k):
    return k + 1, np.zeros(k, np.uint32), np.arange(1, k + 1, dtype=np.uint32)


def _path(n):
    return n, np.arange(n - 1, dtype=np.uint32), np.arange(1, n, dtype=np.uint32)


def _complete(n):
    i, j = np.triu_indices(n, 1)
    return n, i.astype(np.uint32), j.astype(np.uint32)


def _union():
    parts = [_path(300), _complete(40), _star(700), (50, np.zeros(0, np.uint32), np.zeros(0, np.uint32))]
    src, dst, base = [], [], 0
    for n, s, d in parts:
        src.append(s + base)
        dst.append(d + base)
        base += n
    return base, np.concatenate(src), np.concatenate(dst)


CASES = {
    "tiny_er": lambda: graphgen.workload("tiny"),
    "rmat14": lambda: graphgen.rmat_small(14, 16, 101),
    "grid_dropped": lambda: graphgen.grid_small(96, 80, 0.10, 1e-3, 7),
    "grid_full": lambda: graphgen.grid_small(40, 70, 0.0, 0.0, 1),
    "star": lambda: _star(20000),
    "path": lambda: _path(3000),
    "complete": lambda: _complete(160),
    "union": _union,
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, byo):
    n, src, dst = CASES[request.param]()
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev_u32(src), dev_u32(dst))
    yield request.param, n, src, dst, ref, g
    g.close()


def _sources(n, src, dst, ref):
    s = [0]
    s += graphgen.pick_sources(n, src, dst, 2, 555).tolist()
    deg = np.diff(ref.off)
    iso = np.flatnonzero(deg == 0)
    if len(iso):
        s.append(int(iso[0]))
    return s


# ----------------------------------------------------------------------------- container

def test_csr_contents(byo, case):
    _, n, _, _, ref, g = case
    assert g.n == n and g.m == ref.m
    off, col = byo.byo_graph_export_csr(g.handle)
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
    assert np.array_equal(host_u32(col), ref.col)


def test_degree(byo, case):
    _, n, _, _, ref, g = case
    deg = host_u32(byo.byo_degree(g.handle))
    assert np.array_equal(deg.astype(np.uint64), np.diff(ref.off))
    vs = np.array([0, n - 1, n // 2], np.uint32)
    d2 = host_u32(byo.byo_degree(g.handle, dev_u32(vs)))
    assert np.array_equal(d2.astype(np.uint64), np.diff(ref.off)[vs])


def test_offsets64_and_presymmetrised_input(byo):
    n, src, dst = graphgen.rmat_small(13, 8, 9)
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev_u32(src), dev_u32(dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE | byo.BYO_OFFSETS64)
    off, col = byo.byo_graph_export_csr(g.handle)
    assert np.array_equal(off.cpu().numpy().astype(np.uint64), ref.off)
    assert np.array_equal(host_u32(col), ref.col)
    lv, _ = byo.byo_bfs(g.handle, [1])
    assert np.array_equal(host_u32(lv[0]), oracle.bfs(ref, 1)[0])
    g.close()
    # an already symmetric list without BYO_SYMMETRIZE builds the same graph
    rows = np.repeat(np.arange(n, dtype=np.uint32), np.diff(ref.off).astype(np.int64))
    g2 = byo.Graph(n, dev_u32(rows), dev_u32(ref.col), byo.BYO_CSR)
    off2, col2 = byo.byo_graph_export_csr(g2.handle)
    assert np.array_equal(host_u32(col2), ref.col)
    g2.close()


def test_build_errors(byo):
    with pytest.raises(byo.ByoError) as e:
        byo.Graph(4, dev_u32([0, 1]), dev_u32([1, 4]))
    assert e.value.status == byo.BYO_ERR_INVALID_ARG
    with pytest.raises(byo.ByoError) as e:
        byo.Graph(4, dev_u32([0, 1]), dev_u32([1, 2]), byo.BYO_CSR)
    assert e.value.status == byo.BYO_ERR_NOT_SYMMETRIC
    with pytest.raises(byo.ByoError) as e:
        byo.Graph(4, dev_u32([0]), dev_u32([1]), byo.BYO_SYMMETRIZE)
    assert e.value.status == byo.BYO_ERR_INVALID_ARG


def test_empty_graph(byo):
    g = byo.Graph(100, dev_u32(np.zeros(0)), dev_u32(np.zeros(0)))
    assert g.m == 0
    lv, par = byo.byo_bfs(g.handle, [7])
    lv = host_u32(lv[0])
    assert lv[7] == 0 and np.all(np.delete(lv, 7) == INF)
    assert np.array_equal(host_u32(byo.byo_cc(g.handle)), np.arange(100, dtype=np.uint32))
    assert byo.byo_tc(g.handle) == 0
    p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
    assert np.allclose(p.cpu().numpy(), 0.01, rtol=1e-6)
    g.close()


# ----------------------------------------------------------------------------- BFS

# (mode, thr_thread, thr_warp, action, flags); flags 1 = no early exit, 2 = sequential maps (API ablations)
SCHEDS = {"heuristic": (0, 16, 1024, 1, 0), "push": (2, 16, 1024, 1, 0), "pull": (3, 16, 1024, 1, 0),
          "push_thread_only": (2, 1 << 31, 1 << 31, 1, 0), "push_cta_heavy": (2, 1, 2, 1, 0),
          "solo": (4, 16, 1024, 4, 0), "solo_cta_heavy": (4, 1, 2, 4, 0), "push_small_bins": (4, 16, 1024, 2, 0),
          "learned_random": (1, 16, 1024, 1, 0),
          "pull_no_early_exit": (3, 16, 1024, 1, 1), "heuristic_no_early_exit": (0, 16, 1024, 1, 1),
          "push_sequential": (2, 16, 1024, 1, 2), "pull_sequential": (3, 16, 1024, 1, 2),
          "heuristic_both_ablations": (0, 16, 1024, 1, 3), "learned_random_sequential": (1, 16, 1024, 1, 2)}


@pytest.fixture(scope="module")
def random_net(byo):
    m = byo.byo_mlp_create(12345)  # untrained: mixes all five actions
    yield m
    byo.byo_mlp_destroy(m)


@pytest.mark.parametrize("sched", sorted(SCHEDS))
def test_bfs_levels_and_parents(byo, case, sched, random_net):
    name, n, src, dst, ref, g = case
    mode, tt, tw, act, flags = SCHEDS[sched]
    sp = byo.make_sched(mode, tt, tw, mlp=random_net if mode == byo.BYO_SCHED_LEARNED else None, action=act,
                        flags=flags)
    srcs = _sources(n, src, dst, ref)
    lv, par = byo.byo_bfs(g.handle, srcs, sched=sp)
    for i, s in enumerate(srcs):
        want, _ = oracle.bfs(ref, s)
        got = host_u32(lv[i])
        assert np.array_equal(got, want), (name, sched, s, np.flatnonzero(got != want)[:10])
        assert oracle.bfs_check_parents(ref, s, got, host_u32(par[i])) == -1


def test_bfs_trace_and_invalid_source(byo):
    n, src, dst = graphgen.rmat_small(12, 16, 3)
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev_u32(src), dev_u32(dst))
    s = int(graphgen.pick_sources(n, src, dst, 1, 1)[0])
    lv, _ = byo.byo_bfs(g.handle, [s], want_parents=False)
    want, _ = oracle.bfs(ref, s)
    assert np.array_equal(host_u32(lv[0]), want)
    tr = byo.byo_bfs_trace(g.handle)
    depth = int(want[want != INF].max())
    assert len(tr) == depth + 1
    deg = np.diff(ref.off).astype(np.int64)
    for r in tr:
        f = np.flatnonzero(want == r.level)
        assert r.frontier == len(f) and r.frontier_edges == int(deg[f].sum())
        assert r.unvisited == int(np.count_nonzero(want > r.level))
    with pytest.raises(byo.ByoError) as e:
        byo.byo_bfs(g.handle, [n])
    assert e.value.status == byo.BYO_ERR_INVALID_ARG
    g.close()


# ----------------------------------------------------------------------------- CC, PR, TC

def test_cc_labels(byo, case):
    _, _, _, _, ref, g = case
    assert np.array_equal(host_u32(byo.byo_cc(g.handle)), oracle.cc(ref))


def test_pagerank_tolerance(byo, case):
    _, n, _, _, ref, g = case
    p, res = byo.byo_pagerank(g.handle, 0.85, 20)
    want, wres = oracle.pagerank(ref, 0.85, 20)
    got = p.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want) / want) <= PR_MAX_REL
    assert np.sum(np.abs(got - want)) <= PR_L1
    assert abs(res - wres[-1]) <= 1e-6 + 1e-3 * wres[-1]


def test_pagerank_graph_replay_on_side_stream(byo):
    # on a non-default stream the iterations are captured once as a CUDA graph
    # and replayed; replays must give the same ranks, and a new iteration count
    # or a structural change must re-capture
    n, src, dst = graphgen.rmat_small(13, 16, 606)
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev_u32(src), dev_u32(dst), byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        p1, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        p1 = p1.clone()
        p2, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        p7, _ = byo.byo_pagerank(g.handle, 0.85, 7)
        p7 = p7.clone()
    torch.cuda.synchronize()
    assert torch.equal(p1, p2)
    for got, it in ((p1, 20), (p7, 7)):
        want, _ = oracle.pagerank(ref, 0.85, it)
        gotd = got.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(gotd - want) / want) <= PR_MAX_REL and np.sum(np.abs(gotd - want)) <= PR_L1
    ins_s, ins_d = graphgen.rmat(13, 3000, 607)
    byo.byo_insert_batch(g.handle, dev_u32(ins_s), dev_u32(ins_d))
    dg = oracle.DynGraph(n, src, dst)
    dg.insert(ins_s, ins_d)
    with torch.cuda.stream(side):
        p3, _ = byo.byo_pagerank(g.handle, 0.85, 20)
    torch.cuda.synchronize()
    want, _ = oracle.pagerank(dg.csr(), 0.85, 20)
    gotd = p3.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gotd - want) / want) <= PR_MAX_REL and np.sum(np.abs(gotd - want)) <= PR_L1
    g.close()


def test_triangle_count(byo, case):
    _, _, _, _, ref, g = case
    assert byo.byo_tc(g.handle) == oracle.tc(ref)


@pytest.mark.parametrize("light_max,window,bitmap_bits", [(4, 16, 4), (2, 4, 4), (64, 1024, 4), (4, 16, 1 << 30),
                                                          (2, 4, 3000), (64, 1024, 1 << 30)])
def test_triangle_count_cta_path_and_windows(byo, monkeypatch, light_max, window, bitmap_bits):
    # lower the light/heavy split, the window and the bitmap range so that the
    # CTA path, hashed multi-window intersections and the bitmap run on small
    # graphs (4 bits: every CTA centre hashed; 3000: both kinds)
    monkeypatch.setenv("BYO_TC_LIGHT_MAX", str(light_max))
    monkeypatch.setenv("BYO_TC_WINDOW", str(window))
    monkeypatch.setenv("BYO_TC_BITMAP_BITS", str(bitmap_bits))
    for n, src, dst in (graphgen.rmat_small(13, 16, 44), _complete(90), graphgen.workload("tiny")):
        ref = oracle.csr_build(n, src, dst)
        g = byo.Graph(n, dev_u32(src), dev_u32(dst))
        assert byo.byo_tc(g.handle) == oracle.tc(ref)
        g.close()


@pytest.mark.parametrize("light_max,warp_sort_max,sort_max", [(256, 1024, 16384), (4, 32, 16384), (4, 32, 48),
                                                              (64, 64, 40), (4, 4, 4)])
def test_triangle_count_sorted_out_lists(byo, monkeypatch, light_max, warp_sort_max, sort_max):
    # out-lists of 32..sort_max ids are sorted by rank, by one warp up to
    # max(warp_sort_max, light_max) ids and by one CTA above, and the walk of
    # an in-neighbour's sorted out-list starts after the centre; longer lists
    # are walked whole.  K_1100 has out-lists of up to 1,099 ids (the CTA sort
    # at the default limits) and C(1100, 3) triangles.
    monkeypatch.setenv("BYO_TC_LIGHT_MAX", str(light_max))
    monkeypatch.setenv("BYO_TC_WARP_SORT_MAX", str(warp_sort_max))
    monkeypatch.setenv("BYO_TC_SORT_MAX", str(sort_max))
    for n, src, dst in (graphgen.rmat_small(13, 16, 44), _complete(90), _complete(1100)):
        want = n * (n - 1) * (n - 2) // 6 if len(src) == n * (n - 1) // 2 else oracle.tc(oracle.csr_build(n, src, dst))
        g = byo.Graph(n, dev_u32(src), dev_u32(dst))
        assert byo.byo_tc(g.handle) == want
        g.close()


def test_triangle_work_statistics(byo):
    # the byte model of the benchmark's roofline rests on these three sums;
    # recompute them from the oracle's CSR with the (degree, id) orientation
    n, src, dst = graphgen.rmat_small(12, 16, 46)
    ref = oracle.csr_build(n, src, dst)
    off = np.asarray(ref.off, dtype=np.int64)
    col = np.asarray(ref.col, dtype=np.int64)
    deg = np.diff(off)
    row = np.repeat(np.arange(n), deg)
    up = (deg[col] > deg[row]) | ((deg[col] == deg[row]) & (col > row))  # row -> col in the DAG
    a, b = row[up], col[up]
    dp = np.bincount(a, minlength=n)
    dm = np.bincount(b, minlength=n)
    da, db = dp[a], dp[b]
    # at centre b (d+(a) < d+(b)) a sorted out-list of a (32..16384 ids) is
    # walked from the first id above b: the ids of N+(a) ranked above b
    rank = np.empty(n, np.int64)
    rank[np.lexsort((np.arange(n), deg))] = np.arange(n)
    o = np.lexsort((rank[b], a))
    pos = np.empty(len(a), np.int64)
    pos[o] = np.arange(len(a)) - np.searchsorted(a[o], a[o], "left")
    trimmed = np.where((da >= 32) & (da <= 16384), da - 1 - pos, da)
    walked = np.where(da < 2, 0, np.where(db <= da, db, trimmed))
    assert (trimmed < da).any()  # the graph has sorted out-lists that are trimmed
    g = byo.Graph(n, dev_u32(src), dev_u32(dst))
    try:
        assert byo.byo_tc_work(g.handle) == (int((dp * dp).sum()), int((dm * dp).sum()), int(walked.sum()))
    finally:
        g.close()


# ----------------------------------------------------------------------------- schedule network

def _mlp_batch(B=333, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, (B, 12)).astype(np.float32)
    y = rng.integers(0, 5, B).astype(np.int32)
    w = rng.uniform(0.2, 2.0, B).astype(np.float32)
    return X, y, w


def _split(v):
    sizes = [32 * 12, 32, 32 * 32, 32, 5 * 32, 5]
    out, o = [], 0
    for s in sizes:
        out.append(v[o:o + s])
        o += s
    return out


def test_mlp_gradient_matches_oracle(byo):
    m = byo.byo_mlp_create(7)
    P = byo.byo_mlp_get_params(m)
    X, y, w = _mlp_batch()
    loss, grad = byo.byo_mlp_loss_grad(m, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(),
                                       torch.from_numpy(w).cuda())
    L, g64, _ = oracle.mlp_loss(P.astype(np.float64), 12, 32, 32, byo.BYO_NUM_ACTIONS, X.astype(np.float64), y, w.astype(np.float64))
    assert abs(loss - L) <= 1e-4 * max(1.0, abs(L))
    g32 = grad.cpu().numpy().astype(np.float64)
    for a, b in zip(_split(g32), _split(g64)):
        assert np.linalg.norm(a - b) <= 1e-3 * max(np.linalg.norm(b), 1e-6)
    byo.byo_mlp_destroy(m)


def test_mlp_train_and_predict(byo):
    m = byo.byo_mlp_create(3)
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (2000, 12)).astype(np.float32)
    y = (X[:, 0] > X[:, 1]).astype(np.int32) * 2 + (X[:, 2] > 0.5).astype(np.int32)  # 4 separable classes
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0, _ = byo.byo_mlp_loss_grad(m, Xd, yd)
    l1 = byo.byo_mlp_train(m, Xd, yd, None, epochs=400, lr=1e-2)
    assert l1 < 0.5 * l0
    pred = byo.byo_mlp_predict(m, Xd).cpu().numpy()
    P = byo.byo_mlp_get_params(m).astype(np.float64)
    _, _, logits = oracle.mlp_loss(P, 12, 32, 32, byo.BYO_NUM_ACTIONS, X.astype(np.float64), y, None, want_grad=False)
    srt = np.sort(logits, axis=1)
    clear = (srt[:, -1] - srt[:, -2]) > 1e-3                      # skip near-ties (FP32 vs FP64)
    assert np.array_equal(pred[clear], np.argmax(logits, axis=1)[clear])
    assert np.mean(pred == y) > 0.9
    byo.byo_mlp_destroy(m)


# ----------------------------------------------------------------------------- betweenness

def _bc_check(byo, ref, g, s):
    lv, sigma, delta = byo.byo_bc(g.handle, s)
    wl, ws, wd = oracle.bc(ref, s)
    assert np.array_equal(host_u32(lv), wl)
    gs, gd = sigma.cpu().numpy(), delta.cpu().numpy()
    exact = ws < 2.0 ** 53            # path counts are integers, exact in FP64 below 2^53
    assert np.array_equal(gs[exact], ws[exact])
    assert np.all(np.abs(gs[~exact] - ws[~exact]) <= 1e-12 * ws[~exact])
    assert np.all(np.abs(gd - wd) <= 1e-12 * np.maximum(np.abs(wd), 1.0))


def test_bc_sigma_and_delta(byo, case):
    name, n, src, dst, ref, g = case
    if n == 0:
        return
    deg = np.diff(ref.off.astype(np.int64))
    for s in [int(np.argmax(deg)), int(graphgen.pick_sources(n, src, dst, 1, 9)[0]) if ref.m else 0]:
        _bc_check(byo, ref, g, s)


def test_bc_dynamic_container_and_invalid_source(byo):
    n, src, dst = graphgen.rmat_small(12, 16, 33)
    ref = oracle.csr_build(n, src, dst)
    with byo.Graph(n, dev_u32(src), dev_u32(dst), byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE) as g:
        _bc_check(byo, ref, g, int(graphgen.pick_sources(n, src, dst, 1, 5)[0]))
        with pytest.raises(byo.ByoError) as e:
            byo.byo_bc(g.handle, n)
        assert e.value.status == byo.BYO_ERR_INVALID_ARG


def test_pagerank_hub_split_over_chunks(byo):
    # a hub of 150,000 neighbours is summed in several chunks (their partials
    # folded by the last one) -- within the tolerance like every other vertex
    k = 150000
    n = k + 1
    rng = np.random.default_rng(5)
    extra = rng.integers(1, n, size=(40000, 2), dtype=np.int64)
    src = np.concatenate([np.zeros(k, np.uint32), extra[:, 0].astype(np.uint32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.uint32), extra[:, 1].astype(np.uint32)])
    ref = oracle.csr_build(n, src, dst)
    with byo.Graph(n, dev_u32(src), dev_u32(dst)) as g:
        p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        w, _ = oracle.pagerank(ref, 0.85, 20)
        got = p.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - w) / w) <= PR_MAX_REL and np.sum(np.abs(got - w)) <= PR_L1
