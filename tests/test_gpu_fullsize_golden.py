"""Every configuration at its stated size, against reference values of the oracle.

The oracle cannot run these sizes inside a GPU test (its serial CSR build and
PageRank take minutes to an hour on one host core), so
``tests/golden/make_fullsize_golden.py`` computed them once, from the oracle
only, on the same seeded draws (``graphgen``); this file recomputes everything
on the GPU through the C ABI and compares:

* RMAT-25 (the benchmark workload) and RMAT-26 (uint64 offsets, 2.1 G stored
  edges): CSR contents (SHA-256), BFS levels from the eight benchmark sources
  (SHA-256, bit-exact) with every parent checked (one level up, joined by an
  edge of the CSR), CC labels (SHA-256), PageRank per vertex at the sampled
  vertices (relative error <= 1e-5) and its total mass, and the triangle count
  (exact);
* RMAT-22 and the grid: the triangle count (their BFS, CC and PageRank are
  compared element by element in test_gpu_fullsize.py);
* the dynamic container, sorted and hash-indexed (RMAT-24 base, ten rounds of
  1 M inserts and 1 M deletes): after every round the container's contents,
  BFS levels, CC labels and sampled PageRank;
* the 256-graph batch: every member's 64-source level block and CC labels.
"""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import graphgen

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PR_MAX_REL = 1e-5


@pytest.fixture(scope="module")
def byo():
    from paper_2405_11671_gb300 import build
    build.build()
    import paper_2405_11671_gb300 as b
    b.load()
    return b


def gold(name):
    with open(os.path.join(GOLDEN, f"fullsize_{name}.json")) as f:
        return json.load(f)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def sha_u32(t) -> str:
    return hashlib.sha256(t.contiguous().cpu().numpy().view("<u4").tobytes()).hexdigest()


def sha_csr(off, col) -> str:
    h = hashlib.sha256(off.contiguous().cpu().numpy().view("<u8").tobytes())
    h.update(col.contiguous().cpu().numpy().view("<u4").tobytes())
    return h.hexdigest()


def check_parents(off, col, lv, par, s):
    """Every reached vertex but s has a parent one level up that is one of its
    neighbours in the CSR (a BFS tree is not unique; levels are checked by hash)."""
    n = lv.numel()
    L = lv.long() & 0xFFFFFFFF
    P = par.long() & 0xFFFFFFFF
    assert int(L[s]) == 0 and int(P[s]) == s
    v = torch.nonzero((L != 0xFFFFFFFF) & (torch.arange(n, device=lv.device) != s)).squeeze(1)
    pv = P[v]
    assert int((L[pv] + 1 - L[v]).abs().max()) == 0
    assert torch.equal(P[L == 0xFFFFFFFF], torch.full_like(P[L == 0xFFFFFFFF], 0xFFFFFFFF))
    # neighbour test, a chunk of vertices at a time: binary search of pv in N(v)
    c = col.long() & 0xFFFFFFFF
    for i in range(0, v.numel(), 1 << 24):
        vv, pp = v[i:i + (1 << 24)], pv[i:i + (1 << 24)]
        lo, hi = off[vv].clone(), off[vv + 1].clone()
        for _ in range(34):
            mid = (lo + hi) // 2
            go = (lo < hi) & (c[mid.clamp(max=c.numel() - 1)] < pp)
            lo = torch.where(go, mid + 1, lo)
            hi = torch.where(go | (lo >= hi), hi, mid)
        assert torch.equal(c[lo.clamp(max=c.numel() - 1)], pp)


def check_pagerank(p, rec):
    ids = torch.tensor(rec["ids"], dtype=torch.long, device=p.device)
    want = torch.tensor(rec["values"], dtype=torch.float64, device=p.device)
    rel = ((p[ids].double() - want).abs() / want).max().item()
    assert rel <= PR_MAX_REL, rel
    assert abs(float(p.double().sum()) - rec["mass"]) <= 1e-5


@pytest.mark.parametrize("name", ["rmat25", "rmat26"])
def test_rmat_full_size_against_oracle_values(byo, name):
    ref = gold(name)
    n, src, dst = graphgen.workload(name)
    assert len(src) == ref["draws"] and n == ref["n"]
    srcs = graphgen.pick_sources(n, src, dst, 8, graphgen.SEEDS[name] + 1).tolist()
    assert srcs == [b["source"] for b in ref["bfs"]]
    g = byo.Graph(n, dev(src), dev(dst), byo.BYO_CSR | byo.BYO_SYMMETRIZE | byo.BYO_OFFSETS64)
    del src, dst
    try:
        assert g.m == ref["m"]
        off, col = byo.byo_graph_export_csr(g.handle)
        assert sha_csr(off, col) == ref["csr_sha256"]
        for s, want in zip(srcs, ref["bfs"]):
            lv, par = byo.byo_bfs(g.handle, [s])
            assert sha_u32(lv[0]) == want["levels_sha256"], s
            check_parents(off, col, lv[0], par[0], s)
            del lv, par
        del col
        assert sha_u32(byo.byo_cc(g.handle)) == ref["cc_sha256"]
        p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
        check_pagerank(p, ref["pagerank"])
        assert byo.byo_tc(g.handle) == ref["triangles"]
    finally:
        g.close()


@pytest.mark.parametrize("name", ["rmat22", "grid"])
def test_triangle_count_full_size(byo, name):
    ref = gold(name)
    n, src, dst = graphgen.workload(name)
    flags = byo.BYO_CSR | byo.BYO_SYMMETRIZE | (byo.BYO_OFFSETS64 if name.startswith("rmat") else 0)
    with byo.Graph(n, dev(src), dev(dst), flags) as g:
        assert g.m == ref["m"]
        assert byo.byo_tc(g.handle) == ref["triangles"]


@pytest.mark.parametrize("hashed", [False, True], ids=["sorted", "hashed"])
def test_dynamic_rounds_full_size(byo, hashed):
    ref = gold("dynamic")
    n, src, dst = graphgen.workload("rmat24")
    s0 = ref["source"]
    assert s0 == int(graphgen.pick_sources(n, src, dst, 1, graphgen.SEEDS["rmat24"] + 1)[0])
    flags = byo.BYO_DYNAMIC | byo.BYO_SYMMETRIZE | (byo.BYO_DYN_HASH if hashed else 0)
    with byo.Graph(n, dev(src), dev(dst), flags) as g:
        for want, (ins_s, ins_d, del_s, del_d) in zip(ref["rounds"], graphgen.dynamic_rounds(n, src, dst)):
            byo.byo_insert_batch(g.handle, dev(ins_s), dev(ins_d))
            byo.byo_delete_batch(g.handle, dev(del_s), dev(del_d))
            r = want["round"]
            assert g.m == want["m"], r
            off, col = byo.byo_graph_export_csr(g.handle)
            assert sha_csr(off, col) == want["csr_sha256"], r
            del off, col
            lv, _ = byo.byo_bfs(g.handle, [s0], want_parents=False)
            assert sha_u32(lv[0]) == want["bfs"]["levels_sha256"], r
            assert sha_u32(byo.byo_cc(g.handle)) == want["cc_sha256"], r
            p, _ = byo.byo_pagerank(g.handle, 0.85, 20)
            check_pagerank(p, want["pagerank"])
        assert len(ref["rounds"]) == 10


def test_batched_256_graphs_full_size(byo):
    ref = gold("batched")
    members = graphgen.batched_workload(256, 64)
    assert len(members) == len(ref["members"]) == 256
    ns = [m[0] for m in members]
    ks = [len(m[1]) for m in members]
    src = np.concatenate([m[1] for m in members])
    dst = np.concatenate([m[2] for m in members])
    sources = [m[3] for m in members]
    g = byo.byo_batch_build(ns, ks, dev(src), dev(dst))
    try:
        lv = byo.byo_msbfs(g, sources, 64)
        lab = byo.byo_cc(g)
        for i, want in enumerate(ref["members"]):
            base = byo.byo_batch_member_base(g, i)
            n = ns[i]
            assert n == want["n"]
            assert sha_u32(lv[:, base:base + n]) == want["levels_sha256"], i
            assert sha_u32(lab[base:base + n] - base) == want["cc_sha256"], i
    finally:
        byo.byo_graph_destroy(g)
