"""What the trained schedule network gains over the method without it.

The committed network (``paper_2405_11671_gb300/sched_mlp.json``, trained by
``python -m paper_2405_11671_gb300.schedule train`` on generated graphs) is run
on held-out graphs of the three workload shapes.  For every BFS level the
device time of each of the five actions is measured with that action forced
(frontiers do not depend on the schedule), and the per-level choices of the
Beamer heuristic and of the network are scored by their regret: the time they
lose over the best action of each level.  Both choices are scored on the same
timing table, so the comparison carries no run-to-run noise: the network's
per-level total must not exceed the heuristic's on any shape, and both must
give the same levels.
"""
import os

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


HELD_OUT = {
    "grid": lambda: graphgen.grid_small(768, 768, 0.1, 1e-4, 4242),
    "rmat": lambda: graphgen.rmat_small(17, 16, 4243),
    "er": lambda: (1 << 16, *graphgen.er(1 << 16, (1 << 16) * 12, 4244)),
}


@pytest.mark.parametrize("shape", sorted(HELD_OUT))
def test_learned_schedule_regret(byo, shape):
    from paper_2405_11671_gb300 import schedule
    if not os.path.exists(schedule.DEFAULT_PATH):
        pytest.fail("no trained schedule network committed")
    net = schedule.load(byo, schedule.DEFAULT_PATH)
    n, src, dst = HELD_OUT[shape]()
    ref = oracle.csr_build(n, src, dst)
    g = byo.Graph(n, dev(src), dev(dst))
    try:
        srcs = graphgen.pick_sources(n, src, dst, 2, 5).tolist()
        tables = schedule.time_actions(byo, g.handle, srcs, repeats=3)
        heur = byo.make_sched(byo.BYO_SCHED_HEURISTIC)
        learned = byo.make_sched(byo.BYO_SCHED_LEARNED, mlp=net)
        r_h = r_l = best = t_h = t_l = 0.0
        for s, (_, t, _, _) in zip(srcs, tables):
            lv_h, _ = byo.byo_bfs(g.handle, [s], sched=heur, want_parents=False)
            ch = [r.action for r in byo.byo_bfs_trace(g.handle)]
            lv_l, _ = byo.byo_bfs(g.handle, [s], sched=learned, want_parents=False)
            cl = [r.action for r in byo.byo_bfs_trace(g.handle)]
            want, _ = oracle.bfs(ref, s)
            assert np.array_equal(lv_h[0].cpu().numpy().view(np.uint32), want)
            assert np.array_equal(lv_l[0].cpu().numpy().view(np.uint32), want)
            assert len(ch) == len(cl) == len(t)
            r_h += schedule.regret(t, ch)
            r_l += schedule.regret(t, cl)
            best += float(t.min(axis=1).sum())
            t_h += float(sum(t[i, c] for i, c in enumerate(ch)))
            t_l += float(sum(t[i, c] for i, c in enumerate(cl)))
        print(f"\n{shape}: per-level time heuristic {t_h / 1e6:.3f} ms, learned {t_l / 1e6:.3f} ms "
              f"(gain {t_h / max(t_l, 1):.2f}x), best {best / 1e6:.3f} ms")
        assert t_l <= t_h and r_l <= r_h
    finally:
        g.close()
        byo.byo_mlp_destroy(net)
