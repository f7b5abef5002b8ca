"""Host logic of the learned schedule: which actions a level allows, and how
per-level timings become weighted training samples."""
import numpy as np

from paper_2405_11671_gb300 import schedule

INF = np.inf


def test_allowed_masks_pull_on_small_frontiers():
    # |F| = 10, 100 frontier edges, 10,000 unvisited edges, n = 1000:
    # 100 <= 10000 / 15 and 10 < 1000 / 18, so neither Beamer test pulls
    t = schedule.allowed([1.0, 2.0, 3.0, 4.0, 5.0], (10, 100, 10_000, 1000))
    assert t[0] == INF and list(t[1:]) == [2.0, 3.0, 4.0, 5.0]


def test_allowed_pull_by_either_beamer_test():
    by_edges = schedule.allowed([1.0] * 5, (10, 1000, 10_000, 1000))   # 1000 > 10000 / 15
    by_size = schedule.allowed([1.0] * 5, (56, 10, 10_000, 1000))      # 56 >= 1000 / 18
    assert by_edges[0] == 1.0 and by_size[0] == 1.0


def test_allowed_masks_solo_beyond_its_limits():
    lim_e, lim_v = schedule.SOLO_MAX_EDGES, schedule.SOLO_MAX_VERTICES
    assert schedule.allowed([1.0] * 5, (lim_v, lim_e, 1 << 40, 1 << 30))[4] == 1.0
    assert schedule.allowed([1.0] * 5, (lim_v + 1, lim_e, 1 << 40, 1 << 30))[4] == INF
    assert schedule.allowed([1.0] * 5, (lim_v, lim_e + 1, 1 << 40, 1 << 30))[4] == INF


def test_samples_label_fastest_allowed_action_and_weight():
    feats = np.arange(24, dtype=np.float32).reshape(2, 12)
    times = np.array([[0.5, 9.0, 3.0, 6.0, 2.0],        # pull fastest but not allowed; solo allowed
                      [40.0, 80.0, 90.0, 100.0, 1.0]])  # pull allowed (big frontier); solo not
    stats = [(10, 100, 10_000, 1000), (500, 50_000, 60_000, 1000)]
    X, y, w = schedule.samples_from_timings([(feats, times, np.array([100.0, 50_000.0]), stats)])
    assert X.shape == (2, 12) and np.array_equal(X, feats)
    assert list(y) == [4, 0]
    assert np.allclose(w, [np.log(9.0 / 2.0), np.log(100.0 / 40.0)])


def test_regret_is_time_over_the_per_level_best():
    t = np.array([[3.0, 1.0], [2.0, 5.0]])
    assert schedule.regret(t, [0, 0]) == 2.0 and schedule.regret(t, [1, 0]) == 0.0
