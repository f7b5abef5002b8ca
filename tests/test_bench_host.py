"""Host logic of bench.py's roofline: the algorithmic byte models and the
DRAM-traffic table they are reported beside."""
import bench


def test_pagerank_bytes_per_iteration():
    # 8-byte offsets of the degree-ordered copy, 4-byte ids, 16 bytes of
    # contributions and ranks per vertex
    n, m = 1000, 30000
    assert bench.algo_bytes("pr_iter", n, m, 4) == 8 * (n + 1) + 4 * m + 16 * n


def test_cc_sampling_bytes():
    n = 1 << 20
    got = bench.algo_bytes("cc_sample", n, 0, 8)
    assert got == 4 * n + 2 * (8 * (n + 1) + 12 * n) + 8 * n


def test_bfs_bytes_follow_the_trace():
    class R:
        def __init__(self, direction, frontier, unvisited, examined):
            self.direction, self.frontier, self.unvisited, self.edges_examined = direction, frontier, unvisited, examined
    n = 64
    trace = [R(1, 1, 63, 5), R(0, 5, 58, 20)]
    want = 8.0 * n + n / 8.0
    want += 2 * 4 * 1 + 4.0 * 5 + 4.0 * 1                 # push level
    want += 2 * 4 * 58 + 4.0 * 20 + 3 * n / 8.0           # pull level
    want += 12.0 * 5                                      # the pull level's successor frontier
    assert bench.algo_bytes("bfs_persistent", n, 0, 4, trace) == want


def test_traffic_table_is_read():
    assert bench.ncu_traffic("tc_count", "rmat25") > 1e11
    assert bench.ncu_traffic("pr_iter", "rmat22") > 1e8
    assert bench.ncu_traffic("no_such_kernel", "rmat25") is None
