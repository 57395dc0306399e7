"""The batched and serving workloads: seeded, of the stated shapes, the same
arrays for the same seed (the tests and the bench draw them from here)."""
import numpy as np

from paper_2507_11094_gb300 import workloads as wl


def test_batched_rmat_shapes_and_determinism():
    a = wl.batched_rmat(seed=3, k=6)
    b = wl.batched_rmat(seed=3, k=6)
    assert len(a) == 6
    for x, y in zip(a, b):
        assert x.n == y.n and x.n in {2 ** s for s in range(12, 19)}
        assert x.m == 16 * x.n
        np.testing.assert_array_equal(x.col, y.col)
        bx, by = x.batch(0), y.batch(0)
        assert 0.005 * x.m - 2 <= bx.size <= 0.05 * x.m + 2
        np.testing.assert_array_equal(bx.add_dst, by.add_dst)


def test_serving_requests_sizes_and_queries():
    ws = [wl.rmat(scale=10, batch_frac=0.01, seed=1 + i) for i in range(3)]
    reqs = wl.serving_requests(ws, 12, seed=5)
    assert len(reqs) == 12
    for i, (gi, b, q) in enumerate(reqs):
        assert 0 <= gi < 3
        assert 2 <= b.size <= max(2, ws[gi].m // 2)
        assert abs(b.del_src.size - b.add_src.size) <= 1
        if i % 4 == 3:
            assert q.size == 1024 and q.max() < ws[gi].n
        else:
            assert q is None
