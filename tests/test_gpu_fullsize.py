"""GPU parity at the benchmark's full sizes, in the configuration bench.py
times: the graph on its own stream, batches as CUDA tensors, statistics on
(the timed path), repeated batch shapes replayed from the cached CUDA graph,
the invalidation beside the store update, near-far push at the widths the
autotuner picks for these graphs.

- R-MAT scale 20 (1,048,576 vertices, 16,777,216 edges), three 1% batches;
- the 4096 x 4096 grid (16,777,216 vertices, ~67M edges), two 1% batches
  with half of the deletions on shortest-path-tree edges.

The oracle's Dijkstra finishes these sizes in seconds, so every distance is
compared bit for bit after every batch (not a sample); parents are checked by
the shortest-path-tree invariants; the stores against the oracle's edge set.
"""
import numpy as np
import pytest

import oracle
from oracle.invariants import check_sssp
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()
    return t


def _transpose(n, ro, col, w):
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(ro))
    order = np.lexsort((u, col))
    rro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=n), out=rro[1:])
    return rro, u[order].astype(np.int32), w[order]


def _run(torch, W, delta, n_batches, reverse_store):
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    stream = torch.cuda.Stream()
    tree = W.tree_fraction > 0
    with torch.cuda.stream(stream):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
        try:
            g.set_delta(delta)
            g.sssp_init(W.source)
            d = g.get_dist()
            np.testing.assert_array_equal(d, ref.dijkstra(W.source))
            for k in range(n_batches):
                b = W.batch(k, dist=d if tree else None)
                dev = [torch.from_numpy(x).cuda() for x in
                       (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w)]
                stream.synchronize()
                st = g.apply_batch(*dev, stats=True)
                cnt = ref.apply(b)
                assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                        st.n_add_present) == cnt
                d, p = g.get_dist(parent=True)
                want = ref.dijkstra(W.source)
                np.testing.assert_array_equal(d, want)
                ro, col, w = ref.csr()
                check_sssp(W.n, ro, col, w, W.source, d, p)
                assert g.m == col.size
                for a, e in zip(g.export_csr(), (ro, col, w)):
                    np.testing.assert_array_equal(a, e)
                if reverse_store:
                    for a, e in zip(g.export_csr(reverse=True), _transpose(W.n, ro, col, w)):
                        np.testing.assert_array_equal(a, e)
        finally:
            g.close()


def test_rmat20_one_percent_batches(torch):
    W = wl.rmat(scale=20, batch_frac=0.01, seed=1)
    _run(torch, W, delta=800, n_batches=3, reverse_store=True)


def test_grid4096_one_percent_tree_biased_batches(torch):
    W = wl.grid(4096, 4096, batch_frac=0.01, seed=1)
    _run(torch, W, delta=32000, n_batches=2, reverse_store=False)
