"""Batched form on the GPU: many graphs in one handle, multi-source init,
captured CUDA-graph replay, and the schedule autotuner -- all against the
per-graph CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import autotune, batched, sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available()
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()
    return t


def _workloads():
    ws = [wl.rmat(scale=s, batch_frac=f, seed=10 + s) for s, f in
          ((8, 0.05), (9, 0.02), (10, 0.01), (11, 0.005))]
    ws.append(wl.tiny_er(seed=5))
    ws.append(wl.grid(20, 30, batch_frac=0.02, seed=3, tree_fraction=0.0))
    return ws


def test_union_matches_each_graph_oracle(torch):
    ws = _workloads()
    B = batched.BatchedGraphs([(W.n, W.row_off, W.col, W.w) for W in ws],
                              [W.source for W in ws])
    refs = [oracle.OracleGraph(W.n, W.row_off, W.col, W.w) for W in ws]
    B.init()
    for i, W in enumerate(ws):
        np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
    for k in range(3):
        bs = [W.batch(k) for W in ws]
        B.apply(bs)
        for i, W in enumerate(ws):
            refs[i].apply(bs[i])
            np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
    B.close()


def test_multi_source_is_min_over_sources(torch):
    n, ro, col, w = (600,) + wl.er_digraph(600, 3000, 1, 50, seed=9)
    srcs = [3, 77, 400]
    ref = oracle.OracleGraph(n, ro, col, w)
    want = np.min([ref.dijkstra(s) for s in srcs], axis=0)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init_multi(np.array(srcs, np.int32))
        d, p = g.get_dist(parent=True)
        np.testing.assert_array_equal(d, want)
        assert all(p[s] == -1 for s in srcs)


def test_captured_batches_replay_exactly(torch):
    ws = _workloads()
    packed_ws = [(W.n, W.row_off, W.col, W.w) for W in ws]
    B = batched.BatchedGraphs(packed_ws, [W.source for W in ws],
                              stream=torch.cuda.Stream())
    refs = [oracle.OracleGraph(W.n, W.row_off, W.col, W.w) for W in ws]
    B.init()
    rounds = [[W.batch(k) for W in ws] for k in range(3)]
    arrays = [batched.pack_batches(B.packed, r) for r in rounds]
    sizes = {tuple(a.size for a in arr) for arr in arrays}
    assert len(sizes) == 1                      # same sizes every round
    dev = [torch.from_numpy(a).cuda() for a in arrays[0]]
    torch.cuda.synchronize()
    B.g.reserve(sum(a.size for a in arrays[0][:3:2]) + 16)
    ex = B.g.capture(*dev)
    for k, arr in enumerate(arrays):
        for t, a in zip(dev, arr):
            t.copy_(torch.from_numpy(a))
        torch.cuda.synchronize()
        ex.launch()
        st = ex.finish(stats=True)
        for i, W in enumerate(ws):
            cnt = refs[i].apply(rounds[k][i])
            np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
        assert st.n_del_applied + st.n_add_applied > 0
    ex.close()
    B.close()


def test_autotuner_keeps_distances(torch):
    W = wl.grid(40, 40, seed=2)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        res = autotune.tune_schedule(g, lambda h, stats=False: h.sssp_init(W.source, stats=stats),
                                     W.w, reps=1)
        assert res["delta"] in autotune.candidates(W.w)
        np.testing.assert_array_equal(g.get_dist(), ref.dijkstra(W.source))
        b = W.batch(0, dist=g.get_dist())
        g.apply(b)
        ref.apply(b)
        np.testing.assert_array_equal(g.get_dist(), ref.dijkstra(W.source))


def test_autotuned_union_matches_each_graph_oracle(torch):
    """The batched form with the schedule the tuner picks for the union."""
    ws = _workloads()
    B = batched.BatchedGraphs([(W.n, W.row_off, W.col, W.w) for W in ws],
                              [W.source for W in ws])
    refs = [oracle.OracleGraph(W.n, W.row_off, W.col, W.w) for W in ws]
    res = autotune.tune_schedule(B.g, lambda h, stats=False: B.init(stats=stats),
                                 B.packed.w, reps=1)
    assert set(res["schedule"]) == {"delta", "pool_rounds", "small_deg", "local_edges"}
    for k in range(2):
        bs = [W.batch(k) for W in ws]
        B.apply(bs)
        for i, W in enumerate(ws):
            refs[i].apply(bs[i])
            np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
    B.close()
