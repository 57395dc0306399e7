"""GPU parity at the benchmark's full sizes, in the configuration bench.py
times: the graph on its own stream, batches as CUDA tensors, statistics on
(the timed path), repeated batch shapes replayed from the cached CUDA graph,
the invalidation beside the store update, and the push schedule the
autotuner picks for the graph.

- R-MAT scale 20 (1,048,576 vertices, 16,777,216 edges), three 1% batches;
- the 4096 x 4096 grid (16,777,216 vertices, ~67M edges), two batches each
  of 0.1%, 1% and 5%, half of the deletions on shortest-path-tree edges;
- the batched form: 64 R-MAT graphs of scale ~U{12..18} in one handle, each
  with its own batch of 0.5-5% of its edges, replayed through a captured
  sp_capture_apply, every graph against its own oracle after every round;
- the serving form with a scale-22 R-MAT graph (4,194,304 vertices,
  67,108,864 edges) under an HBM budget that forces it out and back in.

The oracle's Dijkstra finishes these sizes in seconds, so every distance is
compared bit for bit after every batch (the serving test checks the queries
after a sample of the scale-22 graph's batches, and the full distances at
the end); parents are checked by the shortest-path-tree invariants; the
stores against the oracle's edge set.
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


def _tune(g, W):
    """The schedule bench.py uses: the autotuner's pick on this graph."""
    from paper_2507_11094_gb300 import autotune
    return autotune.tune_schedule(
        g, lambda h, stats=False: h.sssp_init(W.source, stats=stats), W.w, reps=1)


def _run(torch, W, n_batches, reverse_store):
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    stream = torch.cuda.Stream()
    tree = W.tree_fraction > 0
    with torch.cuda.stream(stream):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
        try:
            _tune(g, W)
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
    _run(torch, W, n_batches=3, reverse_store=True)


@pytest.mark.parametrize("pct", [0.1, 1, 5])
def test_grid4096_tree_biased_batches(torch, pct):
    W = wl.grid(4096, 4096, batch_frac=pct / 100, seed=1)
    _run(torch, W, n_batches=2, reverse_store=False)


def test_batched64_rmat12_18_captured_replay(torch):
    from paper_2507_11094_gb300 import autotune, batched
    ws = wl.batched_rmat(seed=1)
    assert len(ws) == 64 and {W.n for W in ws} <= {2 ** s for s in range(12, 19)}
    stream = torch.cuda.Stream()
    B = batched.BatchedGraphs([(W.n, W.row_off, W.col, W.w) for W in ws],
                              [W.source for W in ws], stream=stream)
    refs = [oracle.OracleGraph(W.n, W.row_off, W.col, W.w) for W in ws]
    try:
        autotune.tune_schedule(B.g, lambda h, stats=False: B.init(stats=stats),
                               B.packed.w, reps=1)
        B.init()
        for i, W in enumerate(ws):
            np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
        rounds = [[W.batch(k) for W in ws] for k in range(3)]
        arrays = [batched.pack_batches(B.packed, r) for r in rounds]
        assert len({tuple(a.size for a in arr) for arr in arrays}) == 1
        fixed = [torch.from_numpy(a).cuda() for a in arrays[0]]
        torch.cuda.synchronize()
        B.g.reserve(int(arrays[0][0].size + arrays[0][2].size) + 16)
        ex = B.g.capture(*fixed)
        try:
            for k, arr in enumerate(arrays):
                for t, a in zip(fixed, arr):
                    t.copy_(torch.from_numpy(a))
                torch.cuda.synchronize()
                ex.launch()
                st = ex.finish(stats=True)
                applied = 0
                for i, W in enumerate(ws):
                    c = refs[i].apply(rounds[k][i])
                    applied += c[0] + c[2]
                    np.testing.assert_array_equal(B.dist(i), refs[i].dijkstra(W.source))
                assert st.n_del_applied + st.n_add_applied == applied
        finally:
            ex.close()
    finally:
        B.close()


def test_serving_scale22_evicted_and_reloaded(torch):
    """A scale-22 R-MAT graph and two scale-16 graphs under a budget that
    holds the big graph and one small one: the big graph is evicted when both
    small ones run and reloaded for its next batch.  Batches of 1k, 100k and
    1M updates; queries of 1,024 vertices after the big graph's first and
    last batches and the full distances at the end equal the oracle's."""
    big = wl.rmat(scale=22, batch_frac=0.001, seed=5150)
    small = [wl.rmat(scale=16, batch_frac=0.01, seed=5151 + i) for i in range(2)]
    rng = np.random.default_rng(7)
    sizes = {"big": [1000, 100_000, 1_000_000], "small": [2000, 5000, 8000]}
    plan = []   # (graph index, batch)
    for k in range(3):
        plan.append((0, big.stream.next(sizes["big"][k] // 2, sizes["big"][k] // 2,
                                        seed=900 + k)))
        for i, W in enumerate(small):
            plan.append((1 + i, W.stream.next(sizes["small"][k] // 2,
                                              sizes["small"][k] // 2, seed=910 + 10 * k + i)))
    works = [big] + small
    # the oracle's distances after each of the big graph's batches that are
    # queried (the first and the last), and every graph's final distances
    refs = [oracle.OracleGraph(W.n, W.row_off, W.col, W.w) for W in works]
    qv = rng.integers(0, big.n, size=1024).astype(np.int32)
    want_q, seen = {}, 0
    for gi, b in plan:
        refs[gi].apply(b)
        if gi == 0:
            seen += 1
            if seen in (1, 3):
                want_q[seen] = refs[0].dijkstra(big.source)[qv]
    final = [r.dijkstra(W.source) for r, W in zip(refs, works)]
    # budget: the big graph's footprint bound plus one small graph's
    est = [sp.footprint_bound(W.n, W.m, 0.25, sizes["big"][-1]) for W in works]
    budget = est[0] + max(est[1:]) + (est[1] + est[2]) // 4
    with sp.Server(hbm_budget_bytes=budget, n_slots=2, max_batch_updates=sizes["big"][-1]) \
            as srv:
        gids = [srv.add_graph(W.n, W.row_off, W.col, W.w, W.source) for W in works]
        pending, seen = [], 0
        for gi, b in plan:
            pending.append((srv.submit(gids[gi], b), None))
            if gi == 0:
                seen += 1
                if seen in (1, 3):
                    pending.append((srv.submit_query(gids[0], qv), seen))
        for rid, q in pending:
            info, out = srv.wait(rid)
            assert info.status == sp.SP_OK, sp.STATUS.get(info.status)
            if q is not None:
                np.testing.assert_array_equal(out, want_q[q])
        for i in range(len(works)):
            np.testing.assert_array_equal(srv.get_dist(gids[i]), final[i])
        st = srv.stats()
        assert st.evictions >= 1 and st.loads >= len(works) + 1
        assert st.max_resident_bytes <= budget
        assert st.recoveries == 0
