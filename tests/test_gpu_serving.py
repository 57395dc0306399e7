"""GPU tests of the serving runtime (sp_server_*): requests of several graphs
run concurrently on worker slots and overlap on the device, graphs are
evicted and reloaded under an HBM budget that the resident graphs never
exceed (reloads restore the checkpointed distances), no repair needs a
recovery (the slots' cooperative grids are co-resident), and every query
answer equals the oracle's distances after the batches submitted before it
on that graph, whatever the mix it ran in."""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()


def make_workloads():
    return [wl.tiny_er(3), wl.rmat(12, batch_frac=0.02, seed=5),
            wl.rmat(13, batch_frac=0.01, seed=6),
            wl.grid(64, 64, batch_frac=0.02, seed=7, tree_fraction=0.0)]


def expected(works, n_batches):
    """Batches per graph and the oracle's distances after each of them
    (index 0 = before any batch)."""
    batches, dists = [], []
    for W in works:
        ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
        bs, ds = [], [ref.dijkstra(W.source)]
        for k in range(n_batches):
            b = W.batch(k)
            ref.apply(b)
            bs.append(b)
            ds.append(ref.dijkstra(W.source))
        batches.append(bs)
        dists.append(ds)
    return batches, dists


def run_mix(srv, works, batches, dists, rng):
    gids = [srv.add_graph(W.n, W.row_off, W.col, W.w, W.source) for W in works]
    pending = []   # (request id, graph index, batch count before it, vertices)
    for k in range(len(batches[0]) + 1):
        for i in rng.permutation(len(works)):
            W = works[i]
            v = rng.integers(0, W.n, size=min(W.n, 257)).astype(np.int32)
            pending.append((srv.submit_query(gids[i], v), i, k, v))
            if k < len(batches[i]):
                pending.append((srv.submit(gids[i], batches[i][k]), i, None, None))
    for rid, i, k, v in pending:
        info, out = srv.wait(rid)
        assert info.status == sp.SP_OK, (i, k, sp.STATUS.get(info.status))
        assert info.done_ms >= info.start_ms >= info.submit_ms
        if k is not None:
            np.testing.assert_array_equal(out, dists[i][k][v])
    for i, W in enumerate(works):
        np.testing.assert_array_equal(srv.get_dist(gids[i]), dists[i][-1])
    return gids


def test_serving_mix_matches_oracle():
    works = make_workloads()
    batches, dists = expected(works, 4)
    with sp.Server(hbm_budget_bytes=8 << 30, n_slots=3) as srv:
        run_mix(srv, works, batches, dists, np.random.default_rng(1))
        st = srv.stats()
        assert st.recoveries == 0
        assert st.max_resident_bytes <= 8 << 30
        assert st.loads == len(works) and st.evictions == 0
        assert st.batches == 4 * len(works)
        assert st.updates == sum(b.size for bs in batches for b in bs)
        assert st.resident_graphs == st.registered_graphs == len(works)


def test_serving_evicts_and_reloads_under_budget():
    works = make_workloads()
    batches, dists = expected(works, 3)
    # size of each graph once it has run a batch, measured on its own
    sizes = []
    with sp.Server(hbm_budget_bytes=8 << 30, n_slots=1) as srv:
        for W, bs in zip(works, batches):
            before = srv.stats().resident_bytes
            g = srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
            srv.wait(srv.submit(g, bs[0]))
            sizes.append(srv.stats().resident_bytes - before)
    big = sorted(sizes)
    budget = big[-1] + big[-2] + big[0] // 2   # never all four at once
    with sp.Server(hbm_budget_bytes=budget, n_slots=2) as srv:
        run_mix(srv, works, batches, dists, np.random.default_rng(2))
        st = srv.stats()
        assert st.evictions > 0 and st.loads == st.evictions + st.resident_graphs
        assert st.resident_graphs < len(works)
        assert st.resident_bytes <= budget and st.max_resident_bytes <= budget
        # reloads restore the checkpointed distances instead of recomputing
        assert st.restores >= 1 and st.restores <= st.loads - len(works)
        assert st.recoveries == 0


def test_serving_graph_over_budget_is_refused():
    """A graph is admitted by the upper bound of its footprint, so one that
    could not fit alone is refused when it is registered, and a batch larger
    than the reserved batch size is refused when it is submitted."""
    W = wl.tiny_er(1)
    bound = sp.footprint_bound(W.n, W.m, 0.25, 64)
    with sp.Server(hbm_budget_bytes=bound - 1, n_slots=1, max_batch_updates=64) as srv:
        with pytest.raises(sp.SpError) as e:
            srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
        assert e.value.code == sp.SP_ENOMEM_BUDGET
    with sp.Server(hbm_budget_bytes=bound, n_slots=1, max_batch_updates=64) as srv:
        g = srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
        with pytest.raises(sp.SpError) as e:
            srv.submit_batch(g, np.zeros(40, np.int32), np.ones(40, np.int32),
                             np.zeros(25, np.int32), np.ones(25, np.int32),
                             np.ones(25, np.int32))
        assert e.value.code == sp.SP_EINVAL
        b = W.batch(0)
        info, _ = srv.wait(srv.submit(g, b))
        assert info.status == sp.SP_OK
        st = srv.stats()
        assert 0 < st.resident_bytes <= bound and st.max_resident_bytes <= bound


def test_footprint_bound_holds():
    """The bound is above what a handle holds once it has reserved its batch
    buffers, on graphs of every kind."""
    for W in (wl.tiny_er(2), wl.rmat(13, batch_frac=0.01, seed=3),
              wl.grid(100, 130, batch_frac=0.01, seed=4)):
        for slack, upd in ((0.25, 1000), (0.0, 50_000), (1.5, 10)):
            with sp.Graph(W.n, W.row_off, W.col, W.w, slack=slack) as g:
                g.reserve(upd)
                held = g.info().device_bytes
            assert held <= sp.footprint_bound(W.n, W.m, slack, upd), (W.name, slack, upd)


def test_requests_of_different_graphs_overlap_on_the_device():
    """Four slots, four graphs (two R-MAT, two grids), every batch submitted
    at once: requests of different graphs on different slots run on the
    device at the same time (their CUDA-event intervals intersect), no repair
    needs a recovery, and the results equal the oracle's."""
    works = [wl.rmat(14, batch_frac=0.01, seed=21), wl.rmat(15, batch_frac=0.005, seed=22),
             wl.grid(256, 256, batch_frac=0.01, seed=23, tree_fraction=0.0),
             wl.grid(200, 300, batch_frac=0.01, seed=24, tree_fraction=0.0)]
    batches, dists = expected(works, 4)
    with sp.Server(hbm_budget_bytes=16 << 30, n_slots=4) as srv:
        gids = [srv.add_graph(W.n, W.row_off, W.col, W.w, W.source) for W in works]
        for i in range(len(works)):      # load every graph first
            srv.wait(srv.submit_query(gids[i], np.arange(4, dtype=np.int32)))
        ids = [(srv.submit(gids[i], batches[i][k]), i) for k in range(4)
               for i in range(len(works))]
        infos = []
        for rid, i in ids:
            info, _ = srv.wait(rid)
            assert info.status == sp.SP_OK
            assert 0 <= info.gpu_start_ms <= info.gpu_done_ms
            infos.append((i, info.slot, info.gpu_start_ms, info.gpu_done_ms))
        overlaps = sum(1 for a in infos for b in infos
                       if a[0] < b[0] and a[1] != b[1] and a[2] < b[3] and b[2] < a[3])
        assert overlaps > 0, infos
        for i, W in enumerate(works):
            np.testing.assert_array_equal(srv.get_dist(gids[i]), dists[i][-1])
        assert srv.stats().recoveries == 0


def test_serving_bad_requests():
    W = wl.tiny_er(2)
    with sp.Server(hbm_budget_bytes=1 << 30, n_slots=2) as srv:
        g = srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
        with pytest.raises(sp.SpError):
            srv.submit_query(g + 1, np.arange(3))
        with pytest.raises(sp.SpError):
            srv.wait(12345)
        # an invalid batch fails alone and leaves the graph as it was
        bad = srv.submit_batch(g, [], [], [0], [W.n], [5])
        q = srv.submit_query(g, np.arange(W.n))
        info, _ = srv.wait(bad)
        assert info.status == sp.SP_EINVAL
        info, d = srv.wait(q)
        assert info.status == sp.SP_OK
        ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
        np.testing.assert_array_equal(d, ref.dijkstra(W.source))
