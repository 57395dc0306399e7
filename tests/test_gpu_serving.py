"""GPU tests of the serving runtime (sp_server_*): requests of several graphs
run concurrently on worker slots, graphs are evicted and reloaded under an
HBM budget, and every query answer equals the oracle's distances after the
batches submitted before it on that graph."""
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
        assert st.resident_bytes <= budget


def test_serving_graph_over_budget_is_refused():
    W = wl.tiny_er(1)
    with sp.Server(hbm_budget_bytes=1 << 16, n_slots=1) as srv:
        with pytest.raises(sp.SpError) as e:   # the lower bound alone is over
            srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
        assert e.value.code == sp.SP_ENOMEM_BUDGET
    with sp.Server(hbm_budget_bytes=1 << 20, n_slots=1) as srv:
        g = srv.add_graph(W.n, W.row_off, W.col, W.w, W.source)
        info, _ = srv.wait(srv.submit_query(g, np.arange(4)))
        assert info.status == sp.SP_ENOMEM_BUDGET
        assert srv.stats().resident_bytes == 0


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
