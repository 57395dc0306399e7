"""GPU parity of dynamic PageRank (sp_pr_*) against the single-precision
oracle (appendix listing "Dynamic PR").

Ranks are compared with a tolerance: a vertex with at most eight in-edges is
summed in in-neighbour order, as the oracle does, but larger in-lists are
summed in parallel parts whose float rounding differs; the difference stays
within a few units in the last place of the sums and is damped by the
factor d < 1 through later steps.  The batch counters, the flagged-vertex
counts and the edge sets must match exactly, and the number of Jacobi
steps may differ by at most one (a step whose difference lies within
rounding of beta)."""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
D, BETA, ITERS = 0.85, 1e-6, 100
RTOL, ATOL = 2e-5, 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()


WORKLOADS = {
    "er1k": lambda: wl.tiny_er(4),
    "rmat12": lambda: wl.rmat(12, batch_frac=0.01, seed=3),
    "grid48": lambda: wl.grid(48, 48, batch_frac=0.01, seed=2, tree_fraction=0.0),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_static_pagerank(name):
    W = WORKLOADS[name]()
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    want, it = ref.pagerank(D, BETA, ITERS)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        st = g.pr_init(D, BETA, ITERS, stats=True)
        got = g.pr_get()
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=ATOL)
    assert abs(st.rounds_push - it) <= 1
    assert st.relaxed_edges == W.m * st.rounds_push


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_dynamic_pagerank_batches(name):
    W = WORKLOADS[name]()
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    want, _ = ref.pagerank(D, BETA, ITERS)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.pr_init(D, BETA, ITERS)
        for k in range(4):
            b = W.batch(k)
            cnt = ref.pagerank_batch(b, want, D, BETA, ITERS)
            st = g.pr_apply(b, stats=True)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt[:4]
            assert st.affected == cnt[4] + cnt[5]
            assert abs(st.rounds_push - (cnt[6] + cnt[7])) <= 2
            np.testing.assert_allclose(g.pr_get(), want, rtol=RTOL, atol=ATOL)
            for x, y in zip(g.export_csr(), ref.csr()):
                np.testing.assert_array_equal(x, y)


def reach(n, ro, col, seeds):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import breadth_first_order
    A = csr_matrix((np.ones(col.size), col, ro), shape=(n, n))
    seen = np.zeros(n, bool)
    for s in np.unique(seeds):
        if not seen[s]:
            seen[breadth_first_order(A, int(s), directed=True,
                                     return_predecessors=False)] = True
    return seen


def test_unflagged_vertices_keep_their_ranks_exactly():
    # a sparse graph with many vertices unreachable from the updates
    n = 3000
    ro, col, w = wl.er_digraph(n, 4500, 1, 9, 11)
    stream = wl.BatchStream(n, ro, col, w, 1, 9, "uniform")
    with sp.Graph(n, ro, col, w) as g:
        g.pr_init(D, BETA, ITERS)
        before = g.pr_get()
        b = stream.next(3, 3, seed=5)
        h = oracle.OracleGraph(n, ro, col, w)
        flagged = reach(n, ro, col, b.del_dst)
        z = np.zeros(0, np.int32)
        h.apply_batch(b.del_src, b.del_dst, z, z, z)
        r1, c1, _ = h.csr()
        flagged |= reach(n, r1, c1, b.add_dst)
        st = g.pr_apply(b, stats=True)
        after = g.pr_get()
        assert 0 < flagged.sum() < n
        assert st.affected <= 2 * flagged.sum()
        np.testing.assert_array_equal(after[~flagged], before[~flagged])


def test_empty_and_invalid_batches():
    W = wl.tiny_er(5)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.pr_init(D, BETA, ITERS)
        before = g.pr_get()
        z = np.zeros(0, np.int32)
        st = g.pr_apply_batch(z, z, z, z, z, stats=True)
        assert st.affected == 0
        np.testing.assert_array_equal(g.pr_get(), before)
        m = g.m
        with pytest.raises(sp.SpError) as e:   # the bad insertion is in phase two
            g.pr_apply_batch(np.array([0], np.int32), np.array([1], np.int32),
                             np.array([0], np.int32), np.array([W.n], np.int32),
                             np.array([3], np.int32))
        assert e.value.code == sp.SP_EINVAL
        assert g.m == m
        np.testing.assert_array_equal(g.pr_get(), before)


def test_pagerank_and_sssp_states():
    W = wl.tiny_er(6)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        with pytest.raises(sp.SpError) as e:
            g.pr_get()
        assert e.value.code == sp.SP_ESTATE
        g.sssp_init(W.source)
        g.pr_init(D, BETA, ITERS)
        g.get_dist()                         # static PR leaves distances valid
        g.pr_apply(W.batch(0))
        with pytest.raises(sp.SpError) as e:
            g.get_dist()
        assert e.value.code == sp.SP_ESTATE
        g.sssp_init(W.source)
        ref = oracle.OracleGraph(W.n, *g.export_csr())
        np.testing.assert_array_equal(g.get_dist(), ref.dijkstra(W.source))
        g.apply(W.batch(1))
        with pytest.raises(sp.SpError) as e:
            g.pr_get()
        assert e.value.code == sp.SP_ESTATE
        with pytest.raises(sp.SpError):
            g.pr_init(1.5, BETA, ITERS)
