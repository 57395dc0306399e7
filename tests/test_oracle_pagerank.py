"""Pins of the PageRank oracle (appendix listing "Dynamic PR": staticPR,
DynPR) against facts that do not come from the oracle itself: closed forms,
a linear solve of the PageRank fixed point, reachability computed by scipy,
and the listing's rule that unflagged vertices keep their ranks."""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import workloads as wl

D = 0.85


def csr_from_edges(n, edges, w=None):
    edges = sorted(set(edges))
    ro = np.zeros(n + 1, np.int64)
    for u, _ in edges:
        ro[u + 1] += 1
    np.cumsum(ro, out=ro)
    col = np.array([v for _, v in edges], np.int32)
    ww = np.ones(len(edges), np.int32) if w is None else np.asarray(w, np.int32)
    return ro, col, ww


def test_cycle_is_uniform():
    n = 50
    g = oracle.OracleGraph(n, *csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)]))
    pr, it = g.pagerank(D, 1e-9, 100)
    np.testing.assert_allclose(pr, 1.0 / n, rtol=2e-7)
    assert it <= 2


def test_star_closed_form():
    k = 20
    n = k + 1
    g = oracle.OracleGraph(n, *csr_from_edges(n, [(0, i) for i in range(1, n)]))
    pr, it = g.pagerank(D, 0.0, 10)
    base = np.float32((np.float32(1) - np.float32(D)) / np.float32(n))
    assert pr[0] == base                                  # no in-edges
    leaf = np.float32(base + np.float32(D) * np.float32(base / np.float32(k)))
    np.testing.assert_array_equal(pr[1:], leaf)
    assert it == 3      # hub, then leaves settle; the third step changes nothing


def fixed_point(ro, col, n, d):
    """(I - d P^T) r = (1 - d)/n, P[u, v] = 1/outdeg(u) (fp64 solve)."""
    deg = np.diff(ro)
    A = np.eye(n)
    for u in range(n):
        for v in col[ro[u]:ro[u + 1]]:
            A[v, u] -= d / deg[u]
    return np.linalg.solve(A, np.full(n, (1 - d) / n))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_static_matches_linear_solve(seed):
    n = 120
    ro, col, w = wl.er_digraph(n, 700, 1, 9, seed)   # dangling vertices allowed
    g = oracle.OracleGraph(n, ro, col, w)
    pr, it = g.pagerank(D, 1e-7, 400)     # float steps settle to about 1e-8
    want = fixed_point(ro, col, n, D)
    np.testing.assert_allclose(pr, want, rtol=3e-5, atol=1e-9)
    assert it < 400


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


@pytest.mark.parametrize("seed", [4, 5])
def test_dynamic_flags_are_reachability_and_the_rest_is_untouched(seed):
    n = 400
    ro, col, w = wl.er_digraph(n, 900, 1, 9, seed)   # sparse: many unreached vertices
    st = wl.BatchStream(n, ro, col, w, 1, 9, "uniform")
    g = oracle.OracleGraph(n, ro, col, w)
    pr, _ = g.pagerank(D, 1e-7, 100)
    for k in range(3):
        before = pr.copy()
        r0, c0, _ = g.csr()
        b = st.next(6, 6, seed=100 * seed + k)
        reach_del = reach(n, r0, c0, b.del_dst) if b.del_dst.size else np.zeros(n, bool)
        # the graph the insertion flags spread over: after the deletions
        h = oracle.OracleGraph(n, r0, c0, np.ones(c0.size, np.int32))
        z = np.zeros(0, np.int32)
        h.apply_batch(b.del_src, b.del_dst, z, z, z)
        r1, c1, _ = h.csr()
        reach_add = reach(n, r1, c1, b.add_dst) if b.add_dst.size else np.zeros(n, bool)
        cnt = g.pagerank_batch(b, pr, D, 1e-7, 100)
        assert cnt[4] == reach_del.sum() and cnt[5] == reach_add.sum()
        untouched = ~(reach_del | reach_add)
        assert untouched.sum() > 0
        np.testing.assert_array_equal(pr[untouched], before[untouched])
        # the batch itself follows the edge-set semantics of the SSSP oracle
        e = oracle.OracleGraph(n, r0, c0, np.ones(c0.size, np.int32))
        assert e.apply(b) == cnt[:4]
        for x, y in zip(e.csr()[:2], g.csr()[:2]):
            np.testing.assert_array_equal(x, y)


def test_dynamic_on_strongly_connected_graph_reaches_static():
    n = 150
    rng = np.random.default_rng(7)
    edges = [(i, (i + 1) % n) for i in range(n)]          # a Hamiltonian cycle
    edges += [(int(a), int(b)) for a, b in rng.integers(0, n, size=(500, 2)) if a != b]
    ro, col, w = csr_from_edges(n, edges)
    g = oracle.OracleGraph(n, ro, col, w)
    pr, _ = g.pagerank(D, 1e-7, 500)
    # delete non-cycle edges only and add fresh ones: still strongly
    # connected, so every vertex is flagged in both phases
    cyc = {(i, (i + 1) % n) for i in range(n)}
    extra = [e for e in sorted(set(edges)) if e not in cyc][:40]
    ds = np.array([u for u, _ in extra], np.int32)
    dd = np.array([v for _, v in extra], np.int32)
    add = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(60, 2))
           if a != b and (int(a), int(b)) not in set(edges)][:30]
    b = wl.Batch(ds, dd, np.array([u for u, _ in add], np.int32),
                 np.array([v for _, v in add], np.int32), np.ones(len(add), np.int32))
    cnt = g.pagerank_batch(b, pr, D, 1e-7, 500)
    assert cnt[4] == n and cnt[5] == n
    assert cnt[6] < 500 and cnt[7] < 500
    fresh = oracle.OracleGraph(n, *g.csr())
    want, _ = fresh.pagerank(D, 1e-7, 500)
    np.testing.assert_allclose(pr, want, rtol=2e-5)
    np.testing.assert_allclose(pr, fixed_point(*g.csr()[:2], n, D), rtol=3e-5)


def test_empty_batch_keeps_ranks():
    W = wl.tiny_er(1)
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    pr, _ = g.pagerank(D, 1e-7, 100)
    before = pr.copy()
    cnt = g.pagerank_batch(wl.Batch.empty(), pr, D, 1e-7, 100)
    assert cnt == (0, 0, 0, 0, 0, 0, 0, 0)
    np.testing.assert_array_equal(pr, before)


def test_invalid_batch_is_rejected_and_changes_nothing():
    W = wl.tiny_er(2)
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    pr, _ = g.pagerank(D, 1e-7, 100)
    before = pr.copy()
    m = g.m
    bad = wl.Batch(np.array([0], np.int32), np.array([W.n], np.int32),
                   np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))
    with pytest.raises(oracle.OracleError):
        g.pagerank_batch(bad, pr, D, 1e-7, 100)
    np.testing.assert_array_equal(pr, before)
    assert g.m == m
