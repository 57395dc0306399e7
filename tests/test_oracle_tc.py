"""Pins of the triangle-count oracle (appendix listing "Dynamic TC",
staticTC): closed forms and trace(A^3) / 6 of the symmetric adjacency
matrix, computed independently with numpy."""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import workloads as wl


def sym_csr(n, pairs):
    e = sorted({(a, b) for a, b in pairs} | {(b, a) for a, b in pairs})
    ro = np.zeros(n + 1, np.int64)
    for u, _ in e:
        ro[u + 1] += 1
    np.cumsum(ro, out=ro)
    return ro, np.array([v for _, v in e], np.int32), np.ones(len(e), np.int32)


def trace_count(n, ro, col):
    A = np.zeros((n, n), np.int64)
    for u in range(n):
        A[u, col[ro[u]:ro[u + 1]]] = 1
    return int(np.trace(A @ A @ A)) // 6


@pytest.mark.parametrize("n", [3, 4, 7, 12])
def test_complete_graph(n):
    g = oracle.OracleGraph(n, *sym_csr(n, [(a, b) for a in range(n) for b in range(a + 1, n)]))
    assert g.triangles() == n * (n - 1) * (n - 2) // 6


@pytest.mark.parametrize("n", [3, 4, 9])
def test_cycle(n):
    g = oracle.OracleGraph(n, *sym_csr(n, [(i, (i + 1) % n) for i in range(n)]))
    assert g.triangles() == (1 if n == 3 else 0)


def test_wheel():
    k = 10                       # hub 0 and a rim cycle 1..k
    pairs = [(0, i) for i in range(1, k + 1)] + [(i, i % k + 1) for i in range(1, k + 1)]
    g = oracle.OracleGraph(k + 1, *sym_csr(k + 1, pairs))
    assert g.triangles() == k


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_symmetric_graphs_and_batches(seed):
    W = wl.sym_er(90, 700, 12, seed)
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    assert g.triangles() == trace_count(W.n, W.row_off, W.col) > 0
    for k in range(3):
        b = W.batch(k)
        g.apply(b)
        ro, col, _ = g.csr()
        assert g.triangles() == trace_count(W.n, ro, col)


def test_symmetric_streams_stay_symmetric():
    W = wl.sym_rmat(9, 8, 0.05, 4)
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    for k in range(3):
        b = W.batch(k)
        cnt = g.apply(b)
        assert cnt[0] == b.del_src.size and cnt[2] == b.add_src.size   # all applied
        ro, col, _ = g.csr()
        u = np.repeat(np.arange(W.n), np.diff(ro))
        fwd = set(zip(u.tolist(), col.tolist()))
        assert all((v, x) in fwd for x, v in fwd)
