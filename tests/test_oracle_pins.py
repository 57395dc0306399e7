"""Pins for the CPU oracle: checks against things other than itself.

The oracle (oracle/oracle.c) is the plain definition: after each batch,
shortest-path distances by Dijkstra.  These tests pin it to
  * independent algorithms written here (Bellman-Ford, Floyd-Warshall, BFS),
  * a library routine (scipy.sparse.csgraph.dijkstra),
  * closed forms (uniform grid, path, star),
  * the batch semantics the paper fixes (deletions before insertions, DynSSSP
    driver, Section 3.2) and the readings for its silent cases,
  * the numbers of the paper's worked example (Section 3.1) and the diff-CSR
    example's edge set (Section 3.5),
  * the invariant checker, which must reject planted mistakes.
"""
import collections
import json
import os

import numpy as np
import pytest

from paper_2507_11094_gb300 import workloads as wl

INF = 2147483647 // 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- references

def bellman_ford(n, row_off, col, w, src):
    """Textbook Bellman-Ford: n-1 rounds of relaxing every edge (numpy)."""
    deg = np.diff(row_off)
    u = np.repeat(np.arange(n), deg)
    v = col.astype(np.int64)
    wt = w.astype(np.int64)
    d = np.full(n, np.iinfo(np.int64).max // 4, dtype=np.int64)
    d[src] = 0
    for _ in range(max(n - 1, 1)):
        cand = d[u] + wt
        nd = d.copy()
        np.minimum.at(nd, v, cand)
        if np.array_equal(nd, d):
            break
        d = nd
    big = np.iinfo(np.int64).max // 4
    return np.where(d >= big, INF, d)


def floyd_warshall(n, row_off, col, w, src):
    """All-pairs Floyd-Warshall on a dense matrix; returns row src."""
    big = np.iinfo(np.int64).max // 4
    D = np.full((n, n), big, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for uu in range(n):
        for e in range(row_off[uu], row_off[uu + 1]):
            D[uu, col[e]] = min(D[uu, col[e]], w[e])
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    r = D[src]
    return np.where(r >= big, INF, r)


def bfs_reachable(n, row_off, col, src):
    seen = np.zeros(n, dtype=bool)
    seen[src] = True
    q = collections.deque([src])
    while q:
        x = q.popleft()
        for e in range(row_off[x], row_off[x + 1]):
            y = col[e]
            if not seen[y]:
                seen[y] = True
                q.append(y)
    return seen


def scipy_dist(n, row_off, col, w, src):
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    A = sp.csr_matrix((w.astype(np.float64), col, row_off), shape=(n, n))
    d = cg.dijkstra(A, directed=True, indices=src)
    return np.where(np.isinf(d), INF, d).astype(np.int64)


def random_digraph(rng, n, m, wmax, self_loops=False):
    m = min(m, n * (n - 1))
    keys = set()
    while len(keys) < m:
        a, b = int(rng.integers(n)), int(rng.integers(n))
        if a != b or self_loops:
            keys.add(a * n + b)
    keys = np.array(sorted(keys), dtype=np.int64)
    u, v = keys // n, (keys % n).astype(np.int32)
    ro = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=ro[1:])
    w = rng.integers(1, wmax + 1, size=keys.size).astype(np.int32)
    return ro, v, w


# ---------------------------------------------------------------- Dijkstra

def test_dijkstra_equals_bellman_ford_on_many_random_digraphs(oracle_mod):
    rng = np.random.default_rng(7)
    for t in range(1000):
        n = int(rng.integers(1, 120))
        m = int(rng.integers(0, 4 * n + 1))
        ro, col, w = random_digraph(rng, n, m, int(rng.choice([1, 3, 100, 1 << 20])))
        src = int(rng.integers(n))
        g = oracle_mod.OracleGraph(n, ro, col, w)
        d = g.dijkstra(src)
        np.testing.assert_array_equal(d, bellman_ford(n, ro, col, w, src),
                                      err_msg=f"case {t}")


def test_dijkstra_equals_floyd_warshall_tiny(oracle_mod):
    rng = np.random.default_rng(11)
    for t in range(200):
        n = int(rng.integers(1, 64))
        m = int(rng.integers(0, 3 * n + 1))
        ro, col, w = random_digraph(rng, n, m, 50)
        src = int(rng.integers(n))
        d = oracle_mod.OracleGraph(n, ro, col, w).dijkstra(src)
        np.testing.assert_array_equal(d, floyd_warshall(n, ro, col, w, src),
                                      err_msg=f"case {t}")


def test_dijkstra_equals_scipy_on_er_and_rmat(oracle_mod):
    for ro, col, w, n in [
        wl.er_digraph(3000, 20000, 1, 100, seed=3) + (3000,),
        wl.rmat_digraph(12, 16 << 12, 1, 100, seed=4)[:3] + (1 << 12,),
    ]:
        src = wl.max_out_degree_source(ro)
        d = oracle_mod.OracleGraph(n, ro, col, w).dijkstra(src)
        np.testing.assert_array_equal(d, scipy_dist(n, ro, col, w, src))


def test_self_loops_never_shorten(oracle_mod):
    rng = np.random.default_rng(5)
    ro, col, w = random_digraph(rng, 40, 120, 20, self_loops=True)
    d = oracle_mod.OracleGraph(40, ro, col, w).dijkstra(0)
    np.testing.assert_array_equal(d, bellman_ford(40, ro, col, w, 0))


def test_closed_form_uniform_grid_from_corner(oracle_mod):
    rows, cols, c = 37, 23, 7
    ro, col, _ = wl.grid_digraph(rows, cols, 1, 1, seed=0)
    w = np.full(col.size, c, dtype=np.int32)
    d = oracle_mod.OracleGraph(rows * cols, ro, col, w).dijkstra(0)
    i, j = np.divmod(np.arange(rows * cols), cols)
    np.testing.assert_array_equal(d, c * (i + j))


def test_closed_form_path_prefix_sums_and_unreachable_prefix(oracle_mod):
    n = 500
    rng = np.random.default_rng(2)
    w = rng.integers(1, 1000, size=n - 1).astype(np.int32)
    ro = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    col = np.arange(1, n, dtype=np.int32)
    g = oracle_mod.OracleGraph(n, ro, col, w)
    np.testing.assert_array_equal(g.dijkstra(0),
                                  np.concatenate([[0], np.cumsum(w)]))
    # from the middle, the vertices before it are unreachable
    d = g.dijkstra(200)
    assert np.all(d[:200] == INF)
    np.testing.assert_array_equal(d[200:],
                                  np.concatenate([[0], np.cumsum(w[200:])]))


def test_closed_form_star(oracle_mod):
    n = 1000
    rng = np.random.default_rng(3)
    w = rng.integers(1, 100, size=n - 1).astype(np.int32)
    ro = np.concatenate([[0], np.full(n, n - 1)]).astype(np.int64)
    col = np.arange(1, n, dtype=np.int32)
    d = oracle_mod.OracleGraph(n, ro, col, w).dijkstra(0)
    np.testing.assert_array_equal(d, np.concatenate([[0], w]))


def test_unreachable_iff_not_found_by_bfs(oracle_mod):
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = int(rng.integers(2, 300))
        ro, col, w = random_digraph(rng, n, int(rng.integers(0, 2 * n)), 9)
        src = int(rng.integers(n))
        d = oracle_mod.OracleGraph(n, ro, col, w).dijkstra(src)
        np.testing.assert_array_equal(d < INF, bfs_reachable(n, ro, col, src))


def test_range_error_when_distance_reaches_inf(oracle_mod):
    # a path of 1100 edges of weight 2^20 exceeds INT_MAX/2
    n = 1101
    ro = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    col = np.arange(1, n, dtype=np.int32)
    w = np.full(n - 1, 1 << 20, dtype=np.int32)
    g = oracle_mod.OracleGraph(n, ro, col, w)
    with pytest.raises(oracle_mod.OracleError) as e:
        g.dijkstra(0)
    assert e.value.code == oracle_mod.ERANGE


def test_rejects_bad_graphs(oracle_mod):
    ro = np.array([0, 2, 2], dtype=np.int64)
    for col, w in [([1, 1], [1, 1]),          # duplicate edge
                   ([1, 2], [1, 1]),          # id out of range
                   ([0, 1], [0, 1]),          # weight 0
                   ([0, 1], [1, (1 << 20) + 1])]:
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.OracleGraph(2, ro, np.array(col, np.int32),
                                   np.array(w, np.int32))


# ---------------------------------------------------------------- batches

def _er(oracle_mod, seed=1):
    ro, col, w = wl.er_digraph(400, 3000, 1, 100, seed)
    return ro, col, w, oracle_mod.OracleGraph(400, ro, col, w)


def test_empty_batch_changes_nothing(oracle_mod):
    ro, col, w, g = _er(oracle_mod)
    d0 = g.dijkstra(0)
    z = np.zeros(0, np.int32)
    assert g.apply_batch(z, z, z, z, z) == (0, 0, 0, 0)
    np.testing.assert_array_equal(g.dijkstra(0), d0)
    for a, b in zip(g.csr(), (ro, col, w)):
        np.testing.assert_array_equal(a, b)


def test_delete_then_reinsert_same_weights_restores(oracle_mod):
    ro, col, w, g = _er(oracle_mod)
    d0 = g.dijkstra(0)
    rng = np.random.default_rng(1)
    pick = rng.choice(col.size, 300, replace=False)
    u = np.repeat(np.arange(400), np.diff(ro))[pick].astype(np.int32)
    v, ww = col[pick], w[pick]
    z = np.zeros(0, np.int32)
    assert g.apply_batch(u, v, z, z, z) == (300, 0, 0, 0)
    assert g.m == col.size - 300
    assert g.apply_batch(z, z, u, v, ww) == (0, 0, 300, 0)
    np.testing.assert_array_equal(g.dijkstra(0), d0)
    for a, b in zip(g.csr(), (ro, col, w)):
        np.testing.assert_array_equal(a, b)


def test_insert_only_equals_dijkstra_on_union(oracle_mod):
    ro, col, w, g = _er(oracle_mod)
    st = wl.BatchStream(400, ro, col, w, 1, 100, "uniform")
    b = st.next(0, 500, seed=5)
    g.apply(b)
    ro2, col2, w2 = st.csr()
    np.testing.assert_array_equal(g.dijkstra(0), scipy_dist(400, ro2, col2, w2, 0))


def test_delete_all_out_edges_of_source(oracle_mod):
    ro, col, w, g = _er(oracle_mod)
    src = 5
    v = col[ro[src]:ro[src + 1]]
    u = np.full(v.size, src, np.int32)
    z = np.zeros(0, np.int32)
    g.apply_batch(u, v, z, z, z)
    d = g.dijkstra(src)
    assert d[src] == 0 and np.all(np.delete(d, src) == INF)


def test_noop_readings_counted(oracle_mod):
    # 0->1 (5), 1->2 (5)
    ro = np.array([0, 1, 2, 2], np.int64)
    col = np.array([1, 2], np.int32)
    w = np.array([5, 5], np.int32)
    g = oracle_mod.OracleGraph(3, ro, col, w)
    a = lambda *x: np.array(x, np.int32)
    # absent deletion (0->2), repeated deletion of 1->2, present insertion 0->1
    # (keeps weight 5), duplicate insertions of 2->0 (smaller w wins)
    c = g.apply_batch(a(0, 1, 1), a(2, 2, 2), a(0, 2, 2), a(1, 0, 0), a(1, 9, 4))
    assert c == (1, 2, 1, 2)
    ro2, col2, w2 = g.csr()
    np.testing.assert_array_equal(ro2, [0, 1, 1, 2])
    np.testing.assert_array_equal(col2, [1, 0])
    np.testing.assert_array_equal(w2, [5, 4])
    # deleting and inserting one edge in a batch leaves it with the new weight
    c = g.apply_batch(a(0), a(1), a(0), a(1), a(8))
    assert c == (1, 0, 1, 0)
    assert list(g.csr()[2]) == [8, 4]


def test_invalid_batch_leaves_graph_untouched(oracle_mod):
    ro, col, w, g = _er(oracle_mod)
    a = lambda *x: np.array(x, np.int32)
    for args in [(a(0), a(400), a(), a(), a()),
                 (a(), a(), a(0), a(1), a(0)),
                 (a(int(np.repeat(np.arange(400), np.diff(ro))[0])), a(int(col[0])),
                  a(-1), a(1), a(3))]:
        with pytest.raises(oracle_mod.OracleError):
            g.apply_batch(*args)
        assert g.m == col.size


def test_sequence_of_batches_matches_scipy_each_step(oracle_mod):
    W = wl.tiny_er(seed=2)
    g = oracle_mod.OracleGraph(W.n, W.row_off, W.col, W.w)
    for k in range(10):
        b = W.batch(k)
        assert g.apply(b) == (32, 0, 32, 0)
        ro, col, w = W.stream.csr()
        got = g.csr()
        for x, y in zip(got, (ro, col, w)):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(g.dijkstra(W.source),
                                      scipy_dist(W.n, ro, col, w, W.source))


# ---------------------------------------------------------------- the paper

def _named_graph(fix, key):
    names = fix["vertices"]
    idx = {s: i for i, s in enumerate(names)}
    n = len(names)
    e = sorted((idx[a], idx[b], c) for a, b, c in fix[key])
    ro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount([x[0] for x in e], minlength=n), out=ro[1:])
    return (n, idx, ro, np.array([x[1] for x in e], np.int32),
            np.array([x[2] for x in e], np.int32))


def test_worked_example_numbers(oracle_mod):
    with open(os.path.join(GOLDEN, "worked_example_sec3.json")) as f:
        fix = json.load(f)
    n, idx, ro, col, w = _named_graph(fix, "edges")
    s = idx[fix["source"]]
    pairs = lambda L: [np.array([idx[x[0]] for x in L], np.int32),
                       np.array([idx[x[1]] for x in L], np.int32)]

    def run(del_, add_):
        g = oracle_mod.OracleGraph(n, ro, col, w)
        d0 = g.dijkstra(s)
        ds, dd = pairs(del_)
        as_, ad = pairs(add_)
        aw = np.array([x[2] for x in add_], np.int32)
        g.apply_batch(ds, dd, as_, ad, aw)
        return d0, g.dijkstra(s)

    d0, _ = run([], [])
    for k, val in fix["before"]["paper_dist"].items():
        assert d0[idx[k]] == val
    d0, d1 = run([], fix["insert_only"]["add"])
    for k, val in fix["insert_only"]["paper_dist"].items():
        assert d1[idx[k]] == val
    for k in fix["insert_only"]["unchanged"]:
        assert d1[idx[k]] == d0[idx[k]]
    _, d1 = run(fix["delete_only"]["del"], [])
    for k, val in fix["delete_only"]["paper_dist"].items():
        assert d1[idx[k]] == val
    _, d1 = run(fix["both"]["del"], fix["both"]["add"])
    for k, val in fix["both"]["paper_dist"].items():
        assert d1[idx[k]] == val


def test_diffcsr_example_edge_set(oracle_mod):
    with open(os.path.join(GOLDEN, "diffcsr_example_sec3.json")) as f:
        fix = json.load(f)
    n, idx, ro, col, w = _named_graph(fix, "g0_edges")
    assert n == 6 and col.size == 7
    assert ro[idx["C"]] == fix["paper_offsets_C"]
    g = oracle_mod.OracleGraph(n, ro, col, w)
    b = fix["batch"]
    a = lambda L, k: np.array([idx[x[k]] if k < 2 else x[k] for x in L], np.int32)
    assert g.apply_batch(a(b["del"], 0), a(b["del"], 1), a(b["add"], 0),
                         a(b["add"], 1), a(b["add"], 2)) == (1, 0, 1, 0)
    _, idx1, ro1, col1, w1 = _named_graph(fix, "g1_edges")
    for x, y in zip(g.csr(), (ro1, col1, w1)):
        np.testing.assert_array_equal(x, y)
