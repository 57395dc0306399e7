"""The invariant checker must accept oracle answers and reject planted mistakes."""
import numpy as np
import pytest

from oracle.invariants import InvariantError, check_sssp
from paper_2507_11094_gb300 import workloads as wl

INF = 2147483647 // 2


def _tree_from_dist(n, ro, col, w, dist, src):
    """Some valid parent array: for each reachable v, the smallest-id tight
    in-neighbour (test helper, independent of any product code)."""
    parent = np.full(n, -1, np.int64)
    deg = np.diff(ro)
    u = np.repeat(np.arange(n), deg)
    tight = (dist[u] < INF) & (dist[u] + w == dist[col])
    for uu, vv in sorted(zip(u[tight], col[tight]), key=lambda t: (t[1], t[0])):
        if vv != src and parent[vv] == -1:
            parent[vv] = uu
    return parent


@pytest.fixture(scope="module")
def case(oracle_mod):
    ro, col, w = wl.er_digraph(300, 1200, 1, 20, seed=4)
    d = oracle_mod.OracleGraph(300, ro, col, w).dijkstra(0).astype(np.int64)
    p = _tree_from_dist(300, ro, col, w, d, 0)
    return ro, col, w, d, p


def test_accepts_oracle_answer(case):
    ro, col, w, d, p = case
    check_sssp(300, ro, col, w, 0, d, p)


@pytest.mark.parametrize("mutate", [
    "src_dist", "src_parent", "lower_one", "raise_one", "parent_not_edge",
    "parent_not_tight", "unreach_parent", "fake_unreachable",
])
def test_rejects_planted_mistakes(case, mutate):
    ro, col, w, d, p = case
    d, p = d.copy(), p.copy()
    reach = np.nonzero((d < INF) & (np.arange(300) != 0))[0]
    v = int(reach[len(reach) // 2])
    if mutate == "src_dist":
        d[0] = 1
    elif mutate == "src_parent":
        p[0] = 3
    elif mutate == "lower_one":
        d[v] -= 1
    elif mutate == "raise_one":
        d[v] += 1
    elif mutate == "parent_not_edge":
        nbr_in = set(np.repeat(np.arange(300), np.diff(ro))[col == v])
        p[v] = next(x for x in range(300) if x not in nbr_in and x != v)
    elif mutate == "parent_not_tight":
        deg = np.diff(ro)
        u = np.repeat(np.arange(300), deg)
        cand = [int(x) for x, y, ww in zip(u, col, w)
                if y == v and d[x] + ww != d[v] and d[x] < INF]
        if not cand:
            pytest.skip("no non-tight in-edge at this vertex")
        p[v] = cand[0]
    elif mutate == "unreach_parent":
        un = np.nonzero(d >= INF)[0]
        if un.size == 0:
            pytest.skip("all reachable")
        p[un[0]] = 0
    elif mutate == "fake_unreachable":
        d[v] = INF
        p[v] = -1
    with pytest.raises(InvariantError):
        check_sssp(300, ro, col, w, 0, d, p)
