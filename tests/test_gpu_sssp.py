"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Distances must equal the oracle's bit for bit after sp_sssp_init and after
every batch; parents must satisfy the shortest-path-tree invariants (ties make
parents non-unique); the stores must equal the oracle's edge set (forward)
and its transpose (reverse); the batch counters must equal the oracle's.
"""
import numpy as np
import pytest

import oracle
from oracle.invariants import check_sssp
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
INF = sp.SP_INF


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()


def transpose(n, ro, col, w):
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(ro))
    key = col.astype(np.int64) * n + u
    order = np.argsort(key, kind="stable")
    rro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(col, minlength=n), out=rro[1:])
    return rro, u[order].astype(np.int32), w[order]


def check_all(g, ref, src, store=True):
    d, p = g.get_dist(parent=True)
    want = ref.dijkstra(src)
    np.testing.assert_array_equal(d, want)
    ro, col, w = ref.csr()
    check_sssp(g.n, ro, col, w, src, d, p)
    assert g.m == col.size
    if store:
        for a, b in zip(g.export_csr(), (ro, col, w)):
            np.testing.assert_array_equal(a, b)
        for a, b in zip(g.export_csr(reverse=True), transpose(g.n, ro, col, w)):
            np.testing.assert_array_equal(a, b)
    return d


def run_workload(W, n_batches, store=True, slack=0.25, setup=None):
    """Every batch against the oracle; returns the stats of each batch."""
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    out = []
    with sp.Graph(W.n, W.row_off, W.col, W.w, slack=slack) as g:
        if setup:
            setup(g)
        g.sssp_init(W.source)
        d = check_all(g, ref, W.source, store)
        for k in range(n_batches):
            b = W.batch(k, dist=d if W.tree_fraction else None)
            st = g.apply(b, stats=True)
            cnt = ref.apply(b)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt
            d = check_all(g, ref, W.source, store)
            out.append(st.as_dict())
    return out


def test_tiny_er_ten_batches():
    run_workload(wl.tiny_er(seed=1), 10)


@pytest.mark.parametrize("seed", [2, 3])
def test_tiny_er_other_seeds(seed):
    run_workload(wl.tiny_er(seed=seed), 10)


def test_rmat_scale14_heavy_rows():
    W = wl.rmat(scale=14, batch_frac=0.01, seed=1)
    assert np.diff(W.row_off).max() > 256      # exercises heavy chunks
    run_workload(W, 5)


def test_rmat_scale12_big_batches():
    run_workload(wl.rmat(scale=12, batch_frac=0.05, seed=5), 4)


def test_grid_tree_biased_deletions():
    run_workload(wl.grid(64, 64, batch_frac=0.02, seed=1), 5)


def test_grid_uniform_pair_insertions():
    run_workload(wl.grid(48, 80, batch_frac=0.01, seed=2, insert_kind="uniform"), 4)


def test_slack_zero_forces_relocation_and_pool_growth():
    n = 300
    ro, col, w = wl.er_digraph(n, 1200, 1, 50, seed=8)
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w, slack=0.0) as g:
        g.sssp_init(0)
        rng = np.random.default_rng(0)
        total_reloc = 0
        for k in range(6):
            # pile insertions onto a few rows
            u = rng.integers(0, 5, size=2000).astype(np.int32)
            v = rng.integers(0, n, size=2000).astype(np.int32)
            ww = rng.integers(1, 50, size=2000).astype(np.int32)
            z = np.zeros(0, np.int32)
            st = g.apply_batch(z, z, u, v, ww, stats=True)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == ref.apply_batch(z, z, u, v, ww)
            total_reloc += st.rows_relocated
            check_all(g, ref, 0)
        assert total_reloc > 0
        assert g.info().pool_used_fwd > 0


def test_pool_growth_rerun_keeps_the_invalidation():
    # batches that cut tree edges and pile insertions onto a few rows of a
    # zero-slack graph: the first attempt runs out of pool (its invalidation
    # has already run beside the store update) and the rerun must keep what
    # that invalidation found
    n = 3000
    ro, col, w = wl.er_digraph(n, 6000, 1, 50, seed=11)
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w, slack=0.0) as g:
        g.sssp_init(0)
        rng = np.random.default_rng(3)
        regrows = 0
        for k in range(8):
            d, p = g.get_dist(parent=True)
            kids = [x for x in rng.permutation(n) if p[x] >= 0][:40]
            ds = np.array([p[x] for x in kids], np.int32)
            dd = np.array(kids, np.int32)
            u = rng.integers(0, 16, size=4000).astype(np.int32)
            v = rng.integers(0, n, size=4000).astype(np.int32)
            ww = rng.integers(1, 50, size=4000).astype(np.int32)
            st = g.apply_batch(ds, dd, u, v, ww, stats=True)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == ref.apply_batch(ds, dd, u, v, ww)
            assert st.n_del_applied == len(kids)
            regrows += st.regrows
            check_all(g, ref, 0)
        assert regrows > 0


# ---------------------------------------------------------------- edge cases

def small_graph(seed=4, n=500, m=4000):
    ro, col, w = wl.er_digraph(n, m, 1, 100, seed)
    return n, ro, col, w


def test_empty_batch():
    n, ro, col, w = small_graph()
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(3)
        z = np.zeros(0, np.int32)
        st = g.apply_batch(z, z, z, z, z, stats=True)
        assert st.n_del_applied == st.n_add_applied == 0
        check_all(g, ref, 3)


def test_delete_then_reinsert_restores_distances():
    n, ro, col, w = small_graph()
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(0)
        d0 = g.get_dist()
        u = np.repeat(np.arange(n), np.diff(ro)).astype(np.int32)
        pick = np.random.default_rng(3).choice(col.size, 800, replace=False)
        z = np.zeros(0, np.int32)
        g.apply_batch(u[pick], col[pick], z, z, z)
        ref.apply_batch(u[pick], col[pick], z, z, z)
        check_all(g, ref, 0)
        g.apply_batch(z, z, u[pick], col[pick], w[pick])
        ref.apply_batch(z, z, u[pick], col[pick], w[pick])
        np.testing.assert_array_equal(check_all(g, ref, 0), d0)


def test_delete_all_out_edges_of_source():
    n, ro, col, w = small_graph()
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w) as g:
        src = 7
        g.sssp_init(src)
        v = col[ro[src]:ro[src + 1]]
        u = np.full(v.size, src, np.int32)
        z = np.zeros(0, np.int32)
        g.apply_batch(u, v, z, z, z)
        ref.apply_batch(u, v, z, z, z)
        d = check_all(g, ref, src)
        assert d[src] == 0 and np.all(np.delete(d, src) == INF)


def test_noop_readings_and_duplicates():
    n, ro, col, w = small_graph(seed=6, n=200, m=1500)
    ref = oracle.OracleGraph(n, ro, col, w)
    u_all = np.repeat(np.arange(n), np.diff(ro)).astype(np.int32)
    rng = np.random.default_rng(1)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(0)
        for k in range(5):
            pick = rng.choice(col.size, 60, replace=False)
            du, dv = u_all[pick], col[pick]
            # absent deletions, repeated deletions
            au = rng.integers(0, n, 40).astype(np.int32)
            av = rng.integers(0, n, 40).astype(np.int32)
            del_s = np.concatenate([du, du[:10], au])
            del_d = np.concatenate([dv, dv[:10], av])
            # present insertions, duplicates with different weights,
            # re-insertion of deleted edges with new weights
            iu = np.concatenate([u_all[pick[10:20]], au[:20], au[:20], du[:15]])
            iv = np.concatenate([col[pick[10:20]], av[:20], av[:20], dv[:15]])
            iw = rng.integers(1, 100, iu.size).astype(np.int32)
            st = g.apply_batch(del_s, del_d, iu, iv, iw, stats=True)
            cnt = ref.apply_batch(del_s, del_d, iu, iv, iw)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt
            check_all(g, ref, 0)
            ro2, col2, w2 = ref.csr()
            u_all = np.repeat(np.arange(n), np.diff(ro2)).astype(np.int32)
            col = col2


def test_invalid_batch_leaves_graph_unchanged():
    n, ro, col, w = small_graph()
    ref = oracle.OracleGraph(n, ro, col, w)
    a = lambda *x: np.array(x, np.int32)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(0)
        for args in [(a(0), a(n), a(), a(), a()),
                     (a(), a(), a(1), a(2), a(0)),
                     (a(), a(), a(1), a(2), a(sp.SP_WMAX + 1)),
                     (a(-1), a(2), a(1), a(2), a(5))]:
            rc, _ = g.apply_batch(*args, raise_on_error=False)
            assert rc == sp.SP_EINVAL
            check_all(g, ref, 0)


def test_state_errors_and_invalid_source():
    n, ro, col, w = small_graph()
    with sp.Graph(n, ro, col, w) as g:
        z = np.zeros(0, np.int32)
        rc, _ = g.apply_batch(z, z, z, z, z, raise_on_error=False)
        assert rc == sp.SP_ESTATE
        with pytest.raises(sp.SpError) as e:
            g.get_dist()
        assert e.value.code == sp.SP_ESTATE
        for bad in (-1, n):
            with pytest.raises(sp.SpError) as e:
                g.sssp_init(bad)
            assert e.value.code == sp.SP_EINVAL


def test_create_rejects_bad_csr_and_sorts_unsorted_rows():
    ro = np.array([0, 2, 3, 3], np.int64)
    with pytest.raises(sp.SpError):
        sp.Graph(3, ro, np.array([1, 1, 0], np.int32), np.array([1, 2, 3], np.int32))
    with pytest.raises(sp.SpError):
        sp.Graph(3, ro, np.array([1, 2, 5], np.int32), np.array([1, 2, 3], np.int32))
    with pytest.raises(sp.SpError):
        sp.Graph(3, ro, np.array([1, 2, 0], np.int32), np.array([1, 0, 3], np.int32))
    # unsorted rows are accepted and stored sorted
    n, ro, col, w = small_graph(seed=9, n=300, m=3000)
    perm_col, perm_w = col.copy(), w.copy()
    rng = np.random.default_rng(2)
    for u in range(n):
        s, e = ro[u], ro[u + 1]
        p = rng.permutation(e - s) + s
        perm_col[s:e], perm_w[s:e] = col[p], w[p]
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, perm_col, perm_w) as g:
        g.sssp_init(0)
        check_all(g, ref, 0)


def test_range_error_and_recovery():
    n = 1101
    ro = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    col = np.arange(1, n, dtype=np.int32)
    w = np.full(n - 1, sp.SP_WMAX, dtype=np.int32)
    with sp.Graph(n, ro, col, w) as g:
        with pytest.raises(sp.SpError) as e:
            g.sssp_init(0)
        assert e.value.code == sp.SP_ERANGE
        assert g.info().state == 2
        g.sssp_init(600)      # 500 edges of 2^20 fit
        d = g.get_dist()
        assert d[-1] == 500 * sp.SP_WMAX and np.all(d[:600] == INF)


def test_round_cap_returns_timeout_and_reinit_recovers():
    n = 400
    ro = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    col = np.arange(1, n, dtype=np.int32)
    w = np.ones(n - 1, dtype=np.int32)
    with sp.Graph(n, ro, col, w) as g:
        g.set_limits(max_rounds=5)
        with pytest.raises(sp.SpError) as e:
            g.sssp_init(0)
        assert e.value.code == sp.SP_ETIMEOUT
        lc = g.loop_counters()   # the bound says where it was hit: a round cap
        assert lc["timeout"] == 1 and lc["timeout_site"] == 1 and lc["timeout_index"] == 5
        assert "site 1" in str(e.value)
        z = np.zeros(0, np.int32)
        rc, _ = g.apply_batch(z, z, z, z, z, raise_on_error=False)
        assert rc == sp.SP_ESTATE
        g.set_limits(0, 0)
        g.sssp_init(0)
        np.testing.assert_array_equal(g.get_dist(), np.arange(n))


def test_device_tensor_inputs_and_outputs():
    import torch
    W = wl.tiny_er(seed=7)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    dev = torch.device("cuda")
    with sp.Graph(W.n, torch.from_numpy(W.row_off).to(dev), torch.from_numpy(W.col).to(dev),
                  torch.from_numpy(W.w).to(dev)) as g:
        g.sssp_init(W.source)
        for k in range(3):
            b = W.batch(k)
            t = [torch.from_numpy(x).to(dev) for x in
                 (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w)]
            g.apply_batch(*t)
            ref.apply(b)
            d = torch.empty(W.n, dtype=torch.int32, device=dev)
            p = torch.empty(W.n, dtype=torch.int32, device=dev)
            g.get_dist(out=(d, p))
            torch.cuda.synchronize()
            np.testing.assert_array_equal(d.cpu().numpy(), ref.dijkstra(W.source))
            ro, col, w = ref.csr()
            check_sssp(W.n, ro, col, w, W.source, d.cpu().numpy(), p.cpu().numpy())


def test_worked_example_numbers_on_gpu():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "worked_example_sec3.json")
    fix = json.load(open(path))
    names = fix["vertices"]
    idx = {s: i for i, s in enumerate(names)}
    n = len(names)
    e = sorted((idx[a], idx[b], c) for a, b, c in fix["edges"])
    ro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount([x[0] for x in e], minlength=n), out=ro[1:])
    col = np.array([x[1] for x in e], np.int32)
    w = np.array([x[2] for x in e], np.int32)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(idx[fix["source"]])
        d = g.get_dist()
        for k, val in fix["before"]["paper_dist"].items():
            assert d[idx[k]] == val
        b = fix["both"]
        arr = lambda L, j: np.array([idx[x[j]] if j < 2 else x[j] for x in L], np.int32)
        g.apply_batch(arr(b["del"], 0), arr(b["del"], 1), arr(b["add"], 0), arr(b["add"], 1),
                      arr(b["add"], 2))
        d = g.get_dist()
        for k, val in b["paper_dist"].items():
            assert d[idx[k]] == val


def test_static_recompute_equals_dynamic():
    W = wl.rmat(scale=13, batch_frac=0.02, seed=3)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.sssp_init(W.source)
        for k in range(3):
            g.apply(W.batch(k))
            d_dyn = g.get_dist()
            g.sssp_init(W.source)
            np.testing.assert_array_equal(g.get_dist(), d_dyn)


def test_merge_tiers_hub_rows():
    """A 15,000-edge hub row (chunked tier, in place via scratch and then
    relocated), a 2,000-edge row (block tier) and small rows in one batch."""
    n = 30000
    rng = np.random.default_rng(11)
    edges = {}
    for v in range(2, n, 2):
        edges[(0, v)] = int(rng.integers(1, 100))
    for v in rng.choice(np.arange(2, n), 2000, replace=False):
        edges[(1, int(v))] = int(rng.integers(1, 100))
    for _ in range(60000):
        a, b = int(rng.integers(n)), int(rng.integers(n))
        if a != b and a > 1:
            edges.setdefault((a, b), int(rng.integers(1, 100)))
    keys = sorted(edges)
    u = np.array([k[0] for k in keys], np.int64)
    ro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=ro[1:])
    col = np.array([k[1] for k in keys], np.int32)
    w = np.array([edges[k] for k in keys], np.int32)
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(0)
        check_all(g, ref, 0)
        for k, n_ins in enumerate((800, 6000)):
            evens = np.arange(2, n, 2)
            dels0 = rng.choice(evens, 700, replace=False).astype(np.int32)
            odds = np.arange(3, n, 2)
            ins0 = rng.choice(odds, n_ins, replace=False).astype(np.int32)
            del_s = np.concatenate([np.zeros(700, np.int32), np.ones(50, np.int32)])
            del_d = np.concatenate([dels0, col[ro[1]:ro[1] + 50]])
            add_s = np.concatenate([np.zeros(n_ins, np.int32), np.ones(300, np.int32)])
            add_d = np.concatenate([ins0, rng.choice(odds, 300, replace=False).astype(np.int32)])
            add_w = rng.integers(1, 100, add_s.size).astype(np.int32)
            st = g.apply_batch(del_s, del_d, add_s, add_d, add_w, stats=True)
            cnt = ref.apply_batch(del_s, del_d, add_s, add_d, add_w)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt
            check_all(g, ref, 0)
            ro2, col2, _ = ref.csr()
            ro, col = ro2, col2
        assert g.info().pool_used_fwd > 0      # the hub row moved on the second batch


def test_store_update_strip_cases():
    """The store update's strips: a 40,000-edge row (157 strips) touched in
    its last strip only and then all over; a 10-edge row that gets 400 items
    (more than a strip stages: runs of duplicate insertions,
    delete-and-reinsert, an absent deletion); a 3,000-edge row with 450
    items inside one strip."""
    n = 90000
    rng = np.random.default_rng(21)
    edges = {}
    for v in range(2, 80002, 2):
        edges[(0, v)] = int(rng.integers(1, 100))
    for v in rng.choice(np.arange(2, n), 10, replace=False):
        edges[(1, int(v))] = int(rng.integers(1, 100))
    for k in range(1, 3001):
        edges[(2, 3 * k)] = int(rng.integers(1, 100))
    for _ in range(80000):
        a, b = int(rng.integers(3, n)), int(rng.integers(n))
        if a != b:
            edges.setdefault((a, b), int(rng.integers(1, 100)))
    keys = sorted(edges)
    u = np.array([k[0] for k in keys], np.int64)
    ro = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(u, minlength=n), out=ro[1:])
    col = np.array([k[1] for k in keys], np.int32)
    w = np.array([edges[k] for k in keys], np.int32)
    ref = oracle.OracleGraph(n, ro, col, w)

    def apply(g, ds, dd, as_, ad, aw):
        ds, dd, as_, ad, aw = (np.asarray(x, np.int32) for x in (ds, dd, as_, ad, aw))
        st = g.apply_batch(ds, dd, as_, ad, aw, stats=True)
        cnt = ref.apply_batch(ds, dd, as_, ad, aw)
        assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                st.n_add_present) == cnt
        check_all(g, ref, 0)

    with sp.Graph(n, ro, col, w) as g:
        g.sssp_init(0)
        check_all(g, ref, 0)
        # row 0, last strip only: five deletions, three insertions
        row0 = col[ro[0]:ro[1]]
        apply(g, [0] * 5, row0[-5:], [0] * 3, [80003, 79999, 80001], [5, 6, 7])
        # row 1: 300 new edges, 60 duplicates of them, delete 5, reinsert 3
        row1 = col[ro[1]:ro[2]]
        absent = np.setdiff1d(np.arange(3, n), np.concatenate([row1, [1]]))
        new1 = rng.choice(absent, 300, replace=False)
        dup = rng.choice(new1, 60)
        add_d = np.concatenate([new1, dup, row1[:3]])
        add_w = rng.integers(1, 100, add_d.size)
        del_d = np.concatenate([row1[:5], [absent[-1]]])
        apply(g, [1] * del_d.size, del_d, [1] * add_d.size, add_d, add_w)
        # row 2: one strip (entries 1280..1535) gets 450 items
        row2 = np.arange(3, 9003, 3)
        span = row2[1280:1536]
        gone = rng.choice(span, 200, replace=False)
        back = gone[:50]
        fresh = rng.choice(np.arange(span[0] + 1, span[-1], 3), 150, replace=False)
        add_d = np.concatenate([back, fresh, fresh[:50]])
        add_w = rng.integers(1, 100, add_d.size)
        apply(g, [2] * gone.size, gone, [2] * add_d.size, add_d, add_w)
        # row 0 all over: 2,000 deletions and 2,000 insertions
        row0 = ref.csr()[1][ref.csr()[0][0]:ref.csr()[0][1]]
        dels = rng.choice(row0, 2000, replace=False)
        ins = rng.choice(np.arange(3, 80003, 2), 2000, replace=False)
        apply(g, [0] * 2000, dels, [0] * 2000, ins, rng.integers(1, 100, 2000))


@pytest.mark.parametrize("delta", [1, 300, 2500])
def test_grid_near_far_matches_oracle(delta):
    W = wl.grid(48, 48, batch_frac=0.03, seed=4)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.set_delta(delta)
        g.sssp_init(W.source)
        d = check_all(g, ref, W.source, store=False)
        for k in range(4):
            b = W.batch(k, dist=d)
            g.apply(b)
            ref.apply(b)
            d = check_all(g, ref, W.source, store=False)


@pytest.mark.parametrize("delta", [7, 60])
def test_rmat_near_far_matches_oracle(delta):
    W = wl.rmat(scale=12, batch_frac=0.02, seed=8)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.set_delta(delta)
        g.sssp_init(W.source)
        check_all(g, ref, W.source, store=False)
        for k in range(4):
            b = W.batch(k)
            g.apply(b)
            ref.apply(b)
            check_all(g, ref, W.source, store=False)


def test_near_far_static_equals_plain_and_does_less_work():
    W = wl.grid(128, 128, seed=6)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        plain = g.sssp_init(W.source, stats=True)
        d_plain = g.get_dist()
        g.set_delta(1500)
        nf = g.sssp_init(W.source, stats=True)
        np.testing.assert_array_equal(g.get_dist(), d_plain)
        assert nf.relaxed_edges < plain.relaxed_edges


# ------------------------------------------- invalidation: rounds vs jumping

@pytest.mark.parametrize("make,deep", [
    (lambda: wl.grid(96, 96, batch_frac=0.01, seed=3), True),
    (lambda: wl.rmat(scale=13, batch_frac=0.02, seed=4), False),
    (lambda: wl.tiny_er(seed=5), False),
], ids=["grid-tree-biased", "rmat13", "er1k"])
def test_invalidation_switch_same_affected_set(make, deep):
    """Frontier rounds only, pointer jumping at once, and switches after 1
    and 3 rounds invalidate the same vertices (the descendants of the cut
    vertices), and every batch matches the oracle."""
    runs = {}
    for sw in (-1, 0, 1, 3):
        W = make()
        runs[sw] = run_workload(W, 4, store=False,
                                setup=lambda g, sw=sw: g.set_inval_switch(sw))
    base = [st["affected"] for st in runs[-1]]
    assert sum(base) > 0
    for sw, sts in runs.items():
        assert [st["affected"] for st in sts] == base, sw
    if deep:   # deep subtrees: log2(depth) passes instead of one round per level
        assert (sum(st["rounds_inval"] for st in runs[0]) <
                sum(st["rounds_inval"] for st in runs[-1]))


# ------------------------------------------------ single-block push rounds

@pytest.mark.parametrize("make", [
    lambda: wl.grid(80, 80, batch_frac=0.01, seed=6),
    lambda: wl.rmat(scale=13, batch_frac=0.01, seed=7),
], ids=["grid", "rmat13"])
@pytest.mark.parametrize("bound,delta", [(0, 0), (64, 0), (4096, 0), (4096, 300), (512, 40)])
def test_local_rounds_any_bound_matches_oracle(make, bound, delta):
    """Push rounds run by one block (frontier bounds 64 .. 4096 edges, with
    and without near-far ordering) give the oracle's distances."""
    def setup(g):
        g.set_local_rounds(bound)
        g.set_delta(delta)
    run_workload(make(), 3, store=False, setup=setup)


# ------------------------------------------------- cached batch CUDA graphs

@pytest.mark.parametrize("make,slack", [
    (lambda: wl.tiny_er(seed=8), 0.25),
    (lambda: wl.rmat(scale=13, batch_frac=0.01, seed=9), 0.25),
    (lambda: wl.rmat(scale=12, batch_frac=0.02, seed=10), 0.0),   # relocations, pool growth
])
def test_repeated_batch_shapes_replay_a_cached_graph(make, slack):
    """On a stream of its own the graph replays repeated batch shapes as a
    CUDA graph; every batch still matches the oracle, with stats on and off
    (which changes the shape and forces a new capture), and around a
    rejected batch."""
    import torch
    W = make()
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, slack=slack, stream=st)
    try:
        g.sssp_init(W.source)
        for k in range(8):
            b = W.batch(k)
            if k == 5:    # a rejected batch of the same shape changes nothing
                bad = wl.Batch(b.del_src, b.del_dst, b.add_src, b.add_dst,
                               np.zeros_like(b.add_w))
                rc, _ = g.apply_batch(bad.del_src, bad.del_dst, bad.add_src, bad.add_dst,
                                      bad.add_w, raise_on_error=False)
                assert rc == sp.SP_EINVAL
            st_ = g.apply(b, stats=(k % 3 == 2))
            cnt = ref.apply(b)
            if st_ is not None:
                assert (st_.n_del_applied, st_.n_del_absent, st_.n_add_applied,
                        st_.n_add_present) == cnt
            check_all(g, ref, W.source, store=(k % 2 == 0))
    finally:
        g.close()


def test_page_locked_host_batches_and_distances():
    """Page-locked host arrays are gathered by a kernel (batch) and written
    in place by the kernel (distances); the results equal the oracle's and
    those of the copy-engine path for pageable arrays of the same batches."""
    import torch
    W = wl.rmat(scale=13, batch_frac=0.01, seed=7)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)

    def pinned(x):
        t = torch.empty(x.size, dtype=torch.int32, pin_memory=True)
        t.numpy()[:] = x
        return t

    with sp.Graph(W.n, W.row_off, W.col, W.w) as g, \
            sp.Graph(W.n, W.row_off, W.col, W.w) as h:
        g.sssp_init(W.source)
        h.sssp_init(W.source)
        dt = torch.empty(W.n, dtype=torch.int32, pin_memory=True)
        pt = torch.empty(W.n, dtype=torch.int32, pin_memory=True)
        for k in range(4):   # the same shape repeats: replayed graphs too
            b = W.batch(k)
            keep = [pinned(x) for x in (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w)]
            st = g.apply_batch(*[t.numpy() for t in keep], stats=True)
            h.apply(b)
            cnt = ref.apply(b)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt
            dt.fill_(-7)
            pt.fill_(-7)
            g.get_dist(out=(dt.numpy(), pt.numpy()))
            want = ref.dijkstra(W.source)
            np.testing.assert_array_equal(dt.numpy(), want)
            ro, col, w = ref.csr()
            check_sssp(g.n, ro, col, w, W.source, dt.numpy(), pt.numpy())
            np.testing.assert_array_equal(h.get_dist(), want)
            for a, c in zip(g.export_csr(), (ro, col, w)):
                np.testing.assert_array_equal(a, c)


@pytest.mark.parametrize("where", ["device", "page-locked", "pageable"])
def test_apply_batch_get_returns_the_repaired_distances(where):
    """One call applies a batch and hands out the distances and parents after
    it (device tensors, page-locked or pageable host arrays); they equal the
    oracle's, and a later get_dist agrees."""
    import torch
    W = wl.rmat(scale=12, batch_frac=0.02, seed=11)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    if where == "device":
        d_out = torch.empty(W.n, dtype=torch.int32, device="cuda")
        p_out = torch.empty(W.n, dtype=torch.int32, device="cuda")
    elif where == "page-locked":
        d_out = torch.empty(W.n, dtype=torch.int32, pin_memory=True).numpy()
        p_out = torch.empty(W.n, dtype=torch.int32, pin_memory=True).numpy()
    else:
        d_out = np.empty(W.n, np.int32)
        p_out = np.empty(W.n, np.int32)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.sssp_init(W.source)
        for k in range(4):   # the same shape repeats: replayed graphs too
            b = W.batch(k)
            arrs = (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w)
            if where == "device":
                arrs = [torch.from_numpy(x).cuda() for x in arrs]
            g.apply_batch_get(*arrs, d_out, p_out if k % 2 else None)
            ref.apply(b)
            want = ref.dijkstra(W.source)
            d = d_out.cpu().numpy() if where == "device" else d_out
            np.testing.assert_array_equal(d, want)
            if k % 2:
                p = p_out.cpu().numpy() if where == "device" else p_out
                ro, col, w = ref.csr()
                check_sssp(g.n, ro, col, w, W.source, d, p)
            np.testing.assert_array_equal(g.get_dist(), want)
        with pytest.raises(sp.SpError):
            g.apply_batch_get(*arrs, np.empty(W.n - 1, np.int32))


def test_device_outputs_must_be_device_memory():
    """Outputs declared as device arrays (out_on_device = 1) that are host
    memory are refused with SP_EINVAL before anything runs; the graph keeps
    working."""
    import ctypes
    W = wl.tiny_er(seed=5)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    lib = sp.load()
    host = np.empty(max(W.n + 1, W.m), np.int64)
    hp = host.ctypes.data_as(ctypes.c_void_p)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.sssp_init(W.source)
        assert lib.sp_get_dist(g._h, hp, None, 1) == sp.SP_EINVAL
        assert lib.sp_export_csr(g._h, 0, hp, hp, hp, 1) == sp.SP_EINVAL
        b = W.batch(0)
        assert lib.sp_apply_batch_get(
            g._h, b.del_src.size, b.del_src.ctypes.data_as(ctypes.c_void_p),
            b.del_dst.ctypes.data_as(ctypes.c_void_p), b.add_src.size,
            b.add_src.ctypes.data_as(ctypes.c_void_p), b.add_dst.ctypes.data_as(ctypes.c_void_p),
            b.add_w.ctypes.data_as(ctypes.c_void_p), 0, hp, None, 1, None) == sp.SP_EINVAL
        # nothing changed: the same batch still applies and matches the oracle
        g.apply(b)
        ref.apply(b)
        np.testing.assert_array_equal(g.get_dist(), ref.dijkstra(W.source))
