"""Seeded input generators: sizes, validity and determinism."""
import numpy as np

from paper_2507_11094_gb300 import workloads as wl


def _check_simple(n, ro, col, w, wlo, whi):
    assert ro[0] == 0 and np.all(np.diff(ro) >= 0) and ro[-1] == col.size
    u = np.repeat(np.arange(n), np.diff(ro))
    assert np.all(u != col), "self-loop"
    keys = u.astype(np.int64) * n + col
    assert np.all(np.diff(keys) > 0), "rows not sorted / duplicates"
    assert w.min() >= wlo and w.max() <= whi


def test_er_exact_size_and_determinism():
    a = wl.er_digraph(1024, 8192, 1, 100, seed=1)
    b = wl.er_digraph(1024, 8192, 1, 100, seed=1)
    _check_simple(1024, *a, 1, 100)
    assert a[1].size == 8192
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_rmat_exact_size_and_skew():
    ro, col, w, _ = wl.rmat_digraph(14, 16 << 14, 1, 100, seed=3)
    _check_simple(1 << 14, ro, col, w, 1, 100)
    assert col.size == 16 << 14
    deg = np.diff(ro)
    assert deg.max() > 20 * deg.mean()      # heavy-tailed out-degrees


def test_grid_edge_count_and_neighbours():
    r, c = 17, 29
    ro, col, w = wl.grid_digraph(r, c, 1, 1000, seed=2)
    _check_simple(r * c, ro, col, w, 1, 1000)
    assert col.size == 4 * r * c - 2 * r - 2 * c
    u = np.repeat(np.arange(r * c), np.diff(ro))
    ui, uj = np.divmod(u, c)
    vi, vj = np.divmod(col, c)
    assert np.all(np.abs(ui - vi) + np.abs(uj - vj) == 1)
    # 4096 x 4096 has 2*2*4096*4095 directed edges
    assert 4 * 4096 * 4096 - 4 * 4096 == 67092480


def test_batches_delete_existing_and_insert_new():
    W = wl.tiny_er(seed=1)
    n = W.n
    keys = set((W.stream.keys).tolist())
    for k in range(10):
        b = W.batch(k)
        assert b.del_src.size == 32 and b.add_src.size == 32
        dk = (b.del_src.astype(np.int64) * n + b.del_dst).tolist()
        ak = (b.add_src.astype(np.int64) * n + b.add_dst).tolist()
        assert all(x in keys for x in dk) and len(set(dk)) == 32
        assert all(x not in keys for x in ak) and len(set(ak)) == 32
        assert np.all(b.add_src != b.add_dst)
        assert b.add_w.min() >= 1 and b.add_w.max() <= 100
        keys = (keys - set(dk)) | set(ak)
        assert keys == set(W.stream.keys.tolist())


def test_batches_deterministic():
    a = wl.tiny_er(seed=4)
    b = wl.tiny_er(seed=4)
    for k in range(3):
        x, y = a.batch(k), b.batch(k)
        for f in ("del_src", "del_dst", "add_src", "add_dst", "add_w"):
            np.testing.assert_array_equal(getattr(x, f), getattr(y, f))


def test_tree_biased_deletions_take_tight_edges():
    W = wl.grid(32, 32, batch_frac=0.05, seed=1)
    # any distance array works for the selection rule; use hop counts
    i, j = np.divmod(np.arange(W.n), 32)
    dist = (i + j).astype(np.int64)
    st = W.stream
    st.wts[:] = 1
    b = W.batch(0, dist=dist)
    d_u, d_v = dist[b.del_src], dist[b.del_dst]
    tight = d_u + 1 == d_v
    assert tight.sum() >= b.del_src.size // 2
