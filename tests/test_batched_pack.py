"""Host-side packing of many graphs into one handle (no GPU)."""
import numpy as np

from paper_2507_11094_gb300 import batched, workloads as wl


def test_pack_graphs_is_the_disjoint_union():
    gs = [wl.er_digraph(50, 200, 1, 9, seed=1), wl.grid_digraph(4, 5, 1, 9, seed=2),
          wl.er_digraph(30, 90, 1, 9, seed=3)]
    graphs = [(50,) + gs[0], (20,) + gs[1], (30,) + gs[2]]
    p = batched.pack_graphs(graphs, [0, 3, 7])
    assert p.n == 100 and list(p.offsets) == [0, 50, 70, 100]
    assert list(p.sources) == [0, 53, 77]
    for i, (n, ro, col, w) in enumerate(graphs):
        o = p.offsets[i]
        for v in range(n):
            a, b = p.row_off[o + v], p.row_off[o + v + 1]
            np.testing.assert_array_equal(p.col[a:b] - o, col[ro[v]:ro[v + 1]])
            np.testing.assert_array_equal(p.w[a:b], w[ro[v]:ro[v + 1]])
    assert p.row_off[-1] == p.col.size == sum(g[2].size for g in graphs)


def test_pack_batches_offsets_ids():
    gs = [(10,) + wl.er_digraph(10, 30, 1, 9, seed=1), (10,) + wl.er_digraph(10, 30, 1, 9, seed=2)]
    p = batched.pack_graphs(gs, [0, 0])
    b0 = wl.Batch(np.array([1], np.int32), np.array([2], np.int32), np.array([3], np.int32),
                  np.array([4], np.int32), np.array([5], np.int32))
    b1 = wl.Batch(np.array([6], np.int32), np.array([7], np.int32), np.array([8], np.int32),
                  np.array([9], np.int32), np.array([1], np.int32))
    ds, dd, as_, ad, aw = batched.pack_batches(p, [b0, b1])
    assert list(ds) == [1, 16] and list(dd) == [2, 17]
    assert list(as_) == [3, 18] and list(ad) == [4, 19] and list(aw) == [5, 1]
