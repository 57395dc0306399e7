"""GPU parity of the dynamic triangle count (sp_tc_*) against the oracle's
staticTC on the same edge set: exact integers after sp_tc_init and after
every batch."""
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


WORKLOADS = {
    "sym-er": lambda: wl.sym_er(1024, 6000, 64, 3),
    "sym-rmat12": lambda: wl.sym_rmat(12, 8, 0.02, 5),
    "sym-rmat10-big-batches": lambda: wl.sym_rmat(10, 8, 0.2, 6),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_dynamic_triangle_count(name):
    W = WORKLOADS[name]()
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        assert g.tc_init() == ref.triangles() > 0
        for k in range(5):
            b = W.batch(k)
            cnt = ref.apply(b)
            c, st = g.tc_apply(b, stats=True)
            assert (st.n_del_applied, st.n_del_absent, st.n_add_applied,
                    st.n_add_present) == cnt
            assert c == ref.triangles()
        for x, y in zip(g.export_csr(), ref.csr()):
            np.testing.assert_array_equal(x, y)
        assert g.tc_init() == c


def complete(n):
    pairs = [(a, b) for a in range(n) for b in range(n) if a != b]
    ro = np.zeros(n + 1, np.int64)
    for u, _ in pairs:
        ro[u + 1] += 1
    np.cumsum(ro, out=ro)
    return ro, np.array([v for _, v in pairs], np.int32), np.ones(len(pairs), np.int32)


def test_complete_graph_delete_and_restore_edges():
    n = 12
    ro, col, w = complete(n)
    with sp.Graph(n, ro, col, w) as g:
        assert g.tc_init() == n * (n - 1) * (n - 2) // 6
        # delete a triangle's three edges (both directions) in one batch:
        # every triangle through them loses 1, 2 or 3 updated edges
        ds = np.array([0, 1, 1, 2, 0, 2], np.int32)
        dd = np.array([1, 0, 2, 1, 2, 0], np.int32)
        z = np.zeros(0, np.int32)
        c = g.tc_apply_batch(ds, dd, z, z, z)
        ref = oracle.OracleGraph(n, *g.export_csr())
        assert c == ref.triangles() == 220 - 1 - 3 * (n - 3)
        c = g.tc_apply_batch(z, z, ds, dd, np.ones(6, np.int32))
        assert c == 220


def test_asymmetric_graph_and_batch_are_rejected():
    n = 5
    ro = np.array([0, 1, 2, 2, 2, 2], np.int64)   # 0 -> 1, 1 -> 0 ... and 1 -> 2 only
    col = np.array([1, 0], np.int32)
    ro2 = np.array([0, 1, 3, 3, 3, 3], np.int64)
    col2 = np.array([1, 0, 2], np.int32)
    with sp.Graph(n, ro2, col2, np.ones(3, np.int32)) as g:
        with pytest.raises(sp.SpError) as e:
            g.tc_init()
        assert e.value.code == sp.SP_EINVAL
    with sp.Graph(n, ro, col, np.ones(2, np.int32)) as g:
        assert g.tc_init() == 0
        m = g.m
        with pytest.raises(sp.SpError) as e:   # 2 -> 3 without 3 -> 2
            g.tc_apply_batch(np.zeros(0, np.int32), np.zeros(0, np.int32),
                             np.array([2], np.int32), np.array([3], np.int32),
                             np.array([1], np.int32))
        assert e.value.code == sp.SP_EINVAL
        assert g.m == m


def test_counts_states():
    W = wl.sym_er(300, 1500, 8, 7)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        with pytest.raises(sp.SpError) as e:
            g.tc_apply(W.batch(0))
        assert e.value.code == sp.SP_ESTATE
        g.sssp_init(0)
        g.tc_init()
        g.apply(W.batch(1))                          # an SSSP batch changes edges
        with pytest.raises(sp.SpError) as e:
            g.tc_apply(W.batch(2))
        assert e.value.code == sp.SP_ESTATE
        ref = oracle.OracleGraph(W.n, *g.export_csr())
        assert g.tc_init() == ref.triangles()
