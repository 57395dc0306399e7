"""Failure detection on the GPU, without a GPU fault.

Bounded waits: every grid-barrier wait of the library's cooperative kernels
ends after the wait bound of sp_set_limits and the call returns SP_ETIMEOUT
with the wait site in the loop counters.  A test hook makes thread block 0
skip its arrival at the barriers of one site, so that every wait of that
barrier runs out: nothing faults or hangs, and the context stays usable.
After a timeout the handle is in SP_ESTATE until sp_sssp_init, which then
gives the oracle's distances on the edge set the batch left (applied when the
bound was hit in the repair, unchanged when it was hit in the batch sort or
count pass, which run before the merge).

Host allocation failures: the binding's allocator refuses chosen device
allocations.  sp_graph_create, sp_reserve and a batch that must grow the
spare pool return SP_ENOMEM, leave the edge set and the distances as they
were, hand back every byte they took, and succeed once the allocator gives
memory again.
"""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

from test_gpu_sssp import check_all

pytestmark = pytest.mark.gpu

SITE_LOOP, SITE_SORT, SITE_COUNT = 2, 4, 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()


def _apply(g, b):
    return g.apply_batch(b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w,
                         raise_on_error=False)


@pytest.mark.parametrize("site", [SITE_LOOP, SITE_SORT, SITE_COUNT])
@pytest.mark.parametrize("stream", [False, True], ids=["sync", "graph-replay"])
def test_missed_barrier_arrival_times_out_and_recovers(site, stream):
    import torch
    W = wl.rmat(scale=13, batch_frac=0.02, seed=11)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    st = torch.cuda.Stream() if stream else None
    g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=st)
    try:
        g.sssp_init(W.source)
        b0 = W.batch(0)
        _apply(g, b0)            # a first batch of this shape (captured on replay)
        ref.apply(b0)
        check_all(g, ref, W.source, store=False)
        g.set_limits(0, 2_000_000)      # 2 ms per wait
        g.inject_missed_arrival(site)
        b1 = W.batch(1)
        rc, _ = _apply(g, b1)
        assert rc == sp.SP_ETIMEOUT
        lc = g.loop_counters()
        assert lc["timeout"] == 2 and lc["timeout_site"] == site, lc
        assert g.info().state == 2
        # SP_ESTATE until a new init; the edge set follows the site
        rc, _ = _apply(g, W.batch(2))
        assert rc == sp.SP_ESTATE
        if site == SITE_LOOP:
            ref.apply(b1)
        g.inject_missed_arrival(0)
        g.set_limits(0, 0)
        g.sssp_init(W.source)
        check_all(g, ref, W.source, store=True)
        for k in (2, 3):         # and the handle keeps working
            b = W.batch(k)
            _apply(g, b)
            ref.apply(b)
            check_all(g, ref, W.source, store=False)
    finally:
        g.close()


def test_tiny_wait_bound_times_out_at_a_barrier():
    """A 1 ns wait bound: some barrier wait of the batch runs out (which one
    depends on arrival order), the call returns SP_ETIMEOUT naming a barrier
    site, and a re-init with the default bound gives the oracle's distances
    on the edge set the batch left."""
    W = wl.grid(96, 96, batch_frac=0.02, seed=5)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.sssp_init(W.source)
        d = g.get_dist()
        g.set_local_rounds(0)
        seen = set()
        for k in range(6):
            g.set_limits(0, 1)
            b = W.batch(k, dist=d)
            rc, _ = _apply(g, b)
            lc = g.loop_counters()
            g.set_limits(0, 0)
            if rc == sp.SP_OK:
                ref.apply(b)
                d = check_all(g, ref, W.source, store=False)
                continue
            assert rc == sp.SP_ETIMEOUT
            assert lc["timeout"] == 2 and lc["timeout_site"] in (2, 3, 4, 5), lc
            seen.add(lc["timeout_site"])
            if lc["timeout_site"] in (2, 3):   # stopped in the repair: merged
                ref.apply(b)
            g.sssp_init(W.source)
            d = check_all(g, ref, W.source, store=True)
        assert seen, "no wait ran out under a 1 ns bound"


def test_missed_arrival_hook_arguments():
    W = wl.tiny_er(seed=2)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        for bad in (1, 3, 6, -1):
            with pytest.raises(sp.SpError):
                g.inject_missed_arrival(bad)


# ----------------------------------------------------- allocation failures

class Refuser:
    """Refuses device allocations once armed: after `after` more successful
    ones, every allocation fails until disarmed."""

    def __init__(self):
        self.after = None
        self.calls = 0
        self.refused = 0

    def __call__(self, nbytes):
        self.calls += 1
        if self.after is None:
            return False
        if self.after > 0:
            self.after -= 1
            return False
        self.refused += 1
        return True


def _held(g):
    return int(g.info().device_bytes)


@pytest.mark.parametrize("after", [0, 1, 3, 7, 15])
def test_create_fails_cleanly_when_allocation_fails(after):
    import torch
    W = wl.rmat(scale=12, batch_frac=0.01, seed=3)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    r = Refuser()
    r.after = after
    with pytest.raises(sp.SpError) as e:
        sp.Graph(W.n, W.row_off, W.col, W.w, refuse_alloc=r)
    assert e.value.code == sp.SP_ENOMEM
    assert r.refused >= 1
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before    # everything handed back
    r.after = None
    with sp.Graph(W.n, W.row_off, W.col, W.w, refuse_alloc=r) as g:   # and it works again
        g.sssp_init(W.source)
        np.testing.assert_array_equal(
            g.get_dist(), oracle.OracleGraph(W.n, W.row_off, W.col, W.w).dijkstra(W.source))


def test_reserve_fails_cleanly_and_recovers():
    W = wl.rmat(scale=12, batch_frac=0.01, seed=4)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    r = Refuser()
    with sp.Graph(W.n, W.row_off, W.col, W.w, refuse_alloc=r) as g:
        g.sssp_init(W.source)
        held = _held(g)
        r.after = 2
        with pytest.raises(sp.SpError) as e:
            g.reserve(4_000_000)
        assert e.value.code == sp.SP_ENOMEM
        assert _held(g) == held
        r.after = None
        check_all(g, ref, W.source, store=True)
        b = W.batch(0)
        g.apply(b)
        ref.apply(b)
        check_all(g, ref, W.source, store=True)
        g.reserve(4_000_000)
        assert _held(g) > held


@pytest.mark.parametrize("beside", [True, False], ids=["inval-beside", "inval-after"])
def test_pool_growth_failure_leaves_graph_unchanged(beside):
    """Zero slack and a batch that cuts tree edges and piles insertions onto
    a few rows: the touched rows must move to the spare pool, which must
    grow.  With the allocator refusing, the batch returns SP_ENOMEM; the edge
    set and the distances are as before (the invalidation that ran beside
    the store update is undone by a recompute); once the allocator gives
    memory again the same batch applies."""
    import torch
    n = 3000
    ro, col, w = wl.er_digraph(n, 6000, 1, 50, seed=11)
    ref = oracle.OracleGraph(n, ro, col, w)
    r = Refuser()
    stream = torch.cuda.Stream()
    g = sp.Graph(n, ro, col, w, slack=0.0, stream=stream, refuse_alloc=r)
    try:
        if not beside:
            g.set_inval_switch(-1)       # frontier rounds after the merge
        g.sssp_init(0)
        d0 = check_all(g, ref, 0, store=True)
        _, p = g.get_dist(parent=True)
        rng = np.random.default_rng(3)
        kids = [x for x in rng.permutation(n) if p[x] >= 0][:40]
        # ~1,700 new edges on each of 32 rows: their relocations alone need
        # more than the initial spare pool (65,536 slots)
        arrs = (np.array([p[x] for x in kids], np.int32), np.array(kids, np.int32),
                rng.integers(0, 32, size=80000).astype(np.int32),
                rng.integers(0, n, size=80000).astype(np.int32),
                rng.integers(1, 50, size=80000).astype(np.int32))
        with torch.cuda.stream(stream):  # device inputs: no staging buffers to grow
            tb = [torch.from_numpy(x).cuda() for x in arrs]
        stream.synchronize()
        g.reserve(80040)
        held = _held(g)
        pool0 = g.info().cap_fwd, g.info().cap_rev
        r.after = 0
        rc, _ = g.apply_batch(*tb, raise_on_error=False)
        assert rc == sp.SP_ENOMEM
        assert r.refused >= 1
        r.after = None
        assert g.info().state == 1
        assert _held(g) == held
        assert (g.info().cap_fwd, g.info().cap_rev) == pool0
        np.testing.assert_array_equal(g.get_dist(), d0)
        check_all(g, ref, 0, store=True)
        st = g.apply_batch(*tb, stats=True)
        assert st.regrows >= 1
        ref.apply_batch(*arrs)
        check_all(g, ref, 0, store=True)
    finally:
        g.close()
