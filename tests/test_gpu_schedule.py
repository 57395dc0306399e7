"""GPU parity of the push fixedPoint's work schedules.

The schedule (small-list degree bound, block-local relaxation sub-rounds,
near-far width, single-block rounds, loop blocks) changes only the order of
the Min relaxations, never the result: every setting must give the oracle's
distances bit for bit after sp_sssp_init and after every batch, with parents
that satisfy the shortest-path-tree invariants.
"""
import numpy as np
import pytest

import oracle
from paper_2507_11094_gb300 import sp
from paper_2507_11094_gb300 import workloads as wl

from test_gpu_sssp import check_all, run_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2507_11094_gb300 import build
    build.build()
    oracle.build()
    sp.load()


MAKERS = {
    "grid": lambda: wl.grid(80, 80, batch_frac=0.01, seed=6),
    "grid-uniform": lambda: wl.grid(40, 96, batch_frac=0.02, seed=3, insert_kind="uniform"),
    "rmat13": lambda: wl.rmat(scale=13, batch_frac=0.01, seed=7),
    "er1k": lambda: wl.tiny_er(seed=4),
}

# (small_deg, pool_rounds, delta, local_edges)
SCHEDULES = [
    (0, 0, 0, 0),          # every vertex as warp-wide edge chunks
    (32, 0, 0, 0),         # thread per vertex up to 32 edges
    (8, 1, 0, 0),          # one block-local sub-round per grid round
    (8, 16, 300, 0),
    (8, 4096, 300, 0),     # blocks run their pools dry
    (16, 64, 2000, 4096),  # pools and single-block rounds together
    (0, 8, 60, 0),
]


@pytest.mark.parametrize("name", sorted(MAKERS))
@pytest.mark.parametrize("small,pool,delta,local", SCHEDULES)
def test_push_schedules_match_oracle(name, small, pool, delta, local):
    def setup(g):
        g.set_schedule(small, pool)
        g.set_delta(delta)
        g.set_local_rounds(local)
    run_workload(MAKERS[name](), 3, store=False, setup=setup)


@pytest.mark.parametrize("blocks", [1, 2, 5])
def test_pool_overflow_with_few_blocks(blocks):
    """With one to five blocks a wide front overflows the 2048-entry pools:
    what does not fit goes to the global frontier, and the distances still
    equal the oracle's."""
    W = wl.grid(160, 160, batch_frac=0.01, seed=9)

    def setup(g):
        g.set_loop_blocks(blocks)
        g.set_schedule(8, 512)
        g.set_delta(4000)
        g.set_local_rounds(0)
    run_workload(W, 2, store=False, setup=setup)


def test_pool_schedule_cuts_grid_rounds():
    """On a high-diameter grid the block-local sub-rounds carry the wave
    across many edges per grid round: the static solve needs far fewer grid
    rounds and gives the same distances."""
    W = wl.grid(256, 256, seed=2)
    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        g.set_delta(3000)
        g.set_local_rounds(0)
        g.sssp_init(W.source)
        plain = g.loop_counters()
        d_plain = g.get_dist()
        np.testing.assert_array_equal(d_plain, ref.dijkstra(W.source))
        g.set_schedule(8, 1024)
        g.sssp_init(W.source)
        pool = g.loop_counters()
        check_all(g, ref, W.source, store=False)
        assert pool["pool_subrounds"] > 0 and pool["pool_entries"] > 0
        assert pool["rounds_push"] * 4 < plain["rounds_push"], (pool, plain)


def test_schedule_arguments_are_checked():
    W = wl.tiny_er(seed=1)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        for bad in ((-1, 0), (65, 0), (8, -1), (8, 16385)):
            with pytest.raises(sp.SpError):
                g.set_schedule(*bad)
        g.set_schedule(64, 16384)
        g.sssp_init(W.source)
        np.testing.assert_array_equal(
            g.get_dist(), oracle.OracleGraph(W.n, W.row_off, W.col, W.w).dijkstra(W.source))


def test_autotuner_schedule_per_graph_kind():
    """The tuner picks the schedule per graph; on a high-diameter grid the
    block-local pools win.  Whatever it picks, the distances after the
    tuning solve and after batches equal the oracle's."""
    from paper_2507_11094_gb300 import autotune
    picked = {}
    for name, W in (("grid", wl.grid(256, 256, batch_frac=0.01, seed=3)),
                    ("rmat", wl.rmat(scale=14, batch_frac=0.01, seed=3))):
        ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
        with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
            res = autotune.tune_schedule(
                g, lambda h, stats=False: h.sssp_init(W.source, stats=stats), W.w, reps=1)
            picked[name] = res["schedule"]
            d = check_all(g, ref, W.source, store=False)
            for k in range(2):
                b = W.batch(k, dist=d if W.tree_fraction else None)
                g.apply(b)
                ref.apply(b)
                d = check_all(g, ref, W.source, store=False)
    assert picked["grid"]["pool_rounds"] > 0, picked


def _grid_with_fifth_edges(rows, cols, every, seed=0):
    """A grid plus, for every `every`-th vertex above the last two rows, one
    extra out-edge two rows down (never a grid edge, so no duplicate)."""
    W = wl.grid(rows, cols, seed=seed)
    n = W.n
    rng = np.random.default_rng(seed)
    u = np.repeat(np.arange(n, dtype=np.int64), np.diff(W.row_off))
    src = np.arange(0, n - 2 * cols, every, dtype=np.int64)
    eu = np.concatenate([u, src])
    ev = np.concatenate([W.col.astype(np.int64), src + 2 * cols])
    ew = np.concatenate([W.w, rng.integers(1, 100, src.size).astype(np.int32)])
    order = np.lexsort((ev, eu))
    row_off = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(eu, minlength=n), out=row_off[1:])
    return n, row_off, ev[order].astype(np.int32), ew[order], W.source


@pytest.mark.parametrize("every,step", [(0, 4), (8, 5)])
def test_pool_step_follows_the_degree_share(every, step):
    """The pool schedule relaxes four edges per lane and step, or five once
    at least 1/64 of the vertices have 5..8 out-edges; either way the
    distances equal the oracle's."""
    if every:
        n, ro, col, w, src = _grid_with_fifth_edges(96, 96, every)
    else:
        W = wl.grid(96, 96, seed=0)
        n, ro, col, w, src = W.n, W.row_off, W.col, W.w, W.source
    ref = oracle.OracleGraph(n, ro, col, w)
    with sp.Graph(n, ro, col, w) as g:
        assert g.info().pool_step == step
        g.set_schedule(8, 64)
        g.set_delta(20000)
        g.set_local_rounds(0)
        g.sssp_init(src)
        assert g.loop_counters()["pool_subrounds"] > 0
        check_all(g, ref, src, store=False)


def test_pool_step_widens_as_batches_add_fifth_edges():
    """Batches of nearby insertions give many grid vertices a fifth edge:
    the pool kernel switches to five-edge steps between batches (a new
    captured graph), and every batch's distances equal the oracle's."""
    W = wl.grid(64, 64, batch_frac=0.05, seed=4)
    steps = []

    def setup(g):
        g.set_schedule(8, 64)
        g.set_delta(20000)
        g.set_local_rounds(0)
        steps.append(g.info().pool_step)

    ref = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    with sp.Graph(W.n, W.row_off, W.col, W.w) as g:
        setup(g)
        g.sssp_init(W.source)
        d = check_all(g, ref, W.source, store=False)
        for k in range(4):
            b = W.batch(k, dist=d)
            g.apply(b)
            ref.apply(b)
            d = check_all(g, ref, W.source, store=False)
            steps.append(g.info().pool_step)
    assert steps[0] == 4 and steps[-1] == 5, steps
