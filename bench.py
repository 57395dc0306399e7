"""Benchmark: dynamic-SSSP batch repair on GB300 (edge-updates/s, p50/p99).

One step = one sp_apply_batch of one update batch (sort, count, merge into
both stores, OnDelete mark + subtree invalidation, pull, OnAdd relax, push
fixedPoint) on the device-resident graph.  Default workload: R-MAT scale 20
(1,048,576 vertices, 16,777,216 edges, a=.57 b=.19 c=.19 d=.05, w~U[1,100],
source = max out-degree vertex), batches of 1% of m (83,886 deletions of
existing edges + 83,886 R-MAT insertions).

Printed JSON line (rank 0): value = edge updates per second over the K timed
steps (inputs resident in HBM, L2 flushed between steps, CUDA events on the
graph's stream, max over ranks; the calls are made as a user makes them,
without the library's per-phase events, whose graph nodes lengthen a step);
the phase breakdown and the rooflines come from K further steps made with
the per-phase events (the "instrumented" entry); e2e = the same through host buffers with the
H2D copy of the batch and the D2H read of all distances inside the timed
region; static = from-scratch GPU SSSP (sp_sssp_init) on the updated graph;
roofline = the dominant kernel's algorithmic bytes / its event-timed duration
against the measured HBM copy bandwidth; cpu_baseline = the CPU oracle
(apply + Dijkstra) on a bounded sample of the same batches.

--impl reference times the CPU oracle as the reference arm.
--gpus N under torchrun runs N independent replicas (one graph per GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_11094_gb300 import workloads as wl  # noqa: E402

METRIC = "dyn-SSSP edge updates/s & p50/p99 batch latency vs GPU static recompute"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat20",
                    help="rmat20 | rmat<scale> | er1k | grid<side>-<pct>[u] (e.g. grid4096-1; "
                         "u: uniform-pair insertions) "
                         "| batched64 | serving")
    ap.add_argument("--batch-pct", type=float, default=None)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--static-reps", type=int, default=3)
    ap.add_argument("--delta", type=int, default=None,
                    help="near-far bucket width of the push loop (default: picked on the "
                         "graph by the autotuner from a few multiples of the mean weight)")
    ap.add_argument("--inval-switch", type=int, default=None,
                    help="frontier rounds of the invalidation before pointer jumping "
                         "(-1 never; default: the library's)")
    ap.add_argument("--local-rounds", type=int, default=None,
                    help="frontier-edge bound of single-block push rounds (0 = off; "
                         "default: picked by the autotuner)")
    ap.add_argument("--pool-rounds", type=int, default=None,
                    help="block-local sub-rounds per push round (0 = off; default: "
                         "picked by the autotuner)")
    ap.add_argument("--small-deg", type=int, default=None,
                    help="out-degree bound of thread-per-vertex expansion (default: "
                         "picked by the autotuner)")
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--algo", default="sssp", choices=["sssp", "pr", "tc"],
                    help="sssp (default), pr (dynamic PageRank on the same workloads) or "
                         "tc (dynamic triangle count on symmetric R-MAT, --workload "
                         "sym-rmat<scale>)")
    ap.add_argument("--serving-big-scale", type=int, default=22)
    ap.add_argument("--serving-requests", type=int, default=48)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-repeats", type=int, default=5,
                    help="sustained phases (fresh requests each) whose rates give the "
                         "serving line's value (median) and spread")
    return ap.parse_args()


def make_workload(name: str, seed: int, pct: float | None):
    if name.startswith("sym-rmat"):
        scale = int(name[8:] or 16)
        frac = (pct if pct is not None else 1.0) / 100.0
        return wl.sym_rmat(scale, 8, frac, seed), {"scale": scale, "edge_factor": 8,
                                                   "symmetric": True}
    if name == "er1k":
        return wl.tiny_er(seed=seed), {"n": 1024, "m": 8192}
    if name.startswith("rmat"):
        scale = int(name[4:] or 20)
        frac = (pct if pct is not None else 1.0) / 100.0
        W = wl.rmat(scale=scale, batch_frac=frac, seed=seed)
        return W, {"scale": scale, "edge_factor": 16}
    if name.startswith("grid"):
        side, p = name[4:].split("-")
        # a trailing "u": insertions join uniform vertex pairs (a sensitivity
        # run: long shortcuts collapse the diameter) instead of 5x5 neighbours
        kind = "uniform" if p.endswith("u") else "local5"
        p = p.rstrip("u")
        frac = (pct if pct is not None else float(p)) / 100.0
        W = wl.grid(int(side), int(side), batch_frac=frac, seed=seed, insert_kind=kind)
        return W, {"rows": int(side), "cols": int(side), "insertions": kind}
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once the sampler is producing samples
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample(W, batches, budget_s: float, min_batches: int = 2):
    """Time the CPU oracle (batch apply + from-scratch Dijkstra, one core) on
    as many of `batches` as fit in about budget_s seconds."""
    import oracle
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    times, sizes = [], []
    t_start = time.perf_counter()
    for i, b in enumerate(batches):
        t0 = time.perf_counter()
        g.apply(b)
        g.dijkstra(W.source)
        times.append(time.perf_counter() - t0)
        sizes.append(b.size)
        if i + 1 >= min_batches and time.perf_counter() - t_start > budget_s:
            break
    g.close()
    return times, sizes


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q))


def aggregate_ranks(distributed: bool, times, works):
    """Whole-job figures of replicas: the max over ranks of each time and the
    sum over ranks of each work count (a barrier on both sides)."""
    if not distributed:
        return [float(x) for x in times], [float(x) for x in works]
    import torch
    import torch.distributed as dist
    dist.barrier()
    t = torch.tensor([float(x) for x in times], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(x) for x in works], dtype=torch.float64)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return t.tolist(), u.tolist()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    W, cfg = make_workload(args.workload, args.seed, args.batch_pct)
    batches = [W.batch(k) for k in range(args.warmup + args.steps)]
    g = oracle.OracleGraph(W.n, W.row_off, W.col, W.w)
    g.dijkstra(W.source)
    lat, ups = [], 0
    for k, b in enumerate(batches):
        t0 = time.perf_counter()
        g.apply(b)
        g.dijkstra(W.source)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            lat.append(dt)
            ups += b.size
    value = ups / sum(lat)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edge_updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(lat) / len(lat), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": W.name, **cfg, "n": W.n, "m": W.m,
                   "batch_updates": W.batch_edges, "source": W.source},
        "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
        "cpu_baseline": {"value": value, "unit": "edge_updates/s", "cores": 1,
                         "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"{len(lat)} full batches of {W.batch_edges} updates: "
                                   "oracle batch apply + binary-heap Dijkstra from scratch"},
        "e2e": {"value": value, "unit": "edge_updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import torch

    from paper_2507_11094_gb300 import sp

    ws, rank, local = dist_env()
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sp.load(build_if_missing=True)

    seed = args.seed + rank
    W, cfg = make_workload(args.workload, seed, args.batch_pct)
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
    from paper_2507_11094_gb300 import autotune
    manual = {"delta": args.delta, "pool_rounds": args.pool_rounds,
              "small_deg": args.small_deg, "local_edges": args.local_rounds}
    if any(v is not None for v in manual.values()):
        sched = {k: (v if v is not None else autotune.DEFAULT[k]) for k, v in manual.items()}
        autotune.apply_schedule(g, sched)
        cfg["schedule_source"] = "command line"
    else:   # the project's autotuner picks the push schedule on this graph
        with torch.cuda.stream(stream):
            tune = autotune.tune_schedule(
                g, lambda h, stats=False: h.sssp_init(W.source, stats=stats), W.w, reps=1)
        sched = tune["schedule"]
        cfg["schedule_source"] = "autotuner (from-scratch solve per candidate)"
        cfg["schedule_tuned_ms"] = dict(sorted(tune["ms"].items(), key=lambda kv: kv[1])[:6])
    cfg["schedule"] = sched
    cfg["delta"] = sched["delta"]
    if args.inval_switch is not None:
        g.set_inval_switch(args.inval_switch)
        cfg["inval_switch"] = args.inval_switch
    g.sssp_init(W.source)

    tree = W.tree_fraction > 0
    # device leg batches (generated against the evolving edge set; tree-biased
    # deletions use the current distances read back between generations)
    def gen(k, dist):
        return W.batch(k, dist=dist if tree else None)

    d_cur = g.get_dist() if tree else None
    dev_batches = []
    # generate all device-leg batches first (the stream tracks the edge set);
    # tree-biased workloads need distances, so they are generated one step ahead
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)

    def to_dev(b):
        return [torch.from_numpy(x).to(dev) for x in
                (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w)]

    lat_ms, sizes, stats_all, launches = [], [], [], 0
    wall_ms, ph_lat_ms = [], []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    # the timed steps run the call as a user does (no per-phase events); the
    # phase breakdown comes from K more steps right after them with the
    # library's phase events (sp_batch_stats), which add graph nodes and so
    # lengthen each step (reported as "instrumented")
    n_dev = Wm + K + 1 + K
    if not tree:
        dev_batches = [to_dev(gen(k, None)) for k in range(n_dev)]
        sizes_all = [int(t[0].numel() + t[2].numel()) for t in dev_batches]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    with clocks:
        for k in range(n_dev):
            if tree:
                b = gen(k, g.get_dist())
                tb = to_dev(b)
                size = b.size
            else:
                tb = dev_batches[k]
                size = sizes_all[k]
            phase_pass = k >= Wm + K
            flush.fill_(k)                      # evict L2 between steps
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev0.record(stream)
            st = g.apply_batch(*tb, stats=phase_pass)
            ev1.record(stream)
            ev1.synchronize()
            t1 = time.perf_counter()
            if Wm <= k < Wm + K:
                lat_ms.append(ev0.elapsed_time(ev1))
                wall_ms.append(1e3 * (t1 - t0))
                sizes.append(size)
            elif k > Wm + K:                    # the first phase step captures its graph
                ph_lat_ms.append(ev0.elapsed_time(ev1))
                stats_all.append(st.as_dict())
    torch.cuda.synchronize()
    total_ms = sum(lat_ms)
    ups = sum(sizes)
    # kernels the timed steps launched (the same pipeline as the phase steps)
    launches = int(round(K * statistics.mean(s["n_launches"] for s in stats_all)))

    # from-scratch GPU SSSP on the updated graph (the comparator), timed as
    # the batches are; one more solve with phase events for its push launch
    static_ms = []
    for _ in range(max(1, args.static_reps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.sssp_init(W.source)
        ev1.record(stream)
        ev1.synchronize()
        static_ms.append(ev0.elapsed_time(ev1))
    flush.fill_(2)
    torch.cuda.synchronize()
    sst = g.sssp_init(W.source, stats=True)

    # end to end through host buffers: H2D of the batch + D2H of all distances
    e2e_batches = [gen(n_dev + k, g.get_dist() if tree else None) for k in range(1 + K)]
    pinned = []
    for b in e2e_batches:
        arrs = []
        for x in (b.del_src, b.del_dst, b.add_src, b.add_dst, b.add_w):
            t = torch.empty(x.size, dtype=torch.int32, pin_memory=True)
            t.numpy()[:] = x
            arrs.append(t.numpy())
        pinned.append(arrs)
    dist_host = torch.empty(W.n, dtype=torch.int32, pin_memory=True).numpy()
    e2e_ms, e2e_sizes = [], []
    for k, arrs in enumerate(pinned):
        flush.fill_(k)
        torch.cuda.synchronize()
        ev0.record(stream)
        # one call: the batch from page-locked host arrays, all distances
        # after it into a page-locked host array
        g.apply_batch_get(*arrs, dist_host)
        ev1.record(stream)
        ev1.synchronize()
        if k >= 1:
            e2e_ms.append(ev0.elapsed_time(ev1))
            e2e_sizes.append(e2e_batches[k].size)
    bi = sum(a.nbytes for a in pinned[1]) if len(pinned) > 1 else 0
    bo = dist_host.nbytes

    # aggregate over ranks: max time, summed work
    (total_ms_all, e2e_ms_all), (ups_all, e2e_ups_all) = aggregate_ranks(
        pg is not None, [total_ms, sum(e2e_ms)], [ups, sum(e2e_sizes)])

    store_ms = [sum(st_["ms_phase"][p] for p in ("sort", "count", "merge", "finish"))
                for st_ in stats_all]
    # dominant kernel: the phase with the largest device time over the steps
    phases = list(sp.PHASES)
    ph_ms = {p: sum(s["ms_phase"][p] for s in stats_all) for p in phases}
    ph_bytes = {p: sum(s["alg_bytes"][p] for s in stats_all) for p in phases}
    dom = max(phases, key=lambda p: ph_ms[p])
    peak, peak_kind = measured_peaks()
    achieved = ph_bytes[dom] / (ph_ms[dom] * 1e-3) / 1e9 if ph_ms[dom] > 0 else 0.0
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        with open(tf) as f:
            tj = json.load(f)
        ent = tj.get(W.name, {}).get(dom)
        if ent and ent.get("valid", False):
            traffic = ent["bytes_per_launch"]

    # the relaxation kernels' own roofline (the push launch: pull, OnAdd and
    # the push fixedPoint), for the dynamic repair and the static recompute
    n_steps = max(1, len(stats_all))
    push_dyn_b = ph_bytes["push"] / n_steps
    push_dyn_ms = ph_ms["push"] / n_steps
    push_st_b = sst.alg_bytes[sp.PHASES.index("push")]
    push_st_ms = sst.ms_phase[sp.PHASES.index("push")]

    def _push_roof(b, ms, traffic_key):
        ach = b / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        tr = None
        if os.path.exists(tf):
            with open(tf) as f:
                ent = json.load(f).get(W.name, {}).get(traffic_key)
            if ent and ent.get("valid", False):
                tr = ent["bytes_per_launch"]
        return {"achieved": ach, "frac": ach / peak if peak else None,
                "alg_bytes_per_launch": b, "ms_per_launch": ms, "traffic": tr,
                "traffic_frac": (tr / (ms * 1e-3) / 1e9 / peak) if (tr and peak and ms > 0)
                else None}

    roof_push = {"bound": "hbm", "unit": "GB/s", "peak": peak, "peak_kind": peak_kind,
                 "dynamic": _push_roof(push_dyn_b, push_dyn_ms, "push"),
                 "static": _push_roof(push_st_b, push_st_ms, "push_static")}

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and ws == 1:
            import oracle
            oracle.build()
            Wc, _ = make_workload(args.workload, seed, args.batch_pct)
            sample = [Wc.batch(k) for k in range(4)] if not tree else []
            if sample:
                times, szs = oracle_sample(Wc, sample, budget_s=12.0)
                cpu = {"value": sum(szs) / sum(times), "unit": "edge_updates/s", "cores": 1,
                       "kind": "oracle", "cpu": cpu_model(), "nproc": os.cpu_count(),
                       "sample": f"first {len(times)} batches of the same workload "
                                 f"({szs[0]} updates each): oracle batch apply + "
                                 "binary-heap Dijkstra from scratch, single-threaded"}
        step_ms = total_ms_all / max(1, len(lat_ms))
        line = {
            "metric": METRIC,
            "value": ups_all / (total_ms_all * 1e-3),
            "unit": "edge_updates/s",
            "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": W.name, **cfg, "n": W.n, "m": W.m,
                       "batch_updates": W.batch_edges, "source": W.source,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "p50_ms": percentile(lat_ms, 50), "p99_ms": percentile(lat_ms, 99),
            "wall_p50_ms": percentile(wall_ms, 50), "wall_p99_ms": percentile(wall_ms, 99),
            "static": {"ms_p50": percentile(static_ms, 50), "ms_min": min(static_ms),
                       "rounds": sst.rounds_push,
                       "speedup_dynamic_vs_static": percentile(static_ms, 50) /
                       percentile(lat_ms, 50),
                       # the paper's static time applies the batch to the
                       # store first, then recomputes (Section 7)
                       "with_store_update_ms_p50": percentile(static_ms, 50) +
                       percentile(store_ms, 50),
                       "speedup_dynamic_vs_static_with_store_update":
                       (percentile(static_ms, 50) + percentile(store_ms, 50)) /
                       percentile(lat_ms, 50)},
            "e2e": {"value": e2e_ups_all / (e2e_ms_all * 1e-3) if e2e_ms_all else None,
                    "unit": "edge_updates/s", "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "p50_ms": percentile(e2e_ms, 50),
                    "p99_ms": percentile(e2e_ms, 99)},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak if peak else None, "traffic": traffic},
            "roofline_push": roof_push,
            "instrumented": {"steps": len(ph_lat_ms), "p50_ms": percentile(ph_lat_ms, 50),
                             "note": "phase_ms, phase_alg_bytes, per_step and both rooflines "
                                     "come from these steps, run right after the timed ones "
                                     "with the library's per-phase CUDA events"},
            "phase_ms": {p: ph_ms[p] / n_steps for p in phases},
            "phase_alg_bytes": {p: ph_bytes[p] / n_steps for p in phases},
            "per_step": {
                "affected": statistics.mean(s["affected"] for s in stats_all),
                "rounds_push": statistics.mean(s["rounds_push"] for s in stats_all),
                "rounds_inval": statistics.mean(s["rounds_inval"] for s in stats_all),
                "relaxed_edges": statistics.mean(s["relaxed_edges"] for s in stats_all),
                "rows_touched": statistics.mean(s["rows_touched"] for s in stats_all),
                "regrows": sum(s["regrows"] for s in stats_all),
            },
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
        if args.json_out:
            with open(args.json_out, "w") as f:
                json.dump(line, f, indent=1)
    g.close()
    if pg:
        pg.destroy_process_group()
    return 0


def batched_workloads(seed: int, k: int = 64):
    return wl.batched_rmat(seed, k)


def run_batched(args):
    """C4: many graphs in one handle, one captured launch sequence per round,
    against the same rounds applied graph by graph on separate handles."""
    import torch

    from paper_2507_11094_gb300 import autotune, batched, sp
    torch.cuda.set_device(0)
    sp.load(build_if_missing=True)
    ws = batched_workloads(args.seed)
    K, Wm = args.steps, args.warmup
    rounds = [[W.batch(k) for W in ws] for k in range(Wm + K)]
    stream = torch.cuda.Stream()
    B = batched.BatchedGraphs([(W.n, W.row_off, W.col, W.w) for W in ws],
                              [W.source for W in ws], stream=stream)
    tune = autotune.tune_schedule(B.g, lambda h, stats=False: h.sssp_init_multi(
        B.packed.sources, stats=stats), B.packed.w, reps=1)
    packed = [batched.pack_batches(B.packed, r) for r in rounds]
    dev_rounds = [[torch.from_numpy(a).cuda() for a in arr] for arr in packed]
    fixed = [torch.empty_like(t) for t in dev_rounds[0]]
    B.g.reserve(int(packed[0][0].size + packed[0][2].size) + 16)
    torch.cuda.synchronize()
    ex = B.g.capture(*fixed)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    ms_b, ups = [], 0
    for k in range(Wm + K):
        flush.fill_(k)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            for t, src in zip(fixed, dev_rounds[k]):
                t.copy_(src)
            ex.launch()
            ev1.record(stream)
        ex.finish()
        if k >= Wm:
            ms_b.append(ev0.elapsed_time(ev1))
            ups += int(packed[k][0].size + packed[k][2].size)
    ex.close()
    B.close()
    # the same rounds, graph by graph on separate handles (plain sp_apply_batch)
    gs = []
    for W in ws:
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
        g.sssp_init(W.source)
        gs.append(g)
    dev_each = [[[torch.from_numpy(x).cuda() for x in (b.del_src, b.del_dst, b.add_src,
                                                      b.add_dst, b.add_w)] for b in r]
                for r in rounds]
    ms_s = []
    for k in range(Wm + K):
        flush.fill_(k)
        torch.cuda.synchronize()
        ev0.record(stream)
        for g, tb in zip(gs, dev_each[k]):
            g.apply_batch(*tb)
        ev1.record(stream)
        ev1.synchronize()
        if k >= Wm:
            ms_s.append(ev0.elapsed_time(ev1))
    for g in gs:
        g.close()
    value = ups / (sum(ms_b) * 1e-3)
    line = {
        "metric": METRIC + " [batched form]", "value": value, "unit": "edge_updates/s",
        "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": sum(ms_b) / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "batched64-rmat12..18", "graphs": len(ws),
                   "n_total": int(sum(W.n for W in ws)), "m_total": int(sum(W.m for W in ws)),
                   "updates_per_round": int(packed[0][0].size + packed[0][2].size),
                   "schedule": tune["schedule"], "delta": tune["delta"],
                   "l2": "flushed between steps"},
        "sequential": {"value": ups / (sum(ms_s) * 1e-3), "ms_per_step": sum(ms_s) / K},
        "speedup_vs_sequential": sum(ms_s) / sum(ms_b),
        "p50_ms": percentile(ms_b, 50), "p99_ms": percentile(ms_b, 99),
        "autotune": tune,
    }
    print(json.dumps(line), flush=True)
    return 0


def serving_workloads(seed: int, big_scale: int = 22):
    return wl.serving_graphs(seed, big_scale)


def serving_requests(ws, count: int, seed: int):
    return wl.serving_requests(ws, count, seed)


def run_serving(args):
    """C5: the serving runtime over 8 graphs under an HBM budget that fits
    about 5 of them.  Sustained edge-updates/s with every request submitted
    at once, then Poisson arrivals at 0.5x and 0.9x of it with
    arrival-to-completion p50/p99."""
    import torch

    from paper_2507_11094_gb300 import sp
    torch.cuda.set_device(0)
    sp.load(build_if_missing=True)
    t_gen = time.perf_counter()
    ws = serving_workloads(args.seed, args.serving_big_scale)
    n_req = args.serving_requests
    reps = max(1, args.serving_repeats)
    names = ["warm"] + [f"sustained{r}" for r in range(reps)] + ["rate0.5", "rate0.9"]
    phases = {name: serving_requests(ws, n_req // 3 if name == "warm" else n_req,
                                     args.seed * 10 + j)
              for j, name in enumerate(names)}
    t_gen = time.perf_counter() - t_gen

    # what the server counts for each graph: the upper bound of its footprint
    # with batch buffers reserved for the largest batch (1e6 updates)
    sizes = []
    with sp.Server(hbm_budget_bytes=200 << 30, n_slots=1, delta=0) as probe:
        for W in ws:
            before = probe.stats().resident_bytes
            gid = probe.add_graph(W.n, W.row_off, W.col, W.w, W.source)
            probe.wait(probe.submit_query(gid, np.arange(4)))
            sizes.append(probe.stats().resident_bytes - before)
    budget = int(sum(sorted(sizes)[-5:]))   # about 5 of the 8 graphs

    srv = sp.Server(hbm_budget_bytes=budget, n_slots=args.serving_slots, delta=0)
    gids = [srv.add_graph(W.n, W.row_off, W.col, W.w, W.source) for W in ws]

    def submit_all(reqs, rate=None, rng=None):
        out = []
        t0 = time.perf_counter()
        t_next = 0.0
        for gi, b, q in reqs:
            if rate:
                t_next += rng.exponential(1.0 / rate)
                dt = t0 + t_next - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
            out.append((srv.submit(gids[gi], b), b.size))
            if q is not None:
                out.append((srv.submit_query(gids[gi], q), 0))
        return out

    def collect(ids):
        infos = []
        for rid, size in ids:
            info, _ = srv.wait(rid)
            if info.status != sp.SP_OK:
                raise SystemExit(f"request failed: {sp.STATUS.get(info.status)}")
            infos.append((info.as_dict(), size))
        return infos

    collect(submit_all(phases["warm"]))
    st0 = srv.stats().as_dict()
    rates, secs, overlap = [], [], 0
    for r in range(reps):
        t0 = time.perf_counter()
        sus = collect(submit_all(phases[f"sustained{r}"]))
        t_sus = time.perf_counter() - t0
        ups = sum(sz for _, sz in sus)
        rates.append(ups / t_sus)
        secs.append(t_sus)
        # requests of different graphs on different slots whose device work
        # intersected in time
        iv = [(i["graph"], i["slot"], i["gpu_start_ms"], i["gpu_done_ms"]) for i, _ in sus
              if i["gpu_start_ms"] >= 0]
        overlap += sum(1 for a in iv for b in iv
                       if a[0] < b[0] and a[1] != b[1] and a[2] < b[3] and b[2] < a[3])
    sustained = statistics.median(rates)
    t_sus = statistics.median(secs)
    st1 = srv.stats().as_dict()
    mean_batch = sum(b.size for r in range(reps) for _, b, _ in phases[f"sustained{r}"]) / \
        (reps * n_req)
    runs = {}
    for name, frac in (("rate0.5", 0.5), ("rate0.9", 0.9)):
        rate = frac * sustained / mean_batch           # batches per second
        t0 = time.perf_counter()
        res = collect(submit_all(phases[name], rate, np.random.default_rng(args.seed + 7)))
        dt = time.perf_counter() - t0
        lat = [i["done_ms"] - i["submit_ms"] for i, sz in res if i["kind"] == 0]
        svc = [i["done_ms"] - i["start_ms"] for i, sz in res if i["kind"] == 0]
        qlat = [i["done_ms"] - i["submit_ms"] for i, sz in res if i["kind"] == 1]
        runs[name] = {"offered_batches_per_s": rate,
                      "achieved_updates_per_s": sum(sz for _, sz in res) / dt,
                      "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                      "service_p50_ms": percentile(svc, 50),
                      "service_p99_ms": percentile(svc, 99),
                      "query_p50_ms": percentile(qlat, 50) if qlat else None,
                      "query_p99_ms": percentile(qlat, 99) if qlat else None,
                      "loads": sum(i["loaded"] for i, _ in res)}
    st2 = srv.stats().as_dict()
    srv.close()
    line = {
        "metric": METRIC + " [serving form]", "value": sustained, "unit": "edge_updates/s",
        "n_gpus": 1, "steps": n_req, "warmup": n_req // 3, "ms_per_step": 1e3 * t_sus / n_req,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"serving-2xrmat{args.serving_big_scale}+6xrmat16..20",
                   "graphs": [{"n": W.n, "m": W.m} for W in ws],
                   "device_bytes": sizes, "hbm_budget_bytes": budget,
                   "slots": args.serving_slots, "requests_per_phase": n_req,
                   "inputs": "host arrays copied by the server (H2D inside every request)"},
        "sustained": {"updates_per_s": sustained, "seconds": t_sus,
                      "repeats": reps, "rates": rates, "min": min(rates), "max": max(rates),
                      "overlapping_request_pairs": overlap,
                      "loads": st1["loads"] - st0["loads"],
                      "evictions": st1["evictions"] - st0["evictions"],
                      "restores": st1["restores"] - st0["restores"]},
        "rates": runs,
        "server_stats": st2,
        "generation_s": t_gen,
    }
    print(json.dumps(line), flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            json.dump(line, f, indent=1)
    return 0


def run_pagerank(args):
    """Dynamic PageRank batches (sp_pr_apply_batch) against a static PageRank
    recompute (sp_pr_init) on the updated graph; CPU oracle beside it."""
    import torch

    from paper_2507_11094_gb300 import sp
    torch.cuda.set_device(0)
    sp.load(build_if_missing=True)
    W, cfg = make_workload(args.workload, args.seed, args.batch_pct)
    damping, beta, iters = 0.85, 1e-6, 100
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
    g.pr_init(damping, beta, iters)
    dev = torch.device("cuda", 0)
    batches = [W.batch(k) for k in range(Wm + K)]
    dev_b = [[torch.from_numpy(x).to(dev) for x in (b.del_src, b.del_dst, b.add_src,
                                                    b.add_dst, b.add_w)] for b in batches]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, sizes, stats = [], [], []
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    with clocks:
        for k in range(Wm + K):
            flush.fill_(k)
            torch.cuda.synchronize()
            ev0.record(stream)
            st = g.pr_apply_batch(*dev_b[k], stats=True)
            ev1.record(stream)
            ev1.synchronize()
            if k >= Wm:
                lat.append(ev0.elapsed_time(ev1))
                sizes.append(batches[k].size)
                stats.append(st.as_dict())
    static = []
    for _ in range(max(1, args.static_reps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        sst = g.pr_init(damping, beta, iters, stats=True)
        ev1.record(stream)
        ev1.synchronize()
        static.append(ev0.elapsed_time(ev1))
    # end to end: host batch in, all ranks back to the host
    e2e_b = [W.batch(Wm + K + k) for k in range(K + 1)]
    e2e = []
    for k, b in enumerate(e2e_b):
        flush.fill_(k)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.pr_apply(b)
        g.pr_get()
        ev1.record(stream)
        ev1.synchronize()
        if k:
            e2e.append(ev0.elapsed_time(ev1))
    peak, peak_kind = measured_peaks()
    alg = sum(sum(s["alg_bytes"].values()) for s in stats)
    achieved = alg / (sum(lat) * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Wc, _ = make_workload(args.workload, args.seed, args.batch_pct)
        ref = oracle.OracleGraph(Wc.n, Wc.row_off, Wc.col, Wc.w)
        pr, _ = ref.pagerank(damping, beta, iters)
        t, n_up = 0.0, 0
        for k in range(4):
            b = Wc.batch(k)
            t0 = time.perf_counter()
            ref.pagerank_batch(b, pr, damping, beta, iters)
            t += time.perf_counter() - t0
            n_up += b.size
            if t > 15.0:
                break
        cpu = {"value": n_up / t, "unit": "edge_updates/s", "cores": 1, "kind": "oracle",
               "cpu": cpu_model(), "sample": f"first batches of the same workload, oracle DynPR "
                                             f"({n_up} updates in {t:.1f} s), single-threaded"}
    line = {
        "metric": "dyn-PR edge updates/s & p50/p99 batch latency vs GPU static recompute",
        "value": sum(sizes) / (sum(lat) * 1e-3), "unit": "edge_updates/s", "n_gpus": 1,
        "steps": K, "warmup": Wm, "ms_per_step": sum(lat) / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": W.name, **cfg, "n": W.n, "m": W.m,
                   "batch_updates": W.batch_edges, "damping": damping, "beta": beta,
                   "max_iter": iters, "l2": "flushed between steps"},
        "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
        "static": {"ms_p50": percentile(static, 50), "steps": sst.rounds_push,
                   "speedup_dynamic_vs_static": percentile(static, 50) / percentile(lat, 50)},
        "e2e": {"value": sum(b.size for b in e2e_b[1:]) / (sum(e2e) * 1e-3),
                "unit": "edge_updates/s", "h2d_bytes_per_step": 20 * W.batch_edges // 2,
                "d2h_bytes_per_step": 4 * W.n},
        "roofline": {"bound": "hbm", "kernel": "whole DynPR batch", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None},
        "per_step": {"flagged": statistics.mean(s["affected"] for s in stats),
                     "jacobi_steps": statistics.mean(s["rounds_push"] for s in stats),
                     "pulled_edges": statistics.mean(s["relaxed_edges"] for s in stats)},
        "gpu_launches": sum(s["n_launches"] for s in stats),
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            json.dump(line, f, indent=1)
    g.close()
    return 0


def run_tc(args):
    """Dynamic triangle count batches (sp_tc_apply_batch) against a static
    recount (sp_tc_init) of the updated graph; CPU oracle (apply + recount)
    beside it."""
    import torch

    from paper_2507_11094_gb300 import sp
    torch.cuda.set_device(0)
    sp.load(build_if_missing=True)
    name = args.workload if args.workload.startswith("sym-rmat") else "sym-rmat16"
    W, cfg = make_workload(name, args.seed, args.batch_pct)
    K, Wm = args.steps, args.warmup
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = sp.Graph(W.n, W.row_off, W.col, W.w, stream=stream)
    count0 = g.tc_init()
    dev = torch.device("cuda", 0)
    batches = [W.batch(k) for k in range(Wm + K)]
    dev_b = [[torch.from_numpy(x).to(dev) for x in (b.del_src, b.del_dst, b.add_src,
                                                    b.add_dst, b.add_w)] for b in batches]
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat, sizes, launches = [], [], 0
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    with clocks:
        for k in range(Wm + K):
            flush.fill_(k)
            torch.cuda.synchronize()
            ev0.record(stream)
            count, st = g.tc_apply_batch(*dev_b[k], stats=True)
            ev1.record(stream)
            ev1.synchronize()
            if k >= Wm:
                lat.append(ev0.elapsed_time(ev1))
                sizes.append(batches[k].size)
                launches += st.n_launches
    static = []
    for _ in range(max(1, args.static_reps)):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        recount = g.tc_init()
        ev1.record(stream)
        ev1.synchronize()
        static.append(ev0.elapsed_time(ev1))
    assert recount == count
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Wc, _ = make_workload(name, args.seed, args.batch_pct)
        ref = oracle.OracleGraph(Wc.n, Wc.row_off, Wc.col, Wc.w)
        t0 = time.perf_counter()
        b = Wc.batch(0)
        ref.apply(b)
        ref.triangles()
        t = time.perf_counter() - t0
        cpu = {"value": b.size / t, "unit": "edge_updates/s", "cores": 1, "kind": "oracle",
               "cpu": cpu_model(), "sample": f"first batch of the same workload ({b.size} "
                                             f"updates): oracle apply + staticTC recount, "
                                             f"single-threaded, {t:.1f} s"}
    line = {
        "metric": "dyn-TC edge updates/s & p50/p99 batch latency vs GPU static recount",
        "value": sum(sizes) / (sum(lat) * 1e-3), "unit": "edge_updates/s", "n_gpus": 1,
        "steps": K, "warmup": Wm, "ms_per_step": sum(lat) / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": W.name, **cfg, "n": W.n, "m": W.m,
                   "batch_updates": W.batch_edges, "l2": "flushed between steps",
                   "triangles_initial": count0, "triangles_final": count},
        "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
        "static": {"ms_p50": percentile(static, 50),
                   "speedup_dynamic_vs_static": percentile(static, 50) / percentile(lat, 50)},
        "gpu_launches": launches, "clocks": clocks.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if args.json_out:
        with open(args.json_out, "w") as f:
            json.dump(line, f, indent=1)
    g.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched64":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.algo == "pr":
        return run_pagerank(args)
    if args.algo == "tc":
        return run_tc(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
