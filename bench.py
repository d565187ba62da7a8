#!/usr/bin/env python3
"""Throughput benchmark of the GB300 BatchLayout path.

Headline workload: exact-mode BatchLayout (Algorithm 2) on a Barabasi-Albert
graph, n = 65,536, m = 4 (262,134 undirected edges), FP32 positions uniform in
[-1,1)^2 from seed 0, minibatch 256. One step = one layout iteration (all 256
minibatches: repulsion over all n, CSR attraction, update, step schedule); a
timed step is one launch of 10 consecutive iterations (as a long run issues
them), with L2 flushed between steps outside the timed events.
Metric: pair-interactions/s = n(n-1) per iteration / device time.

Secondary lines (in "also"): Barnes-Hut on R-MAT scale 20 (vertex-updates/s),
the 32x32 grid for 600 iterations, 4,096 small graphs in one batched launch
(against one graph per launch, at equal stress) and the serving loop
(layouts/s, p50/p99 latency).

--impl reference runs the FP64 CPU oracle on the host cores on a bounded sample
of the same workload (the paper's method has no other runnable implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s & vertex-updates/s per iter; served layouts/s, p50/p99"
SMS = 152
MUFU_PER_CLK_PER_SM = 16      # rcp.approx.f32 lanes per clock per SM


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-also", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only", default=None,
                    choices=["bh_rmat20", "grid32_600it", "batched_4096", "serving", "pair_ceiling"],
                    help="run one secondary workload alone and print its line (profiling)")
    ap.add_argument("--batched-count", type=int, default=4096, help="graphs of the batched line")
    ap.add_argument("--batched-iters", type=int, default=300, help="iterations of the batched line")
    ap.add_argument("--bh-scale", type=int, default=20, help="R-MAT scale of the BH line")
    ap.add_argument("--serve-count", type=int, default=32, help="requests of the serving line")
    ap.add_argument("--serve-rates", default="0.5,0.8,1.0,1.2",
                    help="offered loads of the serving line, as fractions of the saturated rate")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds, world):
    """Whole-job throughput: the units all ranks processed / the slowest rank's
    time (every rank times the same amount of work)."""
    return units_per_rank * world / max_over_ranks(seconds, world)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# headline: exact mode, BA n=65,536, minibatch 256
# ---------------------------------------------------------------------------

BATCH = 256
ITERS_PER_STEP = 10   # one launch of 10 layout iterations per timed step


def exact_graph():
    from paper_2002_08233_gb300 import synth
    return synth.ba_65536()


def run_exact(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2002_08233_gb300 import core, synth

    torch.cuda.set_device(local)
    core.load()
    stream = core.use_torch()
    g = exact_graph()
    n = g.n
    pairs_per_iter = float(n) * float(n - 1)
    G = core.Graph(g)
    x0 = synth.uniform_positions(n, 0)
    L = core.Layout(G, xy=x0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    for _ in range(max(args.warmup, 0)):
        L.run(ITERS_PER_STEP, BATCH, "exact")
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kernel_ms = []
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        L.run(ITERS_PER_STEP, BATCH, "exact")
        ends[k].record(stream)
        kernel_ms.append(L.stats()["last_run_ms"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier(world)
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = whole_job_rate(pairs_per_iter * ITERS_PER_STEP * args.steps, total_ms / 1e3, world)

    # end to end through the public API with pinned host buffers
    host_in = torch.from_numpy(x0.copy()).pin_memory()
    host_out = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    hin = host_in.numpy()
    hout = host_out.numpy()
    e2e_steps = max(3, min(args.steps, 10))
    L2 = core.Layout(G, xy=x0)
    L2.run(ITERS_PER_STEP, BATCH, "exact")
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        L2.set_positions(hin, start_iter=k * ITERS_PER_STEP)
        L2.run(ITERS_PER_STEP, BATCH, "exact")
        L2.positions(out=hout)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = pairs_per_iter * ITERS_PER_STEP * e2e_steps * world / e2e_s

    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_pairs = SMS * MUFU_PER_CLK_PER_SM * sm_max * 1e6
    avg_kernel_s = statistics.mean(kernel_ms) / 1e3
    achieved = pairs_per_iter * ITERS_PER_STEP / avg_kernel_s
    energy = float(L.stats()["energy"])
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "pair-interactions/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": headline_config(g, world),
        "vertex_updates_per_s": n * ITERS_PER_STEP * args.steps * world / (total_ms / 1e3),
        "kernel_ms_mean": statistics.mean(kernel_ms),
        "wall_s": wall,
        "energy_last": energy,
        "e2e": {"value": e2e_value, "unit": "pair-interactions/s",
                "h2d_bytes_per_step": int(host_in.numel() * 4),
                "d2h_bytes_per_step": int(host_out.numel() * 4),
                "steps": e2e_steps},
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak_pairs / 1e9,
                     "unit": "G pair-interactions/s (1 SFU reciprocal per pair)",
                     "frac": achieved / peak_pairs,
                     # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch
                     # (10 iterations) of this kernel on this workload: not taken on
                     # the build that carries the row sums between launches (3,028,992
                     # bytes on the build before it)
                     "traffic": None, "traffic_unit": "bytes per launch",
                     "kernel": "exact_grid_kernel",
                     "peak_source": f"{SMS} SMs x {MUFU_PER_CLK_PER_SM} SFU lanes/clk x "
                                    f"{sm_max:.0f} MHz ({src} sm_max_mhz)"},
        "clocks": clk,
        "gpu_launches": 2 * args.steps,   # engine kernel + energy reduction per step
    }
    return out, g


def headline_config(g, world):
    """The headline workload, as both arms report it (the reference arm times a
    bounded sample of it, described in its cpu_baseline)."""
    return {
        "workload": "exact BatchLayout, Barabasi-Albert n=65,536 m=4 (262,134 edges), "
                    "minibatch 256, 10 iterations per step (one launch)",
        "n": g.n, "nnz": g.nnz, "batch": BATCH, "mode": "exact",
        "iterations_per_step": ITERS_PER_STEP,
        "parallelism": "replicas" if world > 1 else "single",
        "l2": "flushed between steps (256 MB write outside the timed events)",
        "init": "SplitMix64 seed 0, uniform [-1,1)^2",
    }


def _oracle_batches(g, x0, nb, cores):
    """The oracle's forces for the first nb minibatches of iteration 0, each
    followed by Algorithm 2's update, in order."""
    import numpy as np

    import oracle
    xy = x0.astype(np.float64)
    for b in range(nb):
        lo, hi = b * BATCH, min(g.n, (b + 1) * BATCH)
        f, _ = oracle.forces(g, xy, lo=lo, hi=hi, nthreads=cores)
        nf = np.linalg.norm(f, axis=1)
        mv = nf > 0
        xy[lo:hi][mv] += f[mv] / nf[mv, None]
    return xy


def cpu_baseline_exact(g, seconds_target=15.0):
    """The FP64 oracle on all host cores, on a bounded sample of the same
    workload: whole iterations of Algorithm 2 (as many as fit about 15 s after a
    one-iteration probe), timed."""
    import oracle
    from paper_2002_08233_gb300 import synth
    cores = os.cpu_count() or 1
    x0 = synth.uniform_positions(g.n, 0)
    t0 = time.perf_counter()
    x1, _ = oracle.run(g, x0, iters=1, batch=BATCH, nthreads=cores)
    probe = time.perf_counter() - t0
    iters = int(max(1, min(50, round(seconds_target / max(probe, 1e-3)))))
    t0 = time.perf_counter()
    oracle.run(g, x1, iters=iters, batch=BATCH, start_iter=1, nthreads=cores)
    dt = time.perf_counter() - t0
    pairs = iters * float(g.n) * (g.n - 1)
    return {"value": pairs / dt, "unit": "pair-interactions/s", "cores": cores, "kind": "oracle",
            "sample": f"iterations 1..{iters} of the layout ({pairs:.3g} pairs), FP64, OpenMP over "
                      f"each minibatch",
            "seconds": dt}


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step = one sampled minibatch sweep."""
    if rank != 0:
        return None
    import numpy as np

    from paper_2002_08233_gb300 import synth
    g = exact_graph()
    x0 = synth.uniform_positions(g.n, 0)
    cores = os.cpu_count() or 1
    nb = 4
    for _ in range(max(args.warmup, 0)):
        _oracle_batches(g, x0, 1, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_batches(g, x0, nb, cores)
    dt = time.perf_counter() - t0
    pairs = nb * BATCH * float(g.n - 1) * args.steps
    v = pairs / dt
    sample = f"first {nb} minibatches of one iteration per step ({nb * BATCH * (g.n - 1):.3g} pairs)"
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "pair-interactions/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(g, 1),
        "cpu_baseline": {"value": v, "unit": "pair-interactions/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "pair-interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


# ---------------------------------------------------------------------------
# secondary: Barnes-Hut, R-MAT scale 20
# ---------------------------------------------------------------------------

def bh_bytes(n, nnz, nnz_early, nodes):
    """Algorithmic bytes of one Barnes-Hut iteration (what each phase must move at
    least once), by phase. The whole iteration's figure follows the per-unit
    counts of the path: bounding box 8n, Morton codes 12n, four sort passes of 16n
    (keys and values read and written), the tree ~32 B per node plus 8n of codes,
    the CSR work 12 B per edge (column id + neighbour position) plus 16 B per
    vertex; the walk's node records are counted apart (they are L2 reads)."""
    phases = {
        "bbox_morton": 24 * n,                     # bbox read 8n, Morton read 8n, keys+values 8n
        "radix_sort": 4 * 16 * n,
        "tree": 28 * n + 48 * nodes,               # sorted copy 20n, codes 8n, node fields 48 B
        "edge_pass": 12 * nnz + 32 * n,            # every edge once; rowptr, split, S, two outputs
        "sweep": 12 * nnz_early + 48 * n,          # earlier-minibatch edges again; per-row state
        "energy": 8 * n,
    }
    total = 8 * n + 12 * n + 64 * n + (32 * nodes + 8 * n) + 12 * nnz + 16 * n
    return phases, total


def run_bh(args, local, steps=5, warmup=2):
    import numpy as np
    import torch

    from paper_2002_08233_gb300 import core, synth
    core.load()
    stream = core.use_torch()
    g = synth.rmat_scale20() if args.bh_scale == 20 else synth.rmat(args.bh_scale, 16, 0.57, 0.19,
                                                                      0.19, seed=3)
    n = g.n
    G = core.Graph(g)
    L = core.Layout(G, seed=0)
    L.run(warmup, BATCH, "bh", 1.2)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        starts[k].record(stream)
        L.run(1, BATCH, "bh", 1.2)
        ends[k].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    st = L.stats()
    total = sum(ms)
    ms_it = total / steps
    # phases of 3 more iterations (events between phases; not part of the timed steps)
    L.set_phase_timing(True)
    L.run(3, BATCH, "bh", 1.2)
    ph = L.phase_times()
    L.set_phase_timing(False)
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    nnz_early = int(np.count_nonzero(g.colids < (rows // BATCH) * BATCH))
    pbytes, tbytes = bh_bytes(n, g.nnz, nnz_early, ph["nodes"])
    pk, src = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0)) * 1e9
    it = max(ph["iterations"], 1)
    phases = {}
    for name in L.PHASES:
        t_ms = ph[name] / it
        d = {"ms_per_iteration": t_ms, "share": t_ms / (ph["iteration"] / it)}
        if name in pbytes and t_ms > 0:
            d["bytes"] = pbytes[name]
            d["achieved_gbs"] = pbytes[name] / (t_ms / 1e3) / 1e9
            d["frac_hbm"] = pbytes[name] / (t_ms / 1e3) / hbm
        phases[name] = d
    phases["walk"]["node_record_bytes_l1"] = 24 * ph["walk_node_visits"]
    achieved = tbytes / (ms_it / 1e3)
    # end to end through the public API: positions up, one iteration, positions down
    x0 = synth.uniform_positions(n, 0)
    host_in = torch.from_numpy(x0.copy()).pin_memory()
    host_out = torch.empty((n, 2), dtype=torch.float32).pin_memory()
    hin, hout = host_in.numpy(), host_out.numpy()
    L2 = core.Layout(G, seed=0)
    L2.run(1, BATCH, "bh", 1.2)
    torch.cuda.synchronize()
    e2e_steps = 5
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        L2.set_positions(hin, start_iter=k)
        L2.run(1, BATCH, "bh", 1.2)
        L2.positions(out=hout)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    return {
        "workload": f"Barnes-Hut BatchLayout, R-MAT scale {args.bh_scale} (n={n:,}, edge factor "
                    "16, a=.57 b=c=.19), minibatch 256, theta 1.2, one iteration per step",
        "metric": "vertex-updates/s", "value": n * steps / (total / 1e3),
        "ms_per_iteration": ms_it, "steps": steps, "warmup": warmup,
        "n": n, "nnz": g.nnz, "nnz_earlier_minibatch": nnz_early, "tree_nodes": ph["nodes"],
        "tree_walk_far_nodes": st["bh_far_nodes"], "tree_walk_leaf_vertices": st["bh_near_pairs"],
        # far-field nodes accepted plus leaf vertices met (each query's own excluded),
        # per second of whole iteration
        "interactions_per_s": (st["bh_far_nodes"] + st["bh_near_pairs"] - n) / (ms_it / 1e3),
        "roofline": {"bound": "hbm", "achieved": achieved / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                     "frac": achieved / hbm,
                     # ncu dram__bytes_read.sum + dram__bytes_write.sum summed over the 42
                     # kernels of one R-MAT scale-20 iteration (edge pass to energy)
                     "traffic": 736119296 if args.bh_scale == 20 else None,
                     "traffic_unit": "bytes per iteration",
                     "algorithmic_bytes_per_iteration": tbytes,
                     "bytes_note": "172 n + 12 nnz (+ 32 B per tree node over 2n): bbox, Morton, 4 sort "
                                   "passes, tree, CSR; walk node records not counted (L2 reads)",
                     "peak_source": f"{src} hbm_gbs"},
        "phases": phases,
        "e2e": {"value": n * e2e_steps / e2e_s, "unit": "vertex-updates/s",
                "h2d_bytes_per_step": int(host_in.numel() * 4), "d2h_bytes_per_step": int(host_out.numel() * 4),
                "steps": e2e_steps},
        "l2": "working set > L2 (positions, sorted copies and a ~1.3n-node tree)",
    }


def cpu_baseline_bh(g, seconds_target=10.0):
    """The FP64 oracle's Barnes-Hut iteration (Algorithm S5) on all host cores,
    from the seeded start: one probe iteration, then as many as fit ~10 s."""
    import oracle
    from paper_2002_08233_gb300 import synth
    cores = os.cpu_count() or 1
    x0 = synth.uniform_positions(g.n, 0)
    t0 = time.perf_counter()
    x1, _ = oracle.run(g, x0, iters=1, batch=BATCH, mode=oracle.BH, theta=1.2, nthreads=cores)
    probe = time.perf_counter() - t0
    iters = int(max(1, min(20, round(seconds_target / max(probe, 1e-3)))))
    t0 = time.perf_counter()
    oracle.run(g, x1, iters=iters, batch=BATCH, mode=oracle.BH, theta=1.2, start_iter=1, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": g.n * iters / dt, "unit": "vertex-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"iterations 1..{iters} of the Barnes-Hut layout, FP64, OpenMP over each minibatch",
            "seconds": dt}


# ---------------------------------------------------------------------------
# secondary: the 32x32 grid (latency-bound), 600 iterations
# ---------------------------------------------------------------------------

def run_pair_ceiling(args, local):
    """The exact pair loop and rcp.approx alone, against the SFU roofline's 16
    reciprocal lanes per clock per SM (profiling line, not part of the default run)."""
    from paper_2002_08233_gb300 import core
    core.load()
    core.use_torch()
    shapes = {}
    for threads, skip in ((512, False), (384, False), (512, True)):
        r = core.measure_pair_rate(threads, skip)
        r["frac_of_16"] = r["pairs_per_clk_per_sm"] / 16.0
        shapes[f"{threads}_threads" + ("_sp0_idle" if skip else "")] = r
    return {"workload": "one row per thread against a 256-column shared-memory tile, 400 passes, "
                        "every SM; then 8 rcp.approx chains per thread, 512 threads per SM",
            "pair_loop": shapes}


def run_grid(args, local, reps=3):
    import torch

    from paper_2002_08233_gb300 import core, synth
    core.load()
    core.use_torch()
    g = synth.grid_32x32()
    G = core.Graph(g)
    iters, bs = 600, 128
    pairs = float(g.n) * (g.n - 1) * iters
    out = {"workload": "exact BatchLayout, 32x32 grid (n=1,024, 1,984 edges), minibatch 128, "
                       "600 iterations per step (one whole layout)",
           "metric": "pair-interactions/s", "n": g.n, "nnz": g.nnz, "iterations": iters}

    def exact_with(engine):
        def run(L):
            os.environ["BL_EXACT_ENGINE"] = engine
            try:
                L.run(iters, bs, "exact")
            finally:
                os.environ.pop("BL_EXACT_ENGINE", None)
        return run

    for name, run in (("default", lambda L: L.run(iters, bs, "exact")),   # the cluster engine at this size
                      ("cluster_engine", exact_with("cluster")),
                      ("whole_gpu_engine", exact_with("grid")),
                      ("batched_kernel", lambda L: core.run_batch([L], iters, bs))):
        L = core.Layout(G, seed=0)
        run(L)   # warm-up
        ms = []
        for _ in range(reps):
            L = core.Layout(G, seed=0)
            run(L)
            ms.append(L.stats()["last_run_ms"])
        t = statistics.median(ms)
        out[name] = {"ms_per_layout": t, "value": pairs / (t / 1e3),
                     "layouts_per_s": 1e3 / t, "energy_last": float(L.stats()["energy"])}
    out["value"] = out["default"]["value"]
    return out


# ---------------------------------------------------------------------------
# secondary: 4,096 small graphs in one persistent launch
# ---------------------------------------------------------------------------

def run_batched(args, local):
    import numpy as np
    import torch

    from paper_2002_08233_gb300 import core, synth
    core.load()
    core.use_torch()
    gs = synth.small_graph_mix(count=args.batched_count, seed=4)
    Gs = [core.Graph(g) for g in gs]
    seeds = np.arange(len(gs), dtype=np.uint64)
    iters, bs = args.batched_iters, 64
    pairs = float(sum(g.n * (g.n - 1) for g in gs)) * iters
    # resident inputs: layouts created, then one timed batched run
    Ls = core.layout_batch(Gs, seeds, 0, bs)
    core.run_batch(Ls, 5, bs)          # warm-up (autotuner, caches)
    for L in Ls:
        L.close()
    ms = []
    for _ in range(2):
        Ls = core.layout_batch(Gs, seeds, 0, bs)
        torch.cuda.synchronize()
        core.run_batch(Ls, iters, bs)
        ms.append(Ls[0].stats()["last_run_ms"])
        keep = Ls
    t = min(ms) / 1e3
    pk, src = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_pairs = SMS * MUFU_PER_CLK_PER_SM * sm_max * 1e6
    # end to end: seeded positions up, every layout's positions down
    hosts = [np.empty((g.n, 2), dtype=np.float32) for g in gs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Le = core.layout_batch(Gs, seeds, iters, bs)
    for L, h in zip(Le, hosts):
        L.positions(out=h)
    e2e_s = time.perf_counter() - t0
    n_tot = sum(g.n for g in gs)
    # one graph per launch (the whole-GPU engine), on an even sample of 128 graphs
    idx = np.linspace(0, len(gs) - 1, min(128, len(gs))).astype(int)
    plain_ms = 0.0
    for k in idx:
        L = core.Layout(Gs[k], seed=int(seeds[k]))
        L.run(min(30, iters), bs, "exact")
        plain_ms += L.stats()["last_run_ms"]
        L.close()
    plain_s = plain_ms / 1e3 * (len(gs) / len(idx)) * (iters / min(30, iters))
    # stress at the same seeds: batched vs one graph per launch, 16 graphs
    sp, sb = [], []
    for k in idx[::2]:
        L = core.Layout(Gs[k], seed=int(seeds[k]))
        L.run(iters, bs, "exact")
        sp.append(L.quality()["stress"])
        sb.append(keep[k].quality()["stress"])
        L.close()
    sp, sb = np.array(sp), np.array(sb)
    ratio = sb / sp - 1.0
    return {
        "workload": f"{len(gs):,} graphs, n log-uniform [50, 5,000] (grids, random binary trees, "
                    f"ER mean degree U[4,8]; seed 4), exact, minibatch 64, {iters} iterations, one "
                    "persistent launch (CUDA-graph captured)",
        "metric": "pair-interactions/s", "value": pairs / t, "layouts_per_s": len(gs) / t,
        "seconds": t, "graphs": len(gs), "vertices": n_tot,
        "roofline": {"bound": "alu", "achieved": pairs / t / 1e9, "peak": peak_pairs / 1e9,
                     "unit": "G pair-interactions/s", "frac": pairs / t / peak_pairs,
                     "kernel": "batch_kernel", "peak_source": f"{src} sm_max_mhz"},
        "e2e": {"value": pairs / e2e_s, "unit": "pair-interactions/s", "layouts_per_s": len(gs) / e2e_s,
                "h2d_bytes_per_step": int(8 * n_tot), "d2h_bytes_per_step": int(8 * n_tot)},
        "one_graph_per_launch": {"layouts_per_s": len(gs) / plain_s,
                                 "sample": f"{len(idx)} evenly spaced graphs x {min(30, iters)} "
                                           f"iterations, scaled to {len(gs)} x {iters}"},
        "speedup_vs_one_graph_per_launch": plain_s / t,
        # per graph the two FP32 trajectories may settle in different local minima
        # (grids, trees); the ensemble is what must agree
        "stress_vs_one_graph_per_launch": {
            "ratio_of_sums_minus_1": float(sb.sum() / sp.sum() - 1.0),
            "mean_rel_diff": float(ratio.mean()), "median_rel_diff": float(np.median(ratio)),
            "std_err": float(ratio.std(ddof=1) / np.sqrt(len(ratio))), "graphs": int(len(ratio))},
    }


# ---------------------------------------------------------------------------
# secondary: the serving loop
# ---------------------------------------------------------------------------

def run_serving(args, local):
    count = args.serve_count
    import numpy as np
    import torch

    from paper_2002_08233_gb300 import core, synth
    core.load()
    core.use_torch()
    # long streams: graphs drawn in parallel (spawn pool) and uploaded as they
    # arrive, without keeping the host copies
    workers = min(os.cpu_count() or 1, 16) if count > 64 else 1
    reqs, Gs = [], []
    for r in synth.serving_stream(count, 1.0, 1e3, 2e6, seed=5, workers=workers):
        Gs.append(core.Graph(r.graph))
        reqs.append(synth.Request(arrival_s=r.arrival_s, graph=None, seed=r.seed))
    budget = 120 * (1 << 30)

    def serve(arrivals):
        S = core.Server(budget)
        pending = {}
        t0 = time.perf_counter()
        k = 0
        done = 0
        while done < len(reqs):
            now = time.perf_counter() - t0
            while k < len(reqs) and arrivals[k] <= now:
                pending[S.submit(Gs[k], reqs[k].seed, 300, 256, "auto")] = Gs[k].n
                k += 1
            for t, n in list(pending.items()):
                if S.poll(t, n) is not None:
                    del pending[t]
                    done += 1
            time.sleep(0.0005)
        wall = time.perf_counter() - t0
        st = S.stats()
        S.close()
        return wall, st

    wall_sat, st_sat = serve([0.0] * len(reqs))
    thr = len(reqs) / wall_sat
    unit_gaps = np.array([r.arrival_s for r in reqs])   # the seeded unit-rate arrivals
    sweep = {}
    rates = [float(x) for x in args.serve_rates.split(",") if x.strip()]
    if 0.8 not in rates:
        rates.append(0.8)   # the line's headline latency
    for f in rates:   # offered load as a fraction of the saturated rate
        lam_f = f * thr
        wall_f, st_f = serve(list(unit_gaps / lam_f))
        sweep[f"{f}x"] = {"rate_per_s": lam_f, "layouts_per_s": len(reqs) / wall_f,
                          "p50_s": st_f["p50_s"], "p99_s": st_f["p99_s"]}
        if f == 0.8:
            lam, wall_p, st_p = lam_f, wall_f, st_f
    return {
        "workload": f"serving: first {count} requests of the seeded Poisson stream (seed 5), n "
                    "log-uniform [1e3, 2e6], half R-MAT edge factor 8, half triangulated meshes, "
                    "exact below 50K vertices else BH, 300 iterations, budget 120 GB",
        "metric": "served layouts/s", "value": thr,
        "saturated": {"layouts_per_s": thr, "seconds": wall_sat, "p50_s": st_sat["p50_s"],
                      "p99_s": st_sat["p99_s"], "peak_bytes": st_sat["peak_bytes"]},
        "poisson_0.8x": {"rate_per_s": lam, "layouts_per_s": len(reqs) / wall_p, "seconds": wall_p,
                         "p50_s": st_p["p50_s"], "p99_s": st_p["p99_s"],
                         "peak_bytes": st_p["peak_bytes"]},
        "rate_sweep": sweep,
        "vertices": int(sum(g.n for g in Gs)),
    }


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if rank == 0 and out is not None:
            print(json.dumps(out))
        return
    if args.only:
        fn = {"bh_rmat20": run_bh, "grid32_600it": run_grid, "batched_4096": run_batched,
              "serving": run_serving, "pair_ceiling": run_pair_ceiling}[args.only]
        line = fn(args, local)
        if rank == 0:
            print(json.dumps({"only": args.only, **line}))
        return
    out, g = run_exact(args, rank, world, local)
    # the secondary lines are one-GPU measurements: only a single-process run makes them
    if not args.no_also and world == 1:
        also = {}
        for name, fn in (("bh_rmat20", run_bh), ("grid32_600it", run_grid),
                         ("batched_4096", run_batched), ("serving", run_serving)):
            try:
                also[name] = fn(args, local)
            except Exception as e:   # secondary lines never fail the headline
                also[name] = {"error": f"{type(e).__name__}: {e}"}
        out["also"] = also
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            try:
                out["cpu_baseline"] = cpu_baseline_exact(g)
            except Exception as e:   # the baseline is context; never fail the bench on it
                out["cpu_baseline"] = {"error": str(e)}
            bh = out.get("also", {}).get("bh_rmat20")
            if bh is not None and "error" not in bh:
                try:
                    from paper_2002_08233_gb300 import synth
                    bh["cpu_baseline"] = cpu_baseline_bh(synth.rmat_scale20() if args.bh_scale == 20 else
                                                         synth.rmat(args.bh_scale, 16, seed=3))
                except Exception as e:
                    bh["cpu_baseline"] = {"error": str(e)}
        print(json.dumps(out))


if __name__ == "__main__":
    main()
