"""Benchmark of libsgrcolor on one node (one process per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat20]
                    [--mode det|fast] [--impl ours|reference]

A step is one complete coloring (all rounds of Algorithm 7) of the workload
graph, inputs already resident in HBM.  The headline metric is GTEPS: the
edges scanned by FirstFit summed over all rounds (sum of |adj(v)| over v in
W_r, over r), divided by the device time of the step; the color count is
reported against serial first-fit greedy.  Every rank runs its own replica
(coloring one graph has no data-path exchange), so the whole-job value is the
sum of the ranks' work over the slowest rank's time ("scaling": "weak").

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the stream the library launches on; the L2 cache is flushed (a 512 MiB
write) before every step, outside the events.  SM clocks and throttle reasons
are sampled with nvidia-smi during the timed steps.

--impl reference times the CPU oracle (the only reference this method has:
the paper publishes no code) on the host cores, on the same workload, metric
and unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402

METRIC_SINGLE = "GTEPS & #colors vs serial greedy"
HBM_FALLBACK_GBS = 6800.0

WORKLOADS = {
    "rmat20": ("RMAT scale 20, edge factor 16, (0.57,0.19,0.19,0.05), ids permuted, seed 0",
               lambda: gg.rmat20(0)),
    "stencil192": ("3-D 27-point stencil 192^3, natural order", lambda: gg.stencil27(192)),
    "er20k": ("uniform random graph n=20,000, average degree 10, seed 0", lambda: gg.er20k(0)),
    "stencil128": ("3-D 27-point stencil 128^3, natural order (profiling size)",
                   lambda: gg.stencil27(128)),
}
BATCH_WORKLOADS = {
    "batch512": ("512 graphs, n log-uniform in [1k, 200k]: 1/3 uniform (avg degree 4-32), 1/3 R-MAT "
                 "(ef 16, a,b,c,d = 0.57,0.19,0.19,0.05), 1/3 2-D 9-point / 3-D 27-point stencils, seed 0",
                 lambda: gg.batch_mix(512, 1000, 200000, 0)),
    "batch64": ("64 graphs of the same mix, n log-uniform in [1k, 50k], seed 1 (quick check)",
                lambda: gg.batch_mix(64, 1000, 50000, 1)),
}


def workload(name):
    """(description, maker) for a named workload, including the parametric
    er:N:D (uniform random graph, n = N, average degree D, seed 0) and
    rmat:S (R-MAT scale S, edge factor 16, the rmat20 parameters)."""
    if name in WORKLOADS:
        return WORKLOADS[name]
    parts = name.split(":")
    if parts[0] == "er" and len(parts) == 3:
        n, d = int(parts[1]), float(parts[2])
        return (f"uniform random graph n={n}, average degree {d:g}, seed 0",
                lambda: gg.uniform(n, d, 0))
    if parts[0] == "rmat" and len(parts) == 2:
        sc = int(parts[1])
        return (f"RMAT scale {sc}, edge factor 16, (0.57,0.19,0.19,0.05), seed 0",
                lambda: gg.rmat(sc, 16, (0.57, 0.19, 0.19), 0))
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(items, rank, world):
    """The share of independent work items (graphs) a rank colors: every
    world-th item, so each item is colored by exactly one rank."""
    return list(items)[rank::world]


def max_over_ranks(value, device=None):
    """Largest value over all ranks (the job's time is the slowest rank's);
    the identity when no process group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1606_06025_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(workload, mode):
    """DRAM bytes per launch from a committed ncu summary, only if it was taken
    on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    e = d.get(f"{workload}:{mode}")
    if not e or e.get("kernel_sources") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def alg_bytes(st, n, m, mode):
    """Algorithmic DRAM bytes of one coloring launch, as this implementation
    does the work (the byte model; the counts are measured on the device).

    Deterministic mode: 24 B per worklist entry a grid phase visits (entry 4,
    row offsets 8, bitmap word or own color 4, witness or lower-neighbour
    count 4, tentative color or commit write 4), 4 B per col_idx entry the grid
    reads (ConflictResolve scans, commit scatters, dependent scans), 2 B per
    16-bit W-adjacency entry the tail CTA reads (its per-vertex state is in
    shared memory), and for a hand-over 4 B per row entry of the worklist plus
    4 B per vertex (the pass over the colors).  Fast mode, per worklist vertex
    and round, 36 B (entry and row offsets in both phases, color read and
    writes) plus 4 B per entry FirstFit gathers (sum of D_r) and per entry
    ConflictResolve inspects.  Both: the init pass reads col_idx once (4 B per
    entry) and 24 B per vertex.  Neighbour color and bitmap accesses that hit
    the L2-resident arrays are not counted.  Topology-driven schedule
    (Algorithm 6), per iteration: the own color of all n vertices in both
    passes (8n), and per vertex colored tentatively its row offsets in both
    passes (16 B), its tentative write and its commit (8 B) and its row in
    both passes (8 B per entry); the last iteration only reads the n colors
    once."""
    if mode == "topo":
        return 8 * n * st["rounds"] + 4 * n + 24 * st["sum_w"] + 8 * st["sum_d"]
    if mode == "det":
        tail = 4 * st["tail_build"] + 4 * n if st["tail_rounds"] else 0
        return (24 * st["sum_touch"] + 4 * (st["sum_dscan"] + st["sum_scatter"] + st["sum_dep"])
                + 2 * st["tail_entries"] + tail + 4 * m + 24 * n)
    return (36 * st["sum_w"] + 4 * st["sum_d"] + 4 * st["sum_dscan"] + 4 * st["sum_next"]
            + 4 * m + 24 * n)


def paper_bytes(st):
    """Bytes of the same rounds done as Algorithms 4 and 5 print them (every
    round re-reads the whole row of every worklist vertex in FirstFit and in
    ConflictResolve): per round 4|W_r| worklist + 8|W_r| row offsets +
    2 x 4 D_r col_idx + 4|W_r| tentative color + 4|W_r| commit + 4 L_r pushed
    losers."""
    return 20 * st["sum_w"] + 8 * st["sum_d"] + 4 * st["sum_next"]


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling and wait (up to 5 s) for the first sample, so that
        nvidia-smi's own start-up is over before the timed region begins."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.02)
        self.lines.clear()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_info():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return model, os.cpu_count()


def oracle_baseline(g, budget_s=12.0):
    """The CPU oracle as it stands, single-threaded: det-SGR (what the GPU's
    det mode computes) and serial first-fit greedy (the paper's Serial)."""
    import oracle
    t0 = time.perf_counter()
    r = oracle.det_sgr(g)
    t_det = time.perf_counter() - t0
    runs = [t_det]
    while sum(runs) + t_det < budget_s and len(runs) < 5:
        t0 = time.perf_counter()
        oracle.det_sgr(g)
        runs.append(time.perf_counter() - t0)
    ts = []
    k_serial = 0
    while sum(ts) < 2.0 and len(ts) < 10:
        t0 = time.perf_counter()
        _, k_serial = oracle.serial_greedy(g)
        ts.append(time.perf_counter() - t0)
    return r, statistics.median(runs), len(runs), statistics.median(ts), k_serial


def run_reference(args, rank, world):
    if rank != 0:
        return
    desc, make = workload(args.workload)
    g = make()
    import oracle
    # warm-up and timed steps: each step is one full det-SGR run of the oracle
    for _ in range(args.warmup):
        oracle.det_sgr(g)
    times = []
    r = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.det_sgr(g)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = r.sum_d * args.steps / total / 1e9
    model, ncpu = cpu_info()
    line = {
        "impl": "reference", "metric": METRIC_SINGLE, "value": value, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m,
                   "mode": "det", "parallelism": "none (host CPU)"},
        "num_colors": r.num_colors, "rounds": r.rounds,
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"full det-SGR run of the {args.workload} workload per step",
                         "cpu": model, "host_cpus": ncpu},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local):
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.tune:
        fields = [int(x) for x in args.tune.split(",")]
        lm, ch, bps = fields[:3]
        al = fields[3] if len(fields) > 3 else 0
        tv = fields[4] if len(fields) > 4 else 0
        lib.sgr_set_tuning(light_max=lm, chunk=ch, blocks_per_sm=bps, active_lists=al,
                           tail_vertices=tv)
    desc, make = workload(args.workload)
    g = make()
    n, m = g.n, g.m
    ro = torch.from_numpy(g.row_offsets).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    colors = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    mode = args.mode + "+" + args.rule
    tuned = None
    if args.autotune:
        tuned, tuned_ms = lib.sgr_autotune(n, ro, ci, colors, mode, 3000, stream)

    def step():
        return lib.sgr_color(n, ro, ci, colors, mode, stream)

    for _ in range(max(args.warmup, 0)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    step_ms, kern_ms, stats = [], [], []
    k = 0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k = step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        st = lib.sgr_last_stats()
        stats.append(st)
        kern_ms.append(st["device_ms"])
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = max_over_ranks(sum(step_ms), dev)
    if world > 1:
        torch.distributed.barrier()
    st = stats[-1]
    work = st["sum_d"] * args.steps * world
    value = work / (total_ms * 1e-3) / 1e9
    # end to end through the host-buffer entry: H2D of the CSR, coloring, D2H of colors
    ro_h = torch.from_numpy(g.row_offsets).pin_memory().numpy()
    ci_h = torch.from_numpy(g.col_idx).pin_memory().numpy()
    col_h = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    if args.timeline and rank == 0:
        tl = lib.sgr_last_trace()
        with open(args.timeline, "w") as f:
            json.dump({"workload": args.workload, "mode": mode, "init_ns": tl["init_ns"],
                       **{k: v.tolist() for k, v in tl.items() if k != "init_ns"}}, f)
    e2e_ms = []
    for i in range(0 if args.no_e2e else args.warmup + args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lib.sgr_color_host(n, ro_h, ci_h, col_h, mode, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_total = max_over_ranks(sum(e2e_ms) if e2e_ms else float("nan"), dev)
    e2e_value = st["sum_d"] * args.steps * world / (e2e_total * 1e-3) / 1e9
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_src = read_peaks()
    kmean = statistics.mean(kern_ms)
    ab = alg_bytes(st, n, m, args.mode)
    achieved = ab / (kmean * 1e-3) / 1e9
    pb = paper_bytes(st)
    line = {
        "metric": METRIC_SINGLE, "value": value, "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": n, "m": m,
                   "mode": args.mode, "rule": args.rule, "tuning": lib.sgr_get_tuning(),
                   "tuning_source": "autotuned" if tuned else ("--tune" if args.tune else "default"),
                   "l2": "flushed (512 MiB write) before every step",
                   "parallelism": f"replicas x{world}"},
        "num_colors": k, "rounds": st["rounds"], "sum_d": st["sum_d"],
        "useful_gteps": m / (total_ms / args.steps * 1e-3) / 1e9,
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "GTEPS", "ms_per_step": e2e_total / args.steps,
                "h2d_bytes_per_step": 4 * (n + 1) + 4 * m, "d2h_bytes_per_step": 4 * n},
        # per step: the round kernel, then (det) the activation-list kernel and
        # the tail kernel, each of which returns at once when not handed over
        # (topology-driven: two kernels per iteration, and the final one that finds nothing)
        "gpu_launches": args.steps * {"fast": 1, "det": 3}.get(args.mode, 2 * (st["rounds"] + 1)),
        "step_ms": {"min": min(step_ms), "max": max(step_ms)},
        "tail_rounds": st["tail_rounds"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": read_traffic(args.workload, args.mode) if args.rule == "low_keeps" else None,
                     "alg_bytes_per_launch": ab, "kernel_ms": kmean,
                     "paper_model": {"bytes_per_launch": pb, "equivalent_gbs": pb / (kmean * 1e-3) / 1e9,
                                     "frac": pb / (kmean * 1e-3) / 1e9 / peak,
                                     "what": "Algorithms 4/5 as printed: rows re-read every round"},
                     "kernel": ("the coloring launches of one call, timed together on their stream: "
                                "sgr_color_kernel (init, rounds on the grid), its activation-list "
                                "variant, sgr_tail_kernel (last rounds in one CTA)") if args.mode != "topo" else
                               ("the topology-driven iterations of one call (topo_assign_kernel and "
                                "topo_resolve_kernel per iteration, host loop on a flag), event to event"),
                     "peak_source": peak_src + " of measured"
                     if peak_src.startswith("measured") else peak_src},
    }
    if not args.no_cpu_baseline and world == 1:
        r, t_det, runs, t_serial, k_serial = oracle_baseline(g)
        model, ncpu = cpu_info()
        line["cpu_baseline"] = {
            "value": r.sum_d / t_det / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{runs} full det-SGR runs of the workload (median), single thread",
            "cpu": model, "host_cpus": ncpu,
            "serial_greedy_ms": t_serial * 1e3, "serial_greedy_colors": k_serial,
        }
        line["serial_greedy_colors"] = k_serial
        line["colors_vs_serial"] = k / k_serial if k_serial else None
        line["speedup_vs_serial_greedy"] = t_serial * 1e3 / (total_ms / args.steps)
        if args.mode == "det" and args.rule == "low_keeps":
            line["det_matches_oracle"] = bool(
                np.array_equal(colors.cpu().numpy(), r.colors))
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args, rank, world, local):
    """Batched workload: graphs/s of one sgr_color_batch call over the whole mix,
    against the same graphs colored by one sgr_color call each (the plain path)."""
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    desc, make = BATCH_WORKLOADS[args.workload]
    b = make()
    if world > 1:  # shard the graphs by rank: no exchange on the data path
        b = gg.pack(shard(b.graphs, rank, world))
    n, m, G = int(b.vtx_off[-1]), int(b.edge_off[-1]), b.G
    ro = torch.from_numpy(b.row_offsets).to(dev)
    ci = torch.from_numpy(b.col_idx).to(dev)
    colors = torch.empty(n, dtype=torch.int32, device=dev)
    kk = np.zeros(G, dtype=np.int32)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    mode = args.mode

    def step():
        lib.sgr_color_batch(G, b.vtx_off, b.edge_off, ro, ci, colors, kk, mode, stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ms = []
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    st = lib.sgr_last_stats()
    total = max_over_ranks(sum(ms), dev)
    value = G * world * args.steps / (total * 1e-3)
    # the plain path: one sgr_color per graph, same graphs, same device buffers
    seq_ms = []
    offs = [(int(b.vtx_off[i]), int(b.vtx_off[i + 1]), int(b.edge_off[i]), int(b.edge_off[i + 1]))
            for i in range(G)]
    dev_graphs = []
    for i, (v0, v1, e0_, e1_) in enumerate(offs):
        r = torch.from_numpy(b.graphs[i].row_offsets).to(dev)
        c = torch.from_numpy(b.graphs[i].col_idx).to(dev) if e1_ > e0_ else torch.zeros(
            4, dtype=torch.int32, device=dev)
        dev_graphs.append((v1 - v0, r, c))
    out = torch.empty(max(x[0] for x in dev_graphs) + 1, dtype=torch.int32, device=dev)
    for rep in range(2):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for nn, r, c in dev_graphs:
            lib.sgr_color(nn, r, c, out, mode, stream)
        e1.record(stream)
        e1.synchronize()
        if rep == 1:
            seq_ms.append(e0.elapsed_time(e1))
    seq_value = G / (seq_ms[0] * 1e-3)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": "batched graphs/s", "value": value, "unit": "graphs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "graphs": G, "n": n, "m": m,
                   "mode": mode, "l2": "flushed (512 MiB write) before every step",
                   "parallelism": f"graphs sharded by rank x{world}"},
        "rounds": st["rounds"], "sum_d": st["sum_d"], "kernel_ms": st["device_ms"],
        "sequential_graphs_per_s": seq_value, "speedup_vs_sequential": value / seq_value,
        "clocks": clocks, "gpu_launches": args.steps * 5,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve_burst(args, rank, world, local):
    """The 512-graph batch mix submitted at once to the server (host buffers in,
    colors out), against the same graphs colored one at a time through the
    host-buffer entry point: graphs/s, and p50/p99 request latency."""
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    b = gg.batch_mix(512, 1000, 200000, 0)
    graphs = shard(b.graphs, rank, world)
    outs = [np.empty(g.n, dtype=np.int32) for g in graphs]
    for g, o in zip(graphs[:8], outs):  # warm-up
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, o, "det")
    t0 = time.perf_counter()
    for g, o in zip(graphs, outs):
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, o, "det")
    seq_s = time.perf_counter() - t0
    seq_gps = len(graphs) / seq_s
    runs = []
    import threading
    clients = 4  # concurrent submitters, each with a share of the graphs
    with lib.Server(hbm_budget_bytes=int(args.budget_gb * (1 << 30)), mode="det",
                    staging_bytes=8 << 30) as srv:
        for rep in range(max(args.warmup, 1) + args.steps):
            got = [None] * len(graphs)

            def client(c):
                mine = list(range(c, len(graphs), clients))
                ids = [(i, srv.submit(graphs[i].row_offsets, graphs[i].col_idx)) for i in mine]
                for i, rid in ids:
                    got[i] = srv.poll(rid, graphs[i].n, timeout_ms=-1)

            t0 = time.perf_counter()
            th = [threading.Thread(target=client, args=(c,)) for c in range(clients)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            dt = time.perf_counter() - t0
            if rep >= max(args.warmup, 1):
                runs.append(dt)
        st = srv.stats()
    ok = all(np.array_equal(c, o) for (c, _), o in zip(got, outs))
    value = len(graphs) * world / statistics.median(runs)
    if rank != 0:
        return
    line = {
        "metric": "served graphs/s, p50/p99 latency", "value": value, "unit": "graphs/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
        "ms_per_step": statistics.median(runs) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "serve512", "graphs": len(graphs),
                   "submission": "all at once from 4 client threads",
                   "description": BATCH_WORKLOADS["batch512"][0], "mode": "det",
                   "hbm_budget_gb": args.budget_gb},
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "sequential_host_graphs_per_s": seq_gps, "speedup_vs_sequential": value / seq_gps,
        "results_equal_sequential": ok, "launches": st["launches"], "rounds": st["rounds"],
    }
    print(json.dumps(line), flush=True)


def run_serve(args, rank, world, local):
    """Served workload: an open-loop Poisson stream of requests drawn from a
    pool of distinct-seed graphs (sizes log-uniform in [1k, 4M], the batch
    mix's kinds), through the continuous-batching server with its HBM budget,
    against the same requests colored one at a time by sgr_color_host (both
    include the host-device copies)."""
    import threading

    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    specs = gg.mix_specs(args.pool, 1000, 4000000, 7 + rank)
    pool = [gg.mix_graph(s) for s in specs]
    rnd = np.random.default_rng(11 + rank)
    picks = rnd.integers(0, len(pool), size=args.requests)
    # sequential plain path: mean time per request over the pick distribution
    seq = []
    for g in pool:
        out = np.empty(g.n, dtype=np.int32)
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, out, "det")  # warm-up
        t0 = time.perf_counter()
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, out, "det")
        seq.append(time.perf_counter() - t0)
    seq_mean = float(np.mean([seq[j] for j in picks]))
    seq_gps = 1.0 / seq_mean
    budget = int(args.budget_gb * (1 << 30))
    results = {}

    def drain(srv, ids, done):
        for i, rid in ids:
            got = srv.poll(rid, pool[picks[i]].n, timeout_ms=-1)
            done[i] = (time.perf_counter(), got[1])

    with lib.Server(hbm_budget_bytes=budget, mode="det") as srv:
        # capacity: a burst of requests submitted at once
        burst = min(args.requests, 64)
        t0 = time.perf_counter()
        bids = [(i, srv.submit(pool[picks[i]].row_offsets, pool[picks[i]].col_idx))
                for i in range(burst)]
        bdone = {}
        drain(srv, bids, bdone)
        capacity = burst / (time.perf_counter() - t0)
    rate = args.rate if args.rate > 0 else 0.7 * capacity
    gaps = rnd.exponential(1.0 / rate, size=args.requests)
    with lib.Server(hbm_budget_bytes=budget, mode="det") as srv:
        sub_t = {}
        ids = []
        lock = threading.Lock()
        done = {}
        t_start = time.perf_counter()
        t_next = t_start

        def poller():  # non-blocking sweeps, so each completion is seen when it happens
            outstanding = []
            while len(done) < args.requests:
                with lock:
                    outstanding.extend(ids)
                    ids.clear()
                still = []
                for i, rid in outstanding:
                    got = srv.poll(rid, pool[picks[i]].n, timeout_ms=0)
                    if got is None:
                        still.append((i, rid))
                    else:
                        done[i] = (time.perf_counter(), got[1])
                outstanding = still
                time.sleep(0.0002)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        for i in range(args.requests):
            t_next += gaps[i]
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            g = pool[picks[i]]
            sub_t[i] = time.perf_counter()
            rid = srv.submit(g.row_offsets, g.col_idx)
            with lock:
                ids.append((i, rid))
        th.join()
        t_end = max(t for t, _ in done.values())
        st = srv.stats()
    lat = np.array([(done[i][0] - sub_t[i]) * 1e3 for i in range(args.requests)])
    value = args.requests / (t_end - t_start)
    if rank != 0:
        return
    sizes = [pool[j].n for j in picks]
    line = {
        "metric": "served graphs/s, p50/p99 latency", "value": value, "unit": "graphs/s",
        "n_gpus": world, "steps": args.requests, "warmup": burst, "ms_per_step": 1e3 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "serve", "requests": args.requests, "pool": args.pool,
                   "sizes": "log-uniform [1k, 4M] vertices; 1/3 uniform, 1/3 R-MAT, 1/3 stencils",
                   "arrivals": "open-loop Poisson", "arrival_rate_per_s": rate,
                   "hbm_budget_gb": args.budget_gb, "mode": "det",
                   "mean_vertices": float(np.mean(sizes))},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
        # open loop: value follows the arrival rate while the server keeps up,
        # so capacity is compared with capacity
        "burst_capacity_graphs_per_s": capacity, "sequential_graphs_per_s": seq_gps,
        "capacity_vs_sequential": capacity / seq_gps,
        "launches": st["launches"], "rounds": st["rounds"],
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="rmat20",
                    help="rmat20 | stencil192 | er20k | stencil128 | batch512 | batch64 | serve | "
                         "serve512 | er:N:D | rmat:S")
    ap.add_argument("--mode", choices=["det", "fast", "topo"], default="det",
                    help="det: the worklist rounds; fast: racy in place; topo: the deterministic "
                         "rounds on the topology-driven schedule of Algorithm 6 (comparison)")
    ap.add_argument("--rule", choices=["low_keeps", "low_loses", "degree"], default="low_keeps",
                    help="loser rule (Sect. 3.2 heuristic = degree; Alg. 5 as printed = low_loses)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--timeline", default="", help="write the per-round device timeline here")
    ap.add_argument("--tune", default="",
                    help="light_max,chunk,blocks_per_sm[,active_lists[,tail_vertices]] (0 = default)")
    ap.add_argument("--autotune", action="store_true",
                    help="measure the tuning candidates on the workload before timing")
    ap.add_argument("--requests", type=int, default=600, help="serve: requests in the stream")
    ap.add_argument("--pool", type=int, default=24, help="serve: distinct graphs drawn from")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serve: arrivals per second (0: 0.7 x measured capacity)")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serve: server HBM budget")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload in BATCH_WORKLOADS:
        run_batch(args, rank, world, local)
    elif args.workload == "serve":
        run_serve(args, rank, world, local)
    elif args.workload == "serve512":
        run_serve_burst(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
