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

The default run (rmat20, one GPU) also measures the other configurations and
puts them in the same JSON line under "configs": the 192^3 stencil and the
20k uniform graph, the 512-graph batch (graphs/s against one sgr_color call
per graph), the same 512 graphs submitted at once to the server, and an open
Poisson stream of served requests (1k-4M vertices, 64 GB budget) at 0.7 x the
server's burst capacity and at the sequential path's capacity.  Every
deterministic result is checked against the oracle (its colors, or digests
the oracle wrote into tests/golden).  roofline.frac is section 8(d)'s model:
the bytes Algorithms 4/5 as printed would move, over the device time.

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


def golden(name):
    """Oracle-written expected values (tests/golden, written by scripts that
    call only oracle/ and graphgen/)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    with open(path) as f:
        return json.load(f)


def digest(a) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


GOLDEN_SINGLE = {"rmat20": "rmat20", "stencil192": "stencil27_192", "er20k": "er20k"}


def roofline_record(st, n, m, mode, kmean, workload, rule):
    """Section 8(d)'s roofline: the bytes of the printed Algorithms 4/5 per
    call (20 B per worklist vertex and round, 8 B per FirstFit edge visit, 4 B
    per pushed loser, from the device's own counts) over the call's device
    time, against the measured copy bandwidth.  The implementation's own byte
    model is kept beside it as frac_impl."""
    peak, peak_src = read_peaks()
    pb = paper_bytes(st)
    ab = alg_bytes(st, n, m, mode)
    achieved = pb / (kmean * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": read_traffic(workload, mode) if rule == "low_keeps" else None,
            "model": "paper: 20*sum|W_r| + 8*sum D_r + 4*sum L_r bytes per call (Algorithms 4/5 as printed)",
            "bytes_per_launch": pb, "kernel_ms": kmean,
            "frac_impl": ab / (kmean * 1e-3) / 1e9 / peak,
            "impl_model": {"bytes_per_launch": ab, "achieved_gbs": ab / (kmean * 1e-3) / 1e9,
                           "what": "bytes this implementation moves by its own model (bitmaps, "
                                   "witnesses, tail CTA; see alg_bytes)"},
            "kernel": ("the coloring launches of one call, timed together on their stream: "
                       "sgr_color_kernel (init, rounds on the grid), its activation-list variant, "
                       "sgr_tail_kernel (last rounds in one CTA)") if mode != "topo" else
                      ("the topology-driven iterations of one call (topo_assign_kernel and "
                       "topo_resolve_kernel per iteration, host loop on a flag), event to event"),
            "peak_source": peak_src + " of measured" if peak_src.startswith("measured") else peak_src}


def measure_single(lib, dev, stream, name, g, args, steps, warmup, flush, world=1, e2e=True,
                   cpu="det", check=True):
    """One workload graph on the device: K timed steps (L2 flushed before each),
    the section 8(d) roofline, end to end through the host-buffer entry, the
    CPU oracle beside it, and bit-exactness against the oracle."""
    import torch
    n, m = g.n, g.m
    ro = torch.from_numpy(g.row_offsets).to(dev)
    ci = torch.from_numpy(g.col_idx).to(dev)
    colors = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    mode = args.mode + "+" + args.rule
    for _ in range(max(warmup, 0)):
        flush.fill_(1)
        lib.sgr_color(n, ro, ci, colors, mode, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev.index)
    sampler.start()
    step_ms, kern_ms, stats = [], [], []
    k = 0
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k = lib.sgr_color(n, ro, ci, colors, mode, stream)
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
    timeline = lib.sgr_last_trace() if args.timeline else None
    got = colors[:n].cpu().numpy()
    rec = {
        "workload": name, "value": st["sum_d"] * steps * world / (total_ms * 1e-3) / 1e9, "unit": "GTEPS",
        "ms_per_step": total_ms / steps, "n": n, "m": m, "num_colors": k, "rounds": st["rounds"],
        "sum_d": st["sum_d"], "useful_gteps": m / (total_ms / steps * 1e-3) / 1e9, "clocks": clocks,
        "step_ms": {"min": min(step_ms), "max": max(step_ms)}, "tail_rounds": st["tail_rounds"],
        "roofline": roofline_record(st, n, m, args.mode, statistics.mean(kern_ms), name, args.rule),
        "gpu_launches": steps * {"fast": 1, "det": 3}.get(args.mode, 2 * (st["rounds"] + 1)),
    }
    if e2e:
        ro_h = torch.from_numpy(g.row_offsets).pin_memory().numpy()
        ci_h = torch.from_numpy(g.col_idx).pin_memory().numpy()
        col_h = torch.empty(max(n, 1), dtype=torch.int32).pin_memory().numpy()
        e2e_ms = []
        for i in range(warmup + steps):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lib.sgr_color_host(n, ro_h, ci_h, col_h, mode, stream)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                e2e_ms.append(e0.elapsed_time(e1))
        e2e_total = max_over_ranks(sum(e2e_ms), dev)
        rec["e2e"] = {"value": st["sum_d"] * steps * world / (e2e_total * 1e-3) / 1e9, "unit": "GTEPS",
                      "ms_per_step": e2e_total / steps, "h2d_bytes_per_step": 4 * (n + 1) + 4 * m,
                      "d2h_bytes_per_step": 4 * n}
    det = args.mode == "det" and args.rule == "low_keeps"
    if cpu and world == 1:
        model, ncpu = cpu_info()
        if cpu == "det":
            r, t_det, runs, t_serial, k_serial = oracle_baseline(g)
            rec["cpu_baseline"] = {
                "value": r.sum_d / t_det / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                "sample": f"{runs} full det-SGR runs of the workload (median), single thread",
                "cpu": model, "host_cpus": ncpu, "serial_greedy_ms": t_serial * 1e3,
                "serial_greedy_colors": k_serial}
            if det:
                rec["det_matches_oracle"] = bool(np.array_equal(got, r.colors))
        else:  # serial greedy only: the det oracle takes minutes on the largest graphs
            import oracle
            ts = []
            k_serial = 0
            while sum(ts) < 3.0 and len(ts) < 10:
                t0 = time.perf_counter()
                _, k_serial = oracle.serial_greedy(g)
                ts.append(time.perf_counter() - t0)
            t_serial = statistics.median(ts)
            rec["cpu_baseline"] = {
                "value": m / t_serial / 1e9, "unit": "GTEPS (m / time: one pass)", "cores": 1,
                "kind": "oracle", "sample": f"{len(ts)} serial first-fit greedy runs (median), single thread",
                "cpu": model, "host_cpus": ncpu, "serial_greedy_ms": t_serial * 1e3,
                "serial_greedy_colors": k_serial}
        rec["serial_greedy_colors"] = k_serial
        rec["colors_vs_serial"] = k / k_serial if k_serial else None
        rec["speedup_vs_serial_greedy"] = t_serial * 1e3 / (total_ms / steps)
    if det and check and "det_matches_oracle" not in rec and name in GOLDEN_SINGLE:
        gold = golden("configs.json")[GOLDEN_SINGLE[name]]
        rec["det_matches_oracle"] = bool(digest(got) == gold["det_colors_sha256"]
                                         and k == gold["det_num_colors"])
        rec["det_oracle_source"] = "tests/golden/configs.json (written by make_golden.py from the oracle)"
    return rec, timeline


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
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if args.autotune:
        ro = torch.from_numpy(g.row_offsets).to(dev)
        ci = torch.from_numpy(g.col_idx).to(dev)
        colors = torch.empty(g.n, dtype=torch.int32, device=dev)
        tuned, tuned_ms = lib.sgr_autotune(g.n, ro, ci, colors, args.mode + "+" + args.rule, 3000, stream)
        del ro, ci, colors
    rec, timeline = measure_single(lib, dev, stream, args.workload, g, args, args.steps, args.warmup, flush,
                                   world=world, e2e=not args.no_e2e,
                                   cpu=None if args.no_cpu_baseline else "det")
    if args.timeline and rank == 0 and timeline is not None:
        with open(args.timeline, "w") as f:
            json.dump({"workload": args.workload, "mode": args.mode, "init_ns": timeline["init_ns"],
                       **{k: v.tolist() for k, v in timeline.items() if k != "init_ns"}}, f)
    suite = (world == 1 and not args.no_suite and args.workload == "rmat20" and args.mode == "det"
             and args.rule == "low_keeps" and not args.tune and not args.autotune)
    configs = {}
    if suite:
        del g
        configs = run_suite(lib, dev, stream, args, flush)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC_SINGLE, "value": rec["value"], "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": rec["n"], "m": rec["m"],
                   "mode": args.mode, "rule": args.rule, "tuning": lib.sgr_get_tuning(),
                   "tuning_source": "autotuned" if tuned else ("--tune" if args.tune else "default"),
                   "l2": "flushed (512 MiB write) before every step",
                   "parallelism": f"replicas x{world}"},
    }
    for key in ("num_colors", "rounds", "sum_d", "useful_gteps", "clocks", "e2e", "gpu_launches", "step_ms",
                "tail_rounds", "roofline", "cpu_baseline", "serial_greedy_colors", "colors_vs_serial",
                "speedup_vs_serial_greedy", "det_matches_oracle"):
        if key in rec:
            line[key] = rec[key]
    if configs:
        line["configs"] = configs
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_suite(lib, dev, stream, args, flush):
    """The other configurations, each as a sub-record of the headline line:
    the 192^3 stencil and the 20k uniform graph (single graphs), the 512-graph
    batch, the same 512 graphs submitted at once to the server, and the open
    Poisson stream of served requests at two arrival rates."""
    out = {}
    t0 = time.time()
    steps = max(3, min(args.steps, 10))
    g = gg.stencil27(192)
    out["stencil192"], _ = measure_single(lib, dev, stream, "stencil192", g, args, steps, args.warmup, flush,
                                          cpu="serial")
    out["stencil192"]["description"] = WORKLOADS["stencil192"][0]
    del g
    g = gg.er20k(0)
    out["er20k"], _ = measure_single(lib, dev, stream, "er20k", g, args, args.steps, args.warmup, flush, cpu="det")
    out["er20k"]["description"] = WORKLOADS["er20k"][0]
    del g
    out["batch512"] = measure_batch(lib, dev, stream, "batch512", steps, args.warmup, flush)
    out["serve512"] = measure_serve_burst(lib, args.budget_gb, steps, max(args.warmup, 1))
    out["serve"] = measure_serve(lib, args.requests, args.pool, args.rate, args.budget_gb)
    if args.rate == 0:  # also at the sequential path's capacity
        out["serve_at_sequential_rate"] = measure_serve(lib, max(1, args.requests // 2), args.pool,
                                                        -1.0, args.budget_gb)
    out["suite_wall_s"] = time.time() - t0
    return out


def measure_batch(lib, dev, stream, name, steps, warmup, flush, rank=0, world=1, autotune=False):
    """Batched workload: graphs/s of one sgr_color_batch call over the whole mix,
    against the same graphs colored by one sgr_color call each (the plain path),
    with every graph's colors checked against the oracle's digest."""
    import torch
    desc, make = BATCH_WORKLOADS[name]
    b = make()
    if world > 1:  # shard the graphs by rank: no exchange on the data path
        b = gg.pack(shard(b.graphs, rank, world))
    n, m, G = int(b.vtx_off[-1]), int(b.edge_off[-1]), b.G
    ro = torch.from_numpy(b.row_offsets).to(dev)
    ci = torch.from_numpy(b.col_idx).to(dev)
    colors = torch.empty(n, dtype=torch.int32, device=dev)
    kk = np.zeros(G, dtype=np.int32)
    mode = "det"

    def step():
        lib.sgr_color_batch(G, b.vtx_off, b.edge_off, ro, ci, colors, kk, mode, stream)

    tuned = None
    if autotune:
        tuned = lib.sgr_autotune_batch(G, b.vtx_off, b.edge_off, ro, ci, colors, kk, mode, 3000, stream)
    for _ in range(warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(dev.index)
    sampler.start()
    ms, kms = [], []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(lib.sgr_last_stats()["device_ms"])
    clocks = sampler.stop()
    st = lib.sgr_last_stats()
    total = max_over_ranks(sum(ms), dev)
    value = G * world * steps / (total * 1e-3)
    got = colors.cpu().numpy()
    # the plain path: one sgr_color per graph, same graphs, same device buffers
    offs = [(int(b.vtx_off[i]), int(b.vtx_off[i + 1]), int(b.edge_off[i]), int(b.edge_off[i + 1]))
            for i in range(G)]
    dev_graphs = []
    for i, (v0, v1, e0_, e1_) in enumerate(offs):
        r = torch.from_numpy(b.graphs[i].row_offsets).to(dev)
        c = torch.from_numpy(b.graphs[i].col_idx).to(dev) if e1_ > e0_ else torch.zeros(
            4, dtype=torch.int32, device=dev)
        dev_graphs.append((v1 - v0, r, c))
    out = torch.empty(max(x[0] for x in dev_graphs) + 1, dtype=torch.int32, device=dev)
    seq_ms = []
    same_as_alone = True
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
    for i in range(0, G, max(1, G // 16)):  # a sample of graphs, alone, against their batch slice
        nn, r, c = dev_graphs[i]
        lib.sgr_color(nn, r, c, out, mode, stream)
        same_as_alone &= bool(np.array_equal(out[:nn].cpu().numpy(), got[offs[i][0]:offs[i][1]]))
    seq_value = G / (seq_ms[0] * 1e-3)
    rec = {"workload": name, "description": desc, "metric": "batched graphs/s", "value": value,
           "unit": "graphs/s", "ms_per_step": total / steps, "graphs": G, "n": n, "m": m, "mode": mode,
           "rounds": st["rounds"], "sum_d": st["sum_d"], "kernel_ms": statistics.mean(kms),
           "sequential_graphs_per_s": seq_value, "speedup_vs_sequential": value / seq_value,
           "clocks": clocks, "gpu_launches": steps * 5,
           "roofline": roofline_record(st, n, m, "det", statistics.mean(kms), name, "low_keeps"),
           "batch_slices_equal_alone": same_as_alone, "tuning": lib.sgr_get_tuning(),
           "tuning_source": "autotuned (sgr_autotune_batch, 3 s budget)" if tuned else "default"}
    if name == "batch512" and world == 1:
        gold = golden("mix_digests.json")["batch512"]["graphs"]
        bad = sum(1 for i, gr in enumerate(gold)
                  if digest(got[offs[i][0]:offs[i][1]]) != gr["det_colors_sha256"]
                  or kk[i] != gr["det_num_colors"])
        rec["det_matches_oracle"] = bad == 0
        rec["det_oracle_source"] = "tests/golden/mix_digests.json (per-graph digests from the oracle)"
        # the oracle on a bounded sample of the mix, single thread
        import oracle
        t0 = time.perf_counter()
        done = 0
        for g in b.graphs:
            oracle.det_sgr(g)
            done += 1
            if time.perf_counter() - t0 > 10.0:
                break
        el = time.perf_counter() - t0
        model, ncpu = cpu_info()
        rec["cpu_baseline"] = {"value": done / el, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                               "sample": f"det-SGR of the first {done} graphs of the mix, single thread",
                               "cpu": model, "host_cpus": ncpu}
    return rec


def run_batch(args, rank, world, local):
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    rec = measure_batch(lib, dev, stream, args.workload, args.steps, args.warmup, flush, rank, world,
                        autotune=args.autotune)
    if rank == 0:
        line = {"metric": rec.pop("metric"), "value": rec.pop("value"), "unit": rec.pop("unit"),
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": rec.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": args.workload, "description": rec.pop("description"),
                           "graphs": rec["graphs"], "n": rec["n"], "m": rec["m"], "mode": "det",
                           "l2": "flushed (512 MiB write) before every step",
                           "parallelism": f"graphs sharded by rank x{world}"}, **rec}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_serve_burst(lib, budget_gb, steps, warmup, rank=0, world=1):
    """The 512-graph batch mix submitted at once to the server (host buffers in,
    colors out), against the same graphs colored one at a time through the
    host-buffer entry point: graphs/s, and p50/p99 request latency; every result
    checked against the oracle's digest."""
    b = gg.batch_mix(512, 1000, 200000, 0)
    gold = golden("mix_digests.json")["batch512"]["graphs"]
    idx = shard(range(b.G), rank, world)
    graphs = [b.graphs[i] for i in idx]
    outs = [np.empty(g.n, dtype=np.int32) for g in graphs]
    for g, o in zip(graphs[:8], outs):  # warm-up
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, o, "det")
    t0 = time.perf_counter()
    for g, o in zip(graphs, outs):
        lib.sgr_color_host(g.n, g.row_offsets, g.col_idx, o, "det")
    seq_s = time.perf_counter() - t0
    seq_gps = len(graphs) / seq_s
    runs = []
    clients = 4  # concurrent submitters, each with a share of the graphs
    with lib.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)), mode="det", staging_bytes=8 << 30) as srv:
        for rep in range(warmup + steps):
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
            if rep >= warmup:
                runs.append(dt)
        st = srv.stats()
    ok = all(digest(c) == gold[i]["det_colors_sha256"] and k == gold[i]["det_num_colors"]
             for i, (c, k) in zip(idx, got))
    value = len(graphs) * world / statistics.median(runs)
    return {"workload": "serve512", "metric": "served graphs/s, p50/p99 latency", "value": value,
            "unit": "graphs/s", "ms_per_step": statistics.median(runs) * 1e3, "graphs": len(graphs),
            "submission": "all at once from 4 client threads", "description": BATCH_WORKLOADS["batch512"][0],
            "mode": "det", "hbm_budget_gb": budget_gb, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "sequential_host_graphs_per_s": seq_gps, "speedup_vs_sequential": value / seq_gps,
            "det_matches_oracle": ok, "launches": st["launches"], "rounds": st["rounds"],
            "colored_alone": st["direct"], "latency": "submit to completion, host buffers (H2D and D2H included)"}


def run_serve_burst(args, rank, world, local):
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    rec = measure_serve_burst(lib, args.budget_gb, args.steps, max(args.warmup, 1), rank, world)
    if rank != 0:
        return
    line = {"metric": rec.pop("metric"), "value": rec.pop("value"), "unit": rec.pop("unit"), "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 1), "ms_per_step": rec.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": "serve512", "graphs": rec["graphs"],
                                            "hbm_budget_gb": args.budget_gb}, **rec}
    print(json.dumps(line), flush=True)


def measure_serve(lib, requests, pool_size, rate, budget_gb, rank=0):
    """Served workload: an open-loop Poisson stream of requests drawn from a
    pool of distinct-seed graphs (sizes log-uniform in [1k, 4M], the batch
    mix's kinds), through the continuous-batching server with its HBM budget,
    against the same requests colored one at a time by sgr_color_host (both
    include the host-device copies).  rate > 0: arrivals per second; 0: 0.7 x
    the server's measured burst capacity; < 0: the sequential path's
    capacity."""
    specs = gg.mix_specs(pool_size, 1000, 4000000, 7 + rank)
    pool = [gg.mix_graph(s) for s in specs]
    gold = None
    if pool_size == 24 and rank == 0:
        gold = golden("mix_digests.json")["serve_pool"]["graphs"]
    rnd = np.random.default_rng(11 + rank)
    picks = rnd.integers(0, len(pool), size=requests)
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
    budget = int(budget_gb * (1 << 30))

    def drain(srv, ids, done):
        for i, rid in ids:
            got = srv.poll(rid, pool[picks[i]].n, timeout_ms=-1)
            done[i] = (time.perf_counter(), got[1])

    with lib.Server(hbm_budget_bytes=budget, mode="det") as srv:
        # capacity: a burst of requests submitted at once
        burst = min(requests, 64)
        t0 = time.perf_counter()
        bids = [(i, srv.submit(pool[picks[i]].row_offsets, pool[picks[i]].col_idx)) for i in range(burst)]
        bdone = {}
        drain(srv, bids, bdone)
        capacity = burst / (time.perf_counter() - t0)
    if rate > 0:
        lam, rate_src = rate, "stated"
    elif rate == 0:
        lam, rate_src = 0.7 * capacity, "0.7 x measured burst capacity"
    else:
        lam, rate_src = seq_gps, "the sequential path's capacity"
    gaps = rnd.exponential(1.0 / lam, size=requests)
    bad = []
    with lib.Server(hbm_budget_bytes=budget, mode="det") as srv:
        sub_t = {}
        ids = []
        lock = threading.Lock()
        done = {}
        t_start = time.perf_counter()
        t_next = t_start

        def poller():  # non-blocking sweeps, so each completion is seen when it happens
            outstanding = []
            while len(done) < requests:
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
                        if gold is not None:
                            gr = gold[picks[i]]
                            if digest(got[0]) != gr["det_colors_sha256"] or got[1] != gr["det_num_colors"]:
                                bad.append(i)
                outstanding = still
                time.sleep(0.0002)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        for i in range(requests):
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
    lat = np.array([(done[i][0] - sub_t[i]) * 1e3 for i in range(requests)])
    value = requests / (t_end - t_start)
    sizes = [pool[j].n for j in picks]
    rec = {"workload": "serve", "metric": "served graphs/s, p50/p99 latency", "value": value,
           "unit": "graphs/s", "ms_per_step": 1e3 / value, "requests": requests, "pool": pool_size,
           "sizes": "log-uniform [1k, 4M] vertices; 1/3 uniform, 1/3 R-MAT, 1/3 stencils",
           "arrivals": "open-loop Poisson", "arrival_rate_per_s": lam, "arrival_rate": rate_src,
           "hbm_budget_gb": budget_gb, "mode": "det", "mean_vertices": float(np.mean(sizes)),
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "server_p50_ms": st["p50_ms"], "server_p99_ms": st["p99_ms"],
           # open loop: value follows the arrival rate while the server keeps up,
           # so capacity is compared with capacity
           "burst_capacity_graphs_per_s": capacity, "sequential_graphs_per_s": seq_gps,
           "capacity_vs_sequential": capacity / seq_gps, "launches": st["launches"], "rounds": st["rounds"],
           "colored_alone": st["direct"],
           "latency": "submit to completion, host buffers (H2D and D2H included)"}
    if gold is not None:
        rec["det_matches_oracle"] = not bad
        rec["det_oracle_source"] = "tests/golden/mix_digests.json serve_pool (per-graph digests from the oracle)"
    return rec


def run_serve(args, rank, world, local):
    import torch

    from paper_1606_06025_gb300 import sgrcolor as lib

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    rec = measure_serve(lib, args.requests, args.pool, args.rate, args.budget_gb, rank)
    if rank != 0:
        return
    line = {"metric": rec.pop("metric"), "value": rec.pop("value"), "unit": rec.pop("unit"), "n_gpus": world,
            "steps": args.requests, "warmup": 64, "ms_per_step": rec.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": "serve", "requests": args.requests, "pool": args.pool,
                                            "hbm_budget_gb": args.budget_gb}, **rec}
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
    ap.add_argument("--no-suite", action="store_true",
                    help="headline workload only (by default the rmat20 line also carries the other "
                         "configurations as sub-records)")
    ap.add_argument("--requests", type=int, default=10000, help="serve: requests in the stream")
    ap.add_argument("--pool", type=int, default=24, help="serve: distinct graphs drawn from")
    ap.add_argument("--rate", type=float, default=0.0,
                    help="serve: arrivals per second (0: 0.7 x measured capacity; < 0: the sequential capacity)")
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
