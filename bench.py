"""Benchmark: shattered betweenness centrality on one GB300 (or N replicas).

One step = one bcs_bc_shattered call (validate, connected components,
degree-1 removal, biconnected split, identical-vertex merging, Bc-Reach over
all pieces, map-back) on one workload, seeded:

* twins (default, the headline): the identical-vertex heavy social-like graph
  (Chung-Lu core of 500,000 vertices, gamma 2.1, mean degree 12; twin groups
  of 2-8 covering 150,000 vertices; 350,000 pendants; n = 970,060,
  m = 5,024,502), the configuration with the most edges, FP32 dependencies
  as its statement asks;
* articulation: 5,000 Erdos-Renyi blocks (sizes log-uniform 4-512, mean
  degree 6) glued at cut vertices plus 20% dangling chains, FP64;
* road: 1500 x 1500 grid minus 25% of its edges, largest component, trees on
  10% of the perimeter (n = 2,258,525), FP32 dependencies.

metric: effective GTEPS = n * m / T with n, m of the input graph (sources x
undirected edges per second, the work plain Brandes would do) and T the
device time of one step; e2e: the same through host buffers (pinned), with
the host<->device copies inside the timed region.

--impl reference times the CPU oracle (plain Brandes, FP64) on the host
cores over a bounded sample of sources of the same graph.

Multi-GPU: the path needs one GPU; with --gpus N each rank runs its own
replica of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BC GTEPS (sources·m/s), shattered vs plain Brandes on GB300, rel err ≤1e-5"
L2_BYTES = 129 * 1024 * 1024

# workload -> (config id, FP32 dependencies, description)
WORKLOADS = {
    "twins": (3, True, "identical-vertex heavy social-like: Chung-Lu core 500k (gamma 2.1, mean deg 12) + twin "
                       "groups of 2-8 on 15% of vertices + 350k pendants"),
    "articulation": (2, False, "articulation-heavy: 5000 ER blocks (log-uniform 4-512, mean deg 6) + 20% chains"),
    "road": (4, True, "road-like: 1500x1500 grid minus 25% of edges, largest component, trees on 10% of the "
                      "perimeter"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=100, help="workload size in percent (100 = full)")
    ap.add_argument("--plain-sources", type=int, default=4096)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="twins",
                    choices=list(WORKLOADS) + ["batch", "side", "unequal", "twins-batch"],
                    help="twins (the headline), articulation, road; batch: many independent graphs in one call; "
                         "side: the articulation workload with added side vertices, shattered with and without "
                         "the side-vertex step; unequal: a twin-heavy graph whose twins carry pendants, with and "
                         "without merging twins of unequal reach; twins-batch: one 64-source batch of the "
                         "twin workload's largest piece through the whole-GPU kernel, run twice (for profilers)")
    ap.add_argument("--batch-count", type=int, default=20000)
    ap.add_argument("--batch-nmax", type=int, default=4096)
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup(n_gpus: int):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n_gpus > 1 else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name: str, scale: int):
    import graphgen as gg
    cfg_id, fp32, desc = WORKLOADS[name]
    g = gg.config(cfg_id, scale_pct=scale)
    return g, {"workload": desc if scale == 100 else f"{desc}, at {scale}% of its size", "n": g.n, "m": g.m,
               "seed": g.meta["seed"], "delta": "fp32" if fp32 else "fp64"}, fp32


# ncu summaries of the dominant kernels, each keyed by the SHA-1 of the
# sources the kernel compiles from; a figure is used only while they match
PROFILES = {
    "small": ("bcreach_small_articulation.json", ("bcreach.cu", "bc_math.cuh")),
    "wide": ("bcreach_wide_twins.json", ("wide.cu", "bc_math.cuh", "coop.cuh")),
}


def kernel_source_sha1(files) -> str:
    import hashlib
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1209_6007_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(kind: str):
    """The committed ncu summary's record for the kernel, if it was taken on
    the current kernel sources (else None)."""
    fname, files = PROFILES[kind]
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", fname)))
        if rec.get("source_sha1") == kernel_source_sha1(files):
            return rec
    except (OSError, ValueError, KeyError):
        pass
    return None


def cpu_baseline(g, seconds: float) -> dict:
    """The oracle (plain Brandes, FP64) on a bounded sample of sources."""
    import oracle
    cores = oracle.default_threads()
    rng = np.random.default_rng(12345)
    k = max(cores, 64)
    t0 = time.perf_counter()
    oracle.bc_sources(g, rng.choice(g.n, size=k, replace=False), threads=cores)
    dt = time.perf_counter() - t0
    k2 = int(max(k, min(g.n, k * seconds / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.bc_sources(g, rng.choice(g.n, size=k2, replace=False), threads=cores)
    dt = time.perf_counter() - t0
    return {"value": k2 * g.m / dt / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"{k2} seeded sources of the full graph (plain Brandes partial sums), "
                      f"{dt:.1f} s; GTEPS = sources*m/s"}


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return
    name = args.workload if args.workload in WORKLOADS else "twins"
    g, cfg, _ = workload(name, args.scale)
    import oracle
    cores = oracle.default_threads()
    rng = np.random.default_rng(777)
    # size one step to about cpu_seconds / (steps + warmup) of CPU time
    probe = max(cores, 32)
    t0 = time.perf_counter()
    oracle.bc_sources(g, rng.choice(g.n, size=probe, replace=False), threads=cores)
    per_src = (time.perf_counter() - t0) / probe
    budget = max(2.0, min(60.0, 120.0 / max(1, args.steps + args.warmup)))
    k = int(max(cores, min(g.n, budget / max(per_src, 1e-6))))
    for _ in range(args.warmup):
        oracle.bc_sources(g, rng.choice(g.n, size=k, replace=False), threads=cores)
    times = []
    for _ in range(args.steps):
        src = rng.choice(g.n, size=k, replace=False)
        t0 = time.perf_counter()
        oracle.bc_sources(g, src, threads=cores)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = k * g.m * args.steps / T / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {**cfg, "delta": "fp64", "sample": f"{k} sources per step"},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": cores, "kind": "oracle",
                             "sample": f"{k} seeded sources per step of the full graph"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def roofline(st: dict, clk: dict, peaks: dict, n_sm: int) -> dict:
    """Roofline of the call's dominant Bc-Reach kernel.

    Large pieces (the whole-GPU kernel): HBM.  Algorithmic bytes per
    (source, CSR entry) of a piece, with S sources sharing one adjacency
    read: 8/S (the row) + 2/8 (level bits) + f_DAG * 28 (path count written
    and read, coefficient, weights, per shortest-path DAG edge) + (n / 2m) *
    32 (per-vertex state written and read once); f_DAG is the DAG edges the
    call counted over its (source, entry) pairs.  Per launch: the sum over
    processed sources of these bytes, over the kernel's CUDA-event time.

    Shared-memory pieces only: the issue rate, the kernel's warp
    instructions per launch (ncu, committed summary of the same command)
    over its CUDA-event time against 152 SMs x 4 schedulers x 1 warp
    instruction per clock at the sampled clock, with the lanes active per
    instruction beside it; the FP64 figure (2 FLOP per DAG edge plus 9 per
    (source, vertex) against 4 FP64 FLOP/clk per SM) is reported too."""
    dag = float(st["dag_edges"])
    wse, wsv = float(st["work_sources_entries"]), float(st["work_sources_vertices"])
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    if st["ms_bcreach_large"] > st["ms_bcreach_small"]:
        # sources sharing one batch of the whole-GPU kernel (32 or 64)
        S = 64 if st["n_wide_batches"] and st["n_large_sources"] > 32 * st["n_wide_batches"] else 32
        f_dag = dag / wse if wse else 0.0
        by = wse * (8.0 / S + 2.0 / 8.0 + f_dag * 28.0) + wsv * 32.0
        ms = st["ms_bcreach_large"]
        peak = float(peaks.get("hbm_gbs", 6800.0))
        achieved = by / (ms / 1e3) / 1e9
        rec = measured_traffic("wide")
        traffic = rec["dram_bytes_per_batch"] * st["n_wide_batches"] if rec and st["n_wide_batches"] else None
        return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"k_bcreach_wide (whole GPU on one {S}-source batch)",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
                "work": {"bytes": by, "f_dag": f_dag, "sources_x_entries": wse, "sources_x_vertices": wsv,
                         "batches": int(st["n_wide_batches"]), "ms": ms,
                         "traffic_scaled_from": "ncu DRAM bytes of a full launch per batch (profiles/bcreach_wide_twins.json) "
                                                "x this call's batches" if traffic else None}}
    flop = 2.0 * dag + 9.0 * wsv
    ms = st["ms_bcreach_small"]
    fp64_peak = n_sm * 4.0 * sm_mhz * 1e6 / 1e12
    fp64 = flop / (ms / 1e3) / 1e12 if ms > 0 else None
    rec = measured_traffic("small")
    fp64_rec = {"achieved": fp64, "peak": fp64_peak, "unit": "TFLOP/s", "frac": (fp64 / fp64_peak) if fp64 else None,
                "peak_source": f"derived: {n_sm} SMs x 4 FP64 FLOP/clk x {sm_mhz:.0f} MHz (sampled)"}
    work = {"dag_edges": dag, "source_vertices": wsv, "flop": flop, "ms": ms}
    if rec and rec.get("warp_inst_per_launch") and ms > 0:
        inst = float(rec["warp_inst_per_launch"])
        peak = n_sm * 4.0 * sm_mhz * 1e6 / 1e9
        achieved = inst / (ms / 1e3) / 1e9
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp instructions/s",
                "frac": achieved / peak, "traffic": rec["dram_bytes_per_launch"],
                "kernel": "k_bcreach_small (issue rate)",
                "peak_source": f"derived: {n_sm} SMs x 4 schedulers x 1 warp instruction/clk x {sm_mhz:.0f} MHz "
                               "(sampled); instructions per launch from ncu",
                "lane_efficiency": float(rec["thread_inst_per_launch"]) / (32.0 * inst),
                "fp64": fp64_rec, "work": {**work, "warp_instructions": inst}}
    return {"bound": "alu", "achieved": fp64, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": fp64_rec["frac"], "traffic": rec["dram_bytes_per_launch"] if rec else None,
            "kernel": "k_bcreach_small (FP64 dependencies)", "peak_source": fp64_rec["peak_source"], "work": work}


def run_ours(args):
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import paper_1209_6007_gb300 as bcs
    bcs.load()
    g, cfg, fp32 = workload(args.workload, args.scale)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):  # the first call also runs the autotuner
        bcs.bc_shattered(rp, col, delta_fp32=fp32, autotune=True)
    torch.cuda.synchronize()
    stage_sum = {}
    launches = 0
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    dev_ms = 0.0
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the events)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        bc = bcs.bc_shattered(rp, col, delta_fp32=fp32, autotune=True)
        ev1.record(stream)
        ev1.synchronize()
        dev_ms += ev0.elapsed_time(ev1)
        st = bcs.last_stats()
        launches += int(st["kernel_launches"])
        for k, v in st.items():
            if k.startswith("ms_"):
                stage_sum[k] = stage_sum.get(k, 0.0) + v
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    barrier(world)
    clk = clocks.stop()
    T = max_over_ranks(dev_ms / 1e3, world)
    nm = float(g.n) * float(g.m)
    value = world * nm * args.steps / T / 1e9
    stages = {k: v / args.steps for k, v in stage_sum.items()}
    st = bcs.last_stats()

    # end to end through host buffers in pinned memory
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(g.row_ptr).pin_memory().numpy()
        col_h = torch.from_numpy(g.col).pin_memory().numpy()
        ke = max(1, min(args.steps, 3))
        bcs.bc_shattered(rp_h, col_h, delta_fp32=fp32, autotune=True)
        te = 0.0
        for _ in range(ke):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bcs.bc_shattered(rp_h, col_h, delta_fp32=fp32, autotune=True)
            te += time.perf_counter() - t0
        te = max_over_ranks(te, world)
        e2e = {"value": world * nm * ke / te / 1e9, "unit": "GTEPS", "steps": ke,
               "h2d_bytes_per_step": int(g.row_ptr.nbytes + g.col.nbytes), "d2h_bytes_per_step": int(g.n * 8)}

    # the other dependency precision on the same step, and its difference
    # (shared-memory workloads: one untimed call first, which runs that
    # precision's autotuner; a large piece's call is too long to repeat)
    if float(st["ms_bcreach_large"]) < 1000.0:
        bcs.bc_shattered(rp, col, delta_fp32=not fp32, autotune=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    b_other = bcs.bc_shattered(rp, col, delta_fp32=not fp32, autotune=True)
    ev1.record(stream)
    ev1.synchronize()
    t_other = ev0.elapsed_time(ev1) / 1e3
    b32, b64 = (bc, b_other) if fp32 else (b_other, bc)
    err32 = float((b32 - b64).abs().max() / max(1.0, float(b64.abs().max())))
    other = {"delta": "fp64" if fp32 else "fp32", "gteps": nm / t_other / 1e9, "ms": 1e3 * t_other,
             "rel_err_fp32_vs_fp64": err32}

    # plain Brandes on a sample of sources (the same graph, nothing shattered)
    plain = None
    if args.plain_sources > 0:
        rng = np.random.default_rng(99)
        src = rng.choice(g.n, size=min(args.plain_sources, g.n), replace=False)
        bcs.bc_sources(rp, col, src[:64])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        bcs.bc_sources(rp, col, src)
        ev1.record(stream)
        ev1.synchronize()
        tp = ev0.elapsed_time(ev1) / 1e3
        plain = {"gteps": len(src) * g.m / tp / 1e9, "sources": int(len(src)), "seconds": tp, "delta": "fp64"}

    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    roof = roofline(st, clk, peaks, n_sm)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "data": "synthetic",
                "config": {**cfg, "precision": ("dependencies FP32; path counts int64, else FP64; bc FP64"
                                                if fp32 else "dependencies and bc FP64; path counts int64, else FP64"),
                           "l2": "flushed between timed steps (256 MB write)", "parallelism": f"{world} replica(s)"},
                "e2e": e2e, "gpu_launches": launches, "clocks": clk, "roofline": roof,
                "stages_ms": stages, "pieces": int(st["n_pieces"]), "merged_vertices": int(st["n_merged"]),
                "large_sources": int(st["n_large_sources"]), "wide_batches": int(st["n_wide_batches"]),
                "bfs_levels": int(st["bfs_levels"]), "work_nm_pieces": float(st["work_nm"]),
                "raw_gteps": float(st["work_nm"]) * args.steps / (dev_ms / 1e3) / 1e9,
                "other_delta": other, "plain": plain,
                "speedup_vs_plain": (value / plain["gteps"]) if plain else None, "wall_s": wall}
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(g, args.cpu_seconds)
        print(json.dumps(line))


def run_batch(args):
    """Uneven batch (workload 5's generator): `--batch-count` independent
    Chung-Lu graphs (gamma 2.3, mean degree 8) of log-uniform sizes
    16..`--batch-nmax`, packed in one CSR, all shattered and solved by one
    bcs_bc_shattered_batch call per step with FP32 dependencies (the timed
    value); once with FP64 dependencies (its time and the FP32 error, over
    the whole batch and per graph); and the baseline, plain FP64 Brandes
    launched graph by graph (bcs_bc_plain on each graph's own CSR, on the
    device) over a seeded stratified 1% of the graphs (one per stratum of the
    graphs ordered by size), extrapolated to the whole batch stratum by
    stratum.  Work = sum over the graphs of n_i * m_i (every vertex a source
    in its own graph)."""
    import torch
    import graphgen as gg
    import paper_1209_6007_gb300 as bcs
    torch.cuda.set_device(0)
    bcs.load()
    t0 = time.perf_counter()
    g, off = gg.batch(args.batch_count, n_min=16, n_max=args.batch_nmax)
    gen_s = time.perf_counter() - t0
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    n_i = np.diff(off).astype(np.float64)
    m_i = (g.row_ptr[off[1:]] - g.row_ptr[off[:-1]]).astype(np.float64) / 2
    work = float((n_i * m_i).sum())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fp32):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        out = bcs.bc_shattered_batch(off, rp, col, delta_fp32=fp32, autotune=True)
        ev1.record(stream)
        ev1.synchronize()
        return out, ev0.elapsed_time(ev1)

    for _ in range(args.warmup):  # the first call also runs the autotuner
        bcs.bc_shattered_batch(off, rp, col, delta_fp32=True, autotune=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    dev_ms, launches, b32 = 0.0, 0, None
    for _ in range(args.steps):
        b32, ms = timed(True)
        dev_ms += ms
        launches += int(bcs.last_stats()["kernel_launches"])
    clk = clocks.stop()
    st = bcs.last_stats()
    b64, ms64 = timed(False)  # its small-path split is tuned on this first FP64 call
    b32, b64 = b32.cpu().numpy(), b64.cpu().numpy()
    diff = np.abs(b32 - b64)
    err_all = float(diff.max() / max(1.0, float(np.abs(b64).max())))
    err_graph = float(max(diff[off[i]:off[i + 1]].max() / max(1.0, float(np.abs(b64[off[i]:off[i + 1]]).max()))
                          for i in range(len(off) - 1) if off[i + 1] > off[i]))
    # plain FP64 Brandes per graph on a stratified 1% of the graphs
    order = np.argsort(n_i, kind="stable")
    k = max(1, (len(off) - 1) // 100)
    rng = np.random.default_rng(2026)
    strata = np.array_split(order, k)
    est_ms, sampled_ms, sampled = 0.0, 0.0, 0
    for stratum in strata:
        gi = int(rng.choice(stratum))
        a, b = int(off[gi]), int(off[gi + 1])
        rpg = torch.from_numpy((g.row_ptr[a:b + 1] - g.row_ptr[a]).astype(np.int64)).cuda()
        colg = torch.from_numpy((g.col[g.row_ptr[a]:g.row_ptr[b]] - a).astype(np.int32)).cuda()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        bcs.bc_plain(rpg, colg)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        sampled_ms += ms
        sampled += 1
        est_ms += ms * len(stratum)
    T = dev_ms / 1e3
    line = {"metric": "BC GTEPS (sum over the batch's graphs of sources*m / s)", "value": work * args.steps / T / 1e9,
            "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dev_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: {args.batch_count} Chung-Lu graphs (gamma 2.3, mean degree 8), "
                                   f"n log-uniform 16..{args.batch_nmax}", "n": int(g.n), "m": int(g.m),
                       "sum_n_m": work, "delta": "fp32", "l2": "flushed between timed steps (256 MB write)",
                       "generation_s": gen_s},
            "gpu_launches": launches, "clocks": clk,
            "stages_ms": {k2: v for k2, v in st.items() if k2.startswith("ms_")},
            "pieces": st["n_pieces"], "large_sources": st["n_large_sources"], "tuned": st["tuned"],
            "small_limit": st["small_limit"],
            "fp64": {"gteps": work / (ms64 / 1e3) / 1e9, "ms": ms64, "note": "one call, small-path split tuned in it"},
            "rel_err_fp32_vs_fp64": {"batch": err_all, "worst_graph": err_graph},
            "per_graph_fp64_baseline": {"graphs_sampled": sampled, "strata": k, "ms_sampled": sampled_ms,
                                        "ms_extrapolated": est_ms,
                                        "speedup_batched_fp32": est_ms / (dev_ms / args.steps),
                                        "method": "bcs_bc_plain per graph on the device, seeded stratified sample "
                                                  "(one graph per stratum of the graphs ordered by size), each "
                                                  "stratum's time = its sample's time x its graphs"},
            "note": "secondary measurement; the headline line is --workload twins"}
    print(json.dumps(line))


def run_side(args):
    """Side vertices (Section 3.3.2): the articulation workload plus 150,000
    vertices each joined to both ends of a uniform edge and 50,000 more each
    joined to an earlier one and its neighbours (every added vertex has a
    clique for a neighbourhood), shattered with and without the side-vertex
    step.  Work = n * m of the input; value = with the step."""
    import torch
    import graphgen as gg
    import paper_1209_6007_gb300 as bcs
    torch.cuda.set_device(0)
    bcs.load()
    g = gg.with_side_vertices(gg.config(2, scale_pct=args.scale), 0xB0C00006, 150000 * args.scale // 100,
                              50000 * args.scale // 100)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res = {}
    for side in (False, True):
        for _ in range(args.warmup):
            bcs.bc_shattered(rp, col, side=side, autotune=True)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        dev_ms, launches, stages = 0.0, 0, {}
        for _ in range(args.steps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            bcs.bc_shattered(rp, col, side=side, autotune=True)
            ev1.record(stream)
            ev1.synchronize()
            dev_ms += ev0.elapsed_time(ev1)
            st = bcs.last_stats()
            launches += int(st["kernel_launches"])
            for k, v in st.items():
                if k.startswith("ms_"):
                    stages[k] = stages.get(k, 0.0) + v / args.steps
        res[side] = {"ms": dev_ms / args.steps, "launches": launches, "clocks": clocks.stop(), "stages_ms": stages,
                     "n_side": int(st["n_side"]), "pieces": int(st["n_pieces"]), "n_merged": int(st["n_merged"])}
    work = float(g.n) * float(g.m)
    on, off = res[True], res[False]
    line = {"metric": "BC GTEPS (sources*m / s, n and m of the input graph)",
            "value": work / (on["ms"] / 1e3) / 1e9, "unit": "GTEPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": on["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "articulation-heavy + side vertices: 5000 ER blocks + 20% chains, then 150,000 "
                                   "triangle vertices on uniform edges and 50,000 clique-extending vertices",
                       "n": int(g.n), "m": int(g.m), "l2": "flushed between timed steps (256 MB write)"},
            "gpu_launches": on["launches"], "clocks": on["clocks"], "side_step": on,
            "without_side_step": {**off, "gteps": work / (off["ms"] / 1e3) / 1e9},
            "speedup_of_side_step": off["ms"] / on["ms"],
            "note": "secondary measurement; the headline line is --workload twins"}
    print(json.dumps(line))


def run_unequal(args):
    """Identical vertices of unequal reach: a Chung-Lu core (25,000 vertices,
    gamma 2.1, mean degree 12; the twin workload's core at 5 %) plus 7,500
    open twins (copies of a uniform core vertex's neighbour set) and 17,500
    pendants on uniform vertices, twins included, so that twins differ in
    reach.  Shattered with equal-reach classes and with classes of any reach;
    work = n * m of the input; value = with unequal-reach classes."""
    import torch
    import graphgen as gg
    import paper_1209_6007_gb300 as bcs
    torch.cuda.set_device(0)
    bcs.load()
    g = gg.with_twins_and_pendants(gg.chung_lu(25000, 2.1, 12, 0xB0C00007), 0xB0C00007, 7500, 17500)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    res, out = {}, {}
    for unequal in (False, True):
        for _ in range(args.warmup):
            bcs.bc_shattered(rp, col, unequal=unequal, autotune=True)
        torch.cuda.synchronize()
        clocks = ClockSampler(0)
        clocks.start()
        dev_ms, launches, stages = 0.0, 0, {}
        for _ in range(args.steps):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            bc = bcs.bc_shattered(rp, col, unequal=unequal, autotune=True)
            ev1.record(stream)
            ev1.synchronize()
            dev_ms += ev0.elapsed_time(ev1)
            st = bcs.last_stats()
            launches += int(st["kernel_launches"])
            for k, v in st.items():
                if k.startswith("ms_"):
                    stages[k] = stages.get(k, 0.0) + v / args.steps
        out[unequal] = bc
        res[unequal] = {"ms": dev_ms / args.steps, "launches": launches, "clocks": clocks.stop(), "stages_ms": stages,
                        "n_merged": int(st["n_merged"]), "pieces": int(st["n_pieces"]),
                        "large_sources": int(st["n_large_sources"])}
    work = float(g.n) * float(g.m)
    on, off = res[True], res[False]
    diff = float((out[True] - out[False]).abs().max() / out[False].abs().max().clamp(min=1.0))
    line = {"metric": "BC GTEPS (sources*m / s, n and m of the input graph)",
            "value": work / (on["ms"] / 1e3) / 1e9, "unit": "GTEPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": on["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "twins of unequal reach: Chung-Lu core 25,000 (gamma 2.1, mean degree 12) + 7,500 "
                                   "open twins + 17,500 pendants on uniform vertices", "n": int(g.n), "m": int(g.m),
                       "l2": "flushed between timed steps (256 MB write)"},
            "gpu_launches": on["launches"], "clocks": on["clocks"], "unequal_reach_classes": on,
            "equal_reach_classes": {**off, "gteps": work / (off["ms"] / 1e3) / 1e9},
            "speedup_of_unequal_classes": off["ms"] / on["ms"], "max_rel_diff_between_the_two": diff,
            "note": "secondary measurement; the headline line is --workload twins"}
    print(json.dumps(line))


def run_twins_batch(args):
    """One 64-source batch of the twin workload's largest piece (after
    shattering: 423,691 vertices, 5,781,604 entries) through the whole-GPU
    Bc-Reach kernel, FP32 dependencies, run twice; the sources are spread
    over the piece (ids i * 7919 mod n).  A small, fixed launch for ncu."""
    import torch
    import graphgen as gg
    import paper_1209_6007_gb300 as bcs
    torch.cuda.set_device(0)
    bcs.load()
    g = gg.config(3, scale_pct=args.scale)
    c = bcs.shatter(g.row_ptr, g.col)
    sizes = np.diff(c.piece_vtx_off)
    p = int(np.argmax(sizes))
    a, b = int(c.piece_vtx_off[p]), int(c.piece_vtx_off[p + 1])
    rp = (c.row_ptr[a:b + 1] - c.row_ptr[a]).astype(np.int64)
    col = c.col[c.row_ptr[a]:c.row_ptr[b]].astype(np.int32)
    rows = np.repeat(np.arange(b - a), np.diff(rp))
    col = col[np.lexsort((col, rows))]  # the piece's rows in ascending order, as the ABI takes them
    src = (np.arange(64, dtype=np.int64) * 7919) % (b - a)
    rpd, cold = torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()
    ms = []
    for _ in range(2):
        bcs.bc_sources(rpd, cold, src, delta_fp32=True)
        st = bcs.last_stats()
        ms.append(st["ms_bcreach_large"])
    print(json.dumps({"workload": "one 64-source batch of the twin workload's largest piece", "n": int(b - a),
                      "nnz": int(col.size), "wide_batches": int(st["n_wide_batches"]), "ms_bcreach_large": ms}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "side":
        run_side(args)
    elif args.workload == "unequal":
        run_unequal(args)
    elif args.workload == "twins-batch":
        run_twins_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
