"""Benchmark of the pair-distance histogram on GB300.

One step = the three headline frames (N = 1,000,000 particles, 1 species,
uniform at density 0.1, 10,000 bins; no box, orthorhombic and triclinic cell)
through one dh_histogram_batch call (one persistent pair-kernel launch per
minimum-image variant, replayed as a CUDA graph), inputs resident in HBM.  Printed on one JSON line:

  value          Gpairs/s of the batched step (device time, CUDA events)
  pairs_per_step the pairs of one step (every unique pair of the three frames)
  e2e            the same metric through the C ABI with pinned HOST buffers:
                 host->device copy of the coordinates and device->host copy of
                 the histograms inside the timed region
  plain          per-frame dh_histogram Gpairs/s for each box type
  configs        the plain path on C1 (no box, N = 2,000), C2 (orthorhombic, N =
                 100,000) and C3 (clustered triclinic, N = 500,000)
  pipes          measured per-SM throughput of the pipes the pair kernel uses
  roofline       the pair kernel's pairs per second against the minimum over
                 those pipes of measured rate / operations per pair
  batched        the batched step's launch shape, and C4 (256 frames of uneven
                 N in one batched call against one plain call per frame)
  served         C5: p50/p99 latency at offered loads 0.5/0.8/0.95 and the
                 saturated throughput of dh_submit/dh_poll, against the plain path
  cpu_baseline   the FP64 oracle on the host cores, on a bounded sample
  clocks         nvidia-smi SM clocks and throttle reasons during the timed region

``--impl reference`` times the FP64 oracle (the reference arm) on bounded
samples of the same workload instead.  Under torchrun each rank runs its
own replica (frames are independent; no data-path collective) and rank 0
reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402

METRIC = "Gpairs/s binned at N=1M (plain vs batched/served) + p50/p99 frame latency, 1 GB300"
UNIT = "Gpairs/s"
BOXES = (w.BOX_NONE, w.BOX_ORTHO, w.BOX_TRICLINIC)

# Per-pair arithmetic of the pair kernel on the float32 (FMA) pipe, by tile mode,
# as lane operations of each packed kind (FADD2, FMUL2, FFMA2 count two lanes).
# Every mode: d = xj - xi (3 add), r^2 (1 mul, 2 fma), q = S^2 r^2 (1 mul), the
# nearest integer of the root and its residual (2 add, 1 fma), the near-edge
# bound (1 fma).  Orthorhombic tiles with a uniform image shift the j's by the
# image (3 packed adds per 2 j x 4 i: 0.75 lanes per pair; 0.5 with one axis
# wrapped per pair).  A wrapped axis adds a nearest integer and an fma (1 add,
# 2 fma); the per-pair triclinic wrap rounds along c, b, a (3 add, 9 fma).  The
# square root is one MUFU operation per pair and the histogram update one
# shared-memory atomic per pair (the clamp of out-of-range roots runs on the
# integer ALU).
BASE_OPS = {"fadd": 5.0, "fmul": 2.0, "ffma": 4.0}
MODE_OPS = {
    (w.BOX_NONE, "uni"): {}, (w.BOX_NONE, "pair"): {},
    (w.BOX_ORTHO, "uni"): {"fadd": 0.75}, (w.BOX_ORTHO, "axis"): {"fadd": 1.5, "ffma": 2.0},
    (w.BOX_ORTHO, "pair"): {"fadd": 3.0, "ffma": 6.0},
    (w.BOX_TRICLINIC, "uni"): {}, (w.BOX_TRICLINIC, "axis"): {"fadd": 1.0, "ffma": 2.0},
    (w.BOX_TRICLINIC, "pair"): {"fadd": 3.0, "ffma": 9.0},
}
SM_COUNT = 152
PIPE_SET = ("ffma2", "fadd2", "fmul2", "ffma", "sqrt", "frnd", "f2i", "lop3", "iadd", "imad", "dfma", "match",
            "smem_atomic_clustered", "smem_atomic_same", "smem_atomic_sequential")


def measure_pipes(device: int, widths) -> dict:
    """Measured per-SM throughput (operations per clock per SM) of the pipes the
    pair kernel runs on (dh_pipe_rate), with the shared-memory atomic rate on
    uniform random bins for every histogram width in `widths`."""
    import paper_1808_01478_gb300 as dh

    out = {}
    for name in PIPE_SET:
        width = 10000 if name.startswith("smem") else 0
        r = dh.dh_pipe_rate(device, name, width)
        out[name] = {"per_clk_sm": round(r["per_clk_sm"], 3), "mhz": round(r["sm_mhz"], 1)}
    for wd in sorted(set(int(x) for x in widths)):
        r = dh.dh_pipe_rate(device, "smem_atomic_random", min(wd, 57344))
        out[f"smem_atomic_random@{wd}"] = {"per_clk_sm": round(r["per_clk_sm"], 3), "mhz": round(r["sm_mhz"], 1)}
    r = dh.dh_pipe_rate(device, "global_atomic64", 10000)
    out["global_atomic64@10000"] = {"per_clk_sm": round(r["per_clk_sm"], 4), "mhz": round(r["sm_mhz"], 1)}
    return out


def fp32_lane_ops(box_type: int, f_uni: float, f_axis: float) -> dict:
    """Float32 lane operations per pair of each kind, averaged over the tile modes
    with the fractions of pairs the kernel evaluated in each."""
    f_pair = max(0.0, 1.0 - f_uni - f_axis)
    ops = dict(BASE_OPS)
    for mode, frac in (("uni", f_uni), ("axis", f_axis), ("pair", f_pair)):
        for k, v in MODE_OPS.get((box_type, mode), {}).items():
            ops[k] += frac * v
    return ops


def bank_load(f_in: float, trials: int = 4000) -> float:
    """Expected largest number of distinct words one bank receives in a warp's
    shared-memory increment when a fraction f_in of its 32 lanes hits uniform
    random bins and the others their own guard words (one bank each: the
    clamp sends lane l's out-of-range pairs to the word hi + 1 + l)."""
    rng = np.random.default_rng(12345)
    inr = rng.random((trials, 32)) < f_in
    banks = np.where(inr, rng.integers(0, 32, (trials, 32)), np.arange(32)[None, :])
    loads = np.zeros((trials, 32))
    np.add.at(loads, (np.repeat(np.arange(trials), 32), banks.ravel()), 1.0)
    return float(loads.max(axis=1).mean())


def atomic_rate(width: int, f_in: float, pipes: dict) -> float:
    """Shared-memory increments per clock per SM for a histogram of `width`
    bins when a fraction f_in of the pairs is inside r_max: the measured rate
    on uniform random bins (every lane in range), scaled by the expected bank
    load relative to that case, but never above the conflict-free rate."""
    key = f"smem_atomic_random@{width}"
    if key not in pipes:
        return float("nan")
    r_rand, r_free = pipes[key]["per_clk_sm"], pipes["smem_atomic_sequential"]["per_clk_sm"]
    return min(r_free, r_rand * bank_load(1.0) / bank_load(min(1.0, max(0.0, f_in))))


def pair_bound(box_type: int, width: int, f_uni: float, f_axis: float, pipes: dict, f_in: float = 1.0) -> dict:
    """Roofline of the pair kernel for one frame in pairs per clock per SM: the
    minimum over pipes of measured rate / operations per pair (float32 FMA
    pipe, MUFU square root, shared-memory atomic at the frame's width and
    fraction f_in of pairs inside r_max)."""
    ops = fp32_lane_ops(box_type, f_uni, f_axis)
    fp32_clk = (ops["fadd"] / pipes["fadd2"]["per_clk_sm"] + ops["fmul"] / pipes["fmul2"]["per_clk_sm"]
                + ops["ffma"] / pipes["ffma2"]["per_clk_sm"])
    bounds = {"fp32": 1.0 / fp32_clk, "mufu": pipes["sqrt"]["per_clk_sm"],
              "smem_atomic": atomic_rate(width, f_in, pipes)}
    binding = min((v, k) for k, v in bounds.items() if v == v)[1]
    return {"pairs_per_clk_sm": bounds[binding], "binding": binding,
            "fp32_lane_ops_per_pair": round(sum(ops.values()), 3),
            "bounds_pairs_per_clk_sm": {k: round(v, 3) for k, v in bounds.items()}}


def roofline_entry(pairs: float, seconds: float, mhz: float, bound: dict) -> dict:
    """Achieved pairs per clock per SM (at the SM clock sampled under load)
    against the frame's bound; `pairs` are the pairs the kernel evaluated (its
    tiles skipped as out of range or out of the sweep are not counted)."""
    achieved = pairs / seconds / (SM_COUNT * mhz * 1e6)
    return {"achieved_pairs_per_clk_sm": round(achieved, 3), "bound_pairs_per_clk_sm": round(bound["pairs_per_clk_sm"], 3),
            "frac": round(achieved / bound["pairs_per_clk_sm"], 4), "binding": bound["binding"],
            "fp32_lane_ops_per_pair": bound["fp32_lane_ops_per_pair"],
            "bounds_pairs_per_clk_sm": bound["bounds_pairs_per_clk_sm"]}


def load_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


TRAFFIC_FILE = os.path.join("profiles", "pair_kernel_dram_n1m_batch.txt")


def committed_traffic() -> int | None:
    """DRAM bytes of the pair-kernel launches of one headline step, from the
    committed ncu capture, or None once the kernel sources differ from the ones
    the capture was taken with."""
    import hashlib

    try:
        lines = open(os.path.join(ROOT, TRAFFIC_FILE)).read().splitlines()
    except OSError:
        return None
    total = 0
    for line in lines:
        p = line.split()
        if not p or p[0].startswith("#"):
            continue
        if p[0] == "source_sha256":
            try:
                digest = hashlib.sha256(open(os.path.join(ROOT, p[1]), "rb").read()).hexdigest()
            except OSError:
                return None
            if digest != p[2]:
                return None
        elif p[0] == "launch":
            total += int(p[3]) + int(p[4])
    return total or None


# ---------------------------------------------------------------- clocks


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- distributed


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as td

    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    td.init_process_group(backend=backend)
    return td


def max_over_ranks(td, value: float, device=None) -> float:
    if td is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(td, value: float, device=None) -> float:
    if td is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.SUM)
    return float(t.item())


def aggregate_throughput(td, pairs_local: float, seconds_local: float, device=None):
    """Whole-job Gpairs/s: the pairs every rank evaluated over the slowest rank's time.

    Returns (gpairs_s, max_seconds).  Ranks are independent replicas, so the only
    exchange is this pair of reductions on the host-side numbers."""
    t_max = max_over_ranks(td, seconds_local, device)
    all_pairs = sum_over_ranks(td, float(pairs_local), device)
    return all_pairs / t_max / 1e9, t_max


# ---------------------------------------------------------------- oracle timing


def oracle_sample(frames: list, seconds: float, nthreads: int) -> dict:
    """Time the FP64 oracle on leading subsets of each frame (same box, r_max, nbins).

    The subset size is calibrated so the three frames together take about
    `seconds` of wall time on `nthreads` host threads.
    """
    import oracle

    rates = []
    for f in frames:
        n0 = 1500
        sub = w.frame_from(f.coords[:n0], [0, n0], f.box_type, f.box, f.r_max, f.nbins)
        t0 = time.perf_counter()
        oracle.histogram_frame(sub, nthreads=nthreads)
        dt = max(time.perf_counter() - t0, 1e-4)
        rates.append(sub.n_pairs() / dt)
    per = seconds / len(frames)
    total_pairs, total_t, sizes = 0, 0.0, []
    for f, rate in zip(frames, rates):
        n = int(min(f.n, max(2000, math.sqrt(2.0 * rate * per))))
        sub = w.frame_from(f.coords[:n], [0, n], f.box_type, f.box, f.r_max, f.nbins)
        t0 = time.perf_counter()
        oracle.histogram_frame(sub, nthreads=nthreads)
        total_t += time.perf_counter() - t0
        total_pairs += sub.n_pairs()
        sizes.append(n)
    return {"gpairs_s": total_pairs / total_t / 1e9, "seconds": total_t, "pairs": total_pairs,
            "sizes": sizes}


def workload_config(args, world: int) -> dict:
    return {"workload": f"N={args.n} uniform density 0.1, 1 species, {args.nbins} bins; "
                        "one none + one ortho + one triclinic frame per step (dh_histogram_batch)",
            "n": args.n, "nbins": args.nbins, "frames_per_step": 3,
            "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"}


def headline_frames(n: int, nbins: int) -> list:
    return [w.headline_frame(b, seed=11 + b, n=n, nbins=nbins) for b in BOXES]


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    frames = headline_frames(args.n, args.nbins)
    nthreads = os.cpu_count() or 1
    per_step = args.ref_seconds
    # calibrate once, then each step evaluates the same bounded sample
    cal = oracle_sample(frames, per_step, nthreads)
    subs = [w.frame_from(f.coords[:n], [0, n], f.box_type, f.box, f.r_max, f.nbins)
            for f, n in zip(frames, cal["sizes"])]
    pairs_step = sum(s.n_pairs() for s in subs)
    for _ in range(args.warmup):
        for s in subs:
            oracle.histogram_frame(s, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in subs:
            oracle.histogram_frame(s, nthreads=nthreads)
    dt = time.perf_counter() - t0
    value = pairs_step * args.steps / dt / 1e9
    sample = (f"leading subsets N={cal['sizes']} of the three N={args.n} frames "
              f"(none/ortho/triclinic, same box, r_max, {args.nbins} bins)")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, world),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0



# ---------------------------------------------------------------- configurations C1-C3


def config_frames() -> dict:
    """C1: no box, N = 2,000 in a cube of side 10, r_max 17.33, 1,000 bins;
    C2: orthorhombic 60^3, N = 100,000, 2 species, r_max 30, 10,000 bins;
    C3: triclinic 80 A cell (70/80/100 deg), N = 500,000 as 200 Gaussian clusters
    (sigma 2) plus 20 % background, 3 species, r_max 35, 20,000 bins."""
    return {"c1": w.config_small_nobox(seed=1), "c2": w.config_ortho_two_species(seed=2),
            "c3": w.config_triclinic_clusters(seed=3)}


def run_configs(ctx, stream, dev, args, pipes, mhz, flush_l2):
    """The plain path on C1-C3 with device-resident inputs: Gpairs/s of the whole
    call (CUDA events), the pair kernel's share, deferrals and the roofline
    fraction of the pair kernel."""
    import torch

    out = {}
    for name, f in config_frames().items():
        x = torch.from_numpy(f.coords).to(dev)
        o = torch.zeros((f.n_hist, f.nbins), dtype=torch.int64, device=dev)
        ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, o)
        reps = max(3, args.plain_steps) if f.n_pairs() < 1e10 else max(1, args.plain_steps)
        ts, pk = [], []
        for _ in range(reps):
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, o)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            pk.append(ctx.stats()["pair_kernel_ms"])
        st = ctx.stats()
        pairs = f.n_pairs()
        f_cull = st["culled_pairs"] / max(1, st["pairs"] * st["sweeps"])
        ev = pairs * (1.0 - f_cull)
        fu = st["uniform_pairs"] / max(1.0, ev)
        fa_ = st["axis_pairs"] / max(1.0, ev)
        bound = pair_bound(f.box_type, f.nbins, fu, fa_, pipes, int(o.sum().item()) / max(1.0, ev))
        out[name] = {"workload": f.name, "pairs": pairs, "gpairs_s": round(pairs / (statistics.median(ts) / 1e3) / 1e9, 3),
                     "ms": round(statistics.median(ts), 4), "pair_kernel_ms": round(statistics.median(pk), 4),
                     "deferred_frac": round(st["deferred"] / max(1, st["pairs"]), 6),
                     "binary64_frac": round(st["exact_fallback"] / max(1, st["pairs"]), 8),
                     "tile_image_frac": round(fu, 4), "axis_image_frac": round(fa_, 4), "culled_frac": round(f_cull, 4),
                     "roofline": roofline_entry(ev, statistics.median(pk) / 1e3, mhz, bound)}
        del x, o
    return out


# ---------------------------------------------------------------- batched and served legs


def run_batched_c4(ctx, stream, dev, args):
    """C4: orthorhombic frames of uneven N in one dh_histogram_batch (CUDA graph)
    against the same frames through one dh_histogram call each."""
    import torch

    import paper_1808_01478_gb300 as dh

    frames = w.batch_frames(seed=7, n_frames=args.c4_frames)
    pairs = sum(f.n_pairs() for f in frames)
    X = [torch.from_numpy(f.coords).to(dev) for f in frames]
    fas = [dh.FrameArgs(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins) for k, f in enumerate(frames)]
    ctx.histogram_batch(fas)  # first call: measures the launch key's shapes (autotuner), untimed
    st0 = ctx.stats()
    graph = st0["graph_replays"]
    shape = {"tile_j": st0["tile_j"], "hist_depth": st0["hist_depth"], "blocks_per_sm": st0["blocks_per_sm"],
             "autotune_runs": st0["tune_runs"]}
    ts = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.histogram_batch(fas)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    batch_ms = min(ts)
    outs = [torch.zeros_like(fa.out) for fa in fas]
    for k, f in enumerate(frames):  # untimed pass: the per-frame launch keys get tuned here
        ctx.histogram(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins, outs[k])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k, f in enumerate(frames):
        ctx.histogram(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins, outs[k])
    e1.record(stream)
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    same = all(torch.equal(outs[k], fas[k].out) for k in range(len(frames)))
    return {"frames": len(frames), "pairs": pairs, "batch_gpairs_s": round(pairs / (batch_ms / 1e3) / 1e9, 3),
            "batch_ms": round(batch_ms, 3), "cuda_graph": bool(graph), "launch_shape": shape,
            "plain_loop_gpairs_s": round(pairs / (plain_ms / 1e3) / 1e9, 3), "plain_loop_ms": round(plain_ms, 3),
            "identical_to_plain": same}


def _serve(dev_index, fas, pairs, arrivals):
    """Submit request k at arrivals[k] seconds (one client thread) while a poller
    thread records completions; returns latencies (ms), status and the span."""
    import paper_1808_01478_gb300 as dh

    n = len(fas)
    done_t, sub_t, tickets, status = [None] * n, [None] * n, [None] * n, [None] * n
    with dh.Context(dev_index, pool_bytes=8 << 30, max_inflight=64) as sctx:
        f0 = fas[0]
        warm = dh.FrameArgs(f0.coords, f0.offsets, f0.frame.box_type, list(f0.frame.box), f0.frame.r_max,
                            f0.frame.nbins)
        sctx.wait(sctx.submit(warm))  # pool, lanes and kernels warm before the measurement
        stop = threading.Event()
        lock = threading.Lock()

        def poller():
            while not stop.is_set():
                with lock:
                    live = [k for k in range(n) if tickets[k] is not None and done_t[k] is None]
                for k in live:
                    st = sctx.poll(tickets[k])
                    if st != dh.DH_PENDING:
                        done_t[k] = time.perf_counter()
                        status[k] = st
                time.sleep(100e-6)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for k in range(n):
            target = t0 + arrivals[k]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                time.sleep(min(0.0005, target - now))
            sub_t[k] = time.perf_counter()
            t = sctx.submit(fas[k])
            with lock:
                tickets[k] = t
        deadline = time.perf_counter() + 900
        while any(d is None for d in done_t) and time.perf_counter() < deadline:
            time.sleep(0.001)
        stop.set()
        th.join()
    lat = np.array([(d - s_) * 1e3 for d, s_ in zip(done_t, sub_t)])
    return lat, status, max(done_t) - min(sub_t)


def run_served_c5(dev_index, dev, args):
    """C5: Poisson arrivals of frame requests (mixed boxes, 1-3 species, 2^10..2^14
    bins, N log-uniform in [10^3, 10^6]) at offered loads rho x the capacity of
    the plain per-frame path on the same requests, plus all requests at once
    (the server's saturated throughput); coordinates and histograms stay on the
    device."""
    import torch

    import paper_1808_01478_gb300 as dh

    rng = w.rng_for(2024)
    frames = [w.served_request(rng) for _ in range(args.served_requests)]
    pairs = np.array([f.n_pairs() for f in frames], dtype=np.float64)
    fas = [dh.FrameArgs(torch.from_numpy(f.coords).to(dev), f.offsets, f.box_type, f.box, f.r_max, f.nbins)
           for f in frames]
    torch.cuda.synchronize()
    # the plain per-frame path on the same requests, one at a time: capacity and
    # the latency of each request when it has the GPU to itself
    alone_ms = []
    ref = [torch.zeros_like(fa.out) for fa in fas]
    with dh.Context(dev_index) as pctx:
        pctx.histogram(fas[0].coords, frames[0].offsets, frames[0].box_type, frames[0].box, frames[0].r_max,
                       frames[0].nbins, ref[0])
        for k, f in enumerate(frames):
            t0 = time.perf_counter()
            pctx.histogram(fas[k].coords, f.offsets, f.box_type, f.box, f.r_max, f.nbins, ref[k])
            alone_ms.append((time.perf_counter() - t0) * 1e3)
    alone_ms = np.array(alone_ms)
    capacity = pairs.sum() / (alone_ms.sum() / 1e3)
    out = {"requests": len(frames), "pairs": float(pairs.sum()),
           "plain_capacity_gpairs_s": round(capacity / 1e9, 3),
           "plain_alone_p50_ms": round(float(np.percentile(alone_ms, 50)), 3),
           "plain_alone_p99_ms": round(float(np.percentile(alone_ms, 99)), 3), "loads": {}}
    arr_rng = w.rng_for(77)
    for load in args.served_loads:
        lam = load * capacity / pairs.mean()
        arrivals = np.cumsum(arr_rng.exponential(1.0 / lam, size=len(frames)))
        lat, status, span = _serve(dev_index, fas, pairs, arrivals)
        same = all(torch.equal(ref[k], fas[k].out) for k in range(len(frames)))
        out["loads"][str(load)] = {
            "arrival_rate_per_s": round(lam, 3), "p50_ms": round(float(np.percentile(lat, 50)), 3),
            "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
            "p99_slowdown": round(float(np.percentile(lat / alone_ms, 99)), 3),
            "gpairs_s": round(pairs.sum() / span / 1e9, 3),
            "all_ok": all(s_ == dh.DH_OK for s_ in status), "identical_to_plain": same}
    lat, status, span = _serve(dev_index, fas, pairs, np.zeros(len(frames)))
    out["saturated_gpairs_s"] = round(pairs.sum() / span / 1e9, 3)
    out["saturated_identical_to_plain"] = all(torch.equal(ref[k], fas[k].out) for k in range(len(frames)))
    return out

# ---------------------------------------------------------------- GPU arm


def scan_frame(box_name: str, n: int, nbins: int):
    """One frame of the scan: uniform at density 0.1, no box (a cube, r_max its
    diagonal), orthorhombic cube (r_max = L/2) or the 70/80/100-degree cell
    (r_max = 0.95 h_min/2)."""
    if box_name in ("c1", "c2", "c3"):
        return config_frames()[box_name]
    if box_name == "none":
        side = (n / 0.1) ** (1.0 / 3.0)
        f = w.uniform_frame(101, n, w.BOX_ORTHO, w.ortho_box(side), side * math.sqrt(3.0), nbins)
        return w.frame_from(f.coords, f.offsets, w.BOX_NONE, np.zeros(9), side * math.sqrt(3.0), nbins, "none")
    if box_name == "triclinic":
        box = w.scale_box(w.triclinic_box(1.0, 1.0, 1.0, *w.C3_ANGLES), n / 0.1)
        return w.uniform_frame(101, n, w.BOX_TRICLINIC, box, 0.95 * float(w.box_heights(box).min()) / 2.0, nbins)
    side = (n / 0.1) ** (1.0 / 3.0)
    return w.uniform_frame(101, n, w.BOX_ORTHO, w.ortho_box(side), side / 2.0, nbins)


def run_scan(args, world, rank, local):
    """Throughput against histogram width, block shape and private copies (plain
    path, one frame per point): the shared-memory staircase (one more bin sweep
    each time the width exceeds what a block holds) and the block-shape and
    depth tradeoffs.  Shapes are forced through the autotuner's cache file.  One
    JSON line per point; not the bench contract line."""
    import tempfile

    import torch

    import paper_1808_01478_gb300 as dh

    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    tmp = tempfile.mkdtemp(prefix="dh_scan_")
    points = [(b, n, k) for b in args.scan_boxes for n in args.scan_particles for k in args.scan_bins]
    points = list(dict.fromkeys((b, 0, 0) if b.startswith("c") else (b, n, k) for b, n, k in points))
    for box_name, n, nbins in points:
        f = scan_frame(box_name, n, nbins)
        n, nbins = f.n, f.nbins
        x = torch.from_numpy(f.coords).to(dev)
        out = torch.zeros((f.n_hist, nbins), dtype=torch.int64, device=dev)
        with dh.Context(local) as c0:  # default shape: learn the sweep width of this frame
            c0.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
            sweeps = c0.stats()["sweeps"]
        width = -(-nbins // sweeps)
        key = ({w.BOX_NONE: 0, w.BOX_ORTHO: 1}.get(f.box_type, 2), max(0, math.ceil(math.log2(width))),
               math.floor(math.log2(math.sqrt(2.0 * max(f.n_pairs(), 1))) + 0.5), 0)
        ref = None
        for block, depth, agg in args.scan_shapes:
            path = os.path.join(tmp, f"t_{box_name}_{n}_{nbins}_{block}_{depth}_{agg}.txt")
            with open(path, "w") as fh:
                fh.write(f"{sms} {key[0]} {key[1]} {key[2]} {key[3]} 1024 {block} {depth} 32 1.0 {agg}\n")
            with dh.Context(local, flags=dh.DH_CFG_TIMING, tune_cache=path) as ctx:
                ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
                st = ctx.stats()
                if (st["hist_depth"], st["block_threads"], st["warp_agg"]) != (depth, block, agg):
                    continue  # the copies or the larger block do not fit in shared memory
                ms = []
                for _ in range(args.scan_reps):
                    ctx.histogram(x, f.offsets, f.box_type, f.box, f.r_max, f.nbins, out)
                    ms.append(ctx.stats()["pair_kernel_ms"])
                got = out.cpu()
                ref = got if ref is None else ref
                print(json.dumps({"scan": "bins x block x depth", "box": box_name, "n": n, "nbins": nbins,
                                  "sweeps": st["sweeps"], "block_threads": block,
                                  "hist_depth": depth, "warp_agg": agg, "blocks_per_sm": st["blocks_per_sm"],
                                  "pair_kernel_ms": round(min(ms), 3),
                                  "culled_frac": round(st["culled_pairs"] / max(1, st["pairs"] * st["sweeps"]), 4),
                                  "gpairs_s": round(f.n_pairs() / (min(ms) / 1e3) / 1e9, 2),
                                  "same_as_first_shape": bool(torch.equal(got, ref))}), flush=True)
    return 0


def run_pipes(args, world, rank, local):
    """Measured throughput of every pipe dh_pipe_rate covers, one JSON line per
    pipe and width (shared atomics at several histogram widths, cluster atomics
    at several cluster sizes); not the bench contract line."""
    import paper_1808_01478_gb300 as dh

    if rank != 0:
        return 0
    points = [(name, 0) for name in PIPE_SET]
    points += [("smem_atomic_random", wd) for wd in (1024, 4096, 10000, 20000, 50000)]
    points += [("dsmem_atomic_c2", 100000), ("dsmem_atomic_c4", 200000), ("dsmem_atomic_c8", 400000)]
    points += [("global_atomic64", 10000), ("global_atomic64", 1 << 20)]
    for name, wd in points:
        if name.startswith("smem") and wd == 0:
            wd = 10000
        r = dh.dh_pipe_rate(local, name, wd)
        print(json.dumps({"pipe": name, "width": wd, "per_clk_sm": round(r["per_clk_sm"], 3),
                          "per_s": r["per_s"], "sm_mhz": round(r["sm_mhz"], 1), "ms": round(r["ms"], 3)}),
              flush=True)
    return 0


def run_gpu(args, world, rank, local):
    import torch

    import paper_1808_01478_gb300 as dh

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    td = init_dist(world, "nccl")
    frames = headline_frames(args.n, args.nbins)
    pairs = [f.n_pairs() for f in frames]
    pairs_step = sum(pairs)

    ctx = dh.Context(local, flags=dh.DH_CFG_TIMING | (0 if args.no_autotune else dh.DH_CFG_AUTOTUNE))
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream)
    X = [torch.from_numpy(f.coords).to(dev) for f in frames]
    OUT = [torch.zeros((1, f.nbins), dtype=torch.int64, device=dev) for f in frames]
    fas = [dh.FrameArgs(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins, OUT[k])
           for k, f in enumerate(frames)]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    # ---- measured per-pipe peaks (operations per clock per SM)
    pipes = measure_pipes(local, [args.nbins, 1000, 10000, 20000])

    # ---- batched step (headline value); the first warm-up call runs the autotuner
    tune_runs = 0
    for _ in range(args.warmup):
        ctx.histogram_batch(fas)
        tune_runs += ctx.stats()["tune_runs"]
    stats_b = ctx.stats()
    sampler = ClockSampler(local)
    sampler.start()
    if td:
        td.barrier()
    torch.cuda.synchronize()
    step_ms, pair_ms = [], []
    for _ in range(args.steps):
        flush_l2()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.histogram_batch(fas)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pair_ms.append(ctx.stats()["pair_kernel_ms"])
    torch.cuda.synchronize()
    if td:
        td.barrier()
    clocks = sampler.stop()
    value, t_total = aggregate_throughput(td, pairs_step * args.steps, sum(step_ms) / 1e3, dev)
    hist_sums = [int(o.sum().item()) for o in OUT]

    mhz = float(clocks["sm_mhz"]) if clocks else float(load_peaks().get("sm_max_mhz", 2070.0))

    # ---- plain per-frame path (and the pair kernel's own device time per frame)
    plain = {}
    bounds = {}
    evaluated = {}
    for k, f in enumerate(frames):
        ctx.histogram(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins, OUT[k])
        ts, pk = [], []
        for _ in range(max(1, args.plain_steps)):
            flush_l2()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.histogram(X[k], f.offsets, f.box_type, f.box, f.r_max, f.nbins, OUT[k])
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            pk.append(ctx.stats()["pair_kernel_ms"])
        st = ctx.stats()
        fu = st["uniform_pairs"] / max(1, st["pairs"])
        fa_ = st["axis_pairs"] / max(1, st["pairs"])
        f_cull = st["culled_pairs"] / max(1, st["pairs"] * st["sweeps"])  # of the pairs of all sweeps
        evaluated[k] = pairs[k] * (1.0 - f_cull)
        f_in = int(OUT[k].sum().item()) / max(1.0, evaluated[k])  # evaluated pairs inside r_max
        fu, fa_ = fu / (1.0 - f_cull) if f_cull < 1 else 0.0, fa_ / (1.0 - f_cull) if f_cull < 1 else 0.0
        bounds[k] = pair_bound(f.box_type, f.nbins, fu, fa_, pipes, f_in)
        plain[w.BOX_NAMES[f.box_type]] = {
            "gpairs_s": round(pairs[k] / (statistics.mean(ts) / 1e3) / 1e9, 3),
            "ms": round(statistics.mean(ts), 3),
            "pair_kernel_ms": round(statistics.mean(pk), 3),
            "deferred_frac": round(st["deferred"] / max(1, st["pairs"]), 6),
            "tile_image_frac": round(fu, 4),
            "axis_image_frac": round(fa_, 4),
            "culled_frac": round(f_cull, 4),
            "roofline": roofline_entry(evaluated[k], statistics.mean(pk) / 1e3, mhz, bounds[k]),
        }

    # ---- roofline of the pair kernel in the timed batched steps: pairs per
    # second of its launches (CUDA events on their stream) against the bound of
    # the step's frames, min over pipes of measured rate / operations per pair,
    # scaled by the SMs and the median SM clock sampled during the timed steps
    mean_pair_s = statistics.mean(pair_ms) / 1e3
    eval_step = sum(evaluated.values())
    clk_per_step = sum(evaluated[k] / bounds[k]["pairs_per_clk_sm"] for k in range(len(pairs)))  # SM-clocks
    peak_gpairs = eval_step / clk_per_step * SM_COUNT * mhz * 1e6 / 1e9
    achieved_gpairs = eval_step / mean_pair_s / 1e9
    headline_size = (args.n, args.nbins) == (1_000_000, 10_000)
    traffic = committed_traffic() if headline_size else None
    roofline = {"bound": "alu", "achieved": round(achieved_gpairs, 3), "peak": round(peak_gpairs, 3),
                "unit": "Gpairs/s",
                "achieved_basis": ("pairs the pair kernel evaluated (tiles skipped as outside the bins are not "
                                   "counted) over the CUDA-event time of its launches in the timed steps"),
                "frac": round(achieved_gpairs / peak_gpairs, 4), "traffic": traffic,
                "traffic_basis": ("DRAM bytes read + written by the step's three pair-kernel launches (ncu, "
                                  f"{TRAFFIC_FILE}); algorithmic: 3 x (16 B x N + 8 B x nbins)"
                                  if traffic else None),
                "kernel": "dh::pair_kernel",
                "per_frame": {w.BOX_NAMES[f.box_type]: plain[w.BOX_NAMES[f.box_type]]["roofline"] for f in frames},
                "peak_basis": (f"per frame min over pipes of measured rate (dh_pipe_rate, ops/clk/SM) / ops per "
                               f"pair (float32 FMA pipe by tile mode, MUFU sqrt, shared atomic at the width), "
                               f"combined over the step's frames, x {SM_COUNT} SMs x {mhz:.0f} MHz (median SM "
                               f"clock sampled during the timed steps)")}

    # ---- binary64 input coordinates (the same frames, coordinates perturbed below
    # float32 resolution so that they are not float32 values)
    f64 = {}
    if args.f64_steps > 0:
        for k, f in enumerate(frames):
            x64 = torch.from_numpy(f.coords.astype(np.float64)
                                   + w.rng_for(31 + k).random(f.coords.shape) * 1e-5).to(dev)
            ctx.histogram(x64, f.offsets, f.box_type, f.box, f.r_max, f.nbins, OUT[k])
            ts = []
            for _ in range(args.f64_steps):
                flush_l2()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.histogram(x64, f.offsets, f.box_type, f.box, f.r_max, f.nbins, OUT[k])
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            st = ctx.stats()
            f64[w.BOX_NAMES[f.box_type]] = {
                "gpairs_s": round(pairs[k] / (statistics.mean(ts) / 1e3) / 1e9, 3),
                "deferred_frac": round(st["deferred"] / max(1, st["pairs"]), 6),
                "binary64_frac": round(st["exact_fallback"] / max(1, st["pairs"]), 6),
            }
            del x64

    # ---- end to end through the C ABI with pinned host buffers
    hx = [torch.from_numpy(f.coords).pin_memory() for f in frames]
    ho = [torch.zeros((1, f.nbins), dtype=torch.int64).pin_memory() for f in frames]
    hfas = [dh.FrameArgs(hx[k].numpy(), f.offsets, f.box_type, f.box, f.r_max, f.nbins,
                         ho[k].numpy().view(np.uint64)) for k, f in enumerate(frames)]
    ctx.histogram_batch(hfas)
    if td:
        td.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.histogram_batch(hfas)
    torch.cuda.synchronize()
    e2e_val, _ = aggregate_throughput(td, pairs_step * args.e2e_steps, time.perf_counter() - t0, dev)
    e2e_ok = all(int(ho[k].sum()) == hist_sums[k] for k in range(len(frames)))
    h2d = sum(f.n * 12 for f in frames)
    d2h = sum(f.nbins * 8 for f in frames)

    configs = run_configs(ctx, stream, dev, args, pipes, mhz, flush_l2) if args.configs else None
    c4 = run_batched_c4(ctx, stream, dev, args) if args.c4_frames > 0 else None
    served = run_served_c5(local, dev, args) if args.served_requests > 0 else None

    launches_per_step = stats_b["kernel_launches"]
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_total / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (binary64 re-decision of near-edge pairs)", "data": "synthetic",
        "config": workload_config(args, world), "pairs_per_step": pairs_step,
        "e2e": {"value": round(e2e_val, 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps, "matches_device_result": e2e_ok},
        "plain": plain,
        "f64_input": f64 or None,
        "batched": {"gpairs_s": round(value, 3), "deferred_frac": round(stats_b["deferred"] / max(1, stats_b["pairs"]), 6),
                    "cuda_graph": bool(stats_b["graph_replays"]),
                    "launch_shape": {"tile_j": stats_b["tile_j"], "hist_depth": stats_b["hist_depth"],
                                     "blocks_per_sm": stats_b["blocks_per_sm"], "autotune_runs": tune_runs},
                    "c4": c4},
        "served": served,
        "configs": configs,
        "pipes": {"unit": "operations per clock per SM (dh_pipe_rate)", **pipes},
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        nthreads = os.cpu_count() or 1
        cb = oracle_sample(frames, args.cpu_seconds, nthreads)
        c1 = oracle_sample(frames, args.cpu_seconds / 5.0, 1)  # the same oracle on one core
        line["cpu_baseline"] = {"value": round(cb["gpairs_s"], 6), "unit": UNIT, "cores": nthreads,
                                "kind": "oracle",
                                "sample": f"leading subsets N={cb['sizes']} of the three frames, "
                                          f"{cb['pairs']} pairs in {cb['seconds']:.1f} s",
                                "one_core": {"value": round(c1["gpairs_s"], 6), "cores": 1,
                                             "sample": f"leading subsets N={c1['sizes']}, {c1['pairs']} pairs "
                                                       f"in {c1['seconds']:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if td:
        td.destroy_process_group()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["dh", "reference"], default="dh")
    ap.add_argument("--particles", dest="n", type=int, default=1_000_000,
                    help="particles per headline frame")
    ap.add_argument("--nbins", type=int, default=10_000)
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--f64-steps", type=int, default=1, help="timed calls per frame with binary64 coordinates")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shapes instead of measured ones")
    ap.add_argument("--c4-frames", type=int, default=256)
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--no-configs", dest="configs", action="store_false",
                    help="skip the C1-C3 configurations")
    ap.add_argument("--served-loads", type=float, nargs="*", default=[0.5, 0.8, 0.95])
    ap.add_argument("--pipes", action="store_true",
                    help="instead of the bench line: the measured throughput of each pipe (dh_pipe_rate)")
    ap.add_argument("--scan", action="store_true",
                    help="instead of the bench line: throughput against nbins and histogram copies")
    ap.add_argument("--scan-particles", type=int, nargs="*", default=[200_000])
    ap.add_argument("--scan-bins", type=int, nargs="*",
                    default=[1024, 4096, 16384, 32768, 50000, 60000, 100000, 160000, 250000])
    ap.add_argument("--scan-reps", type=int, default=3)
    ap.add_argument("--scan-boxes", nargs="*", default=["ortho", "triclinic"],
                    choices=["none", "ortho", "triclinic", "c1", "c2", "c3"],
                    help="synthetic frames of each box type, or the configurations C1-C3 as they are")
    ap.add_argument("--scan-shapes", nargs="*", default=["256x1", "256x2", "256x4", "512x1", "512x2", "1024x1"],
                    help="threads x histogram copies per block, suffix a: warp-aggregated increments")
    args = ap.parse_args(argv)
    args.scan_shapes = [(int(s.split("x")[0]), int(s.split("x")[1].rstrip("a")), int(s.endswith("a")))
                        for s in args.scan_shapes]
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.scan:
        return run_scan(args, world, rank, local)
    if args.pipes:
        return run_pipes(args, world, rank, local)
    return run_gpu(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
