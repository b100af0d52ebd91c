#!/usr/bin/env python
"""Throughput of the incident-wave reconstruction hot path on GB300.

One step = the whole path over one batch: stage 1 (modes -> zero-padded grid at every level,
for each of the time levels) and stage 2 (space-time interpolation of eta, u, v, w, p onto every
cell and face centre of the mesh). Default workload: 3-D JONSWAP sea, 512 x 256 modes, 64
levels, two time levels, 2.05 M cell centres + 6.18 M face centres of a graded O-grid around a
vertical cylinder (``wavegen.configs.jonswap3d``); inputs are synthetic and seeded.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle (direct modal sum)
on the host cores instead, on bounded samples of the same workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


class L2Flush:
    """Between timed steps: write a buffer larger than L2 (evicts everything the step left), then
    read a second one, so the dirty lines of the write reach DRAM before the next timed step
    rather than inside it: every step starts from a cold, clean L2."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        self.out = torch.empty((), dtype=torch.float32, device=dev)

    def __call__(self):
        import torch
        self.w.zero_()
        torch.amax(self.r, dim=0, out=self.out)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0,
                    help="timed steps (default: 5 for the large sea, 1000 for the smaller workloads)")
    ap.add_argument("--warmup", type=int, default=0,
                    help="untimed warm-up steps, at least 3 (default: 3 large, 10 otherwise)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=["jonswap3d", "stokes2d", "batched", "learned", "e1", "direct",
                                         "large", "relax", "stream", "tank"],
                    default="large")
    ap.add_argument("--pad", type=int, default=1)
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the untuned default launch shape of stage 1")
    ap.add_argument("--tune", default="",
                    help="stage-1 launch shape 'lpc,chunk_mb,row_variant' instead of autotuning "
                         "(e.g. the autotuner's earlier choice, for a profiler run)")
    ap.add_argument("--points", type=int, default=0,
                    help="direct mode: use only the first N near-body points; large mode: N "
                         "points instead of 16 M (small profiling cases)")
    ap.add_argument("--levels", type=int, default=0,
                    help="large mode: number of levels instead of 128 (small profiling case)")
    ap.add_argument("--near", type=int, default=0,
                    help="large mode: N near-body points instead of 1 M (small profiling case)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel from the host instead of replaying CUDA graphs")
    ap.add_argument("--no-pad4", action="store_true",
                    help="large mode: skip the 512x256-mode sea's pad-4 stage breakdown")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="host processes for the CPU oracle (default: every core this process may use)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- workload

def workload(name, pad):
    from wavegen import configs
    if name == "jonswap3d":
        cfg = configs.jonswap3d(pad_n=pad)
        pts = configs.mesh_points(cfg["mesh"])
        desc = (f"jonswap3d: 512x256 modes, 64 levels, pad {pad}, 2 time levels, "
                f"{len(cfg['mesh']['cell_centres'])} cell + {len(cfg['mesh']['face_centres'])} "
                f"face centres (cylinder O-grid)")
    else:
        cfg = configs.stokes2d()
        cfg["pad_n"] = pad
        pts = cfg["points"]
        desc = f"stokes2d: 256 modes (x,z), 33 levels, pad {pad}, 2 time levels, {len(pts)} points"
    return cfg, np.ascontiguousarray(pts, np.float32), desc


def touched_grid_bytes(cfg, pts, nxr, nyr, n_tl):
    """Unique grid bytes the gather reads: the union of every point's 4x4x4 node stencil (float4
    per node and time level) plus its 4x4 eta columns, counted with a bitmap."""
    from wavegen import configs  # noqa: F401  (workload helpers only)
    sea, z = cfg["sea"], np.asarray(cfg["z_levels"], np.float64)
    nz = len(z)
    mark = np.zeros((nz, nyr, nxr), bool)
    col = np.zeros((nyr, nxr), bool)
    for s in range(0, len(pts), 1 << 20):
        p = pts[s:s + (1 << 20)].astype(np.float64)
        ix = np.floor(p[:, 0] * nxr / sea["Lx"]).astype(np.int64)
        iy = np.floor(p[:, 1] * nyr / sea["Ly"]).astype(np.int64) if nyr > 1 else np.zeros(len(p), np.int64)
        j = np.clip(np.searchsorted(z, p[:, 2], side="right") - 1, 0, nz - 2)
        j0 = np.clip(j - 1, 0, nz - 4)
        dys = range(-1, 3) if nyr > 1 else (0,)
        for dx in range(-1, 3):
            xi = (ix + dx) % nxr
            for dy in dys:
                yi = (iy + dy) % nyr
                col[yi, xi] = True
                for dz in range(4):
                    mark[j0 + dz, yi, xi] = True
    return int(mark.sum()) * 16 * n_tl + int(col.sum()) * 4 * n_tl


# ----------------------------------------------------------------------------- clocks

def gpu_uuid(index):
    """nvidia-smi id of torch's device `index`: its UUID ("GPU-..."), which names the same physical
    GPU whatever CUDA_VISIBLE_DEVICES or the enumeration order; the index if torch has no UUID."""
    try:
        import torch
        u = str(torch.cuda.get_device_properties(index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:  # noqa: BLE001  (old torch without .uuid, or no device)
        return str(index)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.gpu_id = gpu_uuid(index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "gpu": self.gpu_id}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "gpu": self.gpu_id}


# ----------------------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(cfg, pts, seconds, seed=1):
    """Direct FP64 modal sum (the oracle) at a seeded sample of the workload's points, sized to
    take about ``seconds`` on one host core. Returns (points/s, n, values, idx)."""
    from oracle import modal
    sea = modal.propagate(cfg["sea"], cfg["t_query"])
    rng = np.random.default_rng(seed)
    probe = rng.choice(len(pts), 16, replace=False)
    t0 = time.perf_counter()
    modal.fields_at_points(sea, pts[probe].astype(np.float64))
    per = (time.perf_counter() - t0) / 16
    n = int(min(max(32, seconds / max(per, 1e-9)), 50_000))
    idx = rng.choice(len(pts), n, replace=False)
    t0 = time.perf_counter()
    vals = modal.fields_at_points(sea, pts[idx].astype(np.float64))
    dt = time.perf_counter() - t0
    return n / dt, n, vals, idx


def n_modes(sea):
    return int(np.count_nonzero((sea["A_eta"] != 0) | (sea["A_phi"] != 0) | (sea["A_phit"] != 0)))


# ----------------------------------------------------------------------------- arms

def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.config == "large":
        run_reference_large(args)
        return
    cfg, pts, desc = workload(args.config, args.pad)
    nm = n_modes(cfg["sea"])
    budget = 120.0 / max(1, args.steps + args.warmup)   # plus a 16-point probe per step
    per_step = []
    n_total = 0
    for s in range(args.warmup + args.steps):
        rate, n, _, _ = cpu_oracle_sample(cfg, pts, min(budget, 20.0), seed=100 + s)
        if s >= args.warmup:
            per_step.append(rate)
            n_total += n
    value = float(np.mean(per_step))
    line = {
        "impl": "reference", "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": value, "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": len(pts) / value * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n_total} seeded points of the workload over {args.steps} "
                                   f"steps; direct FP64 modal sum over {nm} modes; "
                                   f"ms_per_step extrapolated to all {len(pts)} points"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_large(args):
    """The FP64 oracle (direct modal sum) on every host core, each step a bounded sample of the
    large-sea workload's points, timed like the GPU arm's steps; the same config dict."""
    from wavegen import configs
    cfg = configs.large_sea(n_levels=args.levels or 128, n_points=args.points or 16_000_000)
    pts, near = cfg["points"], cfg["near_points"]
    allp = np.concatenate([pts, near])
    cores = args.cpu_cores or host_cores()
    per_step_s = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    rates, n_total = [], 0
    for s_ in range(args.warmup + args.steps):
        rate, n_, _, _, cores = cpu_oracle_pool("large", len(cfg["z_levels"]), cfg["t_query"], allp,
                                                per_step_s, cores, seed=100 + s_)
        if s_ >= args.warmup:
            rates.append(rate)
            n_total += n_
    value = float(np.mean(rates))
    line = {
        "impl": "reference", "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": value, "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": len(allp) / value * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": large_config(cfg, len(pts), len(near)),
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{n_total} seeded points of the workload over {args.steps} timed "
                                   f"steps; direct FP64 modal sum over {n_modes(cfg['sea'])} modes on "
                                   f"{cores} processes; ms_per_step extrapolated to all {len(allp)} points"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(value, world, device=None):
    """Largest value over the ranks (a job's step time is its slowest rank's); N = 1: unchanged."""
    if world <= 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_per_step):
    """Whole-job rate: every rank processes its own replica of the workload (weak scaling)."""
    return world * units_per_rank / (ms_per_step * 1e-3)


GATHER_SOURCES = ("csrc/interp.cu", "csrc/internal.cuh")
GRID_SOURCES = ("csrc/grid_ifft.cu", "csrc/fft.cuh", "csrc/internal.cuh")
GRID_STAGE = "grid_ifft (stage 1: k_propagate, eta k_pass_a/k_pass_b, k_col_t, k_row_t)"


def kernel_source_hash(files=GATHER_SOURCES):
    """Hash of the code a kernel is built from (paths relative to the package): the sources with
    their // comments and blank lines removed, so that a comment edit keeps a capture valid."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.normpath(os.path.join(ROOT, "paper_2005_12716_gb300", f)), encoding="utf-8") as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


# DRAM bytes per launch from ncu captures (dram__bytes_read.sum + dram__bytes_write.sum), with
# the hash of the kernel's sources and the workload they were taken on; a changed kernel or
# workload invalidates them (traffic is then reported as null).
NCU_TRAFFIC = {
    "k_interp_box": {"bytes": 114632192 + 113704704, "hash": "709995ea123f7df2",
                     "workload": "jonswap3d: 512x256 modes, 64 levels, pad 1, 2 time levels, "
                                 "2048000 cell + 6177280 face centres (cylinder O-grid)"},
    # all 13 launches of one step, caches kept between them (--cache-control none), launch shape
    # lpc 4, 64 MB level chunks, row variant 2
    GRID_STAGE: {"bytes": 284673536, "hash": "a8dc3ee11c502d0a",
                 "taken_with": {"lpc": 4, "chunk_bytes": 64 << 20, "row_variant": 2},
                 "workload": "jonswap3d: 512x256 modes, 64 levels, pad 1, 2 time levels, "
                             "2048000 cell + 6177280 face centres (cylinder O-grid)"},
}


DIRECT_KERNEL = "k_direct_tc"
DIRECT_SOURCES = ("csrc/direct_tc.cu", "csrc/tcgen05.cuh", "csrc/tma.cuh", "csrc/internal.cuh")
NCU_TRAFFIC[DIRECT_KERNEL] = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum (caches flushed before the launch),
    # one launch: 1,000,000 near-body points x the 2048 x 1024-mode sea (sources since changed
    # only by a compile-time check of the B column slots)
    "bytes": 59055616 + 9081856, "hash": "f174d5c52843f601",
    "workload": "near-body 1000000 points x 2048x1024 modes"}
# Algorithmic MMA flops of the split-BF16 direct sum (the per-unit figure of the workload's
# definition): per (point, mode) pair of the full nx x ny spectrum, u, v, w and dphi/dt each the
# real part of a complex product (2 MACs over the mode's re/im) in three BF16 products (hi.hi,
# hi.lo, lo.hi): 48 flop
DIRECT_FLOP_PER_PAIR = 4 * 2 * 2 * 3
DIRECT_FLOP_NOTE = ("per (point, mode) pair 48 flop: 4 fields x 2 MACs (re/im of the mode) x 2 flop "
                    "x 3 split products; pairs = near-body points x nx x ny modes (full spectrum)")


def direct_traffic(nn, sea):
    """ncu DRAM bytes of one k_direct_tc launch, when the kernel's sources and the workload are
    those of the capture (else None)."""
    tr = NCU_TRAFFIC.get(DIRECT_KERNEL)
    desc = f"near-body {nn} points x {sea['nx']}x{sea['ny']} modes"
    if tr and tr["hash"] == kernel_source_hash(DIRECT_SOURCES) and tr["workload"] == desc:
        return tr["bytes"]
    return None


def direct_tc_issued_flop(nx, ny, tiles):
    """MMA flops k_direct_tc issues for `tiles` tiles of 128 points (two tiles, one CTA pair, per
    M = 256 MMA): per tile, K-chunk of 32 modes and group of 8 mode-row pairs (n, -n), the
    products hi.hi and lo.hi of 128 x 208 x 64 and hi.lo of 128 x 144 x 64 (the columns with a lo
    half), padded as the kernel pads."""
    mp = -(-(nx // 2) // 64) * 64
    pairs = -(-(ny // 2) // 8) * 8 if ny > 1 else 8
    return tiles * (mp // 32) * (pairs // 8) * (2 * 208 + 144) * 2.0 * 128 * 64


def run_ours(args, rank, world, emit=True):
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg, pts_np, desc = workload(args.config, args.pad)
    sea, z, tl, tq, pad = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"], cfg["pad_n"]
    npts = len(pts_np)
    modes = api.upload_modes(sea, dev)
    grid = api.alloc_grid(modes, z, pad, tl, dev)
    pts = torch.from_numpy(pts_np).to(dev)
    outs = {k: torch.empty(npts, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        api.fields_on_grid(modes, z, pad, tl, out=grid)
        api.interp(grid, tq, pts, out=outs)

    # launch shape of stage 1 chosen by the library's autotuner (untimed, once per grid shape)
    if args.tune:
        lpc_, mb_, rv_ = (int(v) for v in args.tune.split(","))
        S.swense_set_grid_tune(sea["nx"], sea["ny"], pad, len(z), lpc_, mb_ << 20, rv_)
        tune = {"lpc": lpc_, "chunk_bytes": mb_ << 20, "row_variant": rv_, "source": "--tune"}
    elif not args.no_autotune:
        tune = api.autotune_grid(modes, z, pad, tl, out=grid)
    else:
        tune = None

    for _ in range(args.warmup):
        flush()
        step()
    torch.cuda.synchronize()
    # Each stage captured once into a CUDA graph (kernel arguments are captured by value; the
    # library's workspace was sized by the warm-up calls), then replayed per step.
    # Stage 2 runs as its two kernels, the gather plan (point chunks -> stencil boxes) and the
    # gather proper, so the dominant kernel is timed on its own; the plan is remade every step.
    plan = torch.empty(max(1, S.swense_interp_plan_bytes(npts)), dtype=torch.uint8, device=dev)
    launches_c0 = S.swense_launches()
    if not args.no_graph:
        g1, g2a, g2b = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1):
            api.fields_on_grid(modes, z, pad, tl, out=grid)
        launches_s1 = S.swense_launches() - launches_c0
        with torch.cuda.graph(g2a):
            api.interp_plan(grid, pts, out=plan)
        with torch.cuda.graph(g2b):
            api.interp_with_plan(grid, tq, pts, plan, out=outs)
        stage1, stage2a, stage2b = g1.replay, g2a.replay, g2b.replay
        launches_per_step = S.swense_launches() - launches_c0
        launches_s2 = launches_per_step - launches_s1
    else:
        stage1 = lambda: api.fields_on_grid(modes, z, pad, tl, out=grid)  # noqa: E731
        stage2a = lambda: api.interp_plan(grid, pts, out=plan)  # noqa: E731
        stage2b = lambda: api.interp_with_plan(grid, tq, pts, plan, out=outs)  # noqa: E731
        launches_per_step = None
        launches_s1 = launches_s2 = None
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        stage1()
        stage2a()
        stage2b()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    # One step: stage 1, the gather plan, the gather (events between them on the launching
    # stream). Running the plan concurrently with stage 1 on a second stream was measured and
    # gained nothing (both are latency-bound and share the SMs), so the step stays sequential.
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    launches0 = S.swense_launches()
    t_wall = time.perf_counter()
    for s in range(args.steps):
        flush()                     # L2 flush between timed steps (outside the events)
        ev[s][0].record(stream)
        stage1()
        ev[s][1].record(stream)
        stage2a()
        ev[s][2].record(stream)
        stage2b()
        ev[s][3].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = S.swense_launches() - launches0
    if launches_per_step is not None:
        launches = launches_per_step * args.steps
    clk = clocks.stop()
    k1 = np.array([ev[s][0].elapsed_time(ev[s][1]) for s in range(args.steps)])
    k2a = np.array([ev[s][1].elapsed_time(ev[s][2]) for s in range(args.steps)])
    k2b = np.array([ev[s][2].elapsed_time(ev[s][3]) for s in range(args.steps)])
    k2 = k2a + k2b
    total_ms = max_over_ranks(float(sum(ev[s][0].elapsed_time(ev[s][3]) for s in range(args.steps))),
                              world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = job_throughput(npts, world, ms_per_step)

    # ---- algorithmic bytes and roofline
    nxr, nyr = api.grid_dims(modes, pad)
    nz, n_tl = len(z), len(tl)
    nslot = sea["A_eta"].size
    k1_bytes = n_tl * (nz * nyr * nxr * 16 + nyr * nxr * 4) + nslot * (3 * 8 + 8)
    touched = touched_grid_bytes(cfg, pts_np, nxr, nyr, n_tl)
    k2_bytes = touched + npts * (12 + 20)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        with open(peaks_path) as fh:
            hbm = float(json.load(fh)["hbm_gbs"])
        peak_src = "measured"
    else:
        hbm, peak_src = FALLBACK_HBM_GBS, "fallback"
    k1_ms, k2_ms = float(k1.mean()), float(k2.mean())
    k2a_ms, k2b_ms = float(k2a.mean()), float(k2b.mean())
    box_bytes = k2_bytes                                  # the gather reads points, writes fields
    plan_bytes = npts * 12 + (npts + 1023) // 1024 * 16
    src_hash = kernel_source_hash()
    grid_hash = kernel_source_hash(GRID_SOURCES)
    stages = {
        "grid_ifft": {"ms": k1_ms, "algorithmic_bytes": k1_bytes,
                      "achieved_gbs": k1_bytes / (k1_ms * 1e-3) / 1e9,
                      "frac_hbm": k1_bytes / (k1_ms * 1e-3) / 1e9 / hbm,
                      "launches_per_step": launches_s1},
        "interp": {"ms": k2_ms, "algorithmic_bytes": k2_bytes, "touched_grid_bytes": touched,
                   "achieved_gbs": k2_bytes / (k2_ms * 1e-3) / 1e9,
                   "frac_hbm": k2_bytes / (k2_ms * 1e-3) / 1e9 / hbm,
                   "launches_per_step": launches_s2,
                   "k_interp_plan_ms": k2a_ms, "k_interp_plan_bytes": plan_bytes,
                   "k_interp_box_ms": k2b_ms},
    }
    if k2b_ms >= k1_ms:
        kname, dom_bytes, dom_ms, dom_hash = "k_interp_box", box_bytes, k2b_ms, src_hash
    else:
        # the stage as a whole (all its launches of one step, one stream or two)
        kname, dom_bytes, dom_ms, dom_hash = GRID_STAGE, k1_bytes, k1_ms, grid_hash
    tr = NCU_TRAFFIC.get(kname)
    traffic = tr["bytes"] if tr and tr.get("hash") == dom_hash and tr.get("workload") == desc else None
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "traffic_taken_with": (tr or {}).get("taken_with") if traffic is not None else None,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                else "fallback 6.8 TB/s"}
    # the binding resource of the gather: shared-memory reads per point, 16 float4 + 16 eta for
    # the chunks gathered from a z-collapsed plane, 64 float4 + 16 eta for the 3-D boxes, against
    # 128 B/clk/SM x 152 SMs at the maximum SM clock. The chunk kinds are read from the plan the
    # library made (int4 per chunk: w < 0 no tile, bit 30 of z set: flat plane(s), bit 29 as
    # well: two planes).
    pl = plan[: S.swense_interp_plan_bytes(npts)].view(torch.int32).view(-1, 4).cpu().numpy()
    per_chunk = np.full(len(pl), 1024)
    per_chunk[-1] = npts - 1024 * (len(pl) - 1)
    is_flat = (pl[:, 3] >= 0) & ((pl[:, 2] & (1 << 30)) != 0)
    is_box = (pl[:, 3] >= 0) & ~is_flat
    smem_bytes = float(per_chunk[is_flat].sum() * (16 * 16 + 16 * 4) + per_chunk[is_box].sum() * (64 * 16 + 16 * 4))
    smem_peak = 152 * 128 * 2070e6 / 1e9
    smem_gbs = smem_bytes / (k2b_ms * 1e-3) / 1e9
    tb = NCU_TRAFFIC.get("k_interp_box")
    stages["interp"]["k_interp_box_traffic"] = (tb["bytes"] if tb and tb.get("hash") == src_hash
                                               and tb.get("workload") == desc else None)
    is_two = is_flat & ((pl[:, 2] & (1 << 29)) != 0)
    stages["interp"]["chunks"] = {"flat_plane": int((is_flat & ~is_two).sum()),
                                  "flat_two_planes": int(is_two.sum()), "box_3d": int(is_box.sum()),
                                  "global": int((pl[:, 3] < 0).sum())}
    stages["interp"]["k_interp_box_shared_memory"] = {
        "achieved": smem_gbs, "peak": smem_peak, "unit": "GB/s", "frac": smem_gbs / smem_peak,
        "bytes_per_point": smem_bytes / npts}

    line = {
        "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "modes": [sea["nx"], sea["ny"]], "levels": nz, "pad_n": pad,
                   "launch": "host launches" if args.no_graph else "CUDA graph replay per stage",
                   "stage1_tune": tune,
                   "n_tl": n_tl, "points": npts, "fields": 5,
                   "l2": "flushed between timed steps (256 MB write, then a 256 MB read so the "
                         "written lines reach DRAM; both outside the events)",
                   "parallelism": f"replicas x{world}"},
        "points_fields_per_s": value * 5,
        "roofline": roofline,
        "stages": stages,
        "gpu_launches": int(launches),
        "clocks": clk,
        "wall_s_timed": t_wall,
        "kernel_hash": {"gather": src_hash, "grid": grid_hash},
    }

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        h_modes = [pin(modes.A_eta.cpu().numpy()), pin(modes.A_phi.cpu().numpy()),
                   pin(modes.A_phit.cpu().numpy()), pin(modes.omega.cpu().numpy())]
        h_pts = pin(pts_np)
        h_out = {k: torch.empty(npts, dtype=torch.float32).pin_memory() for k in outs}
        h2d = sum(t.numel() * t.element_size() for t in h_modes) + h_pts.numel() * 4
        d2h = sum(t.numel() * 4 for t in h_out.values())

        # Three streams and two buffer sets: step i's host->device copy (modes and points) runs
        # on the copy-in stream while step i-1 computes and step i-2's outputs go back on the
        # copy-out stream. Every step still copies its inputs in and its five fields out.
        s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        s_cmp = stream
        mset = [modes, api.upload_modes(sea, dev)]
        pset = [pts, torch.empty_like(pts)]
        oset = [outs, {k: torch.empty_like(v) for k, v in outs.items()}]
        ev = lambda: torch.cuda.Event()  # noqa: E731
        done_cmp = [None, None]
        done_out = [None, None]

        def e2e_step(i):
            b = i % 2
            m, pd, od = mset[b], pset[b], oset[b]
            with torch.cuda.stream(s_in):
                if done_cmp[b] is not None:
                    s_in.wait_event(done_cmp[b])          # buffers b free again
                for d, h in zip((m.A_eta, m.A_phi, m.A_phit, m.omega), h_modes):
                    d.copy_(h, non_blocking=True)
                pd.copy_(h_pts, non_blocking=True)
                e_in = ev()
                e_in.record(s_in)
            s_cmp.wait_event(e_in)
            if done_out[b] is not None:
                s_cmp.wait_event(done_out[b])             # outputs b copied out
            api.fields_on_grid(m, z, pad, tl, out=grid)
            api.interp(grid, tq, pd, out=od)
            e_c = ev()
            e_c.record(s_cmp)
            done_cmp[b] = e_c
            with torch.cuda.stream(s_out):
                s_out.wait_event(e_c)
                for k in od:
                    h_out[k].copy_(od[k], non_blocking=True)
                e_o = ev()
                e_o.record(s_out)
            done_out[b] = e_o

        for i in range(max(2, args.warmup)):
            e2e_step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ks = max(1, args.steps)
        e0.record(s_cmp)
        s_in.wait_event(e0)
        for i in range(ks):
            e2e_step(i)
        s_cmp.wait_stream(s_out)
        s_cmp.wait_stream(s_in)
        e1.record(s_cmp)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / ks, world, dev)
        line["e2e"] = {"value": job_throughput(npts, world, e_ms), "unit": "points/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": e_ms,
                       "pipeline": "copy-in, compute and copy-out streams overlap across steps"}

    # ---- CPU baseline: the FP64 oracle on a bounded sample, rank 0 at N = 1 only
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.config == "jonswap3d":
            cores = args.cpu_cores or host_cores()
            rate, n, vals, idx, cores = cpu_oracle_pool("jonswap3d", nz, tq, pts_np, args.cpu_seconds,
                                                        cores)
            how = f"numpy, {cores} spawned processes, one thread each"
        else:
            rate, n, vals, idx = cpu_oracle_sample(cfg, pts_np, args.cpu_seconds)
            cores, how = 1, "numpy, one thread"
        line["cpu_baseline"] = {
            "value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{n} seeded points of the {npts}; direct FP64 modal sum over "
                      f"{n_modes(sea)} modes ({how})"}
        # method error of the reconstruction at those points vs the exact modal sum, over the
        # whole sample and over its points below the exact free surface (above it the sum's
        # e^{|k| z} growth is carried by the shortest modes, which the grid resolves least)
        sel = torch.from_numpy(idx).to(dev)
        water = pts_np[idx, 2].astype(np.float64) <= vals["eta"]

        def rel_max(mask):
            err = {}
            for k in ("eta", "u", "v", "w", "p"):
                got = outs[k][sel].cpu().numpy().astype(np.float64)[mask]
                ref = vals[k][mask]
                err[k] = float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)) if ref.size else None
            return err
        line["method_error_vs_exact"] = {
            "norm": "max|gpu-exact|/max|exact| over the sample",
            "fields": rel_max(np.ones(len(idx), bool)),
            "fields_below_surface": rel_max(water),
            "points": int(len(idx)), "points_below_surface": int(water.sum()),
            "pad_n": int(pad)}
    if rank == 0 and emit:
        print(json.dumps(line), flush=True)
    return line


def _time_events(fn, steps, flush=None, clocks=None):
    """Device time per call of fn (CUDA events on the current stream, L2 flushed in between).
    With a dict ``clocks``, the SM clocks and throttle reasons sampled during the timed loop are
    stored in it."""
    import torch
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    sampler = ClockSampler(torch.cuda.current_device()) if clocks is not None else None
    if sampler is not None:
        sampler.start()
    for s in range(steps):
        if flush is not None:
            flush()
        ev[s][0].record(stream)
        fn()
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    if sampler is not None:
        clocks.update(sampler.stop())
    return float(np.mean([a.elapsed_time(b) for a, b in ev]))


def run_batched(args, rank, world):
    """64 uneven instances (grids 128^2 .. 1024^2 modes, 32 levels, 4 time levels, 10k .. 4M
    binned random points each), every instance's reconstruction and gather in one captured
    CUDA graph; autotuned FFT launch shapes. Compared with the same calls launched one by one."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import points as P, seas as W
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(20051273)
    items, nodes_bytes = [], 0
    for i in range(64):
        nx, ny = (int(2 ** rng.integers(7, 11)) for _ in range(2))
        lp = 1.0
        Hs = rng.uniform(0.02, 0.05) * lp
        sea = W.jonswap_sea(nx, ny, nx / 16 * lp, ny / 16 * lp, Hs, lp, heading=rng.uniform(0, 2 * np.pi),
                            seed=int(rng.integers(1 << 30)))
        z = P.levels_surface_clustered(-lp, 1.5 * Hs, 32, n_band=12, band=1.5 * Hs)
        npts = int(np.exp(rng.uniform(np.log(1e4), np.log(4e6))))
        pts = P.uniform_points(npts, (0, 0, -0.95 * lp), (nx / 16 * lp, ny / 16 * lp, 1.4 * Hs),
                               int(rng.integers(1 << 30)))
        Tp = 2 * np.pi / sea["jonswap"]["omega_p"]
        tl = np.arange(4) * Tp / 16
        items.append({"sea": sea, "z_levels": z, "pad_n": 1, "t_levels": tl,
                      "t": float(tl[1] + 0.37 * (tl[2] - tl[1])), "pts": pts, "bin": True})
        nodes_bytes += 4 * (32 * nx * ny * 16 + nx * ny * 4)
    b = api.Batch(items, device=dev)
    b.autotune()
    for _ in range(max(1, args.warmup)):
        b.run()
    torch.cuda.synchronize()
    l0 = S.swense_launches()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b.run()
    launches_per_step = S.swense_launches() - l0
    flush = L2Flush(dev)
    steps = max(3, min(args.steps, 30))
    clocks = ClockSampler(dev.index)
    clocks.start()
    ms_graph = _time_events(g.replay, steps, flush)
    clk = clocks.stop()
    ms_plain = _time_events(b.run, max(3, steps // 3), flush)
    for _ in range(2):
        b.run_individual()
    ms_indiv = _time_events(b.run_individual, max(3, steps // 3), flush)
    npts = b.points()
    algo = nodes_bytes + npts * (12 + 20)
    hbm = _peak_hbm()
    line = {
        "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": npts / (ms_graph * 1e-3), "unit": "points/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched: 64 uneven JONSWAP instances, grids 128^2..1024^2 modes, "
                               f"32 levels, 4 time levels (cubic), {npts} binned random points",
                   "launch": "one CUDA graph per step (all instances)", "l2": "flushed between steps"},
        "batch_call_host_launched_ms": ms_plain,
        "individual_calls_ms": ms_indiv, "speedup_vs_individual_calls": ms_indiv / ms_graph,
        "design": "reconstructions on 4 concurrent library streams (largest first), then one "
                  "planning launch and one persistent gather launch over a device queue of all "
                  "instances' point chunks; one CUDA graph per step",
        "gpu_launches": int(launches_per_step * steps),
        "roofline": {"bound": "hbm", "kernel": "whole batch (grid writes + point I/O)",
                     "achieved": algo / (ms_graph * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                     "frac": algo / (ms_graph * 1e-3) / 1e9 / hbm, "traffic": None},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"])
    return FALLBACK_HBM_GBS


def run_learned(args, rank, world):
    """Learned correction on the 3-D JONSWAP mesh workload: train on random JONSWAP seas with the
    same grid spacing and levels (GPU data + GPU training), then time the learned gather and compare
    its error against plain Lagrange interpolation at sampled points (FP64 oracle in the
    CPU-baseline leg)."""
    import torch
    from paper_2005_12716_gb300 import api, learn
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg, pts_np, desc = workload("jonswap3d", 1)
    sea, z, tl, tq = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    t0 = time.perf_counter()
    x, f, tg = learn.make_dataset(80, 65536, 64, 64, 4.0, 4.0, z, seed=20051274, device=dev,
                                  kind="jonswap")
    mlp = api.Mlp(api.mlp_init(20051275), dev)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = learn.train(mlp, x, f, tg, steps=4000, batch=8192, lr=2e-3, seed=20051276, log_every=500)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, f, tg
    modes = api.upload_modes(sea, dev)
    grid = api.fields_on_grid(modes, z, 1, tl)
    pts = torch.from_numpy(pts_np).to(dev)
    outs_l = {k: torch.empty(len(pts_np), dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    outs_p = {k: torch.empty(len(pts_np), dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    for _ in range(max(1, args.warmup)):
        api.interp_learned(grid, tq, pts, mlp, out=outs_l)
        api.interp(grid, tq, pts, out=outs_p)
    flush = L2Flush(dev)
    steps = max(3, min(args.steps, 20))
    from paper_2005_12716_gb300 import _swense as S
    clocks = ClockSampler(dev.index)
    clocks.start()
    l0 = S.swense_launches()
    ms_l = _time_events(lambda: api.interp_learned(grid, tq, pts, mlp, out=outs_l), steps, flush)
    launches = S.swense_launches() - l0
    clk = clocks.stop()
    ms_p = _time_events(lambda: api.interp(grid, tq, pts, out=outs_p), steps, flush)
    rows = 4 * len(pts_np)
    flops = rows * 2 * (67 * 64 + 64 * 64 + 64 * 4)
    # MMAs issued per 16 rows: layer 1 5 k-tiles x 8 n-tiles, layer 2 4 x 8, layer 3 4 x 1, each
    # twice (hi and lo activations), 4096 flop per m16n8k16
    mma_flops = rows / 16 * 2 * (5 * 8 + 4 * 8 + 4 * 1) * 4096
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as fh:
            peaks = json.load(fh)
    bf16_peak = float(peaks.get("bf16_tflops", 1910.8))
    line = {
        "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": len(pts_np) / (ms_l * 1e-3), "unit": "points/s", "n_gpus": 1, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_l, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 network (fp32 accumulate), f32 gather",
        "data": "synthetic", "config": {"workload": "learned correction on " + desc},
        "plain_gather_ms": ms_p, "train_seconds": t_train, "data_seconds": t_data,
        "train_loss_log": losses,
        "network_tflops_if_all_time_in_mlp": flops / (ms_l * 1e-3) / 1e12,
        "roofline": {"bound": "tensor", "kernel": "k_interp_learned",
                     "achieved": mma_flops / (ms_l * 1e-3) / 1e12, "peak": bf16_peak,
                     "unit": "TFLOP/s", "frac": mma_flops / (ms_l * 1e-3) / 1e12 / bf16_peak,
                     "traffic": None,
                     "note": "m16n8k16 MMA flops issued (split operands, padded shapes) over the "
                             "whole fused kernel time, against the measured dense BF16 peak"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import modal
        rng = np.random.default_rng(5)
        idx = rng.choice(len(pts_np), 4000, replace=False)
        ex = modal.fields_at_points(modal.propagate(sea, tq), pts_np[idx].astype(np.float64))
        sel = torch.from_numpy(idx).to(dev)
        err = {}
        for name, o in (("plain", outs_p), ("learned", outs_l)):
            vs = float(np.max(np.sqrt(ex["u"] ** 2 + ex["v"] ** 2 + ex["w"] ** 2)))
            err[name] = {k: float(np.sqrt(np.mean((o[k][sel].cpu().numpy() - ex[k]) ** 2)) / vs)
                         for k in ("u", "v", "w")}
        line["rms_error_vs_exact_over_vmax"] = err
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_e1(args, rank, world):
    """Divergence of the interpolated velocity on the x-z FV mesh for zero-padding 1, 2, 4, 8."""
    import torch
    from paper_2005_12716_gb300 import api
    from wavegen import configs
    cfg = configs.e1_divergence()
    m = cfg["mesh"]
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    fc = dv(m["face_centres"].astype(np.float32))
    area, cf, vol = dv(m["face_area"].astype(np.float32)), dv(m["cell_faces"]), dv(m["cell_volume"].astype(np.float32))
    below = torch.from_numpy(m["cell_centres"][:, 2] < -cfg["Hs"]).to(dev)
    modes = api.upload_modes(cfg["sea"], dev)
    res = {}
    for pad in (1, 2, 4, 8):
        grid = api.fields_on_grid(modes, cfg["z_levels"], pad, cfg["t_levels"])
        o, _ = api.interp(grid, 0.0, fc)
        d = api.fv_divergence(o["u"], o["v"], o["w"], area, cf, vol)
        res[pad] = float(torch.sqrt(torch.mean(d[below].double() ** 2)).item())
    # the divergence kernel's own speed on the 3-D cylinder mesh (2,048,000 cells, gathered
    # face velocities, areas and cell-face lists)
    from paper_2005_12716_gb300 import _swense as S
    c3 = configs.jonswap3d()
    m3 = c3["mesh"]
    g3 = api.fields_on_grid(api.upload_modes(c3["sea"], dev), c3["z_levels"], 1, c3["t_levels"])
    o3, _ = api.interp(g3, c3["t_query"], dv(m3["face_centres"].astype(np.float32)))
    a3, cf3 = dv(m3["face_area"].astype(np.float32)), dv(m3["cell_faces"])
    v3 = dv(m3["cell_volume"].astype(np.float32))
    div3 = torch.empty(len(m3["cell_volume"]), dtype=torch.float32, device=dev)
    fn = lambda: api.fv_divergence(o3["u"], o3["v"], o3["w"], a3, cf3, v3, out=div3)  # noqa: E731
    for _ in range(3):
        fn()
    l0 = S.swense_launches()
    ms = _time_events(fn, 20, L2Flush(dev))
    launches = S.swense_launches() - l0
    nc = len(m3["cell_volume"])
    nf = len(m3["face_area"])
    nbytes = nf * (12 + 12) + nc * (6 * 4 + 4 + 4)   # each face's u v w and area once; per cell
                                                     # its 6 face indices, volume and output
    line = {"metric": "RMS velocity divergence of the interpolated field [1/s]",
            "config": {"workload": "e1: 2-D JONSWAP Tp 0.7 s, Hs 0.028 m, 128 modes, FV mesh "
                                   "dx = lambda_p/100, dz = Hs/20, cells below -Hs"},
            "rms_by_pad": res, "ratio_pad1_over_pad4": res[1] / res[4],
            "fv_divergence_kernel": {"cells": nc, "ms": ms, "cells_per_s": nc / (ms * 1e-3),
                                     "achieved_gbs": nbytes / (ms * 1e-3) / 1e9,
                                     "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / _peak_hbm(),
                                     "gpu_launches": int(launches),
                                     "mesh": "jonswap3d cylinder O-grid, face values gathered per cell"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_relax(args, rank, world):
    """Incident VOF fraction and relaxation blending on the 2,048,000 cells of the cylinder mesh
    (eta at the cell centres from the gather; a ring zone over the outer quarter of the O-grid
    and three slabs)."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import configs, mesh as M
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = configs.jonswap3d()
    m = cfg["mesh"]
    cc = m["cell_centres"].astype(np.float32)
    lo, hi = M.cell_z_extent(m)
    zext = np.stack([lo, hi], 1).astype(np.float32)
    nc = len(cc)
    grid = api.fields_on_grid(api.upload_modes(cfg["sea"], dev), cfg["z_levels"], 1, cfg["t_levels"])
    d_cc, d_z = torch.from_numpy(cc).to(dev), torch.from_numpy(zext).to(dev)
    eta = api.interp(grid, cfg["t_query"], d_cc)[0]["eta"]
    rng = np.random.default_rng(5)
    alpha = torch.from_numpy(rng.uniform(0, 1, nc).astype(np.float32)).to(dev)
    uc = torch.from_numpy(rng.normal(0, 0.1, (nc, 3)).astype(np.float32)).to(dev)
    xc, yc = cfg["centre"]
    zones = [(S.ZONE_RADIAL, 1.5, 2.0, xc, yc), (S.ZONE_X, xc + 1.2, xc + 2.0, 0.0, 0.0),
             (S.ZONE_X, xc - 1.6, xc - 2.0, 0.0, 0.0), (S.ZONE_Y, yc - 1.7, yc - 2.0, 0.0, 0.0)]
    a_i = torch.empty(nc, dtype=torch.float32, device=dev)
    w = torch.empty(nc, dtype=torch.float32, device=dev)
    fn = lambda: api.relax_cells(d_cc, d_z, eta, zones, alpha=alpha, u_c=uc, out_alpha_i=a_i,  # noqa: E731
                                 out_weight=w)
    for _ in range(max(3, args.warmup)):
        fn()
    l0 = S.swense_launches()
    steps = max(1, args.steps)
    clk = {}
    ms = max_over_ranks(_time_events(fn, steps, L2Flush(dev), clk), world, dev)
    launches = S.swense_launches() - l0
    n_in = int((w > 0).sum().item())
    nbytes = nc * (12 + 8 + 4 + 4 + 4) + n_in * 2 * (4 + 12)    # all cells; blended cells r+w
    hbm = _peak_hbm()
    line = {"metric": "CFD cells per second (incident VOF fraction + relaxation blend)",
            "value": job_throughput(nc, world, ms), "unit": "cells/s", "n_gpus": world,
            "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"relax: jonswap3d cylinder O-grid, {nc} cells, {n_in} in zones "
                                   "(ring 1.5-2.0 lambda_p and three slabs)",
                       "l2": "flushed between timed steps"},
            "roofline": {"bound": "hbm", "kernel": "k_relax_cells", "achieved": nbytes / (ms * 1e-3) / 1e9,
                         "peak": hbm, "unit": "GB/s", "frac": nbytes / (ms * 1e-3) / 1e9 / hbm,
                         "traffic": None},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import relax as R                # the CPU baseline leg only
        t0 = time.perf_counter()
        R.relax_cells(cc, zext[:, 0], zext[:, 1], eta.cpu().numpy(), zones,
                      rng.uniform(0, 1, nc), rng.normal(0, 0.1, (nc, 3)))
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": nc / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                "sample": f"all {nc} cells (numpy FP64)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_stream(args, rank, world):
    """Analytical evaluation of the paper's stream-function wave (T 0.7 s, H 0.058 m, h 0.6 m,
    N = 9) at the 8,225,280 cell and face centres of a cylinder O-grid."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import configs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = configs.progressive_wave()
    pts_np = configs.mesh_points(cfg["mesh"])
    npts = len(pts_np)
    pts = torch.from_numpy(pts_np).to(dev)
    wave = api.stream_wave(cfg["T"], cfg["H"], cfg["h"], n=cfg["n"])
    out = {k: torch.empty(npts, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    fn = lambda: api.stream_eval(wave, cfg["t_query"], pts, p_mode="total", out=out)  # noqa: E731
    for _ in range(max(3, args.warmup)):
        fn()
    l0 = S.swense_launches()
    steps = max(1, args.steps)
    clk = {}
    ms = max_over_ranks(_time_events(fn, steps, L2Flush(dev), clk), world, dev)
    launches = S.swense_launches() - l0
    nbytes = npts * (12 + 20)
    hbm = _peak_hbm()
    # FP32 operations per point: 19 per harmonic (14 instructions, 5 of them FMA) and about 30
    # for the phase, Bernoulli and stores' arithmetic; sincospif and expf are not counted.
    # Peak: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz.
    flops = npts * (19 * cfg["n"] + 30)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    line = {"metric": "wave-field points/sec, stream-function wave (analytical evaluation)",
            "value": job_throughput(npts, world, ms), "unit": "points/s", "n_gpus": world,
            "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"stream: T 0.7 s, H 0.058 m, h 0.6 m, N = {cfg['n']}; {npts} "
                                   "cell + face centres (cylinder O-grid to two wavelengths)",
                       "l2": "flushed between timed steps"},
            "roofline": {"bound": "alu", "kernel": "k_stream_eval",
                         "achieved": flops / (ms * 1e-3) / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": flops / (ms * 1e-3) / 1e12 / fp32_peak, "traffic": None,
                         "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                         "hbm": {"achieved_gbs": nbytes / (ms * 1e-3) / 1e9, "peak_gbs": hbm,
                                 "frac": nbytes / (ms * 1e-3) / 1e9 / hbm},
                         "issue_active_ncu": 0.79},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import stream as O               # the CPU baseline leg only
        o = O.solve(cfg["T"], cfg["H"], cfg["h"], cfg["n"])
        sample = pts_np[:: max(1, npts // 200000)].astype(np.float64)
        t0 = time.perf_counter()
        O.fields_at_points(o, sample, t=cfg["t_query"])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(sample) / dt, "unit": "points/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"{len(sample)} of the {npts} points (numpy FP64)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_tank(args, rank, world):
    """Wave-tank reconstruction: 257 x 129 cosine modes (two snapshots) mapped onto the mirrored
    512 x 256 periodic grid, 64 levels, gathered at the 8,225,280 cell and face centres of a
    cylinder O-grid in the tank. One step = mode mapping + grid + gather."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import configs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = configs.tank3d()
    pts_np = configs.mesh_points(cfg["mesh"])
    npts = len(pts_np)
    pts = torch.from_numpy(pts_np).to(dev)
    dvA = lambda k: torch.from_numpy(np.stack([s[k] for s in cfg["snaps"]]).astype(np.float32)).to(dev)  # noqa: E731
    Ae, Ap, At = dvA("A_eta"), dvA("A_phi"), dvA("A_phit")
    z, tl, tq = cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    modes = api.tank_modes(Ae, Ap, At, cfg["Lx"], cfg["Ly"], cfg["depth"])
    grid = api.fields_on_grid(modes, z, 1, tl)
    outs = {k: torch.empty(npts, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}

    def step():
        m = api.tank_modes(Ae, Ap, At, cfg["Lx"], cfg["Ly"], cfg["depth"])
        api.fields_on_grid(m, z, 1, tl, out=grid)
        api.interp(grid, tq, pts, out=outs)
    for _ in range(max(3, args.warmup)):
        step()
    l0 = S.swense_launches()
    steps = max(1, args.steps)
    clk = {}
    ms = max_over_ranks(_time_events(step, steps, L2Flush(dev), clk), world, dev)
    launches = S.swense_launches() - l0
    line = {"metric": "wave-field points/sec, wave tank (cosine basis on the mirrored grid)",
            "value": job_throughput(npts, world, ms), "unit": "points/s", "n_gpus": world,
            "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"tank3d: 257x129 cosine modes (2 snapshots), mirrored 512x256 grid, "
                                   f"{len(z)} levels, {npts} cell + face centres",
                       "launch": "host launches", "l2": "flushed between timed steps"},
            "clocks": clk, "gpu_launches": int(launches)}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_direct(args, rank, world):
    """Direct modal sums at the near-body points of the 3-D JONSWAP mesh (r < 0.25 lambda_p of the
    cylinder axis), FP32 and split-BF16 tensor-core paths, each checked against the FP64 direct sum
    on a seeded sample of points."""
    import torch
    from oracle import modal
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import configs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = configs.jonswap3d()
    sea, tq = cfg["sea"], cfg["t_query"]
    pts_np = configs.near_body_points(cfg)
    if args.points:
        pts_np = np.ascontiguousarray(pts_np[:args.points])
    npts = len(pts_np)
    nmodes = int((sea["ny"] - 1) * (sea["nx"] // 2))
    modes = api.upload_modes(sea, dev)
    pts = torch.from_numpy(pts_np).to(dev)
    outs = {k: torch.empty(npts, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    sel = np.random.default_rng(20051279).choice(npts, min(192, npts), replace=False)
    ref = modal.fields_at_points(modal.propagate(sea, tq), pts_np[sel].astype(np.float64))
    vs = float(np.max(np.sqrt(ref["u"] ** 2 + ref["v"] ** 2 + ref["w"] ** 2)))
    steps = max(3, min(args.steps, 10))
    res = {}
    clocks = ClockSampler(dev.index)
    clocks.start()
    for prec in ("fp32", "split_bf16"):
        fn = lambda: api.direct(modes, tq, pts, precision=prec, out=outs)  # noqa: E731
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        l0 = S.swense_launches()
        ms = _time_events(fn, steps)
        launches = S.swense_launches() - l0
        err = {}
        for k in ("eta", "u", "v", "w", "p"):
            got = outs[k][torch.from_numpy(sel).to(dev)].cpu().numpy().astype(np.float64)
            scale = vs if k in ("u", "v", "w") else float(np.max(np.abs(ref[k])))
            err[k] = float(np.max(np.abs(got - ref[k])) / scale)
        res[prec] = {"ms": ms, "points_per_s": npts / (ms * 1e-3),
                     "pairs_per_s": npts * nmodes / (ms * 1e-3), "launches": launches,
                     "max_err_vs_fp64": err}
    clk = clocks.stop()
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as fh:
            peaks = json.load(fh)
    bf16_peak = float(peaks.get("bf16_tflops", 1910.8))
    # split path: per 16 points x 8 modes (deep water) three m16n8k16 MMAs of 4096 flop each
    sp = res["split_bf16"]
    mma_tflops = sp["pairs_per_s"] / 128 * 3 * 4096 / 1e12
    line = {
        "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": sp["points_per_s"], "unit": "points/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, args.warmup), "ms_per_step": sp["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (split) / f32 accumulate",
        "data": "synthetic",
        "config": {"workload": f"direct: {npts} near-body mesh points (r < 0.25 lambda_p) x {nmodes} "
                               f"modes of the 512x256 JONSWAP sea, deep water",
                   "l2": "inputs (modes table) are re-read from L2 by design; not flushed"},
        "paths": res,
        "roofline": {"bound": "tensor", "kernel": "k_direct_split", "achieved": mma_tflops,
                     "peak": bf16_peak, "unit": "TFLOP/s", "frac": mma_tflops / bf16_peak,
                     "traffic": None,
                     "note": "MMA flops issued incl. the four zero columns; operand generation on "
                             "the FMA/MUFU pipes binds"},
        "gpu_launches": int(res["split_bf16"]["launches"] * 1),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- CPU oracle pool

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


_POOL_SEA = None
_POOL_Z = None


def _pool_init(kind, n_levels, t):
    """Worker start-up (spawned process): rebuild the workload's sea from its seed, propagated to
    the query time, with one numpy thread per process."""
    global _POOL_SEA, _POOL_Z
    from oracle import modal
    from wavegen import configs
    if kind == "large":
        cfg = configs.large_sea(n_levels=n_levels, n_points=1, n_near=1)
    else:
        cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    _POOL_SEA = modal.propagate(cfg["sea"], t)
    _POOL_Z = cfg["z_levels"]


def _pool_work(pts):
    from oracle import modal
    return modal.fields_at_points(_POOL_SEA, pts, chunk=4)


def _method_level(args):
    """One worker task of the CPU method baseline: the method's grid at level l of the large sea
    (library inverse FFTs of the four modal fields), timed."""
    from oracle import method
    l, pad = args
    t0 = time.perf_counter()
    method.grid_fft(_POOL_SEA, _POOL_Z, pad, levels=[l])
    return time.perf_counter() - t0


def _method_interp(args):
    """One worker task of the CPU method baseline: the oracle's literal space-time interpolation
    of `n` seeded points on a 4-level grid of the 512 x 256-mode sea (two time levels), timed; its
    cost per point does not depend on the grid's size."""
    from oracle import interp, method, modal
    from wavegen import configs
    n, seed = args
    cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    z = np.asarray(cfg["z_levels"], np.float64)[28:32]
    tl = cfg["t_levels"]
    nodes, etas = zip(*(method.grid_fft(modal.propagate(cfg["sea"], t), z, 1) for t in tl))
    rng = np.random.default_rng(seed)
    p = np.stack([rng.uniform(0, cfg["sea"]["Lx"], n), rng.uniform(0, cfg["sea"]["Ly"], n),
                  rng.uniform(z[1], z[2], n)], 1)
    t0 = time.perf_counter()
    interp.interp_points(np.stack(nodes), np.stack(etas), cfg["sea"]["Lx"], cfg["sea"]["Ly"], z, tl, p,
                         cfg["t_query"])
    return time.perf_counter() - t0


def cpu_method_pool(n_levels, n_tl, t, n_points, cores, n_interp=20000):
    """The CPU method baseline on `cores` spawned processes (one numpy thread each): the grid step
    timed on `cores` of the large sea's levels (each a library inverse FFT per modal field) and
    the literal interpolation timed on `cores` x n_interp points; the step's time is extrapolated
    to all n_tl x n_levels level transforms and n_points points."""
    import multiprocessing as mp
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores, initializer=_pool_init, initargs=("large", n_levels, t)) as pool:
            lev = list(np.linspace(0, n_levels - 1, cores).astype(int))
            t0 = time.perf_counter()
            per_level = pool.map(_method_level, [(l, 1) for l in lev])
            grid_wall = time.perf_counter() - t0
            t0 = time.perf_counter()
            per_interp = pool.map(_method_interp, [(n_interp, 7 + c) for c in range(cores)])
            interp_wall = time.perf_counter() - t0
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    grid_s = float(np.mean(per_level)) * n_tl * n_levels / cores
    interp_s = float(np.mean(per_interp)) / n_interp * n_points / cores
    return {"grid_s": grid_s, "interp_s": interp_s, "level_transform_s": float(np.mean(per_level)),
            "interp_points_per_s_per_core": n_interp / float(np.mean(per_interp)),
            "sample_wall_s": grid_wall + interp_wall}


ORACLE_SAMPLE_CAP = 200_000


def oracle_sample_order(n_pts, seed=1):
    """Seeded order of the points the CPU oracle evaluates. A run takes its first n entries, n set
    by the time bound, so runs that admit different n share their first points and their error
    figures compare."""
    return np.random.default_rng(seed).choice(n_pts, min(n_pts, ORACLE_SAMPLE_CAP), replace=False)


def cpu_oracle_pool(kind, n_levels, t, pts, seconds, cores, seed=1):
    """The FP64 oracle's direct modal sum at a seeded sample of ``pts`` on ``cores`` host processes
    (spawned, one numpy thread each), sized to take about ``seconds``: the first n points of
    ``oracle_sample_order``. Returns (points/s, n, values, idx, cores)."""
    import multiprocessing as mp
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        order = oracle_sample_order(len(pts), seed)
        with ctx.Pool(cores, initializer=_pool_init, initargs=(kind, n_levels, t)) as pool:
            probe = pts[order[np.arange(cores) % len(order)]].astype(np.float64)
            pool.map(_pool_work, [probe[i:i + 1] for i in range(cores)])        # warm every worker
            t0 = time.perf_counter()
            pool.map(_pool_work, [probe[i:i + 1] for i in range(cores)])
            per = (time.perf_counter() - t0)                                     # one point per core
            n = int(min(max(cores, seconds / max(per, 1e-9) * cores), len(order)))
            n = min(len(order), max(cores, (n // cores) * cores))
            idx = order[:n]
            sample = pts[idx].astype(np.float64)
            parts = np.array_split(sample, cores * 4)
            t0 = time.perf_counter()
            res = pool.map(_pool_work, parts)
            dt = time.perf_counter() - t0
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    vals = {k: np.concatenate([r[k] for r in res]) for k in res[0]}
    return n / dt, n, vals, idx, cores


# ----------------------------------------------------------------------------- large sea (default)

def large_config(cfg, n, nn):
    """The workload description both arms print (same keys, same values)."""
    z = cfg["z_levels"]
    return {"workload": f"large_sea: JONSWAP k_p Hs/2 = 0.12, 2048x1024 modes, {len(z)} levels, 2 time "
                        f"levels; {n} Morton-order points by grid + space-time interpolation, {nn} "
                        f"near-body points by direct split-BF16 modal sum over all modes",
            "modes": [2048, 1024], "levels": len(z), "pad_n": 1, "n_tl": len(cfg["t_levels"]),
            "points": n, "near_body_points": nn, "fields": 5,
            "l2": "inputs larger than L2 (8.6 GB grid written every step); a 256 MB flush between "
                  "timed steps as well"}


def run_large(args, rank, world):
    """Default workload, the largest single-GPU configuration: large steep sea (2048 x 1024 modes,
    128 levels, two time levels). One step = the grid at both time levels + the gather of 16 M
    points (Morton order) + the split-BF16 direct sum at 1 M near-body points over all modes."""
    import torch
    from paper_2005_12716_gb300 import _swense as S
    from paper_2005_12716_gb300 import api
    from wavegen import configs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    cfg = configs.large_sea(n_levels=args.levels or 128, n_points=args.points or 16_000_000,
                            n_near=args.near or 1_000_000)
    sea, z, tl, tq = cfg["sea"], cfg["z_levels"], cfg["t_levels"], cfg["t_query"]
    pts_np, near_np = cfg["points"], cfg["near_points"]
    n, nn = len(pts_np), len(near_np)
    modes = api.upload_modes(sea, dev)
    grid = api.alloc_grid(modes, z, 1, tl, dev)
    pts = torch.from_numpy(pts_np).to(dev)
    near = torch.from_numpy(near_np).to(dev)
    outs = {k: torch.empty(n, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    outn = {k: torch.empty(nn, dtype=torch.float32, device=dev) for k in ("eta", "u", "v", "w", "p")}
    flush = L2Flush(dev)
    stream = torch.cuda.current_stream(dev)
    if args.tune:
        lpc_, mb_, rv_ = (int(v) for v in args.tune.split(","))
        S.swense_set_grid_tune(sea["nx"], sea["ny"], 1, len(z), lpc_, mb_ << 20, rv_)
        tune = {"lpc": lpc_, "chunk_bytes": mb_ << 20, "row_variant": rv_, "source": "--tune"}
    elif not args.no_autotune:
        tune = api.autotune_grid(modes, z, 1, tl, out=grid)
    else:
        tune = None
    stages = (("grid", lambda: api.fields_on_grid(modes, z, 1, tl, out=grid)),
              ("gather", lambda: api.interp(grid, tq, pts, out=outs)),
              ("direct_near_body", lambda: api.direct(modes, tq, near, precision="split_bf16", out=outn)))
    for _ in range(args.warmup):
        flush()
        for _, fn in stages:
            fn()
    torch.cuda.synchronize()
    S.swense_async_status(reset=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(args.steps)]
    launches0 = S.swense_launches()
    t_wall = time.perf_counter()
    for s_ in range(args.steps):
        flush()                                   # outside the events
        ev[s_][0].record(stream)
        for j, (_, fn) in enumerate(stages):
            fn()
            ev[s_][j + 1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    launches = S.swense_launches() - launches0
    clk = clocks.stop()
    S.swense_async_status(reset=True)             # no bounded device wait gave up
    st_ms = {name: float(np.mean([ev[s_][j].elapsed_time(ev[s_][j + 1]) for s_ in range(args.steps)]))
             for j, (name, _) in enumerate(stages)}
    total_ms = max_over_ranks(float(sum(ev[s_][0].elapsed_time(ev[s_][-1]) for s_ in range(args.steps))),
                              world, dev)
    if world > 1:
        torch.distributed.barrier()
    ms_per_step = total_ms / args.steps
    value = job_throughput(n + nn, world, ms_per_step)

    # ---- algorithmic bytes / flops per stage and the roofline of the dominant kernel
    hbm = _peak_hbm()
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        with open(pp) as fh:
            peaks = json.load(fh)
    nx_r, ny_r = api.grid_dims(modes, 1)
    nz, n_tl = len(z), len(tl)
    nslot = sea["A_eta"].size
    grid_bytes = n_tl * (nz * nx_r * ny_r * 16 + nx_r * ny_r * 4) + nslot * (3 * 8 + 8)
    # the gather: every node of both time levels is in some stencil (16 M uniform points over
    # 268 M nodes; the union of their stencils covers about 98 % of the grid): the whole grid once
    gather_bytes = n_tl * (nz * nx_r * ny_r * 16 + nx_r * ny_r * 4) + n * (12 + 20)
    pairs = float(nn) * sea["nx"] * sea["ny"]
    d_ms = st_ms["direct_near_body"]
    direct_flop = pairs * DIRECT_FLOP_PER_PAIR
    tiles, fb_tiles = S.swense_direct_stats()
    issued = direct_tc_issued_flop(sea["nx"], sea["ny"], tiles - fb_tiles)
    stages_out = {
        "grid": {"ms": st_ms["grid"], "algorithmic_bytes": grid_bytes,
                 "achieved_gbs": grid_bytes / (st_ms["grid"] * 1e-3) / 1e9,
                 "frac_hbm": grid_bytes / (st_ms["grid"] * 1e-3) / 1e9 / hbm},
        "gather": {"ms": st_ms["gather"], "algorithmic_bytes": gather_bytes,
                   "achieved_gbs": gather_bytes / (st_ms["gather"] * 1e-3) / 1e9,
                   "frac_hbm": gather_bytes / (st_ms["gather"] * 1e-3) / 1e9 / hbm,
                   "points_per_s": n / (st_ms["gather"] * 1e-3)},
        "direct_near_body": {"ms": d_ms, "pairs": pairs, "pairs_per_s": pairs / (d_ms * 1e-3),
                             "points_per_s": nn / (d_ms * 1e-3),
                             "algorithmic_tflops": direct_flop / (d_ms * 1e-3) / 1e12,
                             "tiles": tiles, "tiles_per_pair_kernel": fb_tiles,
                             "issued_mma_tflops": issued / (d_ms * 1e-3) / 1e12},
    }
    tens_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    dom = max(st_ms, key=st_ms.get)
    if dom == "direct_near_body":
        ach = direct_flop / (d_ms * 1e-3) / 1e12
        roofline = {"bound": "tensor", "kernel": DIRECT_KERNEL, "achieved": ach, "peak": tens_peak,
                    "unit": "TFLOP/s", "frac": ach / tens_peak,
                    "traffic": direct_traffic(nn, sea),
                    "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops_sustained: the kernel "
                                   "runs for hundreds of ms)" if peaks else "fallback 1.7 PFLOP/s",
                    "algorithmic": DIRECT_FLOP_NOTE}
    else:
        b = stages_out[dom]["algorithmic_bytes"]
        ach = b / (st_ms[dom] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                    "frac": ach / hbm, "traffic": None,
                    "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback"}
    stages_out["direct_near_body"]["frac_tensor"] = stages_out["direct_near_body"]["algorithmic_tflops"] / tens_peak
    stages_out["direct_near_body"]["issued_frac_tensor"] = stages_out["direct_near_body"]["issued_mma_tflops"] / tens_peak
    config = large_config(cfg, n, nn)
    line = {
        "metric": "wave-field points/sec at stated err vs FP64 oracle; % of HBM roofline",
        "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (grid, gather); bf16x3 split / f32 accumulate (near-body direct sum)",
        "data": "synthetic", "config": config,
        "launch": {"stage1_tune": tune, "mode": "host launches, one stream",
                   "parallelism": f"replicas x{world}"},
        "points_fields_per_s": value * 5,
        "roofline": roofline, "stages": stages_out,
        "gpu_launches": int(launches), "clocks": clk, "wall_s_timed": t_wall,
        "kernel_hash": {"direct": kernel_source_hash(DIRECT_SOURCES), "grid": kernel_source_hash(GRID_SOURCES),
                        "gather": kernel_source_hash(GATHER_SOURCES)},
    }

    # ---- end to end through the public API with host buffers
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        h_modes = [pin(modes.A_eta.cpu().numpy()), pin(modes.A_phi.cpu().numpy()),
                   pin(modes.A_phit.cpu().numpy()), pin(modes.omega.cpu().numpy())]
        h_pts, h_near = pin(pts_np), pin(near_np)
        h_out = {k: torch.empty(n, dtype=torch.float32).pin_memory() for k in outs}
        h_outn = {k: torch.empty(nn, dtype=torch.float32).pin_memory() for k in outn}
        h2d = sum(t.numel() * t.element_size() for t in h_modes) + (n + nn) * 12
        d2h = (n + nn) * 4 * 5

        # the 16 M points' copies run on a copy stream: the points' upload under the grid stage,
        # the gathered fields' download under the direct sum (the library calls stay on one
        # stream: they share the library's workspace)
        xs = torch.cuda.Stream(dev)
        ev_pts, ev_gathered, ev_read = (torch.cuda.Event() for _ in range(3))
        ev_gathered.record(stream)
        ev_read.record(stream)

        def e2e_step():
            for d, h in zip((modes.A_eta, modes.A_phi, modes.A_phit, modes.omega), h_modes):
                d.copy_(h, non_blocking=True)
            near.copy_(h_near, non_blocking=True)
            with torch.cuda.stream(xs):
                xs.wait_event(ev_gathered)                 # the last gather has read the points
                pts.copy_(h_pts, non_blocking=True)
                ev_pts.record(xs)
            api.fields_on_grid(modes, z, 1, tl, out=grid)
            stream.wait_event(ev_pts)
            stream.wait_event(ev_read)                     # the last fields are downloaded
            api.interp(grid, tq, pts, out=outs)
            ev_gathered.record(stream)
            with torch.cuda.stream(xs):
                xs.wait_event(ev_gathered)
                for k in outs:
                    h_out[k].copy_(outs[k], non_blocking=True)
                ev_read.record(xs)
            api.direct(modes, tq, near, precision="split_bf16", out=outn)
            for k in outn:
                h_outn[k].copy_(outn[k], non_blocking=True)
        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        stream.wait_event(ev_read)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        line["e2e"] = {"value": job_throughput(n + nn, world, e_ms), "unit": "points/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": e_ms,
                       "pipeline": "pinned host -> device copies of modes and near-body points, the "
                                   "three stages and the near-body fields' download on the compute "
                                   "stream; the 16 M points' upload (under the grid stage) and their "
                                   "fields' download (under the direct sum) on a copy stream"}

    # ---- CPU baseline (the FP64 oracle on every host core, bounded sample) and the error of the
    # timed outputs against it, rank 0 at N = 1 only
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = args.cpu_cores or host_cores()
        allp = np.concatenate([pts_np, near_np])
        rate, m_, vals, idx, cores = cpu_oracle_pool("large", nz, tq, allp, args.cpu_seconds, cores)
        line["cpu_baseline"] = {
            "value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{m_} seeded points of the {n + nn} (mesh and near-body); direct FP64 modal "
                      f"sum over {n_modes(sea)} modes (numpy, {cores} spawned processes, one "
                      f"thread each)"}
        got_all = {k: torch.cat([outs[k], outn[k]]) for k in outs}
        sel = torch.from_numpy(idx).to(dev)
        water = allp[idx, 2].astype(np.float64) <= vals["eta"]
        is_near = idx >= n

        def rel_max(mask):
            err = {}
            for k in ("eta", "u", "v", "w", "p"):
                got = got_all[k][sel].cpu().numpy().astype(np.float64)[mask]
                ref = vals[k][mask]
                err[k] = float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300)) if ref.size else None
            return err
        meth = cpu_method_pool(nz, n_tl, tq, n, cores)
        # the near-body points by the oracle's direct sum at the rate measured above
        near_s = nn / rate
        meth_step = meth["grid_s"] + meth["interp_s"] + near_s
        line["cpu_method_baseline"] = {
            "value": (n + nn) / meth_step, "unit": "points/s", "cores": cores,
            "kind": "method on the CPU: numpy inverse real FFT per level and field + the oracle's "
                    "literal Lagrange interpolation (FP64); near-body points by the direct sum",
            "step_s": meth_step, "grid_s": meth["grid_s"], "interp_s": meth["interp_s"],
            "near_body_s": near_s,
            "sample": f"{cores} level transforms of the large sea and {cores} x 20000 interpolated "
                      f"points timed, extrapolated to {n_tl} x {nz} levels and {n} points"}
        line["error_vs_fp64_oracle"] = {
            "norm": "max|gpu-exact|/max|exact| per field over the sample",
            "near_body_direct": rel_max(is_near), "near_body_points": int(is_near.sum()),
            "gather_all": rel_max(~is_near), "gather_below_surface": rel_max(~is_near & water),
            "gather_points": int((~is_near).sum()),
            "note": "the gather's error is the reconstruction's own interpolation error at pad 1 "
                    "(method error), the direct sum's is its arithmetic error"}

    # ---- context: the 512x256-mode sea at the paper's padding n = 4 (stage breakdown)
    if rank == 0 and world == 1 and not args.no_pad4:
        del grid, outs, outn, pts, near
        torch.cuda.empty_cache()
        sub = argparse.Namespace(**vars(args))
        sub.config, sub.pad, sub.tune, sub.no_e2e = "jonswap3d", 4, "", True
        sub.steps, sub.warmup = max(3, min(args.steps, 20)), max(3, args.warmup)
        sub.cpu_seconds = min(args.cpu_seconds, 10.0)
        line["jonswap3d_pad4"] = run_ours(sub, rank, world, emit=False)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.steps <= 0:
        args.steps = 5 if args.config == "large" else 1000
    if args.warmup <= 0:
        args.warmup = 3 if args.config == "large" else 10
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    try:
        {"batched": run_batched, "learned": run_learned, "e1": run_e1, "direct": run_direct,
         "large": run_large, "relax": run_relax, "stream": run_stream, "tank": run_tank}.get(
            args.config, run_ours)(
            args, rank, world)
    finally:
        if world > 1:
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
