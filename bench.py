"""Benchmark: periodic tricubic B-spline VGH on the paper-shaped workload.

Workload (arXiv:1611.02665, Sec. "Experiments and Results": 48^3 grid,
N up to 4096 orbitals, random positions): 48^3 grid, N = 2048 orbitals, a
smooth plane-wave FP32 table [51][51][51][2048] (1.09 GB), 4096 walkers with
one random position each. One step = one VGH evaluation of the 4096
positions (cell reduction, weights, 64-row gather, FMA accumulation, SoA
stores of 10 x 2048 floats per position). Fresh positions every step; the
table (1.09 GB) is larger than L2, so no explicit flush is needed.

Metric: orbital evaluations per second (positions x orbitals / s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas: the method has no exchange step), timing is the max over ranks and
the value is the sum of all ranks' work over that time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GRID = (48, 48, 48)
NORB = 2048
NPOS = 4096
# general cell of the lattice extra (rows are the lattice vectors): hexagonal a-b plane, tilted c axis
LATTICE_HEX = ((1.3, 0.0, 0.0), (0.65, 1.1258330249197703, 0.0), (0.2, -0.3, 2.1))
METRIC = "VGH orbital evals/s (positions x orbitals)"
UNIT = "orbital-evals/s"
WORKLOAD = "vgh_grid48^3_N2048_4096pos_planewave_fp32"
HBM_FALLBACK_GBS = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def vgh_bytes_per_position(N, esize):
    """Algorithmic bytes of one VGH position: 64 rows of N table elements read, 10 N floats written."""
    return 64 * N * esize + 10 * N * 4


def v_bytes_per_position(N, esize):
    return 64 * N * esize + N * 4


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "samples": len(sm), "reasons": sorted(reasons)}


def aggregate_over_ranks(elapsed_ms, units, dist=None):
    """(max elapsed over ranks, units summed over ranks): the whole job's time and work.

    Each rank evaluates its own positions (replicas; the method has no exchange
    step), so only these two scalars cross ranks.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(elapsed_ms), float(units)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(rank, step):
    """Seed of the positions a rank evaluates at a step: distinct across ranks and steps."""
    return 10_000 * (rank + 1) + step


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_cpu_baseline(coef_np, nsample, seed, kind=2):
    """The FP64 oracle, as it stands, on a bounded sample of the workload's positions."""
    import oracle

    x, y, z = (a[:nsample] for a in _positions(nsample, seed))
    coef64 = coef_np.astype(np.float64)
    t0 = time.perf_counter()
    oracle.eval_periodic(kind, coef64, x, y, z)
    dt = time.perf_counter() - t0
    return nsample * coef_np.shape[-1] / dt, dt, oracle.num_threads()


def run_cpu_baseline_small():
    """The oracle on the small table (16^3 grid, 64 orbitals, uniform coefficients, seed 1): VGH at the
    1024 positions (seed 2) that the L2-resident measurement evaluates, repeated for about a second."""
    import oracle
    from paper_1611_02665_gb300 import inputs

    coef = inputs.uniform_coefs((16, 16, 16), 64, seed=1).astype(np.float64)
    x, y, z = inputs.uniform_positions(1024, seed=2)
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.eval_periodic(oracle.VGH, coef, x, y, z)
        reps += 1
        dt = time.perf_counter() - t0
        if dt > 1.0 or reps >= 200:
            break
    return {"value": reps * 1024 * 64 / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "sample": f"{reps} x 1024 positions x 64 orbitals, VGH, FP64, 16^3 grid, {dt:.2f} s"}


def run_cpu_baseline_precision():
    """The oracle on the reduced-precision workload's table and positions (16^3 grid, 64 orbitals, uniform
    coefficients seed 1, VGH at 16384 positions seed 5), timed once. Its outputs, on the original float32
    coefficients, are what the FP32 / FP16 / BF16 tables' outputs are compared with."""
    import oracle
    from paper_1611_02665_gb300 import inputs

    coef = inputs.uniform_coefs((16, 16, 16), 64, seed=1).astype(np.float64)
    x, y, z = inputs.uniform_positions(16384, seed=5)
    t0 = time.perf_counter()
    ref = oracle.eval_periodic(oracle.VGH, coef, x, y, z)
    dt = time.perf_counter() - t0
    line = {"value": 16384 * 64 / dt, "unit": UNIT, "cores": oracle.num_threads(),
            "sample": f"16384 positions x 64 orbitals, VGH, FP64, 16^3 grid, {dt:.2f} s"}
    return line, ref


def _positions(npos, seed):
    from paper_1611_02665_gb300 import inputs
    return inputs.uniform_positions(npos, seed)


def bench_reference(args):
    """--impl reference: the FP64 CPU oracle timed per step on a bounded sample of the workload."""
    world, rank, local = _dist()
    if rank != 0:
        return
    import oracle
    import torch
    from paper_1611_02665_gb300 import inputs

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    coef = inputs.plane_wave_coefs(GRID, NORB, seed=3, device=dev).cpu().numpy().astype(np.float64)
    nsample = args.ref_sample
    steps = []
    for s in range(args.warmup + args.steps):
        x, y, z = inputs.uniform_positions(nsample, seed=1000 + s)
        t0 = time.perf_counter()
        oracle.eval_periodic(oracle.VGH, coef, x, y, z)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            steps.append(dt)
    t = sum(steps) / len(steps)
    value = nsample * NORB / t
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(GRID), "N": NORB, "npos_per_step": nsample,
                   "sampled": True, "workload_npos_per_step": NPOS, "kind": "VGH",
                   "note": f"FP64 CPU oracle on a bounded sample of {nsample} of the workload's {NPOS} "
                           "positions per step: a rate, not the same batch as the GPU arm"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{nsample} positions x {NORB} orbitals per step, VGH"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_ours(args):
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    kind = capi.VGH
    coef = inputs.plane_wave_coefs(GRID, NORB, seed=3, device="cuda")
    table = capi.Table(GRID, NORB, capi.F32)
    capi.bspline_set_coefs(table.h, coef)
    if args.tune:
        capi.bspline_tune(table.h, kind, NPOS)
    else:
        capi.bspline_set_tuning(table.h, kind, args.variant, args.nb, args.ppc, args.stages, args.order)
    tuning = capi.bspline_get_tuning(table.h, kind)
    stream = torch.cuda.current_stream()

    nsteps = args.warmup + args.steps
    pos = []
    for s in range(nsteps):
        x, y, z = inputs.uniform_positions(NPOS, seed=rank_seed(rank, s))
        pos.append([torch.from_numpy(a).cuda() for a in (x, y, z)])
    v, g, h = table.outputs(kind, NPOS)
    torch.cuda.synchronize()

    def step(s):
        x, y, z = pos[s]
        capi.bspline_eval_vgh(table.h, NPOS, x, y, z, v, g, h, NORB, stream)

    for s in range(args.warmup):
        step(s)
    torch.cuda.synchronize()
    assert capi.bspline_device_status(table.h) == 0

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    # Events only around the whole region: an event recorded between two calls would stop the next call's
    # sort from overlapping the previous evaluation (programmatic dependent launch).
    t_start.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = t_start.elapsed_time(t_end)
    elapsed_ms, units = aggregate_over_ranks(elapsed_ms, args.steps * NPOS * NORB, dist)
    assert capi.bspline_device_status(table.h) == 0
    ms_per_step = elapsed_ms / args.steps
    value = units / (elapsed_ms / 1e3)

    hbm, hbm_src = _peaks()
    bytes_launch = NPOS * vgh_bytes_per_position(NORB, 4)
    # per-launch duration of the evaluation = device time per step over the timed region (it includes the
    # part of the sort that does not overlap the previous evaluation, so it is an upper bound)
    avg_kernel_s = ms_per_step / 1e3
    achieved = bytes_launch / avg_kernel_s / 1e9
    traffic = _profiled_traffic(tuning)

    result = {}
    if rank == 0:
        # End to end through the host-buffer entry point: pinned host positions in, pinned host outputs out.
        e2e = None if args.no_e2e else _e2e(table, kind, args, 0)
        e2e_staged = None if args.no_e2e else _e2e(table, kind, args, 1)
        cpu, precision_ref = None, None
        if not args.no_cpu_baseline:
            rate, dt, cores = run_cpu_baseline(coef.cpu().numpy(), args.cpu_sample, seed=77)
            precision_line, precision_ref = run_cpu_baseline_precision()
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{args.cpu_sample} positions x {NORB} orbitals, VGH, FP64, {dt:.2f} s",
                   "small_table": run_cpu_baseline_small(), "precision_table": precision_line}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": list(GRID), "N": NORB, "npos_per_step": NPOS, "kind": "VGH",
                       "table_dtype": "f32", "table_bytes": table_bytes(GRID, NORB, 4),
                       "l2": "inputs larger than L2 (1.09 GB table, fresh positions each step)",
                       "tuning": tuning, "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         # frac counts every position's 64 stencil rows (the algorithmic bytes), so rows that
                         # cell-sorted positions share through L2 count once per position: it is not an
                         # HBM efficiency. dram_frac (the DRAM bytes ncu measured for one launch of this
                         # kernel, built from these sources, over the same time) is.
                         "frac_algorithmic": achieved / hbm,
                         "traffic_source_hash": eval_source_hash(),
                         "peak_source": f"{hbm_src} hbm_gbs",
                         "algorithmic_bytes_per_launch": bytes_launch,
                         "kernel_ms_avg": avg_kernel_s * 1e3,
                         # the DRAM bytes one launch moves (ncu) over the same time: how close the
                         # kernel runs to the copy peak once L2 reuse is taken out of the bytes
                         "dram_gbs": traffic / avg_kernel_s / 1e9 if traffic else None,
                         "dram_frac": traffic / avg_kernel_s / 1e9 / hbm if traffic else None},
            "e2e": e2e,
            "e2e_staged_copies": e2e_staged,
            "cpu_baseline": cpu,
            # one evaluation kernel per step, plus the cell sort when the positions are ordered
            "gpu_launches": args.steps * (2 if tuning["order"] == 1 else 1),
            "clocks": clk,
        }
        if not args.no_extras:
            result["extras"] = _extras(coef, args, precision_ref)
        print(json.dumps(result), flush=True)
    table.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def table_bytes(grid, N, esize):
    pad = (N + 128 // esize - 1) // (128 // esize) * (128 // esize)
    return (grid[0] + 3) * (grid[1] + 3) * (grid[2] + 3) * pad * esize


# Sources of the headline evaluation (kernels, the sort, their launch code): a DRAM-traffic figure taken
# by ncu holds for the kernel these files build, and for no other.
EVAL_SOURCES = ("bspline_internal.cuh", "bspline_eval_kernels.cuh", "bspline_mma_kernel.cuh",
                "tcgen05_ptx.cuh", "bspline_eval_f32.cu", "bspline_lib.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def eval_source_hash():
    """First 16 hex digits of the SHA-256 of the evaluation's source files, in a fixed order."""
    import hashlib

    h = hashlib.sha256()
    for name in EVAL_SOURCES:
        with open(os.path.join(ROOT, "paper_1611_02665_gb300", "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def _shape_key(tuning):
    return " ".join(str(tuning[k]) for k in ("variant", "nb", "ppc", "stages", "order"))


def _profiled_traffic(tuning):
    """DRAM bytes per launch from the committed ncu capture, if it covers this workload and launch shape AND
    was taken on the sources that built the running library (else None: the figure would be stale)."""
    want = _shape_key(tuning)
    src = eval_source_hash()
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    for line in lines:
        parts = [p.strip() for p in line.split("|")]
        if line.startswith("#") or len(parts) != 5:
            continue
        wl, shape, h, nbytes, _ = parts
        if wl == WORKLOAD and shape == want and h == src:
            return float(nbytes)
    return None


def record_traffic(csv_path, tuning, summary):
    """Write the DRAM bytes of one captured launch (an `ncu -i <rep> --page raw --csv` export holding one
    launch of the evaluation kernel) into the traffic file, keyed by workload, launch shape and the current
    source hash; an older line of the same workload and shape is replaced."""
    import csv

    rows = list(csv.reader(open(csv_path)))
    head = rows[0]
    data = [r for r in rows[1:] if r and r[0].strip().isdigit()]  # skip the units row
    if len(data) != 1:
        raise SystemExit(f"{csv_path}: expected exactly one captured launch, found {len(data)}")
    rec = dict(zip(head, data[0]))
    unit_row = rows[1]
    units = dict(zip(head, unit_row))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    for k in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        if units.get(k, "byte") not in scale:
            raise SystemExit(f"unknown unit {units.get(k)} for {k}")
    nbytes = (float(rec["dram__bytes_read.sum"].replace(",", "")) * scale[units.get("dram__bytes_read.sum", "byte")]
              + float(rec["dram__bytes_write.sum"].replace(",", "")) * scale[units.get("dram__bytes_write.sum", "byte")])
    key = (WORKLOAD, _shape_key(tuning))
    keep = []
    for line in open(TRAFFIC_FILE):
        parts = [p.strip() for p in line.split("|")]
        if not line.startswith("#") and len(parts) == 5 and (parts[0], parts[1]) == key:
            continue
        keep.append(line.rstrip("\n"))
    keep.append(f"{WORKLOAD} | {key[1]} | {eval_source_hash()} | {int(round(nbytes))} | {summary}")
    with open(TRAFFIC_FILE, "w") as f:
        f.write("\n".join(keep) + "\n")
    print(keep[-1])


def _e2e(table, kind, args, mode=0):
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    capi.bspline_set_host_mode(table.h, mode)

    steps = max(3, min(args.steps, 10))
    host = []
    for s in range(steps + 1):
        x, y, z = inputs.uniform_positions(NPOS, seed=500 + s)
        host.append([torch.from_numpy(a).pin_memory() for a in (x, y, z)])
    v = torch.empty((NPOS, NORB), dtype=torch.float32).pin_memory()
    g = torch.empty((NPOS, 3, NORB), dtype=torch.float32).pin_memory()
    h = torch.empty((NPOS, 6, NORB), dtype=torch.float32).pin_memory()

    def one(s):
        x, y, z = host[s]
        capi.bspline_eval_host(table.h, kind, NPOS, x, y, z, v, g, h, NORB)

    one(steps)  # warm-up: allocates the staging buffers
    t0 = time.perf_counter()
    for s in range(steps):
        one(s)
    dt = (time.perf_counter() - t0) / steps
    h2d = NPOS * 3 * 8
    d2h = NPOS * 10 * NORB * 4
    capi.bspline_set_host_mode(table.h, 0)
    return {"value": NPOS * NORB / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": dt * 1e3, "steps": steps,
            "path": {0: "auto (direct access when reachable)", 1: "staged copies", 2: "direct access"}[mode]}


def _time_eval(table, kind, nsteps, npos, seed0, shape=None, lattice=None):
    """Per-launch time (ms) of `kind` over fresh positions (Cartesian r = u L if a lattice is given)."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    if shape:
        capi.bspline_set_tuning(table.h, kind, *shape)

    pos = []
    for s in range(nsteps + 3):
        u = inputs.uniform_positions(npos, seed=seed0 + s)
        if lattice is not None:
            r = np.stack(u, axis=1) @ np.asarray(lattice)
            u = [np.ascontiguousarray(r[:, d]) for d in range(3)]
        pos.append([torch.from_numpy(a).cuda() for a in u])
    v, g, hl = table.outputs(kind, npos)
    stream = torch.cuda.current_stream()
    for s in range(3):
        table.eval(kind, *pos[s], v, g, hl)
    return _region_ms(stream, lambda s: table.eval(kind, *pos[3 + s], v, g, hl), nsteps)


def _region_ms(stream, launch, nsteps):
    """Mean device time (ms) per call of `launch(s)`, s = 0..nsteps-1, back to back on `stream`, with events
    only around the region (so consecutive calls pipeline as they would in a loop), median of 3 regions."""
    import torch

    runs = []
    for _ in range(3):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s in range(nsteps):
            launch(s)
        b.record(stream)
        b.synchronize()
        runs.append(a.elapsed_time(b) / nsteps)
    return statistics.median(runs)


def _set_values(coef):
    """Coefficients from grid samples (the interpolation solve) for the 48^3 x 2048 table."""
    import torch

    from paper_1611_02665_gb300 import capi

    ms = []
    with capi.Table(GRID, NORB, capi.F32) as t:
        for r in range(4):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            capi.bspline_set_values(t.h, coef)  # synchronous: returns with the table filled
            ms.append((time.perf_counter() - t0) * 1e3)
    nbytes = coef.numel() * 4
    return {"ms": statistics.median(ms[1:]), "bytes_samples": nbytes,
            "note": "3 recursive-filter passes (inverse knot operator): samples -> table interior, in place, "
                    "in place plus the periodic copies"}


def _time_ratio(table, kind, nsteps, npos, seed0):
    """Per-call time (ms) of the fused ratio sums (bspline_eval_ratio) over fresh positions."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed0)
    u = torch.randn((npos, table.N), generator=gen, device="cuda") / table.N ** 0.5
    r = torch.empty((npos, capi.NCOMP[kind]), device="cuda")
    stream = torch.cuda.current_stream()
    pos = [[torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=seed0 + s)]
           for s in range(nsteps + 3)]

    def launch(s):
        x, y, z = pos[s]
        capi.bspline_eval_ratio(table.h, kind, npos, x, y, z, u, table.N, r, stream)

    for s in range(3):
        launch(s)
    return _region_ms(stream, lambda s: launch(3 + s), nsteps)


def _ratio_e2e(table, nsteps=10):
    """End to end through the fused ratio consumer: pinned host positions and inverse entries copied in,
    the 10 VGH ratio sums per position copied out, every step (the per-orbital outputs never leave the
    GPU). Wall-clock time per step over nsteps after 2 untimed steps."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    stream = torch.cuda.current_stream()
    gen = np.random.default_rng(9800)
    u_host = torch.from_numpy((gen.normal(size=(NPOS, NORB)) / np.sqrt(NORB)).astype(np.float32)).pin_memory()
    host = [[torch.from_numpy(a).pin_memory() for a in inputs.uniform_positions(NPOS, seed=9810 + s)]
            for s in range(nsteps + 2)]
    dx, dy, dz = (torch.empty(NPOS, dtype=torch.float64, device="cuda") for _ in range(3))
    du = torch.empty((NPOS, NORB), device="cuda")
    dr = torch.empty((NPOS, 10), device="cuda")
    r_host = torch.empty((NPOS, 10)).pin_memory()

    def one(s):
        for d, h in zip((dx, dy, dz), host[s]):
            d.copy_(h, non_blocking=True)
        du.copy_(u_host, non_blocking=True)
        capi.bspline_eval_ratio(table.h, capi.VGH, NPOS, dx, dy, dz, du, NORB, dr, stream)
        r_host.copy_(dr, non_blocking=True)
        stream.synchronize()

    for s in range(2):
        one(nsteps + s)
    t0 = time.perf_counter()
    for s in range(nsteps):
        one(s)
    dt = (time.perf_counter() - t0) / nsteps
    return {"value": NPOS * NORB / dt, "unit": UNIT, "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": NPOS * 3 * 8 + NPOS * NORB * 4, "d2h_bytes_per_step": NPOS * 10 * 4,
            "note": "bspline_eval_ratio, VGH: positions and one row of inverse entries per position in, "
                    "10 sums per position out"}


def _extras(coef, args, precision_ref=None):
    """V throughput and reduced-precision tables on the same workload (reported beside the headline)."""
    from paper_1611_02665_gb300 import capi

    out = {}
    shape = (args.variant, args.nb, args.ppc, args.stages, args.order)
    # V and 16-bit tables load rows into registers (the shared-memory ring is for FP32 VGL and VGH)
    plain = (args.variant, args.nb, args.ppc, 0, args.order)
    out["launch_shape"] = dict(zip(("variant", "nb", "ppc", "stages", "order"), shape))
    with capi.Table(GRID, NORB, capi.F32) as t:
        capi.bspline_set_coefs(t.h, coef)
        ms_vgh = _time_eval(t, capi.VGH, 10, NPOS, 9000, shape)
        ms_v = _time_eval(t, capi.V, 10, NPOS, 9100, plain)
        ms_ratio = _time_ratio(t, capi.VGH, 10, NPOS, 9300)
        ratio_e2e = _ratio_e2e(t)
        capi.bspline_set_lattice(t.h, LATTICE_HEX)
        ms_lat_vgh = _time_eval(t, capi.VGH, 10, NPOS, 9400, shape, LATTICE_HEX)
        ms_lat_vgl = _time_eval(t, capi.VGL, 10, NPOS, 9500, shape, LATTICE_HEX)
        capi.bspline_set_lattice(t.h, None)
    hbm, _ = _peaks()
    out["fp32_vgh_ms"] = ms_vgh
    # fused determinant-ratio consumer: 10 sums per position instead of 10 x 2048 outputs
    rbytes = NPOS * (64 * NORB * 4 + NORB * 4 + 40)
    out["fp32_vgh_ratio"] = {"ms": ms_ratio, "speedup_vs_vgh_outputs": ms_vgh / ms_ratio,
                             "orbital_evals_per_s": NPOS * NORB / (ms_ratio / 1e3),
                             "hbm_frac": rbytes / (ms_ratio / 1e3) / 1e9 / hbm, "e2e": ratio_e2e}
    out["fp32_v"] = {"ms": ms_v, "orbital_evals_per_s": NPOS * NORB / (ms_v / 1e3),
                     "hbm_frac": NPOS * v_bytes_per_position(NORB, 4) / (ms_v / 1e3) / 1e9 / hbm}
    out["lattice_hex"] = {"vgh_ms": ms_lat_vgh, "vgl_ms": ms_lat_vgl, "vgh_slowdown_vs_unit_cube": ms_lat_vgh / ms_vgh,
                          "vgh_orbital_evals_per_s": NPOS * NORB / (ms_lat_vgh / 1e3),
                          "note": "Cartesian positions in a hexagonal cell (a = 1.3, c = 2.1, tilted c axis)"}
    out["set_values"] = _set_values(coef)
    out["l2_resident"] = _l2_resident(precision_ref)
    out["graphite_shape"] = _graphite_shape(out["l2_resident"]["l2_read_gbs"])
    out["n_sweep"] = _n_sweep(out["l2_resident"]["l2_read_gbs"])
    out["batched"] = _batched(args)
    if not args.no_surrogate:
        out["surrogate"] = _surrogate(args)
    # 16-bit tables: the tensor-core variant (2 CTAs per SM, the deepest ring that fits, units of two
    # 128-orbital blocks) and, for comparison, DIRECT
    mma_shape = (capi.VARIANT_MMA, 256, 2, 0, args.order)
    for name, dt, es in (("fp16", capi.F16, 2), ("bf16", capi.BF16, 2)):
        with capi.Table(GRID, NORB, dt) as t:
            capi.bspline_set_coefs(t.h, coef)
            ms = _time_eval(t, capi.VGH, 10, NPOS, 9200, mma_shape)
            mma_tuning = capi.bspline_get_tuning(t.h, capi.VGH)
            ms_ratio16 = _time_ratio(t, capi.VGH, 10, NPOS, 9300)  # the ratio sums follow the VGH shape
            ms_vgl16 = _time_eval(t, capi.VGL, 10, NPOS, 9400, mma_shape)
            ms_direct = _time_eval(t, capi.VGH, 10, NPOS, 9200, plain)
            ms_ratio16_direct = _time_ratio(t, capi.VGH, 10, NPOS, 9300)
        out[f"{name}_vgh"] = {"ms": ms, "launch_shape": mma_tuning,
                              "ratio_ms": ms_ratio16, "ratio_fma_kernel_ms": ms_ratio16_direct,
                              "vgl_ms": ms_vgl16,
                              "direct_ms": ms_direct, "speedup_vs_fp32": ms_vgh / ms,
                              "orbital_evals_per_s": NPOS * NORB / (ms / 1e3),
                              "hbm_frac": NPOS * vgh_bytes_per_position(NORB, es) / (ms / 1e3) / 1e9 / hbm}
    return out


def _l2_resident(oracle_ref=None):
    """Tables that stay in L2: 16^3 grid, 64 orbitals (19^3 x 64 padded, 1.76 MB FP32). FP32 V/VGL/VGH at
    1024 positions, and VGH at 16384 positions for FP32/FP16/BF16 tables. Each time is the mean of 50
    back-to-back launches on warm L2 (the table is meant to stay there), taken 5 times, median; the
    rate is the algorithmic bytes over that time, against the L2 read bandwidth the library's own
    probe measures on a 48 MB buffer. The 1024-position calls are also replayed from a CUDA graph
    (`_graph` lines), which leaves out the host's per-call cost."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    grid, N = (16, 16, 16), 64
    l2 = capi.bspline_measure_read_bandwidth(48 << 20, 20)
    dram = capi.bspline_measure_read_bandwidth(4 << 30, 5)
    coef = torch.from_numpy(inputs.uniform_coefs(grid, N, seed=1)).cuda()
    stream = torch.cuda.current_stream()
    out = {"workload": "grid16^3_N64 (L2-resident table)", "l2_read_gbs": l2, "dram_read_gbs_4GiB": dram}
    out_bytes = {capi.V: 4, capi.VGL: 20, capi.VGH: 40}

    def timed(t, kind, npos, seed):
        x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=seed))
        v, g, hl = t.outputs(kind, npos)
        for _ in range(3):
            t.eval(kind, x, y, z, v, g, hl)
        runs = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(50):
                t.eval(kind, x, y, z, v, g, hl)
            b.record(stream)
            b.synchronize()
            runs.append(a.elapsed_time(b) / 50)
        return statistics.median(runs)

    def graph_timed(t, kind, npos, seed):
        """Per-call device time of 50 calls captured in one CUDA graph (no host launch cost), median of 5."""
        x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=seed))
        v, g, hl = t.outputs(kind, npos)
        t.eval(kind, x, y, z, v, g, hl)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(50):
                t.eval(kind, x, y, z, v, g, hl)
        graph.replay()
        runs = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            graph.replay()
            b.record(stream)
            b.synchronize()
            runs.append(a.elapsed_time(b) / 50)
        return statistics.median(runs)

    def line(ms, kind, npos, esize):
        nbytes = npos * (64 * N * esize + out_bytes[kind] * N)
        return {"us": ms * 1e3, "orbital_evals_per_s": npos * N / (ms / 1e3),
                "l2_frac": nbytes / (ms / 1e3) / 1e9 / l2}

    def vgh_outputs(t, npos, seed):
        x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=seed))
        v, g, hl = t.outputs(capi.VGH, npos)
        t.eval(capi.VGH, x, y, z, v, g, hl)
        torch.cuda.synchronize()
        return {"v": v, "g": g, "h": hl}

    def vs_oracle(got):
        """max |table's output - FP64 oracle on the original coefficients| / max |oracle| per output kind."""
        if oracle_ref is None:
            return None
        return {k: float(np.abs(got[k].cpu().numpy().astype(np.float64) - oracle_ref[k]).max()
                         / np.abs(oracle_ref[k]).max()) for k in ("v", "g", "h")}

    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, coef)
        for kind, name in ((capi.V, "v"), (capi.VGL, "vgl"), (capi.VGH, "vgh")):
            out[f"fp32_{name}_1024pos"] = line(timed(t, kind, 1024, 2), kind, 1024, 4)
            # the same calls replayed from a CUDA graph: the device time without the per-call host cost
            out[f"fp32_{name}_1024pos_graph"] = line(graph_timed(t, kind, 1024, 2), kind, 1024, 4)
        ms32 = timed(t, capi.VGH, 16384, 5)
        ref = vgh_outputs(t, 16384, 5)
        out["fp32_vgh_16384pos"] = dict(line(ms32, capi.VGH, 16384, 4), rel_error_vs_oracle=vs_oracle(ref))
    for name, dt in (("fp16", capi.F16), ("bf16", capi.BF16)):
        with capi.Table(grid, N, dt) as t:
            capi.bspline_set_coefs(t.h, coef)
            ms = timed(t, capi.VGH, 16384, 5)
            got = vgh_outputs(t, 16384, 5)
            shape16 = capi.bspline_get_tuning(t.h, capi.VGH)
        # the table's quantisation error, seen through the outputs: max |16-bit - FP32| / max |FP32| per kind
        err = {k: float((got[k] - ref[k]).abs().max() / ref[k].abs().max()) for k in ref}
        out[f"{name}_vgh_16384pos"] = dict(line(ms, capi.VGH, 16384, 2), speedup_vs_fp32=ms32 / ms,
                                            launch_shape=shape16, rel_error_vs_fp32_table=err,
                                            rel_error_vs_oracle=vs_oracle(got))
    return out


def _graphite_shape(l2_gbs):
    """The grid and orbital count of the paper's graphite workload (48 x 48 x 60, N = 128) with a plane-wave
    FP32 table standing in for its orbitals (51 x 51 x 63 x 128 padded, 84 MB: it fits in L2), VGL and VGH
    at 4096 and 65536 positions, the library's default launch shape. Median of 10 launches on fresh
    positions; the rate is algorithmic bytes over time, against the L2 read bandwidth of the probe."""
    from paper_1611_02665_gb300 import capi, inputs

    grid, N = (48, 48, 60), 128
    coef = inputs.plane_wave_coefs(grid, N, seed=10, device="cuda")
    out = {"workload": "grid48x48x60_N128_planewave_fp32", "table_bytes": table_bytes(grid, N, 4)}
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, coef)
        for kind, name, ob in ((capi.VGL, "vgl", 20), (capi.VGH, "vgh", 40)):
            for npos in (4096, 65536):
                ms = _time_eval(t, kind, 10, npos, 9600 + npos % 7)
                nbytes = npos * (64 * N * 4 + ob * N)
                out[f"{name}_{npos}pos"] = {"us": ms * 1e3, "orbital_evals_per_s": npos * N / (ms / 1e3),
                                            "l2_frac": nbytes / (ms / 1e3) / 1e9 / l2_gbs}
        out["launch_shape"] = capi.bspline_get_tuning(t.h, capi.VGH)
    return out


def _n_sweep(l2_gbs):
    """FP32 VGH throughput against the orbital count at the paper's 48^3 grid (N = 128 ... 4096, the range
    of its throughput-versus-N measurements), 4096 positions per call, the library's default launch shape
    (cell-sorted when the table is larger than L2). The rate is algorithmic bytes over time, against HBM
    for tables larger than L2 and against the probe's L2 read bandwidth otherwise."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    hbm, _ = _peaks()
    l2_size = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    out = {"workload": "vgh_grid48^3_4096pos_planewave_fp32", "positions": NPOS}
    for N in (128, 256, 512, 1024, 2048, 4096):
        coef = inputs.plane_wave_coefs(GRID, N, seed=3, device="cuda")
        with capi.Table(GRID, N, capi.F32) as t:
            capi.bspline_set_coefs(t.h, coef)
            del coef
            ms = _time_eval(t, capi.VGH, 10, NPOS, 9700 + N)
            shape = capi.bspline_get_tuning(t.h, capi.VGH)
        tb = table_bytes(GRID, N, 4)
        rate = NPOS * vgh_bytes_per_position(N, 4) / (ms / 1e3) / 1e9
        ref = "l2" if tb <= l2_size else "hbm"
        out[f"N{N}"] = {"us": ms * 1e3, "orbital_evals_per_s": NPOS * N / (ms / 1e3), "table_bytes": tb,
                        "algorithmic_gbs": rate, f"{ref}_frac": rate / (l2_gbs if ref == "l2" else hbm),
                        "launch_shape": shape}
    return out


def _batched(args):
    """Five uneven tables, walkers with 1..8 positions each, VGL: one persistent launch (CUDA graph)
    against one launch per table."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    work = inputs.batched_workload(seed=9)
    tables, items = [], []
    units = 0
    bytes_alg = 0
    for k, w in enumerate(work):
        N, grid, npos = w["N"], w["grid"], w["npos"]
        t = capi.Table(grid, N, capi.F32)
        coef = inputs.uniform_coefs_device(grid, N, seed=300 + k)
        capi.bspline_set_coefs(t.h, coef)
        del coef
        x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=400 + k))
        v, g, l = t.outputs(capi.VGL, npos)
        items.append({"table": t.h, "npos": npos, "x": x, "y": y, "z": z, "v": v, "g": g, "hl": l, "ld": N})
        tables.append(t)
        units += npos * N
        bytes_alg += npos * (64 * N * 4 + 5 * N * 4)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    plan = capi.bspline_plan_create(items, capi.VGL)

    def timed(fn, reps=10):
        ms = []
        for r in range(reps + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if r >= 3:
                ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    stages = capi.bspline_plan_get_stages(plan)  # a new FP32 plan stages rows through the 4-unit ring
    ms_graph_input_order = timed(lambda: capi.bspline_plan_run_graph(plan, stream))
    capi.bspline_plan_set_order(plan, 1)
    ms_graph = timed(lambda: capi.bspline_plan_run_graph(plan, stream))
    ms_plan = timed(lambda: capi.bspline_plan_run(plan, stream))
    capi.bspline_plan_set_stages(plan, 0)
    ms_graph_registers = timed(lambda: capi.bspline_plan_run_graph(plan, stream))
    capi.bspline_plan_set_stages(plan, stages)

    def separate():
        for t, it in zip(tables, items):
            t.eval(capi.VGL, it["x"], it["y"], it["z"], it["v"], it["g"], it["hl"], it["ld"], stream)

    # five separate launches with the one-launch kernel's shapes: DIRECT, 512 orbitals, cell-sorted, rows
    # into registers and through the 4-unit ring
    for t in tables:
        capi.bspline_set_tuning(t.h, capi.VGL, 1, 512, 1, 0, 1)
    ms_sep = timed(separate)
    for t in tables:
        capi.bspline_set_tuning(t.h, capi.VGL, 1, 512, 1, 4, 1)
    ms_sep_staged = timed(separate)
    # the plan run one table at a time with each table's default shape, then the plan autotuner's pick
    for t in tables:
        capi.bspline_set_tuning(t.h, capi.VGL, 0, 0, 0, 0, 0)
    capi.bspline_plan_set_mode(plan, capi.PLAN_PER_TABLE)
    ms_per_table = timed(lambda: capi.bspline_plan_run_graph(plan, stream))
    mode, order = capi.bspline_plan_tune(plan, 5, stream)
    ms_tuned = timed(lambda: capi.bspline_plan_run_graph(plan, stream))
    tuned_stages = capi.bspline_plan_get_stages(plan)
    capi.bspline_plan_destroy(plan)
    for t in tables:
        t.close()
    hbm, _ = _peaks()
    return {"workload": "vgl_5tables_N256-4096_grid32-64_walkers64-2048x1-8pos_fp32",
            "positions": sum(w["npos"] for w in work), "orbital_evals": units,
            "graph_ms": ms_graph, "plan_ms": ms_plan, "graph_input_order_ms": ms_graph_input_order,
            "stages": stages, "graph_rows_in_registers_ms": ms_graph_registers,
            "separate_launches_ms": ms_sep, "separate_launches_staged_ms": ms_sep_staged,
            "order": "cell-sorted per table (plan_set_order 1)",
            "per_table_graph_ms": ms_per_table,
            "tuned": {"mode": ["one launch", "per table"][mode], "order": order,
                      "stages": tuned_stages, "graph_ms": ms_tuned,
                      "orbital_evals_per_s": units / (ms_tuned / 1e3)},
            "graph_orbital_evals_per_s": units / (ms_graph / 1e3),
            "graph_hbm_frac": bytes_alg / (ms_graph / 1e3) / 1e9 / hbm,
            "speedup_vs_separate": ms_sep / ms_graph}


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["bf16_tflops"]), float(p["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1900.0, 1700.0, "fallback"


def _surrogate(args):
    """Learned surrogate of a 64^3 x 512 plane-wave table (616 MB): trained on 2^22 spline samples,
    then V and VGL (forward mode) on 65536 held-out positions against the FP32 spline."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    grid, N = (64, 64, 64), 512
    coef = inputs.plane_wave_coefs(grid, N, seed=6, device="cuda")
    table = capi.Table(grid, N, capi.F32)
    capi.bspline_set_coefs(table.h, coef)
    del coef
    stream = torch.cuda.current_stream()
    ntrain, B = 1 << 22, 8192
    tx, ty, tz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(ntrain, seed=7))
    target = torch.empty((ntrain, N), device="cuda")
    for lo in range(0, ntrain, 1 << 16):
        sl = slice(lo, lo + (1 << 16))
        capi.bspline_eval_v(table.h, 1 << 16, tx[sl], ty[sl], tz[sl], target[sl], N, stream)
    P = 65536
    hx, hy, hz = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(P, seed=8))

    def timed(fn, reps=10):
        ms = []
        for r in range(reps + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            if r >= 3:
                ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    sv = torch.empty((P, N), device="cuda")
    sg = torch.empty((P, 3, N), device="cuda")
    sl_ = torch.empty((P, N), device="cuda")
    ms_spline_v = timed(lambda: capi.bspline_eval_v(table.h, P, hx, hy, hz, sv, N, stream))
    ms_spline_vgl = timed(lambda: capi.bspline_eval_vgl(table.h, P, hx, hy, hz, sv, sg, sl_, N, stream))
    capi.bspline_eval_v(table.h, P, hx, hy, hz, sv, N, stream)

    with capi.Surrogate(16, 512, 3, N) as s:
        capi.mlp_init(s.h, 12345)
        steps = args.mlp_epochs * (ntrain // B)
        loss = torch.zeros(1, device="cuda")
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for step in range(steps):
            lo = (step * B) % ntrain
            lr = args.mlp_lr * 0.5 * (1 + np.cos(np.pi * step / steps)) + 1e-5
            capi.mlp_train_step(s.h, B, tx[lo:lo + B], ty[lo:lo + B], tz[lo:lo + B], target[lo:lo + B], N, lr,
                                loss, stream)
        t1.record(stream)
        t1.synchronize()
        train_ms = t0.elapsed_time(t1)
        final_loss = loss.item()
        mv = torch.empty((P, N), device="cuda")
        mg = torch.empty((P, 3, N), device="cuda")
        ml = torch.empty((P, N), device="cuda")
        ms_mlp_v = timed(lambda: capi.mlp_eval_v(s.h, P, hx, hy, hz, mv, N, stream))
        ms_mlp_vgl = timed(lambda: capi.mlp_eval_vgl(s.h, P, hx, hy, hz, mv, mg, ml, N, stream))
        capi.mlp_eval_vgl(s.h, P, hx, hy, hz, mv, mg, ml, N, stream)
        fl_train = capi.mlp_flops(s.h, 2, B)
        fl_v = capi.mlp_flops(s.h, 0, P)
        fl_vgl = capi.mlp_flops(s.h, 1, P)
        nparams = capi.mlp_param_count(s.h)
    capi.bspline_eval_vgl(table.h, P, hx, hy, hz, sv, sg, sl_, N, stream)
    torch.cuda.synchronize()

    def rel_rms(a, b):
        return float(torch.sqrt(((a - b) ** 2).mean()) / torch.sqrt((b ** 2).mean()))

    err_v = rel_rms(mv, sv)
    err_vgl = {"v": rel_rms(mv, sv), "g": rel_rms(mg, sg), "l": rel_rms(ml, sl_)}

    # The same network trained on values AND gradients (mlp_train_step_vg): the spline's VGL gradients as
    # targets, lambda puts both terms of the loss on one scale, 4 rows per position (batch 4096 positions =
    # 16384 rows per step).
    del target
    tv = torch.empty((ntrain, N), device="cuda")
    tg = torch.empty((ntrain, 3, N), device="cuda")
    tl = torch.empty((1 << 16, N), device="cuda")
    for lo in range(0, ntrain, 1 << 16):
        sl = slice(lo, lo + (1 << 16))
        capi.bspline_eval_vgl(table.h, 1 << 16, tx[sl], ty[sl], tz[sl], tv[sl], tg[sl], tl, N, stream)
    lam = float((tv[:65536] ** 2).mean() / (tg[:65536] ** 2).mean())
    Bv = 4096
    with capi.Surrogate(16, 512, 3, N) as s:
        capi.mlp_init(s.h, 12345)
        steps_vg = args.mlp_vg_epochs * (ntrain // Bv)
        loss = torch.zeros(1, device="cuda")
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for step in range(steps_vg):
            lo = (step * Bv) % ntrain
            sl = slice(lo, lo + Bv)
            lr = args.mlp_lr * 0.5 * (1 + np.cos(np.pi * step / steps_vg)) + 1e-5
            capi.mlp_train_step_vg(s.h, Bv, tx[sl], ty[sl], tz[sl], tv[sl], tg[sl], N, lam, lr, loss, stream)
        t1.record(stream)
        t1.synchronize()
        vg_train_ms = t0.elapsed_time(t1)
        vg_loss = loss.item()
        capi.mlp_eval_vgl(s.h, P, hx, hy, hz, mv, mg, ml, N, stream)
        torch.cuda.synchronize()
        fl_train_vg = capi.mlp_flops(s.h, 3, Bv)
    del tv, tg
    table.close()
    tf_train_vg = fl_train_vg * steps_vg / (vg_train_ms / 1e3) / 1e12

    peak, peak_sus, src = _bf16_peak()
    tf_v = fl_v / (ms_mlp_v / 1e3) / 1e12
    tf_vgl = fl_vgl / (ms_mlp_vgl / 1e3) / 1e12
    tf_train = fl_train * steps / (train_ms / 1e3) / 1e12
    return {
        "workload": "surrogate_grid64^3_N512_planewave; MLP 96 features -> 3x512 SiLU -> 512, bf16",
        "train": {"samples": ntrain, "epochs": args.mlp_epochs, "lr": args.mlp_lr, "batch": B, "steps": steps,
                  "ms": train_ms,
                  "samples_per_s": steps * B / (train_ms / 1e3), "tflops": tf_train, "final_loss": final_loss},
        "positions": P,
        "v": {"mlp_ms": ms_mlp_v, "spline_fp32_ms": ms_spline_v, "speedup_vs_fp32_spline": ms_spline_v / ms_mlp_v,
              "rel_rms_err_vs_spline": err_v, "tflops": tf_v, "tensor_frac_of_burst_peak": tf_v / peak},
        "vgl": {"mlp_ms": ms_mlp_vgl, "spline_fp32_ms": ms_spline_vgl,
                "speedup_vs_fp32_spline": ms_spline_vgl / ms_mlp_vgl,
                "rel_rms_err_vs_spline": err_vgl,
                "tflops": tf_vgl, "tensor_frac_of_burst_peak": tf_vgl / peak},
        "train_tensor_frac_of_sustained_peak": tf_train / peak_sus,
        "trained_on_values_and_gradients": {
            "samples": ntrain, "epochs": args.mlp_vg_epochs, "batch_positions": Bv, "rows_per_step": 4 * Bv,
            "lr": args.mlp_lr, "lambda": lam, "steps": steps_vg, "ms": vg_train_ms, "final_loss": vg_loss,
            "samples_per_s": steps_vg * Bv / (vg_train_ms / 1e3), "tflops": tf_train_vg,
            "tensor_frac_of_sustained_peak": tf_train_vg / peak_sus,
            "vgl_rel_rms_err_vs_spline": {"v": rel_rms(mv, sv), "g": rel_rms(mg, sg), "l": rel_rms(ml, sl_)}},
        "bf16_peak_tflops": {"burst": peak, "sustained": peak_sus, "source": src},
        "memory_bytes": {"spline_table": table_bytes(grid, N, 4), "mlp_bf16_weights": 2 * nparams,
                         "mlp_fp32_master": 4 * nparams},
    }


# ---------------------------------------------------------------------------
# --profile-case: small, self-contained launch sequences for one kernel family under ncu. Each case builds
# its seeded synthetic inputs, runs --case-reps launches of the path and exits; nothing is timed or printed
# (the timings come from the benchmark itself).
# ---------------------------------------------------------------------------
_DTYPES = {"f32": 0, "f16": 1, "bf16": 2}
_KINDS = {"v": 0, "vgl": 1, "vgh": 2}


def _case_shape(a):
    return tuple(int(v) for v in a.case_shape.split(",")) if a.case_shape else None


def _case_eval(a):
    """One table (--case-grid, --case-n; the 48^3 x 2048 plane-wave table by default, or a uniform table of
    the given shape) evaluated --case-reps times on fresh positions (seeds 100 + rep)."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    grid = tuple(int(v) for v in a.case_grid.split(","))
    N = a.case_n
    t = capi.Table(grid, N, _DTYPES[a.case_dtype])
    if a.case_coefs == "planewave":
        coef = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    else:
        coef = torch.from_numpy(inputs.uniform_coefs(grid, N, seed=1)).cuda()
    capi.bspline_set_coefs(t.h, coef)
    kind = _KINDS[a.case_kind]
    shape = _case_shape(a)
    if shape:
        capi.bspline_set_tuning(t.h, kind, *shape)
    if a.case_lattice == "hex":
        capi.bspline_set_lattice(t.h, np.asarray(LATTICE_HEX))
    v, g, h = t.outputs(kind, a.case_npos)
    for r in range(a.case_reps):
        u = inputs.uniform_positions(a.case_npos, seed=100 + r)
        if a.case_lattice == "hex":  # Cartesian positions r = u L
            rr = np.stack(u, axis=1) @ np.asarray(LATTICE_HEX)
            u = [np.ascontiguousarray(rr[:, d]) for d in range(3)]
        x, y, z = (torch.from_numpy(c).cuda() for c in u)
        t.eval(kind, x, y, z, v, g, h)
    torch.cuda.synchronize()
    t.close()


def _case_ratio(a):
    """The fused determinant-ratio sums (bspline_eval_ratio) on the --case-grid x --case-n table, --case-kind,
    --case-reps calls on fresh positions (seeds 100 + rep), one row of seeded inverse entries per position."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    grid = tuple(int(v) for v in a.case_grid.split(","))
    N = a.case_n
    t = capi.Table(grid, N, _DTYPES[a.case_dtype])
    if a.case_coefs == "planewave":
        coef = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    else:
        coef = torch.from_numpy(inputs.uniform_coefs(grid, N, seed=1)).cuda()
    capi.bspline_set_coefs(t.h, coef)
    kind = _KINDS[a.case_kind]
    shape = _case_shape(a)
    if shape:
        capi.bspline_set_tuning(t.h, kind, *shape)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    u = torch.randn((a.case_npos, N), generator=gen, device="cuda") / N ** 0.5
    r = torch.empty((a.case_npos, capi.NCOMP[kind]), device="cuda")
    for rep in range(a.case_reps):
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(a.case_npos, seed=100 + rep))
        capi.bspline_eval_ratio(t.h, kind, a.case_npos, x, y, z, u, N, r)
    torch.cuda.synchronize()
    t.close()


def _case_batched(a):
    """The five-table VGL batch of the benchmark (or its first --case-tables tables): one plan run as a CUDA
    graph per rep (plan mode --case-plan-mode, order --case-order, staging depth --case-stages, -1 for the
    plan's default), or (--case-separate) one evaluation per table."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    work = inputs.batched_workload(seed=9)[:a.case_tables]
    tables, items = [], []
    for k, w in enumerate(work):
        t = capi.Table(w["grid"], w["N"], capi.F32)
        capi.bspline_set_coefs(t.h, inputs.uniform_coefs_device(w["grid"], w["N"], seed=300 + k))
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(w["npos"], seed=400 + k))
        v, g, l = t.outputs(capi.VGL, w["npos"])
        items.append({"table": t.h, "npos": w["npos"], "x": x, "y": y, "z": z, "v": v, "g": g, "hl": l,
                      "ld": w["N"]})
        tables.append(t)
    if a.case_separate:
        for t in tables:
            capi.bspline_set_tuning(t.h, capi.VGL, 1, 512, 1, 0, a.case_order)
        for _ in range(a.case_reps):
            for t, it in zip(tables, items):
                t.eval(capi.VGL, it["x"], it["y"], it["z"], it["v"], it["g"], it["hl"], it["ld"])
    else:
        plan = capi.bspline_plan_create(items, capi.VGL)
        capi.bspline_plan_set_order(plan, a.case_order)
        capi.bspline_plan_set_mode(plan, a.case_plan_mode)
        if a.case_stages >= 0:
            capi.bspline_plan_set_stages(plan, a.case_stages)
        for _ in range(a.case_reps):
            capi.bspline_plan_run_graph(plan)
        torch.cuda.synchronize()
        capi.bspline_plan_destroy(plan)
    torch.cuda.synchronize()
    for t in tables:
        t.close()


def _case_set_values(a):
    """Coefficients from grid samples (the interpolation solve) for the 48^3 x 2048 table, --case-reps times."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    grid, N = (48, 48, 48), 2048
    samples = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    with capi.Table(grid, N, _DTYPES[a.case_dtype]) as t:
        for _ in range(a.case_reps):
            capi.bspline_set_values(t.h, samples)
    torch.cuda.synchronize()


def _case_mlp(a):
    """The surrogate's inference (mlp_v, mlp_vgl) or training step (mlp_train), --case-reps times."""
    import torch

    from paper_1611_02665_gb300 import capi, inputs

    s = capi.Surrogate(16, 512, 3, 512)
    capi.mlp_init(s.h, 1)
    capi.mlp_set_gemm_kernel(s.h, a.case_gemm_kernel)
    if a.profile_case == "mlp_train":
        B = a.case_batch
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(B, seed=6))
        tgt = torch.rand((B, 512), device="cuda")
        for _ in range(a.case_reps):
            capi.mlp_train_step(s.h, B, x, y, z, tgt, 512, 1e-4)
    else:
        P = a.case_npos
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(P, seed=5))
        v = torch.empty((P, 512), device="cuda")
        g = torch.empty((P, 3, 512), device="cuda")
        l = torch.empty((P, 512), device="cuda")
        for _ in range(a.case_reps):
            if a.profile_case == "mlp_v":
                capi.mlp_eval_v(s.h, P, x, y, z, v, 512)
            else:
                capi.mlp_eval_vgl(s.h, P, x, y, z, v, g, l, 512)
    torch.cuda.synchronize()
    s.close()


def profile_case(a):
    import torch

    torch.cuda.set_device(0)
    if not a.case_npos:
        a.case_npos = {"mlp_v": 65536, "mlp_vgl": 16384}.get(a.profile_case, 4096)
    {"eval": _case_eval, "ratio": _case_ratio, "batched": _case_batched, "set_values": _case_set_values,
     "mlp_v": _case_mlp, "mlp_vgl": _case_mlp, "mlp_train": _case_mlp}[a.profile_case](a)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    # default launch shape: DIRECT, 512 orbitals per CTA, 1 position per CTA, cell-sorted positions
    ap.add_argument("--variant", type=int, default=1)
    ap.add_argument("--nb", type=int, default=512)
    ap.add_argument("--ppc", type=int, default=1)
    ap.add_argument("--stages", type=int, default=4)
    ap.add_argument("--order", type=int, default=1)
    ap.add_argument("--cpu-sample", type=int, default=16384)
    ap.add_argument("--ref-sample", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--mlp-epochs", type=int, default=32)
    ap.add_argument("--mlp-lr", type=float, default=6e-3)
    ap.add_argument("--mlp-vg-epochs", type=int, default=16)
    ap.add_argument("--tune", action="store_true", help="autotune the launch shape before timing")
    ap.add_argument("--record-traffic", metavar="NCU_RAW_CSV",
                    help="write the DRAM bytes of one captured launch of the headline kernel (an ncu raw-page "
                         "CSV export) into profiles/traffic.txt for the launch shape given by --variant etc.")
    ap.add_argument("--traffic-summary", default="", help="the profiles/ summary the --record-traffic figure is from")
    # profiling cases (see profile_case); nothing is timed
    ap.add_argument("--profile-case", choices=["eval", "ratio", "batched", "set_values", "mlp_v", "mlp_vgl",
                                               "mlp_train"])
    ap.add_argument("--case-grid", default="48,48,48")
    ap.add_argument("--case-n", type=int, default=2048)
    ap.add_argument("--case-coefs", choices=["planewave", "uniform"], default="planewave")
    ap.add_argument("--case-kind", choices=sorted(_KINDS), default="vgh")
    ap.add_argument("--case-dtype", choices=sorted(_DTYPES), default="f32")
    ap.add_argument("--case-shape", default="", help="variant,nb,ppc,stages,order (empty: the library default)")
    ap.add_argument("--case-npos", type=int, default=0)
    ap.add_argument("--case-lattice", choices=["none", "hex"], default="none",
                    help="eval case: the hexagonal cell of the lattice extra (Cartesian positions)")
    ap.add_argument("--case-batch", type=int, default=8192)
    ap.add_argument("--case-reps", type=int, default=3)
    ap.add_argument("--case-order", type=int, default=0)
    ap.add_argument("--case-plan-mode", type=int, default=0)
    ap.add_argument("--case-stages", type=int, default=-1)
    ap.add_argument("--case-tables", type=int, default=5)
    ap.add_argument("--case-separate", action="store_true")
    ap.add_argument("--case-gemm-kernel", type=int, default=0,
                    help="surrogate GEMM kernel (mlp_set_gemm_kernel): 0 default, 1 one CTA per tile, 2 CTA pairs")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args)
        return
    if args.record_traffic:
        tuning = dict(zip(("variant", "nb", "ppc", "stages", "order"),
                          (args.variant, args.nb, args.ppc, args.stages, args.order)))
        record_traffic(args.record_traffic, tuning, args.traffic_summary)
        return
    args.warmup = max(3, args.warmup)  # the timing rules want at least 3 untimed steps
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
