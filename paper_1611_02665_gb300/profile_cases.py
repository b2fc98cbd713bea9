"""Small, self-contained launch sequences for profiling one kernel family under ncu.

    python -m paper_1611_02665_gb300.profile_cases vgh [--variant 1 --nb 512 --kind vgh]
    python -m paper_1611_02665_gb300.profile_cases batched [--order 1] [--separate]
    python -m paper_1611_02665_gb300.profile_cases mlp_v [--npos 65536]
    python -m paper_1611_02665_gb300.profile_cases mlp_vgl [--npos 16384]
    python -m paper_1611_02665_gb300.profile_cases mlp_train [--batch 8192]
    python -m paper_1611_02665_gb300.profile_cases set_values [--dtype f32]

Each case builds its inputs (seeded, synthetic), runs `--reps` launches of the
path and exits; nothing is timed here (use bench.py for timings).
"""
from __future__ import annotations

import argparse

import torch

from . import capi, inputs


def vgh(a):
    grid, N = (48, 48, 48), 2048
    t = capi.Table(grid, N, {"f32": capi.F32, "f16": capi.F16, "bf16": capi.BF16}[a.dtype])
    capi.bspline_set_coefs(t.h, inputs.plane_wave_coefs(grid, N, seed=3, device="cuda"))
    kind = {"v": capi.V, "vgl": capi.VGL, "vgh": capi.VGH}[a.kind]
    if a.variant:
        capi.bspline_set_tuning(t.h, kind, a.variant, a.nb, a.ppc, a.stages, a.order)
    v, g, h = t.outputs(kind, a.npos)
    for r in range(a.reps):
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(a.npos, seed=100 + r))
        t.eval(kind, x, y, z, v, g, h)
    torch.cuda.synchronize()
    t.close()


def batched(a):
    """The five-table VGL batch of the benchmark: one plan run as a CUDA graph per rep, or (--separate)
    one evaluation per table."""
    work = inputs.batched_workload(seed=9)
    tables, items = [], []
    for k, w in enumerate(work):
        t = capi.Table(w["grid"], w["N"], capi.F32)
        capi.bspline_set_coefs(t.h, inputs.uniform_coefs_device(w["grid"], w["N"], seed=300 + k))
        x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(w["npos"], seed=400 + k))
        v, g, l = t.outputs(capi.VGL, w["npos"])
        items.append({"table": t.h, "npos": w["npos"], "x": x, "y": y, "z": z, "v": v, "g": g, "hl": l,
                      "ld": w["N"]})
        tables.append(t)
    if a.separate:
        for t in tables:
            capi.bspline_set_tuning(t.h, capi.VGL, 1, 512, 1, 0, a.order)
        for _ in range(a.reps):
            for t, it in zip(tables, items):
                t.eval(capi.VGL, it["x"], it["y"], it["z"], it["v"], it["g"], it["hl"], it["ld"])
    else:
        plan = capi.bspline_plan_create(items, capi.VGL)
        capi.bspline_plan_set_order(plan, a.order)
        for _ in range(a.reps):
            capi.bspline_plan_run_graph(plan)
        torch.cuda.synchronize()
        capi.bspline_plan_destroy(plan)
    torch.cuda.synchronize()
    for t in tables:
        t.close()


def set_values(a):
    """Coefficients from grid samples (the interpolation solve) for the 48^3 x 2048 table, --reps times."""
    grid, N = (48, 48, 48), 2048
    samples = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    with capi.Table(grid, N, {"f32": capi.F32, "f16": capi.F16, "bf16": capi.BF16}[a.dtype]) as t:
        for _ in range(a.reps):
            capi.bspline_set_values(t.h, samples)
    torch.cuda.synchronize()


def _mlp(a):
    s = capi.Surrogate(16, 512, 3, 512)
    capi.mlp_init(s.h, 1)
    return s


def mlp_v(a):
    s = _mlp(a)
    x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(a.npos, seed=5))
    v = torch.empty((a.npos, 512), device="cuda")
    for _ in range(a.reps):
        capi.mlp_eval_v(s.h, a.npos, x, y, z, v, 512)
    torch.cuda.synchronize()
    s.close()


def mlp_vgl(a):
    s = _mlp(a)
    x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(a.npos, seed=5))
    v = torch.empty((a.npos, 512), device="cuda")
    g = torch.empty((a.npos, 3, 512), device="cuda")
    l = torch.empty((a.npos, 512), device="cuda")
    for _ in range(a.reps):
        capi.mlp_eval_vgl(s.h, a.npos, x, y, z, v, g, l, 512)
    torch.cuda.synchronize()
    s.close()


def mlp_train(a):
    s = _mlp(a)
    x, y, z = (torch.from_numpy(c).cuda() for c in inputs.uniform_positions(a.batch, seed=6))
    tgt = torch.rand((a.batch, 512), device="cuda")
    for _ in range(a.reps):
        capi.mlp_train_step(s.h, a.batch, x, y, z, tgt, 512, 1e-4)
    torch.cuda.synchronize()
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["vgh", "batched", "set_values", "mlp_v", "mlp_vgl", "mlp_train"])
    ap.add_argument("--npos", type=int, default=0)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--ppc", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--order", type=int, default=0)
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--kind", choices=["v", "vgl", "vgh"], default="vgh")
    ap.add_argument("--separate", action="store_true")
    a = ap.parse_args()
    if not a.npos:
        a.npos = {"vgh": 4096, "mlp_v": 65536, "mlp_vgl": 16384}.get(a.case, 4096)
    torch.cuda.set_device(0)
    globals()[a.case](a)


if __name__ == "__main__":
    main()
