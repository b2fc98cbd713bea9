"""GPU parity at the sizes the benchmark times, on samples the oracle evaluates one by one.

* The five-table batch as the benchmark builds it (N = 256 ... 4096 on 32^3 ... 64^3 grids, walkers of
  1..8 positions, VGL; the largest table 67^3 x 4096 floats = 4.93 GB, so row offsets pass 2^32 bytes),
  through every way a batch runs: one launch in input and cell-sorted order, the plan's CUDA graph in
  both plan modes, the plan autotuner's pick and the one-call convenience entry point.
* Single tables above 4 GiB: 64^3 x 4096 FP32 (4.93 GB) on the default shape, registers-only DIRECT and
  TMA; 80^3 x 4096 FP16 and BF16 (4.68 GB) on the tensor-core variant and DIRECT; and 48^3 x 4096
  16-bit tables on the tensor-core variant.

Orbitals are independent (Eq. (TricubicValue) holds per orbital) and so are positions, so the FP64 oracle
checks a seeded sample of positions and of orbitals (some in every block of 512, plus the first and the
last) against the same entries of the full outputs; the rest are checked to be finite. The sampled
positions include a few in the far corner of the cell, whose stencil rows sit at the end of the table.
Paper: the walker-level parallelism of Sec. "Baseline and miniQMC" over one shared read-only table.
"""
import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import capi, inputs
from parity_util import assert_parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DIRECT, TMA, MMA = capi.VARIANT_DIRECT, capi.VARIANT_TMA, capi.VARIANT_MMA


def _orbital_sample(N, rng, per_block=3):
    """A few orbitals from every block of 512, plus the first and the last."""
    cols = {0, N - 1}
    for b0 in range(0, N, 512):
        b1 = min(N, b0 + 512)
        cols.update(int(c) for c in rng.choice(np.arange(b0, b1), size=min(per_block, b1 - b0), replace=False))
    return np.array(sorted(cols))


def _position_sample(npos, rng, count=12):
    s = set(int(p) for p in rng.choice(npos, size=min(count, npos), replace=False))
    s.add(npos - 1)
    return np.array(sorted(s))


def _corner_positions(npos, seed, ncorner=4):
    """Uniform positions whose first `ncorner` entries lie in the far corner of the cell."""
    x, y, z = inputs.uniform_positions(npos, seed=seed)
    c = np.random.default_rng(seed + 1).uniform(0.985, 0.9999, size=(3, min(ncorner, npos)))
    for a, cc in zip((x, y, z), c):
        a[:cc.shape[0]] = cc
    return x, y, z


def _ref_table(coef_cols, dtype):
    """Oracle table of the sampled orbitals: the coefficients in FP64, or for a 16-bit table the dequantised
    codes (the per-orbital scale depends on that orbital's column alone, so quantising the sampled columns
    gives the codes the whole table holds)."""
    if dtype == capi.F32:
        return coef_cols.astype(np.float64)
    codes, scale = oracle.quantize(coef_cols, dtype)
    return oracle.dequantize(codes, scale, dtype)


def _gather(kind, outs, rows, cols):
    v, g, hl = outs
    r = torch.as_tensor(rows, device=v.device)
    c = torch.as_tensor(cols, device=v.device)
    got = {"v": v[r][:, c].cpu().numpy()}
    if kind != capi.V:
        got["g"] = g[r][:, :, c].cpu().numpy()
    if kind == capi.VGL:
        got["l"] = hl[r][:, c].cpu().numpy()
    if kind == capi.VGH:
        got["h"] = hl[r][:, :, c].cpu().numpy()
    return got


def _all_finite(outs):
    return all(bool(torch.isfinite(o).all()) for o in outs if o is not None)


# ---------------------------------------------------------------------------
# the five-table batch
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batch5():
    kind = capi.VGL
    work = inputs.batched_workload(seed=9)
    rng = np.random.default_rng(31)
    tables, items, refs, samples = [], [], [], []
    for k, w in enumerate(work):
        N, grid, npos = w["N"], w["grid"], w["npos"]
        t = capi.Table(grid, N, capi.F32)
        coef = inputs.uniform_coefs_device(grid, N, seed=300 + k)
        capi.bspline_set_coefs(t.h, coef)
        cols = _orbital_sample(N, rng)
        coef_cols = coef[..., torch.as_tensor(cols, device="cuda")].cpu().numpy()
        del coef
        x, y, z = _corner_positions(npos, seed=400 + k)
        rows = np.unique(np.concatenate([np.arange(4), _position_sample(npos, rng)]))
        refs.append(oracle.eval_periodic(kind, _ref_table(coef_cols, capi.F32), x[rows], y[rows], z[rows]))
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        v, g, l = t.outputs(kind, npos)
        items.append({"table": t.h, "npos": npos, "x": dx, "y": dy, "z": dz, "v": v, "g": g, "hl": l, "ld": N})
        samples.append((rows, cols))
        tables.append(t)
    torch.cuda.synchronize()
    assert max(capi.bspline_get_info(t.h).table_bytes for t in tables) > 4 << 30
    yield kind, tables, items, refs, samples
    for t in tables:
        t.close()


def _clear(items):
    for it in items:
        for key in ("v", "g", "hl"):
            if it.get(key) is not None:
                it[key].fill_(float("nan"))


def _check_batch(kind, items, refs, samples, label):
    torch.cuda.synchronize()
    for k, (it, ref, (rows, cols)) in enumerate(zip(items, refs, samples)):
        outs = (it["v"], it["g"], it["hl"])
        assert _all_finite(outs), f"{label}: item {k} has non-finite outputs"
        assert_parity(_gather(kind, outs, rows, cols), ref, kind, label=f"{label}, item {k} (N {it['ld']})")
        assert capi.bspline_device_status(it["table"]) == 0


def test_batch5_every_execution(batch5):
    kind, tables, items, refs, samples = batch5
    plan = capi.bspline_plan_create(items, kind)
    try:
        for order in (0, 1):
            capi.bspline_plan_set_order(plan, order)
            _clear(items)
            capi.bspline_plan_run(plan)
            _check_batch(kind, items, refs, samples, f"one launch, order {order}")
            for rep in range(2):  # captured once, then replayed
                _clear(items)
                capi.bspline_plan_run_graph(plan)
                _check_batch(kind, items, refs, samples, f"one-launch graph, order {order}, replay {rep}")
        capi.bspline_plan_set_mode(plan, capi.PLAN_PER_TABLE)
        _clear(items)
        capi.bspline_plan_run(plan)
        _check_batch(kind, items, refs, samples, "per table")
        for rep in range(2):
            _clear(items)
            capi.bspline_plan_run_graph(plan)
            _check_batch(kind, items, refs, samples, f"per-table graph, replay {rep}")
        mode, order = capi.bspline_plan_tune(plan, reps=2)
        _clear(items)
        capi.bspline_plan_run_graph(plan)
        _check_batch(kind, items, refs, samples, f"tuned plan (mode {mode}, order {order})")
    finally:
        capi.bspline_plan_destroy(plan)
    _clear(items)
    capi.bspline_eval_batched(items, kind)
    _check_batch(kind, items, refs, samples, "bspline_eval_batched")


# ---------------------------------------------------------------------------
# single tables above 4 GiB
# ---------------------------------------------------------------------------
def _single_table_case(grid, N, dtype, npos, seed, shapes, kinds):
    rng = np.random.default_rng(seed)
    coef = inputs.uniform_coefs_device(grid, N, seed=seed)
    cols = _orbital_sample(N, rng)
    coef_cols = coef[..., torch.as_tensor(cols, device="cuda")].cpu().numpy()
    x, y, z = _corner_positions(npos, seed=seed + 7)
    rows = np.unique(np.concatenate([np.arange(4), _position_sample(npos, rng, count=20)]))
    ref_tab = _ref_table(coef_cols, dtype)
    dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, coef)
        del coef
        torch.cuda.synchronize()
        info = capi.bspline_get_info(t.h)
        for kind in kinds:
            ref = oracle.eval_periodic(kind, ref_tab, x[rows], y[rows], z[rows])
            outs = t.outputs(kind, npos)
            for shape in shapes:
                capi.bspline_set_tuning(t.h, kind, *(shape or (capi.VARIANT_AUTO,)))
                for o in outs:
                    if o is not None:
                        o.fill_(float("nan"))
                t.eval(kind, dx, dy, dz, *outs)
                torch.cuda.synchronize()
                assert capi.bspline_device_status(t.h) == 0
                assert _all_finite(outs), f"shape {shape} kind {kind}: non-finite outputs"
                errs = assert_parity(_gather(kind, outs, rows, cols), ref, kind,
                                     label=f"{grid} x {N} dtype {dtype} kind {kind} shape {shape}")
                print(f"{grid} x {N} dtype {dtype} kind {kind} shape {shape}: {errs}")
            del outs
    return info


@pytest.mark.parametrize("kind", [capi.V, capi.VGH])
def test_fp32_table_above_4GiB(kind):
    """64^3 x 4096 FP32 (67^3 x 4096 x 4 B = 4.93 GB): the default shape (rows staged through shared
    memory for VGH, cell-sorted), DIRECT with loads into registers in both orders, and TMA boxes."""
    shapes = [None, (DIRECT, 512, 1, 0, 0), (DIRECT, 512, 1, 0, 1), (TMA, 256, 1, 3, 1)]
    info = _single_table_case((64, 64, 64), 4096, capi.F32, 4096, 5100 + kind, shapes, [kind])
    assert info.table_bytes > 4 << 30


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
def test_16bit_table_above_4GiB(dtype):
    """80^3 x 4096 16-bit (83^3 x 4096 x 2 B = 4.68 GB): VGH and VGL on the tensor-core variant (the
    default for rows of 512 orbitals and more) and on DIRECT, V on its default (DIRECT)."""
    shapes = [None, (DIRECT, 512, 1, 0, 1)]
    info = _single_table_case((80, 80, 80), 4096, dtype, 2048, 5200 + dtype, shapes,
                              [capi.V, capi.VGL, capi.VGH])
    assert info.table_bytes > 4 << 30


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
def test_16bit_tensor_core_48cubed_N4096(dtype):
    """48^3 x 4096 16-bit tables (1.09 GB) on the tensor-core variant, VGH at 4096 positions, in both
    position orders: the default (two 128-orbital blocks per unit) and single-block units."""
    shapes = [None, (MMA, 256, 2, 0, 0), (MMA, 128, 2, 0, 1), (MMA, 128, 1, 0, 1)]
    _single_table_case((48, 48, 48), 4096, dtype, 4096, 5300 + dtype, shapes, [capi.VGH])
