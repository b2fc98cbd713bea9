"""GPU parity of the batched launch across walkers and tables.

Several tables of uneven grid and orbital count, each with walkers holding
1..8 positions (the paper's walker-level parallelism, Sec. "Baseline and
miniQMC"), evaluated in one launch, replayed from a CUDA graph, and through
the one-call convenience entry point; checked against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import capi, inputs
from parity_util import assert_parity, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SPECS = [((8, 8, 8), 64), ((10, 9, 7), 100), ((12, 12, 12), 512), ((5, 5, 5), 1), ((6, 7, 6), 700)]


def _ref_table(coef, dtype):
    if dtype == capi.F32:
        return coef.astype(np.float64)
    codes, scale = oracle.quantize(coef, dtype)
    return oracle.dequantize(codes, scale, dtype)


def _build(dtype, kind, seed=0, ld_pad=0, empty_item=False):
    rng = np.random.default_rng(seed)
    tables, items, refs, outs = [], [], [], []
    for k, (grid, N) in enumerate(SPECS):
        coef = inputs.uniform_coefs(grid, N, seed=100 + k)
        t = capi.Table(grid, N, dtype)
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        nw = int(rng.integers(3, 40))
        npos = int(rng.integers(1, 9, size=nw).sum())
        if empty_item and k == 1:
            npos = 0
        x, y, z = inputs.uniform_positions(max(npos, 1), seed=200 + k)
        x, y, z = x[:npos], y[:npos], z[:npos]
        ld = N + ld_pad
        dx, dy, dz = to_device(x, y, z)
        v, g, hl = t.outputs(kind, npos, ld)
        items.append({"table": t.h, "npos": npos, "x": dx, "y": dy, "z": dz, "v": v, "g": g, "hl": hl, "ld": ld})
        refs.append(oracle.eval_periodic(kind, _ref_table(coef, dtype), x, y, z) if npos else None)
        outs.append((v, g, hl, N))
        tables.append(t)
    return tables, items, refs, outs


def _check(kind, refs, outs, label):
    for ref, (v, g, hl, N) in zip(refs, outs):
        if ref is None:
            continue
        got = {"v": v.cpu().numpy()[:, :N]}
        if kind >= 1:
            got["g"] = g.cpu().numpy()[:, :, :N]
        if kind == 1:
            got["l"] = hl.cpu().numpy()[:, :N]
        if kind == 2:
            got["h"] = hl.cpu().numpy()[:, :, :N]
        assert_parity(got, ref, kind, label=label)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
def test_plan_run_and_graph(kind, dtype, order):
    tables, items, refs, outs = _build(dtype, kind, seed=kind * 7 + dtype)
    plan = capi.bspline_plan_create(items, kind)
    capi.bspline_plan_set_order(plan, order)
    try:
        capi.bspline_plan_run(plan)
        torch.cuda.synchronize()
        _check(kind, refs, outs, "plan_run")
        first = [o[0].clone() for o in outs]
        for o in outs:
            o[0].zero_()
        for _ in range(3):  # graph captured once, replayed
            capi.bspline_plan_run_graph(plan)
        torch.cuda.synchronize()
        _check(kind, refs, outs, "graph")
        for a, o in zip(first, outs):
            assert torch.equal(a, o[0])
    finally:
        capi.bspline_plan_destroy(plan)
        for t in tables:
            t.close()


def test_eval_batched_ragged_ld_and_empty_item():
    kind = capi.VGL
    tables, items, refs, outs = _build(capi.F32, kind, seed=3, ld_pad=3, empty_item=True)
    capi.bspline_eval_batched(items, kind)
    _check(kind, refs, outs, "eval_batched")
    for t in tables:
        t.close()


def test_batched_matches_single_table_direct():
    kind = capi.VGH
    tables, items, refs, outs = _build(capi.F32, kind, seed=5)
    capi.bspline_eval_batched(items, kind)
    for t, it, (v, g, hl, N) in zip(tables, items, outs):
        capi.bspline_set_tuning(t.h, kind, capi.VARIANT_DIRECT, 512, 1, 0)
        v2, g2, h2 = t.outputs(kind, it["npos"], it["ld"])
        t.eval(kind, it["x"], it["y"], it["z"], v2, g2, h2)
        torch.cuda.synchronize()
        # same arithmetic in the same order: identical results
        assert torch.equal(v, v2) and torch.equal(g, g2) and torch.equal(hl, h2)
    for t in tables:
        t.close()


def test_order_switch_recaptures_graph():
    kind = capi.VGL
    tables, items, refs, outs = _build(capi.F32, kind, seed=13)
    plan = capi.bspline_plan_create(items, kind)
    try:
        for order in (0, 1, 0, 1):
            capi.bspline_plan_set_order(plan, order)
            for o in outs:
                o[0].fill_(float("nan"))
            capi.bspline_plan_run_graph(plan)
            torch.cuda.synchronize()
            _check(kind, refs, outs, f"order {order}")
        with pytest.raises(capi.BsplineError):
            capi.bspline_plan_set_order(plan, 2)
    finally:
        capi.bspline_plan_destroy(plan)
        for t in tables:
            t.close()


@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
def test_plan_modes_and_tune(dtype, kind):
    """A plan run one table at a time (each table's own launch shape) gives the oracle's values, directly
    and from a graph; the plan autotuner picks one of its three candidates and the plan keeps it."""
    tables, items, refs, outs = _build(dtype, kind, seed=17 + kind, empty_item=kind == capi.VGH)
    plan = capi.bspline_plan_create(items, kind)

    def clear():
        for v, g, hl, _ in outs:
            for o in (v, g, hl):
                if o is not None:
                    o.fill_(float("nan"))

    try:
        assert capi.bspline_plan_get_mode(plan) == (capi.PLAN_ONE_LAUNCH, 0)
        capi.bspline_plan_set_mode(plan, capi.PLAN_PER_TABLE)
        assert capi.bspline_plan_get_mode(plan) == (capi.PLAN_PER_TABLE, 0)
        for run in (capi.bspline_plan_run, capi.bspline_plan_run_graph, capi.bspline_plan_run_graph):
            clear()
            run(plan)
            torch.cuda.synchronize()
            _check(kind, refs, outs, f"per table, {run.__name__}")
        mode, order = capi.bspline_plan_tune(plan, reps=3)
        assert (mode, order) in {(capi.PLAN_ONE_LAUNCH, 0), (capi.PLAN_ONE_LAUNCH, 1), (capi.PLAN_PER_TABLE, 0)}
        assert capi.bspline_plan_get_mode(plan) == (mode, order)
        clear()
        capi.bspline_plan_run_graph(plan)
        torch.cuda.synchronize()
        _check(kind, refs, outs, f"tuned {mode, order}")
        with pytest.raises(capi.BsplineError):
            capi.bspline_plan_set_mode(plan, 2)
        with pytest.raises(capi.BsplineError):
            capi.bspline_plan_tune(plan, reps=0)
    finally:
        capi.bspline_plan_destroy(plan)
        for t in tables:
            t.close()


def test_plan_errors():
    kind = capi.VGH
    tables, items, refs, outs = _build(capi.F32, kind, seed=9)
    with pytest.raises(capi.BsplineError) as e:
        capi.bspline_plan_create([], kind)
    assert e.value.status == capi.ERR_ARG
    with capi.Table((4, 4, 4), 8, capi.BF16) as other:
        bad = dict(items[0])
        bad["table"] = other.h
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_plan_create([bad], kind)
        assert e.value.status == capi.ERR_STATE
        capi.bspline_set_coefs(other.h, torch.zeros((4, 4, 4, 8), device="cuda"))
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_plan_create([items[0], bad], kind)
        assert e.value.status == capi.ERR_DTYPE
    bad = dict(items[0])
    bad["ld"] = 1
    with pytest.raises(capi.BsplineError):
        capi.bspline_plan_create([bad], kind)
    for t in tables:
        t.close()


@pytest.mark.parametrize("stages", [4, 6])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_plan_ring_stages(kind, order, stages):
    """The one-launch kernel with its rows staged through the shared-memory ring gives the oracle's values
    and, doing the same arithmetic in the same order, the register kernel's bit for bit, run directly and
    from the plan's graph; 16-bit plans refuse the ring."""
    tables, items, refs, outs = _build(capi.F32, kind, seed=23 + kind, empty_item=order == 1)
    plan = capi.bspline_plan_create(items, kind)
    try:
        capi.bspline_plan_set_order(plan, order)
        capi.bspline_plan_run(plan)
        torch.cuda.synchronize()
        regs = [tuple(o.clone() if o is not None else None for o in out[:3]) for out in outs]
        capi.bspline_plan_set_stages(plan, stages)
        assert capi.bspline_plan_get_stages(plan) == stages
        for run in (capi.bspline_plan_run, capi.bspline_plan_run_graph, capi.bspline_plan_run_graph):
            for v, g, hl, _ in outs:
                for o in (v, g, hl):
                    if o is not None:
                        o.fill_(float("nan"))
            run(plan)
            torch.cuda.synchronize()
            _check(kind, refs, outs, f"ring {stages}, {run.__name__}")
            for r, o in zip(regs, outs):
                for a, b in zip(r, o[:3]):
                    if a is not None:
                        assert torch.equal(a, b)
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_plan_set_stages(plan, 5)
        assert e.value.status == capi.ERR_ARG
    finally:
        capi.bspline_plan_destroy(plan)
        for t in tables:
            t.close()
    tables, items, refs, outs = _build(capi.F16, kind, seed=29)
    plan = capi.bspline_plan_create(items, kind)
    try:
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_plan_set_stages(plan, stages)
        assert e.value.status == capi.ERR_UNSUPPORTED
    finally:
        capi.bspline_plan_destroy(plan)
        for t in tables:
            t.close()
