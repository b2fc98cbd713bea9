"""The allocation-free batched entry point against the allocating one.

bspline_eval_batched_noalloc is for callers that cannot allocate device memory
around an evaluation (their own memory manager owns the device, or their loop
must never reach cudaMalloc/cudaFree). Its scratch is a fixed array inside the
library, shared by every call. This file is collected last on purpose, and it
builds its own inputs, so it passes both alone in a fresh process and after
the other tests.
"""
import numpy as np
import pytest

from paper_1611_02665_gb300 import capi, inputs
from parity_util import TOL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

SPECS = [((9, 8, 7), 96), ((12, 12, 12), 512), ((6, 5, 6), 33)]


def _setup(kind, dtype=capi.F32):
    rng = np.random.default_rng(77)
    tables, items = [], []
    for k, (grid, N) in enumerate(SPECS):
        t = capi.Table(grid, N, dtype)
        capi.bspline_set_coefs(t.h, torch.from_numpy(inputs.uniform_coefs(grid, N, seed=700 + k)).cuda())
        npos = int(rng.integers(1, 9, size=int(rng.integers(5, 30))).sum())
        x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=800 + k))
        tables.append(t)
        items.append({"table": t.h, "npos": npos, "x": x, "y": y, "z": z, "ld": N})
    return tables, items


def _with_outputs(tables, items, kind):
    out = []
    for t, it in zip(tables, items):
        v, g, hl = t.outputs(kind, it["npos"])
        for b in (v, g, hl):
            if b is not None:
                b.fill_(float("nan"))
        d = dict(it)
        d.update(v=v, g=g, hl=hl)
        out.append(d)
    return out


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).abs().max() / b.abs().max())


def _compare(ref, got, kind, label):
    for r, g in zip(ref, got):
        if r["npos"] == 0:
            continue
        assert _rel(g["v"], r["v"]) <= TOL["v"], label
        if kind != capi.V:
            assert _rel(g["g"], r["g"]) <= TOL["g"], label
            assert _rel(g["hl"], r["hl"]) <= TOL["h" if kind == capi.VGH else "l"], label


@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_noalloc_matches_allocating_entry_point_twice(kind, dtype):
    tables, items = _setup(kind, dtype)
    ref = _with_outputs(tables, items, kind)
    capi.bspline_eval_batched(ref, kind)
    for call in range(2):  # the shared scratch must give the same answer on consecutive calls
        got = _with_outputs(tables, items, kind)
        capi.bspline_eval_batched_noalloc(got, kind)
        torch.cuda.synchronize()
        _compare(ref, got, kind, f"call {call}")
    for t in tables:
        t.close()


def test_noalloc_many_items_with_empty_ones():
    """33..64 items take the kernel's binary-search item lookup (one ballot covers at most 32 items);
    items of zero positions own no work units and must be skipped. The items share the three tables."""
    kind = capi.VGL
    tables, base = _setup(kind)
    rng = np.random.default_rng(78)
    for nitems in (33, capi.NOALLOC_MAX_ITEMS):
        items = []
        for k in range(nitems):
            t = tables[k % len(tables)]
            npos = 0 if k % 5 == 2 else int(rng.integers(1, 12))
            x, y, z = (torch.from_numpy(a).cuda() for a in inputs.uniform_positions(max(npos, 1), seed=900 + k))
            items.append({"table": t.h, "npos": npos, "x": x[:npos], "y": y[:npos], "z": z[:npos], "ld": t.N})
        ref = _with_outputs([tables[k % len(tables)] for k in range(nitems)], items, kind)
        capi.bspline_eval_batched(ref, kind)
        for call in range(2):
            got = _with_outputs([tables[k % len(tables)] for k in range(nitems)], items, kind)
            capi.bspline_eval_batched_noalloc(got, kind)
            torch.cuda.synchronize()
            _compare(ref, got, kind, f"{nitems} items, call {call}")
    for t in tables:
        t.close()


def test_noalloc_refuses_a_capturing_stream():
    """The descriptors come from the call's stack frame, so recording the call in a graph is refused with
    nothing enqueued: the outputs stay as they were after the graph is replayed."""
    kind = capi.V
    tables, items = _setup(kind)
    got = _with_outputs(tables, items, kind)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device="cuda")
    with torch.cuda.graph(graph, stream=side):
        marker.add_(1.0)  # keeps the captured graph non-empty
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_eval_batched_noalloc(got, kind, side)
    assert e.value.status == capi.ERR_UNSUPPORTED
    graph.replay()
    torch.cuda.synchronize()
    assert float(marker.item()) == 1.0
    for g in got:
        assert torch.isnan(g["v"]).all()
    # outside a capture the same call runs
    capi.bspline_eval_batched_noalloc(got, kind)
    torch.cuda.synchronize()
    for g in got:
        assert torch.isfinite(g["v"]).all()
    for t in tables:
        t.close()


def test_noalloc_rejects_too_many_items():
    tables, items = _setup(capi.V)
    many = _with_outputs(tables, items, capi.V)[:1] * (capi.NOALLOC_MAX_ITEMS + 1)
    with pytest.raises(capi.BsplineError) as e:
        capi.bspline_eval_batched_noalloc(many, capi.V)
    assert e.value.status == capi.ERR_ARG
    for t in tables:
        t.close()
