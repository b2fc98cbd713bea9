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


def _setup(kind):
    rng = np.random.default_rng(77)
    tables, items = [], []
    for k, (grid, N) in enumerate(SPECS):
        t = capi.Table(grid, N, capi.F32)
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


@pytest.mark.parametrize("kind", [capi.VGH, capi.VGL])
def test_noalloc_matches_allocating_entry_point_twice(kind):
    tables, items = _setup(kind)
    ref = _with_outputs(tables, items, kind)
    capi.bspline_eval_batched(ref, kind)
    for call in range(2):  # the shared scratch must give the same answer on consecutive calls
        got = _with_outputs(tables, items, kind)
        capi.bspline_eval_batched_noalloc(got, kind)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            assert _rel(g["v"], r["v"]) <= TOL["v"], f"call {call}"
            assert _rel(g["g"], r["g"]) <= TOL["g"], f"call {call}"
            assert _rel(g["hl"], r["hl"]) <= TOL["h" if kind == capi.VGH else "l"], f"call {call}"
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
