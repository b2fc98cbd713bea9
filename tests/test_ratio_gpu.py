"""GPU parity of the fused determinant-ratio consumer (bspline_eval_ratio).

Sec. "QMC and B-spline-based SPOs": the ratio of a one-electron move is
sum_n phi_n(r') A^-1(n,e), and the gradient ratio the same sum over grad phi_n.
The kernel forms these sums for every output component without writing the
per-orbital values. Error bound per component q at position p:

    |gpu - oracle| <= TOL_K max|c_K(phi)| sum_n |u_n| + 32 * 2^-24 sum_n |c_q(phi_n) u_n|

the first term from the per-orbital float32 tolerance of the evaluation (TOL_K
as in parity_util), the second from the float32 summation (at most about 25
roundings deep: 16 terms per thread, 5 shuffle levels, 4 warps).
"""
import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import capi, inputs
from parity_util import TOL, run_eval

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KIND_KEYS = {0: ["v"], 1: ["v", "g", "g", "g", "l"], 2: ["v", "g", "g", "g"] + ["h"] * 6}


def _ref_table(coef, dtype):
    if dtype == capi.F32:
        return coef.astype(np.float64)
    codes, scale = oracle.quantize(coef, dtype)
    return oracle.dequantize(codes, scale, dtype)


def _check(kind, got, coef64, x, y, z, u):
    out = oracle.eval_periodic(kind, coef64, x, y, z)
    comps = oracle.ratio_components(kind, out)
    ref = np.stack([np.einsum("pn,pn->p", c, u) for c in comps], axis=1)
    au = np.abs(u).sum(axis=1)
    for q, (c, key) in enumerate(zip(comps, KIND_KEYS[kind])):
        kmax = np.abs(out[key]).max()
        bound = TOL[key] * kmax * au + 32 * 2.0 ** -24 * np.einsum("pn,pn->p", np.abs(c), np.abs(u))
        err = np.abs(got[:, q] - ref[:, q])
        assert (err <= bound).all(), f"component {q}: max err/bound {(err / bound).max():.3f}"
    return ref


def _run(table, kind, x, y, z, u, ldu=None):
    N = table.N
    ldu = N if ldu is None else ldu
    npos = x.shape[0]
    uu = np.zeros((npos, ldu), np.float32)
    uu[:, :N] = u
    dx, dy, dz, du = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, z, uu))
    nc = capi.NCOMP[kind]
    r = torch.full((npos, nc), float("nan"), device="cuda")
    capi.bspline_eval_ratio(table.h, kind, npos, dx, dy, dz, du, ldu, r)
    torch.cuda.synchronize()
    return r.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("dtype", [capi.F32, capi.F16, capi.BF16])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_ratio_matches_oracle(kind, dtype, order):
    grid, N, npos = (16, 16, 16), 64, 1024
    coef = inputs.uniform_coefs(grid, N, seed=1)
    x, y, z = inputs.uniform_positions(npos, seed=2)
    u = (np.random.default_rng(3).normal(size=(npos, N)) / np.sqrt(N)).astype(np.float32)
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_tuning(t.h, kind, capi.VARIANT_DIRECT, 512, 1, 0, order)
        got = _run(t, kind, x, y, z, u)
    _check(kind, got, _ref_table(coef, dtype), x, y, z, u.astype(np.float64))


@pytest.mark.parametrize("grid,N,npos,ldu_pad", [((5, 7, 3), 37, 333, 3), ((9, 4, 6), 700, 129, 0),
                                                 ((3, 3, 3), 1, 5, 1), ((12, 10, 8), 2048, 64, 0)])
def test_ratio_ragged(grid, N, npos, ldu_pad):
    coef = inputs.uniform_coefs(grid, N, seed=21)
    x, y, z = inputs.uniform_positions(npos, seed=22)
    u = np.random.default_rng(23).normal(size=(npos, N)).astype(np.float32)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for kind in (capi.V, capi.VGL, capi.VGH):
            got = _run(t, kind, x, y, z, u, N + ldu_pad)
            _check(kind, got, coef.astype(np.float64), x, y, z, u.astype(np.float64))


def test_ratio_matches_per_orbital_outputs():
    """The fused sums equal the sums of the library's own per-orbital outputs (float32 summation apart)."""
    grid, N, npos = (10, 11, 12), 300, 200
    coef = inputs.uniform_coefs(grid, N, seed=41)
    x, y, z = inputs.uniform_positions(npos, seed=42)
    u = np.random.default_rng(43).normal(size=(npos, N)).astype(np.float32)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        got = _run(t, capi.VGH, x, y, z, u)
        per = run_eval(t, capi.VGH, x, y, z)
    comps = oracle.ratio_components(capi.VGH, {k: v.astype(np.float64) for k, v in per.items()})
    for q, c in enumerate(comps):
        ref = np.einsum("pn,pn->p", c, u.astype(np.float64))
        scale = np.einsum("pn,pn->p", np.abs(c), np.abs(u.astype(np.float64)))
        assert (np.abs(got[:, q] - ref) <= 32 * 2.0 ** -24 * scale).all()


def test_ratio_errors_and_empty():
    with capi.Table((4, 4, 4), 8, capi.F32) as t:
        r = torch.zeros((4, 1), device="cuda")
        x = torch.zeros(4, dtype=torch.float64, device="cuda")
        u = torch.zeros((4, 8), device="cuda")
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_eval_ratio(t.h, capi.V, 4, x, x, x, u, 8, r)
        assert e.value.status == capi.ERR_STATE
        capi.bspline_set_coefs(t.h, torch.zeros((4, 4, 4, 8), device="cuda"))
        with pytest.raises(capi.BsplineError):
            capi.bspline_eval_ratio(t.h, capi.V, 4, x, x, x, u, 7, r)
        with pytest.raises(capi.BsplineError):
            capi.bspline_eval_ratio(t.h, 3, 4, x, x, x, u, 8, r)
        capi.bspline_eval_ratio(t.h, capi.V, 0, None, None, None, None, 8, None)


def test_ratio_deterministic_and_scratch_reuse():
    """Partial sums of several orbital blocks are combined in a fixed order: repeated calls give the same
    bits, also after the scratch grows (a larger batch) and its arrival counters are reused."""
    grid, N = (9, 10, 11), 1500  # three 512-orbital blocks per position
    coef = inputs.uniform_coefs(grid, N, seed=51)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for npos in (100, 700, 300):
            x, y, z = inputs.uniform_positions(npos, seed=52 + npos)
            u = np.random.default_rng(53).normal(size=(npos, N)).astype(np.float32)
            first = _run(t, capi.VGH, x, y, z, u)
            for _ in range(3):
                np.testing.assert_array_equal(_run(t, capi.VGH, x, y, z, u), first)
            _check(capi.VGH, first, coef.astype(np.float64), x, y, z, u.astype(np.float64))


@pytest.mark.parametrize("nb,N", [(128, 700), (256, 700), (256, 580)])
@pytest.mark.parametrize("lattice", [False, True])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_ratio_tensor_core_variant(kind, dtype, order, lattice, nb, N):
    """Ratio sums on the tensor-core variant: running sums over the position's 128-orbital blocks (the last
    half empty: N = 700), in units of one or two blocks (N = 580: an odd number of blocks, the last unit
    one block), reduced across the four epilogue warps in a fixed order. Same bound as above; repeated
    calls give the same bits."""
    grid, npos = (11, 9, 10), 300
    coef = inputs.uniform_coefs(grid, N, seed=61)
    x, y, z = inputs.uniform_positions(npos, seed=62)
    u = (np.random.default_rng(63).normal(size=(npos, N)) / np.sqrt(N)).astype(np.float32)
    L = np.array([[1.3, 0.0, 0.0], [0.65, 1.1258330249197703, 0.0], [0.2, -0.3, 2.1]])
    if lattice:
        r = np.stack([x, y, z], axis=1) @ L
        x, y, z = (np.ascontiguousarray(r[:, d]) for d in range(3))
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        if lattice:
            capi.bspline_set_lattice(t.h, L)
        capi.bspline_set_tuning(t.h, kind, capi.VARIANT_MMA, nb, 2, 0, order)
        got = _run(t, kind, x, y, z, u)
        np.testing.assert_array_equal(_run(t, kind, x, y, z, u), got)
        assert capi.bspline_device_status(t.h) == 0
    tab = _ref_table(coef, dtype)
    if not lattice:
        _check(kind, got, tab, x, y, z, u.astype(np.float64))
        return
    out = oracle.eval_lattice(kind, tab, L, x, y, z)
    comps = oracle.ratio_components(kind, out)
    u64 = u.astype(np.float64)
    au = np.abs(u64).sum(axis=1)
    for q, (c, key) in enumerate(zip(comps, KIND_KEYS[kind])):
        ref = np.einsum("pn,pn->p", c, u64)
        bound = 2 * TOL[key] * np.abs(out[key]).max() * au + 32 * 2.0 ** -24 * np.einsum("pn,pn->p", np.abs(c),
                                                                                          np.abs(u64))
        err = np.abs(got[:, q] - ref)
        assert (err <= bound).all(), f"component {q}: max err/bound {(err / bound).max():.3f}"
