"""GPU parity: V / VGL / VGH through the C ABI against the FP64 oracle.

Eq. (TricubicValue) of arXiv:1611.02665 evaluated by every kernel variant
and table type on seeded inputs: the 16^3 x 64 uniform table at 1024
positions, ragged orbital counts and position counts, tiny grids, padded
non-periodic fields, positions outside the cell and on knots, and the full
48^3 x 2048 plane-wave table at 4096 positions in the benchmark's launch
shape (checked on sampled positions).
"""
import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import capi, inputs
from parity_util import (assert_lattice_parity, assert_parity, assert_rounding_bound, lattice_bounds, run_eval,
                         to_device)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU hosts too; skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

DIRECT = capi.VARIANT_DIRECT
TMA = capi.VARIANT_TMA
SHAPES = [
    (DIRECT, 512, 1, 0, 0), (DIRECT, 256, 3, 0, 0), (DIRECT, 1024, 2, 0, 0),
    (TMA, 256, 1, 3, 0), (TMA, 128, 2, 2, 0), (TMA, 256, 1, 2, 0),
    (DIRECT, 512, 1, 0, 1), (DIRECT, 256, 3, 0, 1), (TMA, 256, 1, 3, 1),
]


def _oracle_ref(kind, coef64, x, y, z):
    return oracle.eval_periodic(kind, coef64, x, y, z)


def _table(grid, N, dtype, coef):
    t = capi.Table(grid, N, dtype)
    capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
    return t


def _reference_table(coef, dtype):
    """Values the stored table stands for: the float32 input, or the oracle's own quantisation of it."""
    if dtype == capi.F32:
        return coef.astype(np.float64)
    codes, scale = oracle.quantize(coef, dtype)
    return oracle.dequantize(codes, scale, dtype)


@pytest.fixture(scope="module")
def cfg1():
    coef = inputs.uniform_coefs((16, 16, 16), 64, seed=1)
    x, y, z = inputs.uniform_positions(1024, seed=2)
    return coef, x, y, z


@pytest.mark.parametrize("dtype", [capi.F32, capi.F16, capi.BF16])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_cfg1_all_shapes(cfg1, dtype, kind):
    coef, x, y, z = cfg1
    ref = _oracle_ref(kind, _reference_table(coef, dtype), x, y, z)
    with _table((16, 16, 16), 64, dtype, coef) as t:
        for shape in SHAPES:
            capi.bspline_set_tuning(t.h, kind, *shape)
            got = run_eval(t, kind, x, y, z)
            assert_parity(got, ref, kind, label=f"dtype={dtype} shape={shape}")


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
def test_quantised_codes_bit_exact(cfg1, dtype):
    coef = cfg1[0]
    codes, scale = oracle.quantize(oracle.pad(coef).astype(np.float32), dtype)
    with _table((16, 16, 16), 64, dtype, coef) as t:
        got = np.zeros(codes.shape, dtype=np.uint16)
        gs = np.zeros(64, dtype=np.float32)
        capi.bspline_get_table(t.h, got, gs)
    np.testing.assert_array_equal(gs, scale)
    np.testing.assert_array_equal(got, codes)


def _abs_weight_sums(x, y, z, grid):
    """Per position, the sum over the 64 stencil points of |weight| of each output component (VGH order
    v, gx, gy, gz, xx, xy, xz, yy, yz, zz, then the Laplacian), from the oracle's cell reduction and basis."""
    out = np.zeros((len(x), 11))
    for p in range(len(x)):
        s = []  # per axis: sums of |w|, |w'| n, |w''| n^2
        for c, n in zip((x[p], y[p], z[p]), grid):
            _, t = oracle.cell(c, n)
            w, dw, d2w = oracle.basis(t)
            s.append((np.abs(w).sum(), np.abs(dw).sum() * n, np.abs(d2w).sum() * n * n))
        (a0, a1, a2), (b0, b1, b2), (c0, c1, c2) = s
        hxx, hyy, hzz = a2 * b0 * c0, a0 * b2 * c0, a0 * b0 * c2
        out[p] = (a0 * b0 * c0, a1 * b0 * c0, a0 * b1 * c0, a0 * b0 * c1,
                  hxx, a1 * b1 * c0, a1 * b0 * c1, hyy, a0 * b1 * c1, hzz, hxx + hyy + hzz)
    return out


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
def test_16bit_table_error_against_fp64_oracle_on_original_coefficients(dtype):
    """The 16-bit table's own error (16^3 x 64 uniform table, VGH and VGL at 16384 positions) against the
    FP64 oracle on the ORIGINAL float32 coefficients, not on the dequantised codes. Each stored code is
    p / s_n rounded to nearest even, |p / s_n| <= 1, so it is off by at most half a unit in the last place
    at 1: u = 2^-12 (FP16, 11 significant bits) or 2^-9 (BF16, 8 bits), plus the float32 division's 2^-24.
    An output is a weighted sum of 64 coefficients, so its error is at most u s_n sum |w| over the stencil
    (the weights of that output component) plus the float32 evaluation error allowed on every path."""
    grid, N, npos = (16, 16, 16), 64, 16384
    coef = inputs.uniform_coefs(grid, N, seed=1)
    x, y, z = inputs.uniform_positions(npos, seed=5)
    u = (2.0 ** -12 if dtype == capi.F16 else 2.0 ** -9) + 2.0 ** -24
    scale = np.abs(coef).reshape(-1, N).max(axis=0).astype(np.float64)
    wsum = _abs_weight_sums(x, y, z, grid)
    comps = {"v": [0], "g": [1, 2, 3], "h": [4, 5, 6, 7, 8, 9], "l": [10]}
    from parity_util import TOL
    with _table(grid, N, dtype, coef) as t:
        for kind in (capi.VGH, capi.VGL):
            ref = _oracle_ref(kind, coef.astype(np.float64), x, y, z)
            got = run_eval(t, kind, x, y, z)
            errs = {}
            for k in got:
                r = ref[k]
                bound_w = wsum[:, comps[k]]  # [npos, ncomp]
                bound = u * bound_w[:, :, None] * scale[None, None, :]
                if r.ndim == 2:
                    bound = bound[:, 0, :]
                slack = TOL[k] * np.abs(r).max()
                diff = np.abs(got[k].astype(np.float64) - r)
                assert (diff <= bound + slack).all(), f"dtype {dtype} kind {kind} {k}: max excess " \
                    f"{(diff - bound - slack).max():.3e}"
                errs[k] = float(diff.max() / np.abs(r).max())
            print(f"dtype {dtype} kind {kind}: max error / max |oracle| {errs}")


def test_f32_table_padding_exact(cfg1):
    coef = cfg1[0]
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        got = np.zeros((19, 19, 19, 64), dtype=np.float32)
        capi.bspline_get_table(t.h, got)
    np.testing.assert_array_equal(got, oracle.pad(coef).astype(np.float32))


@pytest.mark.parametrize("grid,N,npos", [((5, 7, 3), 37, 333), ((1, 2, 4), 1, 17), ((9, 4, 6), 300, 129),
                                         ((3, 3, 3), 100, 1)])
@pytest.mark.parametrize("dtype", [capi.F32, capi.BF16])
def test_ragged_and_tiny(grid, N, npos, dtype):
    coef = inputs.uniform_coefs(grid, N, seed=21)
    x, y, z = inputs.uniform_positions(npos, seed=22)
    ref_tab = _reference_table(coef, dtype)
    with _table(grid, N, dtype, coef) as t:
        for kind in (capi.V, capi.VGL, capi.VGH):
            ref = _oracle_ref(kind, ref_tab, x, y, z)
            for shape in SHAPES:
                capi.bspline_set_tuning(t.h, kind, *shape)
                got = run_eval(t, kind, x, y, z)
                assert_parity(got, ref, kind, label=f"grid={grid} N={N} shape={shape}")


def test_leading_dimension_and_untouched_tail():
    grid, N = (6, 5, 7), 45
    coef = inputs.uniform_coefs(grid, N, seed=31)
    x, y, z = inputs.uniform_positions(200, seed=32)
    ref = _oracle_ref(capi.VGH, coef.astype(np.float64), x, y, z)
    with _table(grid, N, capi.F32, coef) as t:
        for ld in (N, 47, 64):
            for shape in SHAPES:
                capi.bspline_set_tuning(t.h, capi.VGH, *shape)
                dx, dy, dz = to_device(x, y, z)
                v, g, h = t.outputs(capi.VGH, 200, ld)
                for buf in (v, g, h):
                    buf.fill_(12345.0)
                t.eval(capi.VGH, dx, dy, dz, v, g, h, ld)
                torch.cuda.synchronize()
                got = {"v": v.cpu().numpy()[:, :N], "g": g.cpu().numpy()[:, :, :N], "h": h.cpu().numpy()[:, :, :N]}
                assert_parity(got, ref, capi.VGH, label=f"ld={ld} {shape}")
                if ld > N:
                    assert (v[:, N:] == 12345.0).all() and (g[:, :, N:] == 12345.0).all()
                    assert (h[:, :, N:] == 12345.0).all()


def test_positions_outside_cell_and_on_knots():
    grid, N = (8, 6, 10), 40
    coef = inputs.uniform_coefs(grid, N, seed=41)
    rng = np.random.default_rng(42)
    knots = rng.integers(0, 10, size=(64, 3)) / np.array(grid)
    shifts = rng.integers(-3, 4, size=(64, 3))
    pts = np.concatenate([knots, knots + shifts, rng.uniform(-5, 5, size=(64, 3)),
                          np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0], [-1e-20, 1 - 1e-17, 2.0]])])
    x, y, z = pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy()
    with _table(grid, N, capi.F32, coef) as t:
        for kind in (capi.V, capi.VGL, capi.VGH):
            ref = _oracle_ref(kind, coef.astype(np.float64), x, y, z)
            for shape in SHAPES:
                capi.bspline_set_tuning(t.h, kind, *shape)
                assert_parity(run_eval(t, kind, x, y, z), ref, kind, label=f"{shape}")


def _knot_field(grid, f):
    nx, ny, nz = grid
    k = [(np.arange(n + 3) - 1.0) / n for n in grid]
    X, Y, Z = np.meshgrid(*k, indexing="ij")
    return f(X, Y, Z)


def test_padded_polynomial_fields():
    # Non-periodic fields stored directly in padded rows. Their curvature is small next to
    # n^2 |p|, so the check is the float32 rounding bound of the stencil sums rather than
    # the relative-to-max tolerance used for random tables.
    grid = (12, 10, 14)
    fields = [lambda X, Y, Z: 0.3 - 1.7 * X + 2.1 * Y + 0.9 * Z,
              lambda X, Y, Z: X * X + Y * Y + Z * Z,
              lambda X, Y, Z: X * Y - 0.5 * Y * Z]
    pad = np.stack([_knot_field(grid, f) for f in fields], axis=-1).astype(np.float32)
    x, y, z = inputs.uniform_positions(300, seed=51)
    ref = oracle.eval_padded(capi.VGH, pad.astype(np.float64), x, y, z)
    with capi.Table(grid, 3, capi.F32) as t:
        capi.bspline_set_coefs_padded(t.h, torch.from_numpy(pad).cuda())
        for shape in SHAPES:
            capi.bspline_set_tuning(t.h, capi.VGH, *shape)
            got = run_eval(t, capi.VGH, x, y, z)
            assert_rounding_bound(got, ref, capi.VGH, np.abs(pad).max(), grid, label=f"{shape}")
            # closed forms: the quadratic's Hessian is 2*I, the linear field's gradient is constant
            np.testing.assert_allclose(got["h"][:, [0, 3, 5], 1], 2.0, atol=2e-3)
            np.testing.assert_allclose(got["g"][:, 0, 0], -1.7, atol=1e-4)


@pytest.mark.timeout(300)
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("shape", [None, (DIRECT, 512, 1, 0, 1), (TMA, 256, 1, 3, 0), (TMA, 128, 2, 2, 1)])
def test_host_buffers_match_device_path(cfg1, shape, mode):
    coef, x, y, z = cfg1
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        capi.bspline_set_host_mode(t.h, mode)
        for kind in (capi.V, capi.VGL, capi.VGH):
            if shape:
                capi.bspline_set_tuning(t.h, kind, *shape)
            dev = run_eval(t, kind, x, y, z)
            nc = {0: 1, 1: 5, 2: 10}[kind]
            v = np.zeros((1024, 64), np.float32)
            g = np.zeros((1024, 3, 64), np.float32) if kind else None
            hl = None if kind == 0 else np.zeros((1024, 64) if kind == 1 else (1024, 6, 64), np.float32)
            try:
                capi.bspline_eval_host(t.h, kind, 1024, x, y, z, v, g, hl, 64)
            except capi.BsplineError as err:
                if mode == 2 and err.status == capi.ERR_UNSUPPORTED:
                    pytest.skip("this GPU cannot address pageable host memory")
                raise
            np.testing.assert_array_equal(v, dev["v"])
            if kind:
                np.testing.assert_array_equal(g, dev["g"])
                np.testing.assert_array_equal(hl, dev["l" if kind == 1 else "h"])
            assert nc


def test_argument_errors_and_state(cfg1):
    coef, x, y, z = cfg1
    dx, dy, dz = to_device(x, y, z)
    with capi.Table((16, 16, 16), 64, capi.F32) as t:
        v, g, h = t.outputs(capi.VGH, 1024)
        with pytest.raises(capi.BsplineError) as e:
            t.eval(capi.VGH, dx, dy, dz, v, g, h)
        assert e.value.status == capi.ERR_STATE
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_eval_vgh(t.h, 1024, dx, dy, dz, v, g, h, 63)
        assert e.value.status == capi.ERR_ARG
        with pytest.raises(capi.BsplineError):
            capi.bspline_eval_vgh(t.h, 1024, dx, dy, dz, v, None, h, 64)
        with pytest.raises(capi.BsplineError):
            capi.bspline_eval_v(t.h, -1, dx, dy, dz, v, 64)
        with pytest.raises(capi.BsplineError):
            capi.bspline_set_tuning(t.h, capi.VGH, capi.VARIANT_TMA, 512, 1, 3)
        with pytest.raises(capi.BsplineError):
            capi.bspline_set_tuning(t.h, capi.VGH, capi.VARIANT_DIRECT, 512, 1, 0, 2)
        capi.bspline_eval_v(t.h, 0, None, None, None, None, 64)  # empty batch is a no-op
        assert capi.bspline_device_status(t.h) == 0


def test_autotuner_and_wisdom(cfg1, tmp_path):
    coef, x, y, z = cfg1
    wisdom = str(tmp_path / "wisdom.jsonl")
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        best = capi.bspline_tune(t.h, capi.VGH, 1024, wisdom)
        assert best["variant"] in (DIRECT, TMA)
        assert capi.bspline_get_tuning(t.h, capi.VGH) == best
        ref = _oracle_ref(capi.VGH, coef.astype(np.float64), x, y, z)
        assert_parity(run_eval(t, capi.VGH, x, y, z), ref, capi.VGH)
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        again = capi.bspline_tune(t.h, capi.VGH, 1024, wisdom)  # read back without timing
        assert again == best
    assert open(wisdom).read().count("\n") == 1


@pytest.fixture(scope="module")
def cfg2():
    """48^3 grid, 2048 plane-wave orbitals, 4096 positions: the benchmark workload."""
    grid, N = (48, 48, 48), 2048
    coef = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    x, y, z = inputs.uniform_positions(4096, seed=4)
    return grid, N, coef, x, y, z


@pytest.mark.parametrize("kind", [capi.V, capi.VGH])
def test_cfg2_full_size_sampled(cfg2, kind):
    grid, N, coef, x, y, z = cfg2
    sample = np.random.default_rng(5).choice(4096, size=24, replace=False)
    coef64 = coef.cpu().numpy().astype(np.float64)
    ref = _oracle_ref(kind, coef64, x[sample], y[sample], z[sample])
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, coef)
        for shape in [None, (TMA, 256, 1, 3, 0), (DIRECT, 512, 1, 0, 0), (DIRECT, 512, 1, 0, 1), (TMA, 256, 1, 3, 1)]:
            if shape:
                capi.bspline_set_tuning(t.h, kind, *shape)
            got = run_eval(t, kind, x, y, z)
            sub = {k: v[sample] for k, v in got.items()}
            errs = assert_parity(sub, ref, kind, label=f"{shape}")
            assert all(np.isfinite(v).all() for v in got.values())
            print(f"cfg2 kind={kind} shape={shape} rel errors {errs}")


def test_default_shape_sorts_tables_larger_than_l2():
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    with capi.Table((48, 48, 48), 2048, capi.F32) as big, capi.Table((16, 16, 16), 64, capi.F32) as small:
        assert capi.bspline_get_info(big.h).table_bytes > l2 >= capi.bspline_get_info(small.h).table_bytes
        for kind in (capi.V, capi.VGL, capi.VGH):
            assert capi.bspline_get_tuning(big.h, kind)["order"] == 1
            assert capi.bspline_get_tuning(small.h, kind)["order"] == 0


@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_graphite_shape_sampled(kind):
    """The grid and orbital count of the paper's graphite workload (48 x 48 x 60, N = 128; plane-wave
    orbitals stand in for its DFT orbitals), 4096 positions, default and explicit launch shapes, on a
    sample of positions the oracle evaluates one by one."""
    grid, N = (48, 48, 60), 128
    coef = inputs.plane_wave_coefs(grid, N, seed=10, device="cuda")
    x, y, z = inputs.uniform_positions(4096, seed=11)
    sample = np.random.default_rng(12).choice(4096, size=64, replace=False)
    ref = _oracle_ref(kind, coef.cpu().numpy().astype(np.float64), x[sample], y[sample], z[sample])
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, coef)
        for shape in [None, (DIRECT, 512, 1, 0, 0), (DIRECT, 256, 2, 0, 1), (DIRECT, 512, 1, 6, 1),
                      (TMA, 128, 1, 3, 1)]:
            if shape:
                capi.bspline_set_tuning(t.h, kind, *shape)
            got = run_eval(t, kind, x, y, z)
            assert_parity({k: v[sample] for k, v in got.items()}, ref, kind, label=f"{shape}")
            assert all(np.isfinite(v).all() for v in got.values())


@pytest.mark.parametrize("npos", [8192, 8193, 40000])
@pytest.mark.parametrize("dtype,shape", [(capi.F32, (DIRECT, 512, 1, 0)), (capi.F32, (DIRECT, 512, 1, 4)),
                                         (capi.F16, (capi.VARIANT_MMA, 128, 2, 0))])
@pytest.mark.parametrize("lattice", [None, ((1.3, 0.0, 0.0), (0.65, 1.1258330249197703, 0.0), (0.2, -0.3, 2.1))])
def test_sorted_order_many_positions(npos, dtype, shape, lattice):
    """Above 8192 positions the cell sort runs on many CTAs (keys, histogram, scan, atomic scatter). Its
    permutation must cover every position exactly once: the sorted evaluation writes every output, equal
    bit for bit to the input-order evaluation of the same positions (outputs start as NaN)."""
    grid, N = (20, 24, 28), 600
    coef = inputs.plane_wave_coefs(grid, N, seed=41, device="cuda")
    u = inputs.uniform_positions(npos, seed=42)
    if lattice is not None:
        r = np.stack(u, axis=1) @ np.asarray(lattice)
        u = [np.ascontiguousarray(r[:, d]) for d in range(3)]
    x, y, z = (torch.from_numpy(a).cuda() for a in u)
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, coef)
        if lattice is not None:
            capi.bspline_set_lattice(t.h, lattice)
        for kind in (capi.V, capi.VGH):
            if kind == capi.V and shape[0] == capi.VARIANT_MMA:
                continue
            res = []
            for order in (0, 1, 1):
                capi.bspline_set_tuning(t.h, kind, *shape, order)
                out = [o.fill_(float("nan")) if o is not None else None for o in t.outputs(kind, npos)]
                t.eval(kind, x, y, z, *out)
                torch.cuda.synchronize()
                res.append([o for o in out if o is not None])
            for sorted_run in res[1:]:
                for got, ref in zip(sorted_run, res[0]):
                    assert torch.equal(got, ref)
        assert capi.bspline_device_status(t.h) == capi.OK


@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
def test_sorted_calls_back_to_back(dtype):
    """Cell-sorted calls queued back to back on one stream: each call's sort may start while the previous
    evaluation drains (programmatic dependent launch). Every call's outputs equal those of the same
    positions evaluated alone in input order, bit for bit; a call that reuses the previous call's output
    buffers leaves its own results there; and a torch kernel that rewrites the positions in place between
    two calls is seen by the second."""
    grid, N, npos, K = (32, 32, 32), 768, 4096, 6
    coef = inputs.plane_wave_coefs(grid, N, seed=21, device="cuda")
    pos = [[torch.from_numpy(a).cuda() for a in inputs.uniform_positions(npos, seed=300 + k)] for k in range(K)]
    stream = torch.cuda.current_stream()
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, coef)
        capi.bspline_set_tuning(t.h, capi.VGH, 0, 0, 0, 0, 0)
        default = capi.bspline_get_tuning(t.h, capi.VGH)
        plain = dict(default, order=0)
        capi.bspline_set_tuning(t.h, capi.VGH, *plain.values())
        refs = []
        for k in range(K):
            v, g, h = t.outputs(capi.VGH, npos)
            t.eval(capi.VGH, *pos[k], v, g, h)
            torch.cuda.synchronize()
            refs.append((v, g, h))
        capi.bspline_set_tuning(t.h, capi.VGH, *dict(default, order=1).values())
        outs = [t.outputs(capi.VGH, npos) for _ in range(K)]
        shared = t.outputs(capi.VGH, npos)
        for rep in range(2):
            for k in range(K):
                t.eval(capi.VGH, *pos[k], *outs[k])
                t.eval(capi.VGH, *pos[k], *shared)
        torch.cuda.synchronize()
        for k in range(K):
            for got, ref in zip(outs[k], refs[k]):
                assert torch.equal(got, ref), f"call {k}"
        for got, ref in zip(shared, refs[K - 1]):
            assert torch.equal(got, ref)
        # positions rewritten in place by a torch kernel right before the call
        x, y, z = (c.clone() for c in pos[0])
        t.eval(capi.VGH, x, y, z, *outs[0])
        x.copy_(pos[1][0]), y.copy_(pos[1][1]), z.copy_(pos[1][2])
        t.eval(capi.VGH, x, y, z, *outs[0])
        torch.cuda.synchronize()
        for got, ref in zip(outs[0], refs[1]):
            assert torch.equal(got, ref)
        assert capi.bspline_device_status(t.h) == capi.OK
        assert stream is not None


def test_bounded_wait_times_out_and_context_survives(cfg1):
    """A wait on a flag nothing sets gives up after its limit and reports it; the GPU stays usable."""
    coef, x, y, z = cfg1
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        assert capi.bspline_device_status(t.h) == capi.OK
        capi.bspline_selftest_wait_timeout(t.h, 1000)
        assert capi.bspline_device_status(t.h, reset=True) == capi.ERR_TIMEOUT
        assert capi.bspline_device_status(t.h) == capi.OK
        ref = _oracle_ref(capi.VGH, coef.astype(np.float64), x, y, z)
        capi.bspline_set_tuning(t.h, capi.VGH, TMA, 256, 1, 3, 1)
        assert_parity(run_eval(t, capi.VGH, x, y, z), ref, capi.VGH)


def test_host_path_many_sorted_positions():
    """The host-buffer path on 30000 positions with the cell sort: staged chunks of about 13000 positions
    and the whole batch at once both take the many-CTA sort in their own scratch."""
    grid, N, npos = (16, 16, 16), 64, 30000
    coef = inputs.uniform_coefs(grid, N, seed=51)
    x, y, z = inputs.uniform_positions(npos, seed=52)
    with _table(grid, N, capi.F32, coef) as t:
        capi.bspline_set_tuning(t.h, capi.VGH, DIRECT, 512, 1, 0, 0)
        dev = run_eval(t, capi.VGH, x, y, z)
        capi.bspline_set_tuning(t.h, capi.VGH, DIRECT, 512, 1, 0, 1)
        px, py, pz = (torch.from_numpy(a).pin_memory() for a in (x, y, z))
        for mode in (1, 2, 0):
            capi.bspline_set_host_mode(t.h, mode)
            v = torch.full((npos, N), float("nan")).pin_memory()
            g = torch.full((npos, 3, N), float("nan")).pin_memory()
            h = torch.full((npos, 6, N), float("nan")).pin_memory()
            try:
                capi.bspline_eval_host(t.h, capi.VGH, npos, px, py, pz, v, g, h, N)
            except capi.BsplineError as err:
                if mode == 2 and err.status == capi.ERR_UNSUPPORTED:
                    continue  # no direct access to host memory on this system
                raise
            np.testing.assert_array_equal(v.numpy(), dev["v"])
            np.testing.assert_array_equal(g.numpy(), dev["g"])
            np.testing.assert_array_equal(h.numpy(), dev["h"])
        assert capi.bspline_device_status(t.h) == capi.OK


def test_host_path_pinned_buffers(cfg1):
    coef, x, y, z = cfg1
    with _table((16, 16, 16), 64, capi.F32, coef) as t:
        dev = run_eval(t, capi.VGH, x, y, z)
        px, py, pz = (torch.from_numpy(a).pin_memory() for a in (x, y, z))
        for mode in (1, 2, 0):
            capi.bspline_set_host_mode(t.h, mode)
            v = torch.zeros((1024, 64)).pin_memory()
            g = torch.zeros((1024, 3, 64)).pin_memory()
            h = torch.zeros((1024, 6, 64)).pin_memory()
            capi.bspline_eval_host(t.h, capi.VGH, 1024, px, py, pz, v, g, h, 64)
            np.testing.assert_array_equal(v.numpy(), dev["v"])
            np.testing.assert_array_equal(g.numpy(), dev["g"])
            np.testing.assert_array_equal(h.numpy(), dev["h"])


@pytest.mark.parametrize("grid,N", [((5, 7, 6), 37), ((1, 2, 3), 5), ((16, 16, 16), 64), ((12, 40, 9), 200),
                                    ((2, 1, 66), 33), ((3, 65, 4), 40)])
def test_set_values_interpolates(grid, N):
    """bspline_set_values: coefficients equal the oracle's FFT solve; the spline reproduces the samples.
    Device samples are solved in the padded table itself, host samples on a scratch copy: both give the
    same table, bit for bit.

    Bound: each of the three passes is an n-term float32 sum with sum|G| < 2 (G the inverse of the
    knot circulant), so the coefficient error is below 3 * n * 2^-24 * 2 * 8 * max|f|; the spline's
    knot values add the float32 evaluation error (2e-6 of max|v|, the V tolerance).
    """
    f = inputs.uniform_coefs(grid, N, seed=61)
    nx, ny, nz = grid
    cref = oracle.interpolate(f.astype(np.float64))
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_values(t.h, torch.from_numpy(f).cuda())
        tab = np.zeros((nx + 3, ny + 3, nz + 3, N), np.float32)
        capi.bspline_get_table(t.h, tab)
        got = tab[1:nx + 1, 1:ny + 1, 1:nz + 1].astype(np.float64)
        n = max(grid)
        bound = 48 * n * 2.0 ** -24 * np.abs(f).max()
        assert np.abs(got - cref).max() <= bound
        np.testing.assert_array_equal(tab, oracle.pad(got).astype(np.float32))  # padded periodically
        I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        x, y, z = (I / nx).ravel(), (J / ny).ravel(), (K / nz).ravel()
        v = run_eval(t, capi.V, x, y, z)["v"]
        assert np.abs(v - f.reshape(-1, N)).max() <= bound * 2 + 2e-6 * np.abs(f).max()
    # host input gives the same table
    with capi.Table(grid, N, capi.F32) as t2:
        capi.bspline_set_values(t2.h, f)
        tab2 = np.zeros_like(tab)
        capi.bspline_get_table(t2.h, tab2)
    np.testing.assert_array_equal(tab, tab2)


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
@pytest.mark.parametrize("grid,N", [((6, 5, 7), 70), ((3, 66, 4), 20)])
def test_set_values_16bit(dtype, grid, N):
    """16-bit tables from grid samples: the solve's FP32 coefficients go through the same per-orbital
    quantisation as bspline_set_coefs, so the table equals the one set from the FP32 table's coefficients
    (checked against the oracle's solve here), bit for bit."""
    f = inputs.uniform_coefs(grid, N, seed=62)
    nx, ny, nz = grid
    with capi.Table(grid, N, capi.F32) as t32:
        capi.bspline_set_values(t32.h, torch.from_numpy(f).cuda())
        tab = np.zeros((nx + 3, ny + 3, nz + 3, N), np.float32)
        capi.bspline_get_table(t32.h, tab)
    c32 = np.ascontiguousarray(tab[1:nx + 1, 1:ny + 1, 1:nz + 1])
    cref = oracle.interpolate(f.astype(np.float64))
    assert np.abs(c32 - cref).max() <= 48 * max(grid) * 2.0 ** -24 * np.abs(f).max()
    tabs = []
    for setter, src in ((capi.bspline_set_values, f), (capi.bspline_set_coefs, c32)):
        with capi.Table(grid, N, dtype) as t:
            setter(t.h, torch.from_numpy(src).cuda())
            codes = np.zeros((nx + 3, ny + 3, nz + 3, N), np.uint16)
            scale = np.zeros(N, np.float32)
            capi.bspline_get_table(t.h, codes, scale)
            tabs.append((codes, scale))
    np.testing.assert_array_equal(tabs[0][0], tabs[1][0])
    np.testing.assert_array_equal(tabs[0][1], tabs[1][1])


@pytest.mark.parametrize("N", [1, 31, 33, 96, 129, 200, 255, 500, 513])
@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
def test_small_n_position_groups(N, dtype):
    """Orbital counts around the lane boundaries of the grouped layout: when a table's padded row fits in
    fewer than the CTA's lanes, one CTA evaluates several positions side by side. Every CTA width, up to
    8 positions per group (capped at 32 per CTA), both position orders, a ragged position count."""
    grid, npos = (7, 9, 5), 333
    coef = inputs.uniform_coefs(grid, N, seed=81)
    x, y, z = inputs.uniform_positions(npos, seed=82)
    ref_tab = _reference_table(coef, dtype)
    with _table(grid, N, dtype, coef) as t:
        for kind in (capi.V, capi.VGH):
            ref = _oracle_ref(kind, ref_tab, x, y, z)
            for nb in (256, 512, 1024):
                for ppc, order in ((1, 0), (3, 1), (8, 0)):
                    capi.bspline_set_tuning(t.h, kind, DIRECT, nb, ppc, 0, order)
                    got = run_eval(t, kind, x, y, z, ld=N + 3)
                    assert_parity(got, ref, kind, label=f"N={N} nb={nb} ppc={ppc} order={order}")
            if dtype == capi.F32:  # rows staged through shared memory (grouped for rows of <= 256 orbitals)
                for ppc, order in ((0, 0), (1, 1), (3, 0), (8, 1)):
                    capi.bspline_set_tuning(t.h, kind, DIRECT, 512, ppc, 4, order)
                    got = run_eval(t, kind, x, y, z, ld=N + 3)
                    assert_parity(got, ref, kind, label=f"N={N} staged ppc={ppc} order={order}")


def test_read_bandwidth_probe():
    """The probe returns a finite rate; an L2-sized buffer reads faster than a DRAM-sized one; bad arguments fail."""
    l2 = capi.bspline_measure_read_bandwidth(32 << 20, 5)
    dram = capi.bspline_measure_read_bandwidth(1 << 30, 3)
    assert np.isfinite(l2) and np.isfinite(dram) and l2 > dram > 100.0
    for nbytes, reps in ((0, 5), (24, 5), (1 << 20, 0)):
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_measure_read_bandwidth(nbytes, reps)
        assert e.value.status == capi.ERR_ARG


@pytest.mark.parametrize("dtype", [capi.F32, capi.F16])
def test_maximum_orbital_count(dtype):
    """N = 2^20 (the largest a table takes): 64-bit row offsets, 2048 blocks of 512 orbitals (DIRECT) or
    8192 units of 128 (the 16-bit default). Orbitals are independent, so the oracle checks a sample."""
    grid, N = (2, 3, 2), 1 << 20
    coef = inputs.uniform_coefs_device(grid, N, seed=61)
    x, y, z = inputs.uniform_positions(3, seed=62)
    cols = np.random.default_rng(63).choice(N, size=2048, replace=False)
    sub = coef.cpu().numpy()[..., cols]
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, coef)
        if dtype == capi.F32:
            ref_tab = sub.astype(np.float64)
        else:  # an orbital's scale and codes depend on its own column only: the oracle quantises the sample
            codes, scale = oracle.quantize(sub, dtype)
            ref_tab = oracle.dequantize(codes, scale, dtype)
        for kind in (capi.V, capi.VGH):
            got = run_eval(t, kind, x, y, z)
            sub_got = {k: v[..., cols] for k, v in got.items()}
            assert_parity(sub_got, oracle.eval_periodic(kind, ref_tab, x, y, z), kind, label=f"kind {kind}")


def test_many_positions_sorted():
    """2^21 positions (sorted on many CTAs), sampled against the oracle; the sorted outputs equal the
    input-order ones bit for bit."""
    grid, N, npos = (8, 8, 8), 32, 1 << 21
    coef = inputs.uniform_coefs(grid, N, seed=64)
    x, y, z = inputs.uniform_positions(npos, seed=65)
    sample = np.random.default_rng(66).choice(npos, size=256, replace=False)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        outs = []
        for order in (0, 1):
            capi.bspline_set_tuning(t.h, capi.VGH, DIRECT, 512, 1, 0, order)
            got = run_eval(t, capi.VGH, x, y, z)
            ref = _oracle_ref(capi.VGH, coef.astype(np.float64), x[sample], y[sample], z[sample])
            assert_parity({k: v[sample] for k, v in got.items()}, ref, capi.VGH, label=f"order {order}")
            outs.append(got)
        for k in outs[0]:
            np.testing.assert_array_equal(outs[1][k], outs[0][k])
        assert capi.bspline_device_status(t.h) == capi.OK


def test_long_axis():
    """1024 intervals along one axis (the most the interpolation solve takes), both position orders."""
    grid, N, npos = (1024, 3, 5), 64, 2000
    coef = inputs.uniform_coefs(grid, N, seed=67)
    x, y, z = inputs.uniform_positions(npos, seed=68)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for kind in (capi.V, capi.VGL, capi.VGH):
            ref = _oracle_ref(kind, coef.astype(np.float64), x, y, z)
            for order in (0, 1):
                capi.bspline_set_tuning(t.h, kind, DIRECT, 512, 1, 0, order)
                assert_parity(run_eval(t, kind, x, y, z), ref, kind, label=f"kind {kind} order {order}")


@pytest.mark.parametrize("stages", [3, 4, 6, 8])
def test_direct_rows_staged_through_shared_memory(stages):
    """DIRECT with each thread's stencil rows staged through a shared-memory ring (FP32, stages = ring
    units): every kind, ragged orbital counts, several positions per CTA, both orders, a general cell;
    16-bit tables report the shape as unsupported."""
    for grid, N, npos in (((7, 9, 5), 37, 333), ((12, 10, 14), 1100, 200)):
        coef = inputs.uniform_coefs(grid, N, seed=71)
        x, y, z = inputs.uniform_positions(npos, seed=72)
        with _table(grid, N, capi.F32, coef) as t:
            for kind in (capi.V, capi.VGL, capi.VGH):
                ref = _oracle_ref(kind, coef.astype(np.float64), x, y, z)
                for ppc, order in ((1, 1), (3, 0)):
                    capi.bspline_set_tuning(t.h, kind, DIRECT, 512, ppc, stages, order)
                    assert_parity(run_eval(t, kind, x, y, z, ld=N + 2), ref, kind,
                                  label=f"N={N} stages={stages} ppc={ppc} order={order}")
            L = np.array([[2.0, 0.3, -0.4], [-0.5, 1.7, 0.2], [0.6, 0.4, 1.5]])
            r = np.stack([x, y, z], axis=1) @ L
            xr, yr, zr = (np.ascontiguousarray(r[:, d]) for d in range(3))
            capi.bspline_set_lattice(t.h, L)
            capi.bspline_set_tuning(t.h, capi.VGH, DIRECT, 512, 1, stages, 1)
            assert_lattice_parity(run_eval(t, capi.VGH, xr, yr, zr),
                                  oracle.eval_lattice(capi.VGH, coef.astype(np.float64), L, xr, yr, zr),
                                  lattice_bounds(coef.astype(np.float64), L, xr, yr, zr))
    with capi.Table((4, 4, 4), 64, capi.F16) as t:
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_set_tuning(t.h, capi.VGH, DIRECT, 512, 1, stages, 0)
        assert e.value.status == capi.ERR_UNSUPPORTED


def test_binding_current_stream_is_torchs():
    """The binding's default stream (no stream argument) is torch's current stream, inside a stream
    context too, and an evaluation enqueued there is ordered with torch work on it."""
    s = torch.cuda.Stream()
    assert capi._stream(None) == torch.cuda.current_stream().cuda_stream
    with torch.cuda.stream(s):
        assert capi._stream(None) == s.cuda_stream
    assert capi._stream(None) == torch.cuda.current_stream().cuda_stream
    coef = inputs.uniform_coefs((6, 6, 6), 40, seed=91)
    x, y, z = inputs.uniform_positions(50, seed=92)
    ref = _oracle_ref(capi.V, coef.astype(np.float64), x, y, z)
    with _table((6, 6, 6), 40, capi.F32, coef) as t:
        dx, dy, dz = to_device(x, y, z)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            v = torch.full((50, 40), float("nan"), device="cuda")
            t.eval(capi.V, dx, dy, dz, v)
            got = v.cpu().numpy()  # ordered after the evaluation on s
        assert_parity({"v": got}, ref, capi.V)


@pytest.mark.parametrize("N", [1, 33, 64, 128, 256])
@pytest.mark.parametrize("npos", [1, 100, 1024])
def test_small_launch_stages_whole_stencil(N, npos):
    """FP32 calls whose grouped grid fits in one CTA per SM, on the default shape (positions per CTA left
    to the call), stage all 16 units of a position's stencil at once (a 16-unit ring, packed VGH). Checked
    against the oracle, and bit for bit against the grouped kernel with rows in registers (same
    arithmetic in the same order)."""
    grid = (7, 6, 9)
    coef = inputs.uniform_coefs(grid, N, seed=170 + N)
    x, y, z = inputs.uniform_positions(npos, seed=171 + npos)
    with _table(grid, N, capi.F32, coef) as t:
        for kind in (capi.V, capi.VGL, capi.VGH):
            ref = _oracle_ref(kind, coef.astype(np.float64), x, y, z)
            capi.bspline_set_tuning(t.h, kind, capi.VARIANT_AUTO)
            assert capi.bspline_get_tuning(t.h, kind)["ppc"] == 0
            got = run_eval(t, kind, x, y, z)
            assert_parity(got, ref, kind, label=f"N={N} npos={npos} kind={kind}")
            capi.bspline_set_tuning(t.h, kind, DIRECT, 512, 1, 0, 0)
            regs = run_eval(t, kind, x, y, z)
            for k in got:
                np.testing.assert_array_equal(got[k], regs[k])
