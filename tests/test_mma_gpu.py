"""GPU parity of the tensor-core variant (BSPLINE_VARIANT_MMA) for 16-bit tables.

Each position's outputs are the 64-point stencil sum of Eq. (TricubicValue)
computed as a matrix product on the tensor cores: the 16-bit table codes times
the weights split into 16-bit parts (22 significant bits for FP16, 24 for
BF16), FP32 accumulation. Products of 16-bit numbers are exact in FP32, so the
result is the FP32 stencil sum up to rounding order and the weight split
(below 2^-22 relative), inside the same tolerances as the FMA path (TOL of
parity_util), against the oracle on the dequantised table.
"""
import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import capi, inputs
from parity_util import assert_lattice_parity, assert_parity, lattice_bounds, run_eval, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

MMA = capi.VARIANT_MMA
# (variant, nb, CTAs per SM, stages, order); nb = 256: units of two 128-orbital blocks
SHAPES = [(MMA, 128, 2, 4, 0), (MMA, 128, 1, 2, 0), (MMA, 128, 2, 3, 1), (MMA, 128, 1, 8, 1), (MMA, 256, 2, 2, 1),
          (MMA, 256, 1, 4, 0)]


def _dequantised(coef, dtype):
    codes, scale = oracle.quantize(coef, dtype)
    return oracle.dequantize(codes, scale, dtype)


@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_mma_cfg1(kind, dtype):
    grid, N = (16, 16, 16), 64
    coef = inputs.uniform_coefs(grid, N, seed=1)
    x, y, z = inputs.uniform_positions(1024, seed=2)
    ref = oracle.eval_periodic(kind, _dequantised(coef, dtype), x, y, z)
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for shape in SHAPES:
            capi.bspline_set_tuning(t.h, kind, *shape)
            got = run_eval(t, kind, x, y, z)
            errs = assert_parity(got, ref, kind, label=f"dtype={dtype} shape={shape}")
            print(f"kind={kind} dtype={dtype} shape={shape} rel errors {errs}")


@pytest.mark.parametrize("grid,N,npos", [((5, 7, 3), 37, 333), ((1, 2, 4), 1, 17), ((9, 4, 6), 300, 129),
                                         ((3, 3, 3), 100, 1), ((6, 5, 7), 700, 64), ((4, 4, 4), 129, 200)])
@pytest.mark.parametrize("dtype", [capi.F16, capi.BF16])
def test_mma_ragged(grid, N, npos, dtype):
    """Orbital counts that leave the upper half of the last 128-orbital block empty (not loaded) or partly
    filled, several blocks, tiny and ragged grids, ld > N."""
    coef = inputs.uniform_coefs(grid, N, seed=91)
    x, y, z = inputs.uniform_positions(npos, seed=92)
    tab = _dequantised(coef, dtype)
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for kind in (capi.V, capi.VGL, capi.VGH):
            ref = oracle.eval_periodic(kind, tab, x, y, z)
            for shape in SHAPES[:3]:
                capi.bspline_set_tuning(t.h, kind, *shape)
                got = run_eval(t, kind, x, y, z, ld=N + 5)
                assert_parity(got, ref, kind, label=f"grid={grid} N={N} shape={shape}")


def test_mma_positions_outside_cell_and_on_knots():
    grid, N = (8, 6, 10), 40
    coef = inputs.uniform_coefs(grid, N, seed=93)
    rng = np.random.default_rng(94)
    knots = rng.integers(0, 10, size=(64, 3)) / np.array(grid)
    pts = np.concatenate([knots, knots + rng.integers(-3, 4, size=(64, 3)), rng.uniform(-5, 5, size=(64, 3))])
    x, y, z = pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy()
    tab = _dequantised(coef, capi.F16)
    with capi.Table(grid, N, capi.F16) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        for kind in (capi.V, capi.VGL, capi.VGH):
            capi.bspline_set_tuning(t.h, kind, *SHAPES[0])
            assert_parity(run_eval(t, kind, x, y, z), oracle.eval_periodic(kind, tab, x, y, z), kind)


def test_mma_matches_direct_path():
    """Both 16-bit paths read the same codes and compute the same stencil sums: they agree to FP32 rounding."""
    grid, N, npos = (12, 10, 14), 512, 500
    coef = inputs.uniform_coefs(grid, N, seed=95)
    x, y, z = inputs.uniform_positions(npos, seed=96)
    with capi.Table(grid, N, capi.BF16) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_tuning(t.h, capi.VGH, capi.VARIANT_DIRECT, 512, 1, 0, 0)
        direct = run_eval(t, capi.VGH, x, y, z)
        capi.bspline_set_tuning(t.h, capi.VGH, *SHAPES[0])
        mma = run_eval(t, capi.VGH, x, y, z)
    for k in ("v", "g", "h"):
        scale = np.abs(direct[k]).max()
        assert np.abs(mma[k] - direct[k]).max() <= 4e-6 * scale, k


@pytest.mark.parametrize("kind", [capi.V, capi.VGH])
def test_mma_full_size_sampled(kind):
    """48^3 grid, 2048 plane-wave orbitals, 4096 positions in the benchmark's FP16 launch shape, sampled."""
    grid, N = (48, 48, 48), 2048
    coef = inputs.plane_wave_coefs(grid, N, seed=3, device="cuda")
    x, y, z = inputs.uniform_positions(4096, seed=4)
    sample = np.random.default_rng(5).choice(4096, size=24, replace=False)
    ref = oracle.eval_periodic(kind, _dequantised(coef.cpu().numpy(), capi.F16), x[sample], y[sample], z[sample])
    with capi.Table(grid, N, capi.F16) as t:
        capi.bspline_set_coefs(t.h, coef)
        for shape in (SHAPES[0], SHAPES[2], SHAPES[4]):
            capi.bspline_set_tuning(t.h, kind, *shape)
            got = run_eval(t, kind, x, y, z)
            assert all(np.isfinite(v).all() for v in got.values())
            assert_parity({k: v[sample] for k, v in got.items()}, ref, kind, label=f"{shape}")


def test_mma_errors():
    with capi.Table((4, 4, 4), 16, capi.F32) as t:
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_set_tuning(t.h, capi.VGH, *SHAPES[0])
        assert e.value.status == capi.ERR_UNSUPPORTED
    with capi.Table((4, 5, 6), 16, capi.F16) as t:
        for bad in ((MMA, 512, 1, 2, 0), (MMA, 256, 2, 4, 0), (MMA, 128, 3, 4, 0), (MMA, 128, 1, 1, 0),
                    (MMA, 128, 1, 9, 0), (MMA, 128, 2, 8, 0)):
            with pytest.raises(capi.BsplineError) as e:
                capi.bspline_set_tuning(t.h, capi.VGH, *bad)
            assert e.value.status == capi.ERR_ARG, bad
        capi.bspline_set_coefs(t.h, torch.from_numpy(inputs.uniform_coefs((4, 5, 6), 16, seed=97)).cuda())
        capi.bspline_set_tuning(t.h, capi.VGH, *SHAPES[0])
        x, y, z = to_device(*inputs.uniform_positions(8, seed=98))
        v, g, hl = t.outputs(capi.VGH, 8)
        t.eval(capi.VGH, x, y, z, v, g, hl)
        torch.cuda.synchronize()
        assert capi.bspline_device_status(t.h) == 0


def test_mma_default_and_autotune():
    """16-bit tables default to the tensor-core variant for VGL/VGH (also in a general cell) once rows
    hold 512 orbitals (FP16) or more than 512 (BF16), shorter rows and V to DIRECT; the autotuner's
    candidates include it, and whatever it picks stays within the tolerances."""
    for dtype, N, variant in ((capi.F16, 448, capi.VARIANT_DIRECT), (capi.F16, 512, MMA),
                              (capi.BF16, 512, capi.VARIANT_DIRECT), (capi.BF16, 576, MMA)):
        with capi.Table((4, 4, 4), N, dtype) as t:
            assert capi.bspline_get_tuning(t.h, capi.VGH)["variant"] == variant, (dtype, N)
            assert capi.bspline_get_tuning(t.h, capi.V)["variant"] == capi.VARIANT_DIRECT
    grid, N = (10, 12, 9), 600
    coef = inputs.uniform_coefs(grid, N, seed=99)
    x, y, z = inputs.uniform_positions(300, seed=100)
    tab = _dequantised(coef, capi.F16)
    with capi.Table(grid, N, capi.F16) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        assert capi.bspline_get_tuning(t.h, capi.VGH)["variant"] == MMA
        assert capi.bspline_get_tuning(t.h, capi.VGL)["variant"] == MMA
        assert capi.bspline_get_tuning(t.h, capi.V)["variant"] == capi.VARIANT_DIRECT
        for kind in (capi.V, capi.VGL, capi.VGH):
            assert_parity(run_eval(t, kind, x, y, z), oracle.eval_periodic(kind, tab, x, y, z), kind)
        best = capi.bspline_tune(t.h, capi.VGH, 300)
        assert best["variant"] in (capi.VARIANT_DIRECT, capi.VARIANT_TMA, MMA)
        assert_parity(run_eval(t, capi.VGH, x, y, z), oracle.eval_periodic(capi.VGH, tab, x, y, z), capi.VGH)
        capi.bspline_set_tuning(t.h, capi.VGH)  # back to the default
        L = np.diag([1.5, 1.0, 2.0])
        capi.bspline_set_lattice(t.h, L)
        assert capi.bspline_get_tuning(t.h, capi.VGH)["variant"] == MMA
        r = np.stack([x, y, z], axis=1) @ L
        xr, yr, zr = (np.ascontiguousarray(r[:, d]) for d in range(3))
        assert_lattice_parity(run_eval(t, capi.VGH, xr, yr, zr), oracle.eval_lattice(capi.VGH, tab, L, xr, yr, zr),
                              lattice_bounds(tab, L, xr, yr, zr))
