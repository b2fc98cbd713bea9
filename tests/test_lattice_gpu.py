"""GPU parity of evaluation in a general (non-orthorhombic) cell: bspline_set_lattice.

Eq. (TricubicValue) is defined on the fractional coordinates u = r L^-1 of a
Cartesian position r (lattice vectors as the rows of L); gradients and
Hessians come back Cartesian by the chain rule, g = G g_u and H = G H_u G^T
with G = L^-1, and the Laplacian is trace(H). The oracle is
oracle.eval_lattice, pinned on the CPU against Cartesian finite differences.

Tolerance, derived from the transform. The fractional outputs carry at most
the fractional path's error, TOL_K (parity_util) times the largest fractional
magnitude of their kind. With |G| the largest row sum of |G| and M = G^T G:
  g = G g_u             error <= |G| (TOL_g max|g_u| + rounding)
  H = G H_u G^T         error <= |G|^2 (TOL_h max|H_u| + rounding)
  L = sum M_de H_u,de   error <= sum |M| (TOL_h max|H_u| + rounding)
where the rounding of the float32 transform (G rounded to float, then 3 or 9
products summed) is a few units of 2^-24 of the same magnitudes. So the
error relative to the largest Cartesian magnitude is at most
(TOL_K + rounding) x |G|^k max|frac_K| / max|cart_K|, computed per case from
the oracle's fractional and Cartesian outputs (parity_util.lattice_bounds). V is
not transformed and keeps TOL_v.
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

# hexagonal a-b plane with a tilted c axis, and a triclinic cell with a negative off-diagonal
HEX = np.array([[1.3, 0.0, 0.0], [0.65, 1.1258330249197703, 0.0], [0.2, -0.3, 2.1]])
TRICLINIC = np.array([[2.0, 0.3, -0.4], [-0.5, 1.7, 0.2], [0.6, 0.4, 1.5]])
KIND_KEYS = {0: ["v"], 1: ["v", "g", "g", "g", "l"], 2: ["v", "g", "g", "g"] + ["h"] * 6}


def _cartesian_positions(npos, lattice, seed):
    """Fractional coordinates uniform over [-0.5, 1.5)^3 (so some wrap), mapped to Cartesian r = u L."""
    u = np.random.default_rng(seed).uniform(-0.5, 1.5, size=(npos, 3))
    r = u @ lattice
    return [np.ascontiguousarray(r[:, d]) for d in range(3)]


def _ref_table(coef, dtype):
    if dtype == capi.F32:
        return coef.astype(np.float64)
    codes, scale = oracle.quantize(coef, dtype)
    return oracle.dequantize(codes, scale, dtype)


@pytest.mark.parametrize("lattice", [HEX, TRICLINIC], ids=["hex", "triclinic"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("dtype,variant,stages", [(capi.F32, capi.VARIANT_DIRECT, 0), (capi.F32, capi.VARIANT_DIRECT, 4),
                                                  (capi.F16, capi.VARIANT_DIRECT, 0), (capi.F16, capi.VARIANT_MMA, 0),
                                                  (capi.BF16, capi.VARIANT_MMA, 0)])
@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_lattice_matches_oracle(kind, dtype, variant, stages, order, lattice):
    """FP32 on DIRECT with rows in registers (stages 0) and staged through the 4-unit ring, 16-bit tables
    on DIRECT and on the tensor-core variant."""
    grid, N, npos = (12, 10, 14), 200, 700
    coef = inputs.uniform_coefs(grid, N, seed=61)
    x, y, z = _cartesian_positions(npos, lattice, seed=62)
    shape = (variant, 512, 1, stages, order) if variant == capi.VARIANT_DIRECT else (variant, 128, 2, 0, order)
    with capi.Table(grid, N, dtype) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_lattice(t.h, lattice)
        capi.bspline_set_tuning(t.h, kind, *shape)
        got = run_eval(t, kind, x, y, z, ld=N + 4)
    ref_tab = _ref_table(coef, dtype)
    ref = oracle.eval_lattice(kind, ref_tab, lattice, x, y, z)
    assert_lattice_parity(got, ref, lattice_bounds(ref_tab, lattice, x, y, z),
                          label=f"kind {kind} dtype {dtype} shape {shape}")


@pytest.mark.parametrize("stages", [0, 3, 4])
@pytest.mark.parametrize("grid,N,npos,ppc", [((5, 7, 3), 37, 333, 2), ((9, 4, 6), 700, 129, 4),
                                             ((3, 3, 3), 1, 5, 1)])
def test_lattice_ragged(grid, N, npos, ppc, stages):
    """Ragged grids and orbital counts, several positions per CTA; rows in registers, or staged through a
    ring of 3 (the plain layout, also for short rows) or 4 units (the grouped layout for short rows)."""
    coef = inputs.uniform_coefs(grid, N, seed=63)
    x, y, z = _cartesian_positions(npos, TRICLINIC, seed=64)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_lattice(t.h, TRICLINIC)
        for kind in (capi.V, capi.VGL, capi.VGH):
            capi.bspline_set_tuning(t.h, kind, capi.VARIANT_DIRECT, 512, ppc, stages, 1)
            got = run_eval(t, kind, x, y, z)
            ref = oracle.eval_lattice(kind, coef.astype(np.float64), TRICLINIC, x, y, z)
            assert_lattice_parity(got, ref, lattice_bounds(coef.astype(np.float64), TRICLINIC, x, y, z),
                                  label=f"{grid} N={N} kind {kind}")


def test_identity_lattice_and_reset():
    """The unit cube as a lattice gives the fractional results bit for bit (V, VGH); None restores them."""
    grid, N, npos = (8, 9, 10), 130, 257
    coef = inputs.uniform_coefs(grid, N, seed=65)
    x, y, z = inputs.uniform_positions(npos, seed=66)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        base = {k: run_eval(t, k, x, y, z) for k in (capi.V, capi.VGL, capi.VGH)}
        capi.bspline_set_lattice(t.h, np.eye(3))
        for k in (capi.V, capi.VGH):
            got = run_eval(t, k, x, y, z)
            for key in got:
                np.testing.assert_array_equal(got[key], base[k][key])
        got = run_eval(t, capi.VGL, x, y, z)
        assert_parity(got, oracle.eval_periodic(capi.VGL, coef.astype(np.float64), x, y, z), capi.VGL)
        capi.bspline_set_lattice(t.h, HEX)
        assert not np.array_equal(run_eval(t, capi.VGH, x, y, z)["g"], base[capi.VGH]["g"])
        capi.bspline_set_lattice(t.h, None)
        for k in (capi.V, capi.VGL, capi.VGH):
            got = run_eval(t, k, x, y, z)
            for key in got:
                np.testing.assert_array_equal(got[key], base[k][key])


@pytest.mark.parametrize("kind", [capi.V, capi.VGL, capi.VGH])
def test_lattice_ratio(kind):
    """Fused determinant-ratio sums in a general cell; bound as in the fractional ratio test."""
    grid, N, npos = (11, 13, 9), 300, 400
    coef = inputs.uniform_coefs(grid, N, seed=67)
    x, y, z = _cartesian_positions(npos, HEX, seed=68)
    u = (np.random.default_rng(69).normal(size=(npos, N)) / np.sqrt(N)).astype(np.float32)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_lattice(t.h, HEX)
        capi.bspline_set_tuning(t.h, kind, capi.VARIANT_DIRECT, 512, 1, 0, 1)
        dx, dy, dz, du = to_device(x, y, z, u)
        r = torch.full((npos, capi.NCOMP[kind]), float("nan"), device="cuda")
        capi.bspline_eval_ratio(t.h, kind, npos, dx, dy, dz, du, N, r)
        torch.cuda.synchronize()
        got = r.cpu().numpy().astype(np.float64)
    out = oracle.eval_lattice(kind, coef.astype(np.float64), HEX, x, y, z)
    bounds = lattice_bounds(coef.astype(np.float64), HEX, x, y, z)  # per-orbital relative bounds
    comps = oracle.ratio_components(kind, out)
    u64 = u.astype(np.float64)
    au = np.abs(u64).sum(axis=1)
    for q, (c, key) in enumerate(zip(comps, KIND_KEYS[kind])):
        ref = np.einsum("pn,pn->p", c, u64)
        bound = bounds[key] * np.abs(out[key]).max() * au + 32 * 2.0 ** -24 * np.einsum("pn,pn->p", np.abs(c),
                                                                                         np.abs(u64))
        err = np.abs(got[:, q] - ref)
        assert (err <= bound).all(), f"component {q}: max err/bound {(err / bound).max():.3f}"


def test_lattice_host_buffers():
    grid, N, npos = (7, 8, 9), 64, 300
    coef = inputs.uniform_coefs(grid, N, seed=70)
    x, y, z = _cartesian_positions(npos, TRICLINIC, seed=71)
    with capi.Table(grid, N, capi.F32) as t:
        capi.bspline_set_coefs(t.h, torch.from_numpy(coef).cuda())
        capi.bspline_set_lattice(t.h, TRICLINIC)
        v = np.zeros((npos, N), np.float32)
        g = np.zeros((npos, 3, N), np.float32)
        h = np.zeros((npos, 6, N), np.float32)
        capi.bspline_eval_host(t.h, capi.VGH, npos, x, y, z, v, g, h, N)
    ref = oracle.eval_lattice(capi.VGH, coef.astype(np.float64), TRICLINIC, x, y, z)
    assert_lattice_parity({"v": v, "g": g, "h": h}, ref,
                          lattice_bounds(coef.astype(np.float64), TRICLINIC, x, y, z))


def test_lattice_errors():
    with capi.Table((4, 5, 6), 16, capi.F32) as t:
        for bad in (np.zeros((3, 3)), np.array([[1, 0, 0], [0, 1, 0], [1, 1, 0.0]]),
                    np.array([[np.nan, 0, 0], [0, 1, 0], [0, 0, 1.0]]),
                    np.array([[np.inf, 0, 0], [0, 1, 0], [0, 0, 1.0]])):
            with pytest.raises(capi.BsplineError) as e:
                capi.bspline_set_lattice(t.h, bad)
            assert e.value.status == capi.ERR_ARG
        coef = torch.from_numpy(inputs.uniform_coefs((4, 5, 6), 16, seed=72)).cuda()
        capi.bspline_set_coefs(t.h, coef)
        capi.bspline_set_lattice(t.h, HEX)
        x, y, z = to_device(*inputs.uniform_positions(8, seed=73))
        v, g, hl = t.outputs(capi.VGH, 8)
        capi.bspline_set_tuning(t.h, capi.VGH, capi.VARIANT_TMA, 256, 1, 0, 0)
        with pytest.raises(capi.BsplineError) as e:
            t.eval(capi.VGH, x, y, z, v, g, hl)
        assert e.value.status == capi.ERR_UNSUPPORTED
        capi.bspline_set_tuning(t.h, capi.VGH)
        t.eval(capi.VGH, x, y, z, v, g, hl)
        item = {"table": t.h, "npos": 8, "x": x, "y": y, "z": z, "v": v, "g": g, "hl": hl, "ld": 16}
        for call in (capi.bspline_eval_batched, capi.bspline_eval_batched_noalloc):
            with pytest.raises(capi.BsplineError) as e:
                call([item], capi.VGH)
            assert e.value.status == capi.ERR_UNSUPPORTED
        with pytest.raises(capi.BsplineError) as e:
            capi.bspline_plan_create([item], capi.VGH)
        assert e.value.status == capi.ERR_UNSUPPORTED
        torch.cuda.synchronize()
        assert capi.bspline_device_status(t.h) == 0
