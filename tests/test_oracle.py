"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

Each check below is independent of the oracle's own stencil code: textbook
rational values, closed-form sums written with numpy, exact polynomial
reproduction, a brute-force sum over every knot, finite differences,
periodicity and library rounding. A plausible mistake in the oracle (a wrong
piece, sign, derivative factor, stencil offset or wrap) fails at least one.
Paper: arXiv:1611.02665, Sec. "QMC and B-spline-based SPOs", Eq. (SplineFunc)
and Eq. (TricubicValue).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1611_02665_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_basis_golden():
    rows = []
    with open(os.path.join(GOLDEN, "cubic_bspline_basis.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = [p.split() for p in line.split("|")]
            t = float(Fraction(parts[0][0]))
            vals = [np.array([float(Fraction(s)) for s in p]) for p in parts[1:]]
            rows.append((t, *vals))
    return rows


def test_basis_matches_golden_rationals():
    rows = _read_basis_golden()
    assert len(rows) == 4
    for t, w, dw, d2w in rows:
        ow, odw, od2w = oracle.basis(t)
        np.testing.assert_allclose(ow, w, rtol=0, atol=1e-15)
        np.testing.assert_allclose(odw, dw, rtol=0, atol=1e-15)
        np.testing.assert_allclose(od2w, d2w, rtol=0, atol=1e-15)


def test_basis_partition_of_unity():
    for t in np.random.default_rng(0).random(200):
        w, dw, d2w = oracle.basis(t)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(dw.sum()) < 1e-15
        assert abs(d2w.sum()) < 1e-14
        assert (w >= 0).all()


def test_basis_c2_across_knot():
    # At t=1 the interval ends on knot i+1; piece a there is piece a-1 of the next interval at t=0.
    w1, dw1, d2w1 = oracle.basis(1.0)
    w0, dw0, d2w0 = oracle.basis(0.0)
    for a in range(1, 4):
        assert abs(w1[a] - w0[a - 1]) < 1e-15
        assert abs(dw1[a] - dw0[a - 1]) < 1e-15
        assert abs(d2w1[a] - d2w0[a - 1]) < 1e-15
    assert abs(w1[0]) < 1e-15 and abs(dw1[0]) < 1e-15 and abs(d2w1[0]) < 1e-15


def test_basis_is_derivative_of_itself():
    # dw and d2w are the t-derivatives of w (central differences of the pieces).
    eps = 1e-6
    for t in np.random.default_rng(1).uniform(0.01, 0.99, 50):
        wp, dwp, _ = oracle.basis(t + eps)
        wm, dwm, _ = oracle.basis(t - eps)
        _, dw, d2w = oracle.basis(t)
        np.testing.assert_allclose((wp - wm) / (2 * eps), dw, atol=1e-9)
        np.testing.assert_allclose((dwp - dwm) / (2 * eps), d2w, atol=1e-9)


def test_centred_bspline_unit_mass_and_variance():
    # B is four unit boxes convolved: integral 1, second moment 4 * (1/12) = 1/3.
    s = np.linspace(-2.5, 2.5, 500001)
    b = np.array([oracle.centred_bspline(v)[0] for v in s[::50]])
    ds = s[50] - s[0]
    assert abs(np.trapezoid(b, dx=ds) - 1.0) < 1e-6
    assert abs(np.trapezoid(b * s[::50] ** 2, dx=ds) - 1.0 / 3.0) < 1e-6


@pytest.mark.parametrize("x,n,i,t", [
    (0.5, 16, 8, 0.0), (0.0, 16, 0, 0.0), (1.0, 16, 0, 0.0), (1.25, 16, 4, 0.0),
    (-0.25, 16, 12, 0.0), (-1e-20, 16, 0, 0.0), (0.53125, 16, 8, 0.5), (2.0 - 2**-40, 48, 47, None),
])
def test_cell_reduction(x, n, i, t):
    ci, ct = oracle.cell(x, n)
    assert ci == i
    assert 0.0 <= ct < 1.0
    if t is not None:
        assert ct == t


@pytest.mark.parametrize("grid,N", [((4, 4, 4), 3), ((5, 4, 6), 2), ((4, 5, 5), 3)])
@pytest.mark.parametrize("kind", [oracle.V, oracle.VGL, oracle.VGH])
def test_stencil_matches_bruteforce(grid, N, kind):
    coef = inputs.uniform_coefs(grid, N, seed=11)
    x, y, z = inputs.uniform_positions(40, seed=12)
    a = oracle.eval_periodic(kind, coef, x, y, z)
    b = oracle.eval_bruteforce(kind, coef, x, y, z)
    for key in a:
        scale = max(1.0, np.abs(b[key]).max())
        np.testing.assert_allclose(a[key], b[key], rtol=0, atol=1e-12 * scale)


def test_padded_equals_periodic():
    coef = inputs.uniform_coefs((5, 6, 7), 5, seed=3)
    pad = oracle.pad(coef)
    # pad[a] holds knot (a-1) mod n: check three planes by hand.
    np.testing.assert_array_equal(pad[0, 1:7, 1:8], coef[4])
    np.testing.assert_array_equal(pad[1:6, 1:7, 1:8], coef)
    np.testing.assert_array_equal(pad[6:8, 1:7, 1:8], coef[0:2])
    x, y, z = inputs.uniform_positions(30, seed=4)
    a = oracle.eval_periodic(oracle.VGH, coef, x, y, z)
    b = oracle.eval_padded(oracle.VGH, pad, x, y, z)
    for key in a:
        np.testing.assert_array_equal(a[key], b[key])


def _knot_field(grid, N, f):
    """Padded table whose row (a,b,c) holds f at knot ((a-1)/nx, (b-1)/ny, (c-1)/nz), for N copies."""
    nx, ny, nz = grid
    kx = (np.arange(nx + 3) - 1.0) / nx
    ky = (np.arange(ny + 3) - 1.0) / ny
    kz = (np.arange(nz + 3) - 1.0) / nz
    X, Y, Z = np.meshgrid(kx, ky, kz, indexing="ij")
    vals = f(X, Y, Z)
    return np.repeat(vals[..., None], N, axis=-1)


def test_linear_fields_exact():
    grid = (6, 7, 5)
    c0, cx, cy, cz = 0.3, -1.7, 2.1, 0.9
    pad = _knot_field(grid, 2, lambda X, Y, Z: c0 + cx * X + cy * Y + cz * Z)
    x, y, z = inputs.uniform_positions(50, seed=5)
    out = oracle.eval_padded(oracle.VGH, pad, x, y, z)
    np.testing.assert_allclose(out["v"][:, 0], c0 + cx * x + cy * y + cz * z, atol=1e-13)
    for d, c in enumerate((cx, cy, cz)):
        np.testing.assert_allclose(out["g"][:, d, 0], c, atol=1e-12)
    np.testing.assert_allclose(out["h"], 0.0, atol=1e-10)


def test_quadratic_fields_with_variance_shift():
    # Cubic B-spline moments: sum_j (s-j)^2 B(s-j) = 1/3, so knot values x_j^2 give x^2 + h^2/3.
    grid = (8, 6, 10)
    h2 = [1.0 / g ** 2 for g in grid]
    x, y, z = inputs.uniform_positions(50, seed=6)
    pad = _knot_field(grid, 1, lambda X, Y, Z: X * X + Y * Y + Z * Z)
    out = oracle.eval_padded(oracle.VGH, pad, x, y, z)
    np.testing.assert_allclose(out["v"][:, 0], x * x + y * y + z * z + sum(h2) / 3.0, atol=1e-13)
    np.testing.assert_allclose(out["g"][:, 0, 0], 2 * x, atol=1e-12)
    np.testing.assert_allclose(out["g"][:, 1, 0], 2 * y, atol=1e-12)
    np.testing.assert_allclose(out["g"][:, 2, 0], 2 * z, atol=1e-12)
    np.testing.assert_allclose(out["h"][:, [0, 3, 5], 0], 2.0, atol=1e-10)
    np.testing.assert_allclose(out["h"][:, [1, 2, 4], 0], 0.0, atol=1e-10)
    # The same shift written as a correction: knot values x_j^2/2 - h^2/6 reproduce x^2/2 exactly.
    pad = _knot_field(grid, 1, lambda X, Y, Z: 0.5 * X * X - h2[0] / 6.0)
    out = oracle.eval_padded(oracle.V, pad, x, y, z)
    np.testing.assert_allclose(out["v"][:, 0], 0.5 * x * x, atol=1e-13)
    # Mixed products have no shift (the first moment vanishes).
    pad = _knot_field(grid, 1, lambda X, Y, Z: X * Y)
    out = oracle.eval_padded(oracle.VGH, pad, x, y, z)
    np.testing.assert_allclose(out["v"][:, 0], x * y, atol=1e-13)
    np.testing.assert_allclose(out["g"][:, 0, 0], y, atol=1e-12)
    np.testing.assert_allclose(out["g"][:, 1, 0], x, atol=1e-12)
    np.testing.assert_allclose(out["h"][:, 1, 0], 1.0, atol=1e-10)
    np.testing.assert_allclose(out["h"][:, [0, 2, 3, 4, 5], 0], 0.0, atol=1e-10)


def test_knot_closed_forms():
    # At a knot (t = 0 on every axis) the stencil reduces to the textbook three-point forms:
    # value (c_{j-1} + 4 c_j + c_{j+1})/6, slope (c_{j+1} - c_{j-1})/(2h), curvature (c_{j-1} - 2c_j + c_{j+1})/h^2,
    # tensorised over the three axes.
    grid = (6, 5, 7)
    nx, ny, nz = grid
    coef = inputs.uniform_coefs(grid, 3, seed=7).astype(np.float64)
    rng = np.random.default_rng(8)
    idx = rng.integers(0, [nx, ny, nz], size=(20, 3))
    x, y, z = idx[:, 0] / nx, idx[:, 1] / ny, idx[:, 2] / nz
    out = oracle.eval_periodic(oracle.VGH, coef, x, y, z)

    def op(c, axis, kind, n):
        m, p = np.roll(c, 1, axis), np.roll(c, -1, axis)  # c_{j-1}, c_{j+1}
        if kind == 0:
            return (m + 4 * c + p) / 6.0
        if kind == 1:
            return (p - m) * n / 2.0
        return (m - 2 * c + p) * n * n

    def field(kx, ky, kz):
        f = op(coef, 0, kx, nx)
        f = op(f, 1, ky, ny)
        return op(f, 2, kz, nz)

    sel = (idx[:, 0], idx[:, 1], idx[:, 2])
    np.testing.assert_allclose(out["v"], field(0, 0, 0)[sel], atol=1e-13)
    for d, o in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        np.testing.assert_allclose(out["g"][:, d], field(*o)[sel], atol=1e-12)
    for d, o in enumerate([(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]):
        np.testing.assert_allclose(out["h"][:, d], field(*o)[sel], atol=1e-10)


def test_periodicity():
    coef = inputs.uniform_coefs((5, 7, 6), 4, seed=9).astype(np.float64)
    x, y, z = inputs.uniform_positions(30, seed=10)
    base = oracle.eval_periodic(oracle.VGH, coef, x, y, z)
    for sx, sy, sz in [(1, 0, 0), (0, -1, 0), (0, 0, 3), (-2, 1, 1)]:
        sh = oracle.eval_periodic(oracle.VGH, coef, x + sx, y + sy, z + sz)
        for key in base:
            np.testing.assert_allclose(sh[key], base[key], rtol=0, atol=1e-9 * np.abs(base[key]).max())


def test_finite_differences():
    grid = (8, 7, 9)
    coef = inputs.uniform_coefs(grid, 3, seed=13).astype(np.float64)
    rng = np.random.default_rng(14)
    # keep away from knots so every difference stencil stays inside one cubic piece
    cells = rng.integers(0, grid, size=(25, 3))
    frac = rng.uniform(0.05, 0.95, size=(25, 3))
    r = (cells + frac) / np.array(grid)
    out = oracle.eval_periodic(oracle.VGH, coef, r[:, 0], r[:, 1], r[:, 2])

    def V(dr):
        q = r + dr
        return oracle.eval_periodic(oracle.V, coef, q[:, 0], q[:, 1], q[:, 2])["v"]

    e = np.eye(3)
    h1 = 1e-6
    gmax = np.abs(out["g"]).max()
    for d in range(3):
        fd = (V(h1 * e[d]) - V(-h1 * e[d])) / (2 * h1)
        np.testing.assert_allclose(out["g"][:, d], fd, atol=1e-7 * gmax)
    h2 = 1e-4
    hmax = np.abs(out["h"]).max()
    pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    v0 = V(0 * e[0])
    for q, (a, b) in enumerate(pairs):
        if a == b:
            fd = (V(h2 * e[a]) - 2 * v0 + V(-h2 * e[a])) / h2 ** 2
        else:
            fd = (V(h2 * (e[a] + e[b])) - V(h2 * (e[a] - e[b])) - V(h2 * (e[b] - e[a]))
                  + V(-h2 * (e[a] + e[b]))) / (4 * h2 * h2)
        np.testing.assert_allclose(out["h"][:, q], fd, atol=1e-6 * hmax)
    np.testing.assert_allclose(out["l"], out["h"][:, 0] + out["h"][:, 3] + out["h"][:, 5], atol=1e-9)


def test_vgl_and_v_agree_with_vgh():
    coef = inputs.uniform_coefs((6, 6, 6), 4, seed=15).astype(np.float64)
    x, y, z = inputs.uniform_positions(20, seed=16)
    vgh = oracle.eval_periodic(oracle.VGH, coef, x, y, z)
    vgl = oracle.eval_periodic(oracle.VGL, coef, x, y, z)
    v = oracle.eval_periodic(oracle.V, coef, x, y, z)
    np.testing.assert_array_equal(v["v"], vgh["v"])
    np.testing.assert_array_equal(vgl["g"], vgh["g"])
    np.testing.assert_allclose(vgl["l"], vgh["h"][:, 0] + vgh["h"][:, 3] + vgh["h"][:, 5], rtol=1e-14,
                               atol=1e-12)


@pytest.mark.parametrize("dtype", [oracle.F16, oracle.BF16])
def test_quantize_matches_library_rounding(dtype):
    import torch

    p = inputs.uniform_coefs((4, 5, 3), 7, seed=17) * np.float32(3.0)
    p[..., 2] = 0.0  # an all-zero orbital takes scale 1
    codes, scale = oracle.quantize(p, dtype)
    s = np.abs(p).reshape(-1, 7).max(axis=0)
    s[s == 0] = 1.0
    np.testing.assert_array_equal(scale, s.astype(np.float32))
    q = (p / s.astype(np.float32)).astype(np.float32)
    if dtype == oracle.F16:
        ref = q.astype(np.float16).view(np.uint16)
    else:
        ref = torch.from_numpy(q).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(codes, ref)
    deq = oracle.dequantize(codes, scale, dtype)
    if dtype == oracle.F16:
        back = ref.view(np.float16).astype(np.float64) * s.astype(np.float32).astype(np.float64)
    else:
        back = torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16).double().numpy() * s.astype(
            np.float32).astype(np.float64)
    np.testing.assert_array_equal(deq, back)


def test_ratio_is_determinant_ratio():
    # Matrix determinant lemma: replacing electron e's column of the Slater matrix A[n][i] = phi_n(r_i)
    # changes det(A) by the factor sum_n (A^-1)[e][n] phi_n(r'), the paper's ratio formula; its gradient
    # in r' is the same sum over grad phi_n (checked by central differences of the determinant ratio).
    grid, N = (5, 6, 4), 6
    coef = inputs.uniform_coefs(grid, N, seed=31).astype(np.float64)
    x, y, z = inputs.uniform_positions(N, seed=32)
    A = oracle.eval_periodic(oracle.V, coef, x, y, z)["v"].T  # [orbital n][electron i]
    Ainv = np.linalg.inv(A)
    rng = np.random.default_rng(33)
    moves = rng.random((4, 3))
    for e, (xn, yn, zn) in zip([0, 2, 5, 3], moves):
        u = Ainv[e][None, :]
        got = oracle.ratio(oracle.VGL, coef, [xn], [yn], [zn], u)[0]

        def det_ratio(px, py, pz):
            A2 = A.copy()
            A2[:, e] = oracle.eval_periodic(oracle.V, coef, [px], [py], [pz])["v"][0]
            return np.linalg.det(A2) / np.linalg.det(A)

        assert abs(got[0] - det_ratio(xn, yn, zn)) < 1e-10 * max(1.0, abs(got[0]))
        h = 1e-6
        fd = [(det_ratio(*(np.array([xn, yn, zn]) + h * d)) - det_ratio(*(np.array([xn, yn, zn]) - h * d))) / (2 * h)
              for d in np.eye(3)]
        np.testing.assert_allclose(got[1:4], fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(got[1:4]).max()))


@pytest.mark.parametrize("grid", [(5, 7, 6), (1, 2, 3), (8, 8, 8)])
def test_interpolation_reproduces_samples(grid):
    # The coefficients from oracle.interpolate make the spline (evaluated by the stencil code)
    # equal the samples at every grid point.
    N = 3
    f = inputs.uniform_coefs(grid, N, seed=51).astype(np.float64)
    c = oracle.interpolate(f)
    nx, ny, nz = grid
    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    out = oracle.eval_periodic(oracle.V, c, (I / nx).ravel(), (J / ny).ravel(), (K / nz).ravel())
    np.testing.assert_allclose(out["v"], f.reshape(-1, N), atol=1e-12)


def test_interpolation_matches_dense_solve():
    # Same coefficients as solving the Kronecker product of the three circulant knot matrices.
    grid, N = (4, 5, 3), 2
    f = inputs.uniform_coefs(grid, N, seed=52).astype(np.float64)

    def circ(n):
        m = np.zeros((n, n))
        for j in range(n):
            m[j, (j - 1) % n] += 1 / 6
            m[j, j] += 4 / 6
            m[j, (j + 1) % n] += 1 / 6
        return m

    K = np.kron(np.kron(circ(grid[0]), circ(grid[1])), circ(grid[2]))
    c = np.linalg.solve(K, f.reshape(-1, N)).reshape(f.shape)
    np.testing.assert_allclose(oracle.interpolate(f), c, atol=1e-12)


SKEWED = np.array([[1.3, 0.0, 0.0], [0.65, 1.1258330249197703, 0.0], [0.2, -0.3, 2.1]])


def test_lattice_derivatives_match_cartesian_finite_differences():
    coef = inputs.uniform_coefs((7, 6, 8), 3, seed=71).astype(np.float64)
    rng = np.random.default_rng(72)
    u = rng.uniform(0.05, 0.95, size=(20, 3))
    u = (np.floor(u * [7, 6, 8]) + rng.uniform(0.1, 0.9, size=(20, 3))) / [7, 6, 8]  # away from knots
    r = u @ SKEWED
    out = oracle.eval_lattice(oracle.VGH, coef, SKEWED, r[:, 0], r[:, 1], r[:, 2])

    def V(dr):
        q = r + dr
        return oracle.eval_lattice(oracle.V, coef, SKEWED, q[:, 0], q[:, 1], q[:, 2])["v"]

    e = np.eye(3)
    h1, h2 = 1e-6, 1e-4
    for d in range(3):
        np.testing.assert_allclose(out["g"][:, d], (V(h1 * e[d]) - V(-h1 * e[d])) / (2 * h1),
                                   atol=1e-7 * np.abs(out["g"]).max())
    v0 = V(0 * e[0])
    for q, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        if a == b:
            fd = (V(h2 * e[a]) - 2 * v0 + V(-h2 * e[a])) / h2 ** 2
        else:
            fd = (V(h2 * (e[a] + e[b])) - V(h2 * (e[a] - e[b])) - V(h2 * (e[b] - e[a]))
                  + V(-h2 * (e[a] + e[b]))) / (4 * h2 * h2)
        np.testing.assert_allclose(out["h"][:, q], fd, atol=1e-6 * np.abs(out["h"]).max())
    np.testing.assert_allclose(out["l"], out["h"][:, 0] + out["h"][:, 3] + out["h"][:, 5], atol=1e-9)
    vgl = oracle.eval_lattice(oracle.VGL, coef, SKEWED, r[:, 0], r[:, 1], r[:, 2])
    np.testing.assert_allclose(vgl["l"], out["l"], atol=1e-9)


def test_lattice_special_cases():
    coef = inputs.uniform_coefs((5, 6, 7), 2, seed=73).astype(np.float64)
    x, y, z = inputs.uniform_positions(15, seed=74)
    frac = oracle.eval_periodic(oracle.VGH, coef, x, y, z)
    ident = oracle.eval_lattice(oracle.VGH, coef, np.eye(3), x, y, z)
    for k in ("v", "g", "h"):
        np.testing.assert_allclose(ident[k], frac[k], atol=1e-10)
    a, b, c = 2.0, 3.0, 0.5  # orthorhombic: d/dx = (1/a) d/du0 etc.
    ortho = oracle.eval_lattice(oracle.VGH, coef, np.diag([a, b, c]), a * x, b * y, c * z)
    np.testing.assert_allclose(ortho["g"][:, 0], frac["g"][:, 0] / a, atol=1e-10)
    np.testing.assert_allclose(ortho["h"][:, 4], frac["h"][:, 4] / (b * c), atol=1e-8)
    # lattice translations leave everything unchanged
    r = np.stack([x, y, z], axis=1) @ SKEWED
    base = oracle.eval_lattice(oracle.VGH, coef, SKEWED, r[:, 0], r[:, 1], r[:, 2])
    shifted = r + SKEWED[0] - 2 * SKEWED[2]
    sh = oracle.eval_lattice(oracle.VGH, coef, SKEWED, shifted[:, 0], shifted[:, 1], shifted[:, 2])
    for k in ("v", "g", "h"):
        np.testing.assert_allclose(sh[k], base[k], atol=1e-8 * np.abs(base[k]).max())
