"""FP64 CPU oracle for periodic tricubic B-spline orbital evaluation.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. It shares no code with the CUDA library and the CUDA library never
calls it.

The arithmetic lives in ``bspline_oracle.c`` (plain C11, double precision,
OpenMP over positions). This module only compiles it with gcc and marshals
numpy arrays through ctypes. Paper: Mathuriya et al., arXiv:1611.02665,
Sec. "QMC and B-spline-based SPOs", Eq. (SplineFunc) and Eq. (TricubicValue);
Sec. "Baseline and miniQMC", Fig. (baselineCode) for the V / VGL / VGH outputs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bspline_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_bspline.so")
_lock = threading.Lock()
_lib = None

V, VGL, VGH = 0, 1, 2
F16, BF16 = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: the same source builds on x86-64 and aarch64)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i, p, sz = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
        lib.orc_basis.argtypes = [d, p, p, p]
        lib.orc_centred_bspline.argtypes = [d, p]
        lib.orc_cell.argtypes = [d, i, p, p]
        for name in ("orc_eval_periodic", "orc_eval_padded", "orc_eval_bruteforce"):
            getattr(lib, name).argtypes = [i, i, i, i, i, p, i, p, p, p, p, p, p, p]
        lib.orc_pad.argtypes = [i, i, i, i, p, p]
        lib.orc_quantize.argtypes = [sz, i, p, i, p, p]
        lib.orc_dequantize.argtypes = [sz, i, p, p, i, p]
        lib.orc_num_threads.restype = i
        lib.orc_set_num_threads.argtypes = [i]
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def basis(t: float):
    """(w, dw, d2w): the four cubic pieces of Eq. (SplineFunc) at offset t and their t-derivatives."""
    w, dw, d2w = np.zeros(4), np.zeros(4), np.zeros(4)
    _load().orc_basis(float(t), _ptr(w), _ptr(dw), _ptr(d2w))
    return w, dw, d2w


def centred_bspline(s: float):
    """(B, B', B'') of the centred cubic B-spline at s."""
    out = np.zeros(3)
    _load().orc_centred_bspline(float(s), _ptr(out))
    return out


def cell(x: float, n: int):
    """(i, t): lower-bound cell index and offset of Eq. (SplineFunc) after periodic wrap."""
    i = ctypes.c_int(0)
    t = ctypes.c_double(0.0)
    _load().orc_cell(float(x), int(n), ctypes.byref(i), ctypes.byref(t))
    return i.value, t.value


def _eval(fn, kind, grid, table, x, y, z, N):
    nx, ny, nz = grid
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    npos = x.shape[0]
    table = np.ascontiguousarray(table, dtype=np.float64)
    v = np.zeros((npos, N))
    g = np.zeros((npos, 3, N)) if kind >= VGL else None
    h = np.zeros((npos, 6, N)) if kind == VGH else None
    lap = np.zeros((npos, N)) if kind >= VGL else None
    fn(kind, nx, ny, nz, N, _ptr(table), npos, _ptr(x), _ptr(y), _ptr(z),
       _ptr(v), _ptr(g), _ptr(h), _ptr(lap))
    out = {"v": v}
    if kind >= VGL:
        out["g"] = g
        out["l"] = lap
    if kind == VGH:
        out["h"] = h
    return out


def eval_periodic(kind, coef, x, y, z):
    """Eq. (TricubicValue) on a periodic table coef[nx][ny][nz][N] (knot indices mod n)."""
    nx, ny, nz, N = coef.shape
    return _eval(_load().orc_eval_periodic, kind, (nx, ny, nz), coef, x, y, z, N)


def eval_padded(kind, pad, x, y, z):
    """Eq. (TricubicValue) on a padded table [nx+3][ny+3][nz+3][N] (rows i..i+3, no wrap)."""
    px, py, pz, N = pad.shape
    return _eval(_load().orc_eval_padded, kind, (px - 3, py - 3, pz - 3), pad, x, y, z, N)


def eval_bruteforce(kind, coef, x, y, z):
    """Sum over every knot and periodic image with the closed-form centred B-spline (tiny grids)."""
    nx, ny, nz, N = coef.shape
    return _eval(_load().orc_eval_bruteforce, kind, (nx, ny, nz), coef, x, y, z, N)


def pad(coef):
    """Padded table with pad[a][b][c] = coef[(a-1) mod nx][(b-1) mod ny][(c-1) mod nz]."""
    nx, ny, nz, N = coef.shape
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    out = np.zeros((nx + 3, ny + 3, nz + 3, N))
    _load().orc_pad(nx, ny, nz, N, _ptr(coef), _ptr(out))
    return out


def quantize(table_f32, dtype):
    """(codes uint16, scale float32): per-orbital scale s_n = max|p| and round-to-nearest-even codes of p/s_n."""
    t = np.ascontiguousarray(table_f32, dtype=np.float32)
    N = t.shape[-1]
    cnt = t.size // N
    codes = np.zeros(t.shape, dtype=np.uint16)
    scale = np.zeros(N, dtype=np.float32)
    _load().orc_quantize(cnt, N, _ptr(t), int(dtype), _ptr(codes), _ptr(scale))
    return codes, scale


def dequantize(codes, scale, dtype):
    """Exact double value of each code times its orbital's scale."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    scale = np.ascontiguousarray(scale, dtype=np.float32)
    N = codes.shape[-1]
    out = np.zeros(codes.shape)
    _load().orc_dequantize(codes.size // N, N, _ptr(codes), _ptr(scale), int(dtype), _ptr(out))
    return out


def ratio_components(kind, out):
    """Per-orbital output components of `kind` in the library's order: V: v; VGL: v, g(3), l; VGH: v, g(3), h(6)."""
    comps = [out["v"]]
    if kind >= VGL:
        comps += [out["g"][:, d] for d in range(3)]
    if kind == VGL:
        comps.append(out["l"])
    if kind == VGH:
        comps += [out["h"][:, d] for d in range(6)]
    return comps


def ratio(kind, coef, x, y, z, u):
    """Determinant-ratio sums of Sec. "QMC and B-spline-based SPOs": r[p, q] = sum_n c_q(phi_n)(r_p) u[p, n].

    u[p, n] are the inverse entries that multiply phi_n (row e of A^-1 for A[n][i] = phi_n(r_i)).
    """
    out = eval_periodic(kind, coef, x, y, z)
    u = np.asarray(u, dtype=np.float64)
    return np.stack([np.einsum("pn,pn->p", c, u) for c in ratio_components(kind, out)], axis=1)


def interpolate(values):
    """Coefficients c[nx][ny][nz][N] of the periodic cubic B-spline that equals `values` at the grid points.

    At a knot the spline is the tensor product over axes of (c[j-1] + 4 c[j] + c[j+1]) / 6 (the knot
    weights of Eq. (SplineFunc)); that circulant is diagonal in the discrete Fourier basis with symbol
    (4 + 2 cos(2 pi k / n)) / 6, so the solve divides the 3-D FFT of the values by the product of the
    three symbols (numpy FFTs in double precision).
    """
    f = np.asarray(values, dtype=np.float64)
    nx, ny, nz = f.shape[:3]
    sym = [(4.0 + 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n)) / 6.0 for n in (nx, ny, nz)]
    den = sym[0][:, None, None, None] * sym[1][None, :, None, None] * sym[2][None, None, :, None]
    return np.real(np.fft.ifftn(np.fft.fftn(f, axes=(0, 1, 2)) / den, axes=(0, 1, 2)))


def eval_lattice(kind, coef, lattice, x, y, z):
    """Eq. (TricubicValue) in a general cell: Cartesian positions r, lattice vectors as rows of L.

    u = r L^-1 (fractional coordinates, then the periodic evaluation); derivatives by the chain rule:
    g = G g_u, H = G H_u G^T with G = L^-1, Laplacian = trace(H). numpy in double precision.
    """
    L = np.asarray(lattice, dtype=np.float64).reshape(3, 3)
    G = np.linalg.inv(L)
    r = np.stack([np.asarray(c, dtype=np.float64) for c in (x, y, z)], axis=1)
    u = r @ G
    out = eval_periodic(VGH if kind >= VGL else V, coef, u[:, 0].copy(), u[:, 1].copy(), u[:, 2].copy())
    res = {"v": out["v"]}
    if kind == V:
        return res
    res["g"] = np.einsum("id,pdn->pin", G, out["g"])
    hu = out["h"]
    H = np.empty((hu.shape[0], 3, 3, hu.shape[2]))
    for q, (a, b) in enumerate([(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]):
        H[:, a, b] = hu[:, q]
        H[:, b, a] = hu[:, q]
    Hc = np.einsum("id,pden,je->pijn", G, H, G)
    lap = Hc[:, 0, 0] + Hc[:, 1, 1] + Hc[:, 2, 2]
    if kind == VGL:
        res["l"] = lap
    else:
        res["h"] = np.stack([Hc[:, a, b] for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]], axis=1)
        res["l"] = lap
    return res
