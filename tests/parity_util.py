"""Shared helpers for parity tests: tolerances, error metric, device input upload.

Tolerance (float32 paths vs the FP64 oracle): per output kind K,
max |gpu - oracle| / max |oracle_K| over all positions and orbitals must be at
most 2e-6 for values, 1e-5 for gradients (all three components together) and
5e-5 for Hessians (all six) and Laplacians.

In a general cell (Cartesian outputs g = G g_u, H = G H_u G^T, L = trace H with G = L^-1), the bound
follows from the transform: the fractional outputs carry at most TOL_K of their largest magnitude,
and the float32 transform adds a few units of 2^-24, so relative to the largest Cartesian magnitude
the error is at most (TOL_K + rounding) x |G|^k max|frac_K| / max|cart_K| (lattice_bounds), with |G|
the largest row sum of |G| (k = 1 for gradients, 2 for Hessians; the Laplacian takes sum |G^T G|).
"""
import numpy as np

import oracle

TOL = {"v": 2e-6, "g": 1e-5, "h": 5e-5, "l": 5e-5}
KEYS = {0: ("v",), 1: ("v", "g", "l"), 2: ("v", "g", "h")}


def rel_errors(gpu, ref, keys):
    out = {}
    for k in keys:
        r = np.asarray(ref[k], dtype=np.float64)
        g = np.asarray(gpu[k], dtype=np.float64)
        denom = np.abs(r).max()
        out[k] = float(np.abs(g - r).max() / (denom if denom > 0 else 1.0))
    return out


def assert_parity(gpu, ref, kind, scale=1.0, label=""):
    errs = rel_errors(gpu, ref, KEYS[kind])
    for k, e in errs.items():
        assert e <= TOL[k] * scale, f"{label} {k}: rel err {e:.3e} > {TOL[k] * scale:.1e} (all: {errs})"
    return errs


def to_device(*arrays):
    import torch
    return [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in arrays]


def run_eval(table, kind, x, y, z, ld=None, npos=None):
    """Evaluate through the C ABI on device tensors; returns numpy dict trimmed to N."""
    import torch
    from paper_1611_02665_gb300 import capi
    N = table.N
    ld = N if ld is None else ld
    dx, dy, dz = to_device(x, y, z)
    npos = dx.shape[0] if npos is None else npos
    v, g, hl = table.outputs(kind, npos, ld)
    table.eval(kind, dx, dy, dz, v, g, hl, ld)
    torch.cuda.synchronize()
    assert capi.bspline_device_status(table.h) == 0
    out = {"v": v.cpu().numpy()[:, :N]}
    if kind >= 1:
        out["g"] = g.cpu().numpy()[:, :, :N]
    if kind == 1:
        out["l"] = hl.cpu().numpy()[:, :N]
    if kind == 2:
        out["h"] = hl.cpu().numpy()[:, :, :N]
    return out


def assert_rounding_bound(gpu, ref, kind, pmax, grid, label=""):
    """Float32 summation bound for fields whose derivatives cancel heavily.

    Each output is a sum of 64 products W_x W_y W_z p. With |p| <= pmax the sum
    of |terms| is at most pmax for values, n * pmax for first derivatives
    (sum |dW| <= 1 per axis before the n scale) and 4 n^2 pmax for second
    derivatives (sum |d2W| <= 4), n the largest grid count. The float32 result
    may differ from the exact one by a small multiple of 2^-24 of that sum; 32
    ulps of headroom covers the factorised summation depth (about 10 roundings)
    and the rounded weights.
    """
    n = max(grid)
    eps = 2.0 ** -24
    bound = {"v": 32 * eps * pmax, "g": 32 * eps * n * pmax, "h": 32 * eps * 4 * n * n * pmax,
             "l": 32 * eps * 12 * n * n * pmax}
    for k in KEYS[kind]:
        err = np.abs(np.asarray(gpu[k], np.float64) - np.asarray(ref[k], np.float64)).max()
        assert err <= bound[k], f"{label} {k}: abs err {err:.3e} > bound {bound[k]:.3e}"


def lattice_bounds(ref_tab, lattice, x, y, z):
    """Per-kind relative error bounds of Cartesian outputs (see the module docstring)."""
    G = np.linalg.inv(np.asarray(lattice, dtype=np.float64))
    r = np.stack([x, y, z], axis=1)
    u = r @ G
    frac = oracle.eval_periodic(oracle.VGH, ref_tab, *(np.ascontiguousarray(u[:, d]) for d in range(3)))
    cart = oracle.eval_lattice(oracle.VGH, ref_tab, lattice, x, y, z)
    gnorm = np.abs(G).sum(axis=1).max()
    msum = np.abs(G.T @ G).sum()
    eps = 2.0 ** -24
    return {"v": TOL["v"],
            "g": (TOL["g"] + 4 * eps) * gnorm * np.abs(frac["g"]).max() / np.abs(cart["g"]).max(),
            "h": (TOL["h"] + 12 * eps) * gnorm ** 2 * np.abs(frac["h"]).max() / np.abs(cart["h"]).max(),
            "l": (TOL["h"] + 12 * eps) * msum * np.abs(frac["h"]).max() / np.abs(cart["l"]).max()}


def assert_lattice_parity(got, ref, bounds, label=""):
    for k in got:
        err = np.abs(np.asarray(got[k], np.float64) - ref[k]).max() / np.abs(ref[k]).max()
        assert err <= bounds[k], f"{label} {k}: rel err {err:.3e} > derived bound {bounds[k]:.3e}"
