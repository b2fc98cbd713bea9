"""Shared helpers for parity tests: tolerances, error metric, device input upload.

Tolerance (float32 paths vs the FP64 oracle): per output kind K,
max |gpu - oracle| / max |oracle_K| over all positions and orbitals must be at
most 2e-6 for values, 1e-5 for gradients (all three components together) and
5e-5 for Hessians (all six) and Laplacians.
"""
import numpy as np

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
