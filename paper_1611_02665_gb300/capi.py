"""Thin ctypes binding of the C ABI declared in ``include/bspline_gb300.h``.

Every function here has the name of the C entry point it calls and only
marshals arguments: torch tensors (device memory, streams) or numpy arrays
(host memory) become raw pointers and sizes. All arithmetic runs in the CUDA
library. If the library has not been built, every call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB_PATH

F32, F16, BF16 = 0, 1, 2
V, VGL, VGH = 0, 1, 2
VARIANT_AUTO, VARIANT_DIRECT, VARIANT_TMA, VARIANT_MMA = 0, 1, 2, 3
NCOMP = {V: 1, VGL: 5, VGH: 10}

OK = 0
ERR_ARG, ERR_ALLOC, ERR_CUDA, ERR_DTYPE, ERR_STATE, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_BOUNDS = 1, 2, 3, 4, 5, 6, 7, 8


class BsplineError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {bspline_status_str(status)} (status {status})")


class bspline_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("N", ctypes.c_int),
                ("Npad", ctypes.c_int), ("dtype", ctypes.c_int), ("table_bytes", ctypes.c_size_t),
                ("has_coefs", ctypes.c_int)]


class bspline_tuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("nb", ctypes.c_int), ("ppc", ctypes.c_int), ("stages", ctypes.c_int),
                ("order", ctypes.c_int)]

    def as_dict(self):
        return {"variant": self.variant, "nb": self.nb, "ppc": self.ppc, "stages": self.stages, "order": self.order}


class bspline_batch_item(ctypes.Structure):
    _fields_ = [("table", ctypes.c_void_p), ("npos", ctypes.c_int),
                ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("g", ctypes.c_void_p), ("hl", ctypes.c_void_p), ("ld", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_P, _I, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p
_SIGS = {
    "bspline_abi_version": ([], _I),
    "bspline_status_str": ([_I], _S),
    "bspline_create": ([_I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "bspline_destroy": ([_P], _I),
    "bspline_set_coefs": ([_P, _P, _I, _P], _I),
    "bspline_set_coefs_padded": ([_P, _P, _I, _P], _I),
    "bspline_set_values": ([_P, _P, _I, _P], _I),
    "bspline_set_lattice": ([_P, _P], _I),
    "bspline_get_info": ([_P, ctypes.POINTER(bspline_info)], _I),
    "bspline_get_table": ([_P, _P, _P], _I),
    "bspline_eval_v": ([_P, _I, _P, _P, _P, _P, _I, _P], _I),
    "bspline_eval_vgl": ([_P, _I, _P, _P, _P, _P, _P, _P, _I, _P], _I),
    "bspline_eval_vgh": ([_P, _I, _P, _P, _P, _P, _P, _P, _I, _P], _I),
    "bspline_eval_host": ([_P, _I, _I, _P, _P, _P, _P, _P, _P, _I], _I),
    "bspline_eval_ratio": ([_P, _I, _I, _P, _P, _P, _P, _I, _P, _P], _I),
    "bspline_device_status": ([_P, _P, _I], _I),
    "bspline_set_host_mode": ([_P, _I], _I),
    "bspline_selftest_wait_timeout": ([_P, _I, _P], _I),
    "bspline_measure_read_bandwidth": ([ctypes.c_size_t, _I, ctypes.POINTER(ctypes.c_double), _P], _I),
    "bspline_set_tuning": ([_P, _I, ctypes.POINTER(bspline_tuning)], _I),
    "bspline_get_tuning": ([_P, _I, ctypes.POINTER(bspline_tuning)], _I),
    "bspline_tune": ([_P, _I, _I, _S, ctypes.POINTER(bspline_tuning)], _I),
    "bspline_plan_create": ([ctypes.POINTER(bspline_batch_item), _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "bspline_plan_run": ([_P, _P], _I),
    "bspline_plan_run_graph": ([_P, _P], _I),
    "bspline_plan_destroy": ([_P], _I),
    "bspline_plan_set_order": ([_P, _I], _I),
    "bspline_plan_set_mode": ([_P, _I], _I),
    "bspline_plan_get_mode": ([_P, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "bspline_plan_set_stages": ([_P, _I], _I),
    "bspline_plan_get_stages": ([_P, ctypes.POINTER(_I)], _I),
    "bspline_plan_tune": ([_P, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "bspline_eval_batched": ([ctypes.POINTER(bspline_batch_item), _I, _I, _P], _I),
    "bspline_eval_batched_noalloc": ([ctypes.POINTER(bspline_batch_item), _I, _I, _P], _I),
}
NOALLOC_MAX_ITEMS = 64

_F, _SZ, _D, _ULL = ctypes.c_float, ctypes.c_size_t, ctypes.c_double, ctypes.c_ulonglong
_SIGS.update({
    "mlp_create": ([_I, _I, _I, _I, ctypes.POINTER(ctypes.c_void_p)], _I),
    "mlp_destroy": ([_P], _I),
    "mlp_param_count": ([_P], _SZ),
    "mlp_feature_count": ([_P], _I),
    "mlp_init": ([_P, _ULL], _I),
    "mlp_set_gemm_kernel": ([_P, _I], _I),
    "mlp_device_status": ([_P, _P, _I], _I),
    "mlp_get_params": ([_P, _P, _SZ], _I),
    "mlp_set_params": ([_P, _P, _SZ], _I),
    "mlp_get_grads": ([_P, _P, _SZ], _I),
    "mlp_train_step": ([_P, _I, _P, _P, _P, _P, _I, _F, _P, _P], _I),
    "mlp_train_step_vg": ([_P, _I, _P, _P, _P, _P, _P, _I, _F, _F, _P, _P], _I),
    "mlp_eval_v": ([_P, _I, _P, _P, _P, _P, _I, _P], _I),
    "mlp_eval_vgl": ([_P, _I, _P, _P, _P, _P, _P, _P, _I, _P], _I),
    "mlp_save": ([_P, _S], _I),
    "mlp_load": ([_P, _S], _I),
    "mlp_gemm_bf16": ([_P, _P, _P, _I, _I, _I, _I, _I, _P], _I),
    "mlp_gemm_bf16_ex": ([_P, _P, _P, _I, _I, _I, _I, _I, _I, _P], _I),
    "mlp_flops": ([_P, _I, _I], _D),
})


def library_path() -> str:
    return LIB_PATH


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"GB300 B-spline library not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            missing = [name for name in _SIGS if not hasattr(L, name)]
            if missing:
                raise RuntimeError(f"{LIB_PATH} is stale (missing {missing}); run __graft_entry__.build()")
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


def _check(st, where):
    if st != OK:
        raise BsplineError(st, where)


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None stays NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _on_device(a):
    return bool(getattr(a, "is_cuda", False))


_raw_stream = None


def _current_stream():
    """cudaStream_t of torch's current stream on the current device. torch.cuda.current_stream() builds a
    Stream object (about 3 us per call); torch's raw-stream query returns the handle alone, so it is used
    when this torch has it."""
    global _raw_stream
    import torch
    if _raw_stream is None:
        q = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        _raw_stream = (lambda: q(torch._C._cuda_getDevice())) if q is not None else \
            (lambda: torch.cuda.current_stream().cuda_stream)
    return _raw_stream()


def _stream(stream):
    if stream is None:
        return _current_stream()
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def bspline_abi_version() -> int:
    return lib().bspline_abi_version()


def bspline_status_str(status) -> str:
    return lib().bspline_status_str(int(status)).decode()


def bspline_create(nx, ny, nz, N, dtype=F32):
    h = ctypes.c_void_p()
    _check(lib().bspline_create(int(nx), int(ny), int(nz), int(N), int(dtype), ctypes.byref(h)), "bspline_create")
    return h.value


def bspline_destroy(h):
    _check(lib().bspline_destroy(h), "bspline_destroy")


def bspline_set_coefs(h, coefs, stream=None):
    """coefs: float32 [nx][ny][nz][N], contiguous, torch (host or device) or numpy."""
    s = _stream(stream) if _on_device(coefs) else None
    _check(lib().bspline_set_coefs(h, _ptr(coefs), int(_on_device(coefs)), s), "bspline_set_coefs")


def bspline_set_coefs_padded(h, padded, stream=None):
    """padded: float32 [nx+3][ny+3][nz+3][N], contiguous."""
    s = _stream(stream) if _on_device(padded) else None
    _check(lib().bspline_set_coefs_padded(h, _ptr(padded), int(_on_device(padded)), s),
           "bspline_set_coefs_padded")


def bspline_set_values(h, values, stream=None):
    """values: float32 [nx][ny][nz][N] orbital samples on the grid (torch host/device or numpy)."""
    s = _stream(stream) if _on_device(values) else None
    _check(lib().bspline_set_values(h, _ptr(values), int(_on_device(values)), s), "bspline_set_values")


def bspline_set_lattice(h, lattice=None):
    """lattice: 3x3 lattice vectors as rows (Cartesian), or None for the unit cube."""
    if lattice is None:
        _check(lib().bspline_set_lattice(h, None), "bspline_set_lattice")
        return
    import numpy as np
    L = np.ascontiguousarray(np.asarray(lattice, dtype=np.float64).reshape(9))
    _check(lib().bspline_set_lattice(h, L.ctypes.data), "bspline_set_lattice")


def bspline_get_info(h) -> bspline_info:
    info = bspline_info()
    _check(lib().bspline_get_info(h, ctypes.byref(info)), "bspline_get_info")
    return info


def bspline_get_table(h, dst, scale=None):
    """dst: host array of (nx+3)*(ny+3)*(nz+3)*N elements of the stored type; scale: host float32[N]."""
    _check(lib().bspline_get_table(h, _ptr(dst), _ptr(scale)), "bspline_get_table")


def bspline_eval_v(h, npos, x, y, z, v, ld, stream=None):
    _check(lib().bspline_eval_v(h, int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), int(ld), _stream(stream)),
           "bspline_eval_v")


def bspline_eval_vgl(h, npos, x, y, z, v, g, l, ld, stream=None):
    _check(lib().bspline_eval_vgl(h, int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), _ptr(g), _ptr(l), int(ld),
                                  _stream(stream)), "bspline_eval_vgl")


def bspline_eval_vgh(h, npos, x, y, z, v, g, hh, ld, stream=None):
    _check(lib().bspline_eval_vgh(h, int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), _ptr(g), _ptr(hh), int(ld),
                                  _stream(stream)), "bspline_eval_vgh")


def bspline_eval_ratio(h, kind, npos, x, y, z, uinv, ldu, ratio, stream=None):
    _check(lib().bspline_eval_ratio(h, int(kind), int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(uinv), int(ldu),
                                    _ptr(ratio), _stream(stream)), "bspline_eval_ratio")


def bspline_eval_host(h, kind, npos, x, y, z, v, g, hl, ld):
    _check(lib().bspline_eval_host(h, int(kind), int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), _ptr(g), _ptr(hl),
                                   int(ld)), "bspline_eval_host")


def bspline_set_host_mode(h, mode):
    _check(lib().bspline_set_host_mode(h, int(mode)), "bspline_set_host_mode")


def bspline_device_status(h, stream=None, reset=False) -> int:
    return lib().bspline_device_status(h, _stream(stream), int(bool(reset)))


def bspline_measure_read_bandwidth(nbytes, reps=20, stream=None) -> float:
    """GB/s of repeated full reads of a device buffer of nbytes (L2 bandwidth when it fits in L2)."""
    out = ctypes.c_double(0.0)
    _check(lib().bspline_measure_read_bandwidth(int(nbytes), int(reps), ctypes.byref(out), _stream(stream)),
           "bspline_measure_read_bandwidth")
    return out.value


def bspline_selftest_wait_timeout(h, limit_us, stream=None):
    _check(lib().bspline_selftest_wait_timeout(h, int(limit_us), _stream(stream)), "bspline_selftest_wait_timeout")


def bspline_set_tuning(h, kind, variant=0, nb=0, ppc=0, stages=0, order=0):
    tu = bspline_tuning(int(variant), int(nb), int(ppc), int(stages), int(order))
    _check(lib().bspline_set_tuning(h, int(kind), ctypes.byref(tu)), "bspline_set_tuning")


def bspline_get_tuning(h, kind) -> dict:
    tu = bspline_tuning()
    _check(lib().bspline_get_tuning(h, int(kind), ctypes.byref(tu)), "bspline_get_tuning")
    return tu.as_dict()


def bspline_tune(h, kind, npos_hint=0, wisdom_path=None) -> dict:
    tu = bspline_tuning()
    wp = wisdom_path.encode() if wisdom_path else None
    _check(lib().bspline_tune(h, int(kind), int(npos_hint), wp, ctypes.byref(tu)), "bspline_tune")
    return tu.as_dict()


def _items(items):
    arr = (bspline_batch_item * len(items))()
    for k, it in enumerate(items):
        arr[k] = bspline_batch_item(it["table"], int(it["npos"]), _ptr(it["x"]), _ptr(it["y"]), _ptr(it["z"]),
                                    _ptr(it["v"]), _ptr(it.get("g")), _ptr(it.get("hl")), int(it["ld"]))
    return arr


def bspline_plan_create(items, kind):
    """items: list of dicts with table, npos, x, y, z, v, g, hl, ld (device tensors)."""
    arr = _items(items)
    h = ctypes.c_void_p()
    _check(lib().bspline_plan_create(arr, len(items), int(kind), ctypes.byref(h)), "bspline_plan_create")
    return h.value


def bspline_plan_run(plan, stream=None):
    _check(lib().bspline_plan_run(plan, _stream(stream)), "bspline_plan_run")


def bspline_plan_run_graph(plan, stream=None):
    _check(lib().bspline_plan_run_graph(plan, _stream(stream)), "bspline_plan_run_graph")


def bspline_plan_set_order(plan, order):
    _check(lib().bspline_plan_set_order(plan, int(order)), "bspline_plan_set_order")


PLAN_ONE_LAUNCH, PLAN_PER_TABLE = 0, 1


def bspline_plan_set_mode(plan, mode):
    _check(lib().bspline_plan_set_mode(plan, int(mode)), "bspline_plan_set_mode")


def bspline_plan_get_mode(plan):
    """(mode, order) of the plan."""
    m, o = ctypes.c_int(), ctypes.c_int()
    _check(lib().bspline_plan_get_mode(plan, ctypes.byref(m), ctypes.byref(o)), "bspline_plan_get_mode")
    return m.value, o.value


def bspline_plan_set_stages(plan, stages):
    _check(lib().bspline_plan_set_stages(plan, int(stages)), "bspline_plan_set_stages")


def bspline_plan_get_stages(plan) -> int:
    st = ctypes.c_int()
    _check(lib().bspline_plan_get_stages(plan, ctypes.byref(st)), "bspline_plan_get_stages")
    return st.value


def bspline_plan_tune(plan, reps=5, stream=None):
    """Time the plan's candidate executions and keep the fastest; returns (mode, order)."""
    m, o = ctypes.c_int(), ctypes.c_int()
    _check(lib().bspline_plan_tune(plan, int(reps), _stream(stream), ctypes.byref(m), ctypes.byref(o)),
           "bspline_plan_tune")
    return m.value, o.value


def bspline_plan_destroy(plan):
    _check(lib().bspline_plan_destroy(plan), "bspline_plan_destroy")


def bspline_eval_batched(items, kind, stream=None):
    arr = _items(items)
    _check(lib().bspline_eval_batched(arr, len(items), int(kind), _stream(stream)), "bspline_eval_batched")


def bspline_eval_batched_noalloc(items, kind, stream=None):
    """Batched evaluation whose scratch is a fixed device array inside the library (no allocation).

    For callers that cannot allocate device memory around an evaluation. At most
    NOALLOC_MAX_ITEMS items; calls that overlap on the GPU race on the shared array.
    """
    arr = _items(items)
    _check(lib().bspline_eval_batched_noalloc(arr, len(items), int(kind), _stream(stream)),
           "bspline_eval_batched_noalloc")


# ---- learned surrogate (include/mlp_surrogate.h) ----

def mlp_create(nfreq, hidden, layers, nout):
    h = ctypes.c_void_p()
    _check(lib().mlp_create(int(nfreq), int(hidden), int(layers), int(nout), ctypes.byref(h)), "mlp_create")
    return h.value


def mlp_destroy(m):
    _check(lib().mlp_destroy(m), "mlp_destroy")


def mlp_param_count(m) -> int:
    return int(lib().mlp_param_count(m))


def mlp_feature_count(m) -> int:
    return int(lib().mlp_feature_count(m))


def mlp_init(m, seed):
    _check(lib().mlp_init(m, int(seed)), "mlp_init")


def mlp_set_gemm_kernel(m, kernel):
    _check(lib().mlp_set_gemm_kernel(m, int(kernel)), "mlp_set_gemm_kernel")


def mlp_device_status(m, stream=None, reset=False) -> int:
    return lib().mlp_device_status(m, _stream(stream), int(bool(reset)))


def mlp_get_params(m, host):
    """host: float32 numpy array of mlp_param_count elements (filled in place)."""
    _check(lib().mlp_get_params(m, _ptr(host), host.size), "mlp_get_params")


def mlp_set_params(m, host):
    _check(lib().mlp_set_params(m, _ptr(host), host.size), "mlp_set_params")


def mlp_get_grads(m, host):
    _check(lib().mlp_get_grads(m, _ptr(host), host.size), "mlp_get_grads")


def mlp_train_step(m, batch, x, y, z, target, ld_target, lr, loss_out=None, stream=None):
    _check(lib().mlp_train_step(m, int(batch), _ptr(x), _ptr(y), _ptr(z), _ptr(target), int(ld_target), float(lr),
                                _ptr(loss_out), _stream(stream)), "mlp_train_step")


def mlp_train_step_vg(m, batch, x, y, z, target_v, target_g, ld_target, lam, lr, loss_out=None, stream=None):
    """One Adam step on the value-and-gradient loss; target_g is [batch][3][ld_target]."""
    _check(lib().mlp_train_step_vg(m, int(batch), _ptr(x), _ptr(y), _ptr(z), _ptr(target_v), _ptr(target_g),
                                   int(ld_target), float(lam), float(lr), _ptr(loss_out), _stream(stream)),
           "mlp_train_step_vg")


def mlp_eval_v(m, npos, x, y, z, v, ld, stream=None):
    _check(lib().mlp_eval_v(m, int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), int(ld), _stream(stream)),
           "mlp_eval_v")


def mlp_eval_vgl(m, npos, x, y, z, v, g, l, ld, stream=None):
    _check(lib().mlp_eval_vgl(m, int(npos), _ptr(x), _ptr(y), _ptr(z), _ptr(v), _ptr(g), _ptr(l), int(ld),
                              _stream(stream)), "mlp_eval_vgl")


def mlp_save(m, path):
    _check(lib().mlp_save(m, str(path).encode()), "mlp_save")


def mlp_load(m, path):
    _check(lib().mlp_load(m, str(path).encode()), "mlp_load")


def mlp_gemm_bf16(A, B, C, M, N, K, ldc, splitk=1, stream=None):
    _check(lib().mlp_gemm_bf16(_ptr(A), _ptr(B), _ptr(C), int(M), int(N), int(K), int(ldc), int(splitk),
                               _stream(stream)), "mlp_gemm_bf16")


GEMM_AUTO, GEMM_ONE_CTA, GEMM_CTA_PAIR, GEMM_TWO_CTAS = 0, 1, 2, 3


def mlp_gemm_bf16_ex(A, B, C, M, N, K, ldc, splitk=1, kernel=GEMM_AUTO, stream=None):
    _check(lib().mlp_gemm_bf16_ex(_ptr(A), _ptr(B), _ptr(C), int(M), int(N), int(K), int(ldc), int(splitk),
                                  int(kernel), _stream(stream)), "mlp_gemm_bf16_ex")


def mlp_flops(m, what, n) -> float:
    return float(lib().mlp_flops(m, int(what), int(n)))


class Surrogate:
    """Owning wrapper of a surrogate handle."""

    def __init__(self, nfreq, hidden, layers, nout):
        self.shape = (int(nfreq), int(hidden), int(layers), int(nout))
        self.h = mlp_create(*self.shape)

    def close(self):
        if self.h:
            mlp_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Table:
    """Owning wrapper of a table handle (create on enter / destroy on close)."""

    def __init__(self, grid, N, dtype=F32):
        self.grid = tuple(int(g) for g in grid)
        self.N = int(N)
        self.dtype = int(dtype)
        self.h = bspline_create(*self.grid, self.N, self.dtype)

    def close(self):
        if self.h:
            bspline_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, kind, npos, ld=None, device="cuda"):
        """Allocate device outputs (v, g, hl) for kind with leading dimension ld (default N)."""
        import torch
        ld = self.N if ld is None else ld
        v = torch.empty((npos, ld), dtype=torch.float32, device=device)
        g = torch.empty((npos, 3, ld), dtype=torch.float32, device=device) if kind != V else None
        hl = None
        if kind == VGL:
            hl = torch.empty((npos, ld), dtype=torch.float32, device=device)
        elif kind == VGH:
            hl = torch.empty((npos, 6, ld), dtype=torch.float32, device=device)
        return v, g, hl

    def eval(self, kind, x, y, z, v, g=None, hl=None, ld=None, stream=None):
        ld = self.N if ld is None else ld
        npos = x.shape[0]
        if kind == V:
            bspline_eval_v(self.h, npos, x, y, z, v, ld, stream)
        elif kind == VGL:
            bspline_eval_vgl(self.h, npos, x, y, z, v, g, hl, ld, stream)
        else:
            bspline_eval_vgh(self.h, npos, x, y, z, v, g, hl, ld, stream)
