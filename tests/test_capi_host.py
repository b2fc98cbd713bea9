"""Host-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that the headers in include/ declare; argument checks
that run before any CUDA call reject bad input. No kernel runs here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bspline_gb300.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    from paper_1611_02665_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions(headers=(HEADER,)):
    names = set()
    for h in headers:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b((?:bspline|mlp)_\w+)\s*\(", src,
                                flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bspline_create", "bspline_destroy", "bspline_set_coefs", "bspline_eval_v",
                     "bspline_eval_vgl", "bspline_eval_vgh", "bspline_eval_batched", "bspline_tune"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions(HEADERS)
    assert "mlp_train_step" in names and "mlp_gemm_bf16_ex" in names and "mlp_set_gemm_kernel" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_host_side_argument_checks(lib):
    from paper_1611_02665_gb300 import capi
    assert capi.bspline_abi_version() == 2
    assert capi.bspline_status_str(capi.ERR_TIMEOUT) == "device wait timed out"
    assert capi.bspline_status_str(capi.ERR_BOUNDS) == "device-side index check failed"
    h = ctypes.c_void_p()
    L = capi.lib()
    assert L.bspline_create(0, 4, 4, 8, 0, ctypes.byref(h)) == capi.ERR_ARG
    assert L.bspline_create(4, 4, 4, 0, 0, ctypes.byref(h)) == capi.ERR_ARG
    assert L.bspline_create(4, 4, 4, 8, 7, ctypes.byref(h)) == capi.ERR_DTYPE
    assert L.bspline_create(4, 4, 4, 8, 0, None) == capi.ERR_ARG
    assert L.bspline_destroy(None) == capi.ERR_ARG
    assert L.bspline_eval_v(None, 1, None, None, None, None, 8, None) == capi.ERR_ARG
    assert L.bspline_plan_run(None, None) == capi.ERR_ARG
    assert L.bspline_eval_batched(None, 0, 2, None) == capi.ERR_ARG
    assert L.bspline_plan_set_mode(None, capi.PLAN_PER_TABLE) == capi.ERR_ARG
    assert L.bspline_plan_get_mode(None, None, None) == capi.ERR_ARG
    assert L.bspline_plan_tune(None, 3, None, None, None) == capi.ERR_ARG
    assert L.bspline_plan_set_order(None, 1) == capi.ERR_ARG
    assert L.mlp_set_gemm_kernel(None, 1) == capi.ERR_ARG
    assert L.mlp_device_status(None, None, 0) == capi.ERR_ARG
    assert L.mlp_gemm_bf16_ex(None, None, None, 128, 256, 64, 256, 1, 2, None) == capi.ERR_ARG


def test_package_raises_without_library(monkeypatch, tmp_path):
    from paper_1611_02665_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.lib()
