"""The C-ABI library builds, loads and exports every declared symbol (CPU only).

Also checks the host-side argument validation, which returns before any
CUDA call, so it runs without a GPU.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1808_06992_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", h)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            if m.group(1) not in ("if", "for", "while", "sizeof", "return"):
                names.append(m.group(1))
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = native.lib()
    names = _declared_functions()
    assert "uoi_lasso_fit" in names and "lasso_admm_batch" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert set(native.EXPORTED) <= set(names)


def test_status_strings():
    lib = native.lib()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -8):
        s = lib.uoi_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.uoi_status_string(12345).decode() == "unknown status"


def test_params_default():
    prm, _ = native.make_params()
    assert prm.struct_size == C.sizeof(native.UoiParams)
    assert prm.rho == 1.0 and prm.max_iter == 1000 and prm.train_frac == 0.8


@pytest.mark.parametrize("kw,code", [
    (dict(B1=0), native.ERR_INVALID_ARG),
    (dict(q=0), native.ERR_INVALID_ARG),
    (dict(rho=0.0), native.ERR_INVALID_ARG),
    (dict(train_frac=1.0), native.ERR_INVALID_ARG),
    (dict(max_iter=0), native.ERR_INVALID_ARG),
    (dict(warm_start=7), native.ERR_INVALID_ARG),
    (dict(B2=200), native.ERR_UNSUPPORTED),
])
def test_invalid_parameters_rejected_on_host(kw, code):
    X = np.zeros((10, 3))
    y = np.zeros(10)
    with pytest.raises(native.UoiError) as ei:
        native.uoi_lasso_fit(X, y, **kw)
    assert ei.value.status == code


@pytest.mark.parametrize("N,order", [(10, 0), (10, -1), (4, 3), (2, 1)])
def test_var_order_and_length_rejected(N, order):
    # rejected before any device work: order >= 1 and N - order >= 2
    with pytest.raises(native.UoiError) as ei:
        native.uoi_var_fit(np.zeros((N, 3)), order=order, B1=2, B2=2, q=2)
    assert ei.value.status == native.ERR_INVALID_ARG


def test_intercept_argument_checks():
    # only 0/1, and only on entries that have an output for mu
    with pytest.raises(native.UoiError) as ei:
        native.uoi_var_fit(np.zeros((10, 3)), order=2, B1=2, B2=2, q=2, intercept=2)
    assert ei.value.status == native.ERR_INVALID_ARG
    with pytest.raises(native.UoiError) as ei:
        native.uoi_lasso_fit(np.zeros((10, 3)), np.zeros(10), B1=2, B2=2, q=2, intercept=1)
    assert ei.value.status == native.ERR_UNSUPPORTED


def test_block_mode_checked():
    with pytest.raises(native.UoiError) as ei:
        native.uoi_var_fit(np.zeros((10, 3)), order=1, B1=2, B2=2, q=2, block_mode=2)
    assert ei.value.status == native.ERR_INVALID_ARG


def test_params_struct_matches_header():
    # the binding's struct ends with the intercept field, as uoi.h declares it
    prm, _ = native.make_params()
    assert prm.struct_size == C.sizeof(native.UoiParams)
    assert native.UoiParams.intercept.offset + 4 <= C.sizeof(native.UoiParams)
    assert native.UoiParams.block_mode.offset == native.UoiParams.intercept.offset + 4


def test_null_pointer_rejected():
    lib = native.lib()
    prm, _ = native.make_params()
    st = lib.uoi_lasso_fit(None, None, 10, 3, C.byref(prm), None, None, None)
    assert st == native.ERR_INVALID_ARG
    assert "NULL" in native.last_error()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the CUDA library the loader and every entry point raise
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native._build, "build", lambda *a, **k: str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        native.lib()
    with pytest.raises(RuntimeError, match="missing"):
        native.uoi_lasso_fit(np.zeros((10, 3)), np.zeros(10), B1=2, B2=2, q=2)
