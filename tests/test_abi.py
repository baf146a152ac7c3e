"""The C ABI library builds, loads without a GPU, exports every entry point
that include/mm.h declares, and rejects bad plan descriptions on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_02842_gb300 import build as b
    b.build()
    from paper_2003_02842_gb300 import _lib
    return _lib.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mm_[a-z_0-9]+)\s*\(", src))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"mm_plan_create", "mm_coeffs", "mm_cov", "mm_corr", "mm_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    import paper_2003_02842_gb300 as mm
    assert mm.mm_version() >= 100
    for s in range(12):
        assert mm.mm_status_string(s)


@pytest.mark.parametrize("field,value", [
    ("D", 0), ("N_max", -1), ("tol", 0.0), ("tol", 0.7), ("kernel", 7), ("basis", 3), ("prec", 9),
    ("max_events", -5), ("spread_tile", -1), ("spread_algo", 4), ("spread_algo", -1),
    ("fft_algo", 6), ("fft_algo", 3), ("fft_algo", -1),
])
def test_bad_desc_rejected_on_host(lib, field, value):
    from paper_2003_02842_gb300 import _lib
    d = _lib.PlanDesc()
    d.D, d.N_max, d.max_events, d.tol, d.kernel, d.basis, d.prec = 4, 10, 100, 1e-6, 2, 0, 1
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.mm_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1  # MM_ERR_INVALID_ARG
    assert not h.value


def test_reserved_fields_must_be_zero(lib):
    from paper_2003_02842_gb300 import _lib
    d = _lib.PlanDesc()
    d.D, d.N_max, d.max_events, d.tol, d.kernel, d.basis, d.prec = 4, 10, 100, 1e-6, 2, 0, 1
    d.reserved[2] = 1
    h = ctypes.c_void_p()
    assert lib.mm_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
    d.reserved[2] = 0
    d.gram_algo = 3  # no such contraction variant
    assert lib.mm_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1


def test_null_arguments_rejected(lib):
    assert lib.mm_plan_create(None, None) == 1
    assert lib.mm_destroy(None) == 1
    assert lib.mm_plan_sync(None) == 1
    assert lib.mm_coeffs(None, None, None, None, 5, 0.0, 0.0, None, None, None) == 1


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_2003_02842_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()


@pytest.mark.parametrize("field,value,code", [
    ("reps", 0, 1), ("D", 0, 1), ("N_max", 0, 1), ("max_events", -1, 1), ("reserved0", 1, 1),
    ("D", 13, 11), ("prec", 7, 1), ("spread_algo", 4, 1), ("spread_algo", -1, 1),
])
def test_bad_batch_desc_rejected_on_host(lib, field, value, code):
    from paper_2003_02842_gb300 import _lib
    d = _lib.BatchDesc()
    d.reps, d.D, d.N_max, d.max_events, d.tol, d.kernel, d.basis, d.prec = 4, 3, 10, 100, 1e-6, 2, 0, 1
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.mm_batch_create(ctypes.byref(d), ctypes.byref(h)) == code
    assert not h.value


@pytest.mark.parametrize("field,value", [
    ("D", 0), ("D", 5000), ("N_max", 0), ("max_events", 0), ("max_slots", 0), ("max_slots", 65), ("cache_rows", -1),
])
def test_bad_server_desc_rejected_on_host(lib, field, value):
    from paper_2003_02842_gb300 import _lib
    d = _lib.ServerDesc()
    d.D, d.N_max, d.max_events, d.max_slots, d.tol, d.kernel, d.basis, d.prec = 4, 10, 100, 2, 1e-6, 2, 1, 1
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert lib.mm_server_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert not h.value
