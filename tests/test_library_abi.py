"""The C ABI without a GPU: libvrm.so builds (nvcc cross-compiles for
sm_103a), loads, and exports every function include/vrm.h declares; the
ctypes binding declares the same set; host-only calls work; the binding
refuses to run without the library (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vrm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:vrm_status|void|char\s*\*|int64_t|int32_t)\s*\*?\s*(vrm_\w+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_06379_gb300 import builder
    path = builder.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vrm_build_neighbourhoods", "vrm_solve_weights", "vrm_insert_reduce", "vrm_apply", "vrm_step",
                     "vrm_step_batched", "vrm_rk3_step", "vrm_mlp_train_step", "vrm_set_mlp"):
        assert required in names
    assert len(names) >= 30


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1508_06379_gb300 import binding
    assert set(binding.SIGNATURES) == set(declared_functions())


def test_host_only_calls(lib):
    from paper_1508_06379_gb300 import binding
    lib.vrm_status_string.restype = ctypes.c_char_p
    assert lib.vrm_status_string(0) == b"ok" and lib.vrm_status_string(2) == b"capacity too small"
    p = binding.Params()
    lib.vrm_default_params(ctypes.byref(p))
    assert (p.r, p.R, p.order, p.k_cap, p.max_rounds) == (0.5, 2.0, 1, 32, 8)
    # argument checks happen before any device work
    lib.vrm_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    bad = binding.Params()
    lib.vrm_default_params(ctypes.byref(bad))
    bad.h = -1.0
    assert lib.vrm_create(ctypes.byref(bad), ctypes.byref(out)) == 1
    bad.h, bad.order = 1.0, 3
    assert lib.vrm_create(ctypes.byref(bad), ctypes.byref(out)) == 4


def test_binding_refuses_without_the_library(monkeypatch, tmp_path):
    from paper_1508_06379_gb300 import binding, builder
    monkeypatch.setattr(builder, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(binding, "_LIB", None)
    with pytest.raises(RuntimeError):
        binding._lib_handle()
