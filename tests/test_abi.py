"""The C-ABI library loads and exports every entry point declared in
include/sharp.h; host-side argument checks work without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sharp.h")
LIB = os.path.join(ROOT, "paper_1602_01448_gb300", "_lib", "libsharp.so")


@pytest.fixture(scope="session")
def lib():
    if not os.path.exists(LIB):
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "sharp_build", os.path.join(ROOT, "paper_1602_01448_gb300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()
    return ctypes.CDLL(LIB)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int|void)\s+(sharp_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for required in ("sharp_q_gather", "sharp_fourier_project", "sharp_overlap_project",
                     "sharp_raar_step", "sharp_probe_update", "sharp_plan_create", "sharp_amp_loss",
                     "sharp_amp_loss_backward"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_defaults_without_gpu(lib):
    lib.sharp_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sharp_version()

    class Params(ctypes.Structure):
        _fields_ = [("beta", ctypes.c_float), ("wrap", ctypes.c_int), ("probe_every", ctypes.c_int),
                    ("residual_every", ctypes.c_int), ("precision", ctypes.c_int)]
    p = Params()
    lib.sharp_default_params(ctypes.byref(p))
    assert abs(p.beta - 0.75) < 1e-7 and p.wrap == 0 and p.residual_every == 1


def test_plan_create_rejects_bad_arguments_on_host(lib):
    lib.sharp_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    f = lib.sharp_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert f(ctypes.byref(h), 0, 64, 256, 256, dummy, None, None) == 1      # K < 1
    assert b"K" in lib.sharp_last_error()
    assert f(ctypes.byref(h), 4, 64, 32, 256, dummy, None, None) == 1       # object smaller than frame
    assert f(ctypes.byref(h), 4, 96, 256, 256, dummy, None, None) == 2      # no kernel for m=96
    assert f(ctypes.byref(h), 4, 64, 256, 256, None, None, None) == 1       # NULL positions

    class Params(ctypes.Structure):
        _fields_ = [("beta", ctypes.c_float), ("wrap", ctypes.c_int), ("probe_every", ctypes.c_int),
                    ("residual_every", ctypes.c_int), ("precision", ctypes.c_int)]
    # RAAR's relaxation range is (0.5, 1] (Sec. 2.2): at 1/2 the new state
    # carries no trace of P_a z, below it the method is not RAAR
    for beta in (0.5, 0.3, 0.0, -1.0, 1.01, float("nan")):
        p = Params()
        lib.sharp_default_params(ctypes.byref(p))
        p.beta = beta
        assert f(ctypes.byref(h), 4, 64, 256, 256, dummy, ctypes.byref(p), None) == 1, beta
        assert b"beta" in lib.sharp_last_error()
    lib.sharp_plan_destroy.argtypes = [ctypes.c_void_p]
    assert lib.sharp_plan_destroy(None) == 0
    lib.sharp_plan_set_wait_limit.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    assert lib.sharp_plan_set_wait_limit(None, 5) == 1                        # NULL plan
