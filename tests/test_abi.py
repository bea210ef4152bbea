"""The C-ABI library builds, loads and exports every function include/ocmc.h declares
(CPU: no compute calls); argument validation that needs no device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(ocmc_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_01722_gb300 import build
    return C.CDLL(build.build())


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params(lib):
    from paper_1503_01722_gb300 import ocmc
    p = ocmc.default_params()
    assert abs(p.e_abs_e - 0.2) < 1e-7 and abs(p.e_abs_g - 0.01) < 1e-9
    assert abs(p.w_cc - 0.2) < 1e-7 and abs(p.w_cb - 0.01) < 1e-9
    assert p.n_batches == 10 and p.flags == 0
    assert abs(p.e_class_split - 2.0) < 1e-7


@pytest.mark.parametrize("field,value", [("e_abs_e", 0.0), ("f_maxe", 0.9), ("n_batches", 0),
                                         ("block_threads", 100), ("stack_capacity", 8), ("e_class_split", -1.0),
                                         ("e_class_split", 40.0)])
def test_invalid_params_rejected_before_device(lib, field, value):
    from paper_1503_01722_gb300 import ocmc
    p = ocmc.default_params()
    setattr(p, field, value)
    with pytest.raises(ocmc.OcmcError) as e:
        ocmc.Engine(0, params=p)
    assert e.value.status == ocmc.ERR_ARG


def test_init_without_device_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1503_01722_gb300 import ocmc
    with pytest.raises(ocmc.OcmcError) as e:
        ocmc.Engine(0)
    assert e.value.status == ocmc.ERR_CUDA
    assert "CUDA" in str(e.value) or "device" in str(e.value)


def test_null_context_calls_fail_cleanly(lib):
    lib.ocmc_run.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p]
    assert lib.ocmc_run(None, 10, 1, None) == 1
    lib.ocmc_destroy.argtypes = [C.c_void_p]
    lib.ocmc_destroy(None)
