"""The C-ABI library builds, loads and exports every symbol include/lpk.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

from paper_1604_07491_gb300 import build, lpk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lpk.h")).read()
    return sorted(set(re.findall(r"LPK_API\s+[\w\s\*]+?\b(lpk_\w+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared_symbols() == sorted(lpk.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_binding_loads_and_defaults():
    build.build()
    o = lpk.default_options()
    assert o.tol == 1e-8 and o.max_ipm == 99 and abs(o.sigma_max - 0.208) < 1e-15
    assert 0.9 <= o.eta < 1.0 and o.phi == 1e-5 and o.eps_in0 == 1e-6


def test_missing_device_is_an_error_not_a_crash():
    import torch
    if torch.cuda.is_available():
        return
    lib = lpk.load()
    h = ctypes.c_void_p()
    assert lib.lpk_create(ctypes.byref(h), 0, None) != 0
