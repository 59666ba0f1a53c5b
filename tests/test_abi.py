"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/weno_gb300.h declares.  No compute call is made (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "weno_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(weno_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("weno_init", "weno_rhs", "weno_ssprk3_step", "weno_cross_eval", "weno_sums", "weno_run"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2405_12301_gb300 import build, weno
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(weno.EXPORTS) == set(_declared())


def test_init_rejects_bad_arguments_without_touching_the_gpu():
    """Argument checks run before any CUDA call."""
    from paper_2405_12301_gb300 import build, weno
    build.build()
    L = weno.lib()
    h = ctypes.c_void_p()
    p = weno.weno_params()
    p.gamma, p.eps_weno, p.cfl = 0.9, 1e-6, 0.5  # gamma <= 1 is invalid
    assert L.weno_init(ctypes.byref(h), None, ctypes.byref(p), None) == weno.ERR_ARG
    assert b"gamma" in L.weno_last_error(None)
    p.gamma = 1.4
    p.alpha_mode = 7  # not a weno_alpha_mode
    assert L.weno_init(ctypes.byref(h), None, ctypes.byref(p), None) == weno.ERR_ARG
    p.alpha_mode = weno.ALPHA_GLOBAL_NORM
    p.bc[0][1] = 9    # not a weno_bc
    assert L.weno_init(ctypes.byref(h), None, ctypes.byref(p), None) == weno.ERR_ARG
    p.bc[0][1] = weno.BC_INFLOW
    p.model = 5       # not a weno_model
    assert L.weno_init(ctypes.byref(h), None, ctypes.byref(p), None) == weno.ERR_ARG
    p.model, p.precision = weno.MODEL_BURGERS, weno.FP32_BULK  # scalar laws are FP64 only
    assert L.weno_init(ctypes.byref(h), None, ctypes.byref(p), None) == weno.ERR_UNSUPPORTED
