"""The C-ABI library builds, loads and exports every entry point that
include/scgr.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scgr.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SCGR_EXPORT\s+[\w\s\*]+?\b(scgr_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    names = declared_symbols()
    assert "scgr_run" in names and "scgr_forces" in names and len(names) >= 20


def test_binding_constants_match_the_header():
    """Every integer SCGR_* constant of the binding has the header's value,
    and every tuning knob the header defines is in the binding."""
    from paper_1902_01061_gb300 import scgr
    defined = {k: int(v) for k, v in re.findall(r"#define\s+(SCGR_\w+)\s+(-?\d+)\b", open(HEADER).read())}
    knobs = [k for k in defined if k.startswith("SCGR_TUNE_")]
    assert len(knobs) >= 13
    for k in knobs:
        assert hasattr(scgr, k), k
    for k, v in defined.items():
        if hasattr(scgr, k):
            assert getattr(scgr, k) == v, k


def test_library_exports_every_declared_symbol(scgr_lib):
    from paper_1902_01061_gb300 import scgr
    out = subprocess.run(["nm", "-D", "--defined-only", scgr.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (scgr_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    assert set(scgr.EXPORTED) == set(declared_symbols())
    for n in declared_symbols():
        assert hasattr(scgr_lib, n)


def test_default_params(scgr_lib):
    from paper_1902_01061_gb300 import scgr
    p = scgr.scgr_default_params()
    assert (p.k, p.p, p.g_mode, p.G1, p.step_mode, p.eta0, p.scale_mode) == (16, 1.0, 1, 1e4, 0, 0.5, 0)


def test_create_rejects_bad_params_before_touching_the_gpu(scgr_lib):
    from paper_1902_01061_gb300 import scgr
    for bad in (dict(k=2), dict(k=33), dict(p=0.5), dict(eta0=0.0), dict(g_mode=2), dict(scale_mode=3),
                dict(G1=-1.0), dict(step_mode=2)):
        p = scgr.scgr_default_params(**bad)
        out = ctypes.c_void_p()
        st = scgr_lib.scgr_create(ctypes.byref(p), None, ctypes.byref(out))
        assert st == 1, bad                 # SCGR_ERR_INVALID_ARG
        assert out.value is None
        assert scgr_lib.scgr_last_error(None)


def test_null_arguments(scgr_lib):
    assert scgr_lib.scgr_default_params(None) == 1
    assert scgr_lib.scgr_create(None, None, None) == 1
    assert scgr_lib.scgr_run(None, 1) == 1
    assert scgr_lib.scgr_launch_count(None) == -1
    scgr_lib.scgr_destroy(None)
