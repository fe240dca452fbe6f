"""The C ABI library loads and exports every symbol include/pf.h declares (no GPU needed;
no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1506_01684_gb300 import build, pf
from paper_1506_01684_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "pf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", text))
    names -= {"pf_alloc_fn", "pf_free_fn"}
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    L = ctypes.CDLL(path)
    declared = _declared()
    assert "pf_create" in declared and "pf_step" in declared
    for name in declared:
        assert hasattr(L, name), name
    # the binding wraps every declared entry point under the same name
    for name in declared:
        assert name in pf.SIGNATURES, name
        assert callable(getattr(pf, name)), name


def test_host_only_entry_points():
    # calls that touch no device: defaults, error strings, argument checks
    p = pf.pf_default_params()
    assert p.version == pf.PF_PARAMS_VERSION and p.eps == 4.0 and p.gamma3[2] == 15.0
    assert abs(p.T0 - (1.0 - 8e-3 - 0.15)) < 1e-15
    assert pf.pf_strerror(pf.PF_E_UNSTABLE).startswith("non-finite")
    L = pf.lib()
    h = ctypes.c_void_p()
    assert L.pf_create(0, 4, 4, ctypes.byref(p), None, ctypes.byref(h)) == pf.PF_E_INVAL
    bad = pf.pf_default_params()
    bad.version = 99
    assert L.pf_create(4, 4, 4, ctypes.byref(bad), None, ctypes.byref(h)) == pf.PF_E_INVAL
    assert L.pf_step(None, 1) == pf.PF_E_INVAL
    assert L.pf_default_params(None) == pf.PF_E_INVAL
    # general thermodynamics: curvature matrices must be positive definite, pair times all set or none
    for change in ({"Am": [[1.0, 2.0, 1.0]] + [[0.0, 0.0, 0.0]] * 3},
                   {"Am": [[1.0, 0.1, -1.0]] + [[0.0, 0.0, 0.0]] * 3},
                   {"tau_ab": [1.0, 1.0, 0.0, 1.0, 1.0, 1.0]}):
        q = pf.params_from_dict(dict(W.symmetric_params(), **change))
        assert L.pf_create(8, 8, 8, ctypes.byref(q), None, ctypes.byref(h)) == pf.PF_E_INVAL


def test_default_params_match_the_workload_parameter_set():
    from paper_1506_01684_gb300 import workloads as W
    d = W.symmetric_params()
    p = pf.pf_default_params()
    q = pf.params_from_dict(d)
    for f, _ in pf.pf_params._fields_:
        a, b = getattr(p, f), getattr(q, f)
        if isinstance(a, (int, float)):
            assert a == b, f
        else:
            assert list(map(lambda x: list(x) if hasattr(x, "__len__") else x, a)) == \
                list(map(lambda x: list(x) if hasattr(x, "__len__") else x, b)), f


def test_host_side_checks_of_the_split_batch_and_checkpoint_calls():
    # argument checks that return before any device call
    L = pf.lib()
    p = pf.params_from_dict(W.symmetric_params(), pf.PF_FP64)
    h = ctypes.c_void_p()
    # slabs: at least one, at most one a row; compensated FP32 is not offered
    assert L.pf_split_create(8, 6, 8, ctypes.byref(p), 0, ctypes.byref(h)) == pf.PF_E_INVAL
    assert L.pf_split_create(8, 6, 8, ctypes.byref(p), 7, ctypes.byref(h)) == pf.PF_E_INVAL
    assert L.pf_split_create(0, 6, 8, ctypes.byref(p), 2, ctypes.byref(h)) == pf.PF_E_INVAL
    c = pf.params_from_dict(W.symmetric_params(), pf.PF_FP32_COMP)
    assert L.pf_split_create(8, 6, 8, ctypes.byref(c), 2, ctypes.byref(h)) == pf.PF_E_INVAL
    assert L.pf_split_create(8, 6, 8, ctypes.byref(p), 2, None) == pf.PF_E_INVAL
    for name in ("pf_split_destroy", "pf_split_sync"):
        assert getattr(L, name)(None) == pf.PF_E_INVAL
    assert L.pf_split_step(None, 1) == pf.PF_E_INVAL
    assert L.pf_split_init(None, 0) == pf.PF_E_INVAL
    assert L.pf_split_read_fields(None, None, None, 0) == pf.PF_E_INVAL
    assert L.pf_split_stats(None, None, None, None, None) == pf.PF_E_INVAL
    # the batch's launch shape and byte tally, and the single-precision checkpoint, of no object
    assert L.pf_batch_config(None, None, None, None, None) == pf.PF_E_INVAL
    assert L.pf_batch_set_config(None, 0, 2, 1, 8) == pf.PF_E_INVAL
    assert L.pf_batch_step_bytes(None, None) == pf.PF_E_INVAL
    assert L.pf_checkpoint_write_f32(None, b"x") == pf.PF_E_INVAL
