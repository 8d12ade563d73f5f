"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ctr_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    from paper_2210_03699_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("ctr_ibim_setup", "ctr_ibim_matvec", "ctr_ibim_solve", "ctr_ibim_energy"):
        assert required in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, missing


def test_status_strings_and_defaults(library):
    library.ctr_status_string.restype = ctypes.c_char_p
    assert library.ctr_status_string(0) == b"ok"
    assert library.ctr_status_string(-2) == b"empty tube"
    import paper_2210_03699_gb300 as ctr
    o = ctr._Options()
    ctr.lib.ctr_default_options(ctypes.byref(o))
    assert o.tol == 1e-10 and o.restart == 64 and o.precision == ctr.FP64
    assert o.farfield == ctr.FARFIELD_DIRECT and o.tree_degree == 10 and o.tree_theta == 0.8
    assert o.tree_leaf == 128 and o.tree_degree_fp32 == 6 and o.tree_theta_fp32 == 0.9
    # the binding's mirror of ctr_options has the C layout: its defaults match the library's
    d = ctr.Options()
    assert (d.tree_degree, d.tree_theta, d.tree_leaf, d.tree_degree_fp32, d.tree_theta_fp32) == (
        o.tree_degree, o.tree_theta, o.tree_leaf, o.tree_degree_fp32, o.tree_theta_fp32)
    # server options: the binding's struct has the C layout (defaults written by the library)
    so = ctr._ServerOptions(0, 7, -1.0)
    ctr.lib.ctr_default_server_options(ctypes.byref(so))
    assert (so.max_slots, so.hbm_budget_bytes, so.step_quantum_ms) == (16, 0, 20.0)


def test_invalid_arguments_rejected_without_gpu(library):
    import paper_2210_03699_gb300 as ctr
    h = ctypes.c_void_p()
    st = ctr.lib.ctr_ibim_setup(None, None, 0, 1.0, 80.0, 0.1, 0, None, None, None, None, ctypes.byref(h))
    assert st == -1 and h.value is None
    assert b"NULL" in ctr.lib.ctr_last_error()
    # inspection entry points reject missing handles and arguments before touching the GPU
    i64 = ctypes.c_int64()
    assert ctr.lib.ctr_ibim_pair_schedule(None, ctr.FP32_REFINE, ctypes.byref(i64), None, None, None) == -1
    v = ctypes.c_int()
    assert ctr.lib.ctr_tuning_info(None, ctypes.byref(v), ctypes.byref(v)) == -1
    assert ctr.lib.ctr_ibim_matvec(None, None, None, ctr.FP32_REFINE, 0) == -1
    assert ctr.lib.ctr_ibim_farfield_info(None, ctr.FP32_REFINE, None, None, None, None, None) == -1
    d = ctypes.c_double()
    assert ctr.lib.ctr_ibim_time_operator(None, ctr.FP32_REFINE, 1, ctypes.byref(d), None, None, None) == -1
    assert ctr.lib.ctr_farfield_plan(0, None, None, None, 2, 10, 0.8, 128, 256, 0, None, None, None, None, None,
                                     None, None, None) == -1
    # server options are validated before any device call
    sv = ctypes.c_void_p()
    for bad in (ctr._ServerOptions(0, 0, 20.0), ctr._ServerOptions(4, 0, -1.0),
                ctr._ServerOptions(4, 0, float("nan")), ctr._ServerOptions(4, 0, float("inf"))):
        assert ctr.lib.ctr_server_create(ctypes.byref(bad), ctypes.byref(sv)) == -1 and sv.value is None
