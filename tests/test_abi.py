"""The C-ABI library builds, loads and exports every symbol include/gint.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gint.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(gint_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["gint_setup", "gint_destroy", "gint_pattern", "gint_vlocal", "gint_rho", "gint_force_stress",
              "gint_sync", "gint_last_error", "gint_set_precision", "gint_get_info"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2409_09399_gb300 import gint
    L = gint.load()
    out = subprocess.run(["nm", "-D", "--defined-only", L._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gint_[a-z_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(L, n)
    assert set(gint.SYMBOLS) <= set(declared_functions())


def test_host_validation_without_gpu():
    """Argument errors are reported by status before any device work."""
    from paper_2409_09399_gb300 import gint
    L = gint.load()
    out = ctypes.c_void_p()
    # n_atoms = 0 is rejected before touching a device
    st = L.gint_setup(0, None, None, None, 1, None, None, None, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert b"n_atoms" in L.gint_last_error()
    assert L.gint_vlocal(None, None, None, 0, None) == 1
    assert L.gint_rho(None, None, None, None) == 1
    assert L.gint_force_stress(None, None, None, None, None, None, None, None) == 1
    assert L.gint_set_precision(None, 0) == 1
    L.gint_destroy(None)  # no-op


def test_host_validation_of_the_other_entry_points():
    """NULL handles and empty batches are refused by status on the host (no device touched)."""
    from paper_2409_09399_gb300 import gint
    L = gint.load()
    i64 = ctypes.c_int64
    assert L.gint_check(None) == 1
    assert L.gint_vlocal_static(None, None, None, None) == 1
    k = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert L.gint_fold_k(None, None, ctypes.byref(k), None, 0, None) == 1
    assert b"gint_fold_k" in L.gint_last_error()
    out = ctypes.c_void_p()
    assert L.gint_batch_create(0, None, ctypes.byref(out)) == 1 and out.value is None
    assert L.gint_batch_run(None, None, None, None, None, None, None, None, None) == 1
    L.gint_batch_destroy(None)  # no-op
    assert L.gint_sync(None, None) == 1
    assert L.gint_get_info(None, None) == 1
    a, b = i64(), i64()
    assert L.gint_work_stats(None, ctypes.byref(a), ctypes.byref(b)) == 1
    assert L.gint_pattern(None, None, None, None, None) == 1


def test_host_validation_of_geometry_and_adjoint_entry_points():
    """The position update, brick selection, adjoint, wait-limit and allocation-hook entry points
    refuse bad arguments by status on the host."""
    from paper_2409_09399_gb300 import gint
    L = gint.load()
    assert L.gint_energy_grads(None, None, None, None, None, None, None, None, None, None) == 1
    assert b"gint_energy_grads" in L.gint_last_error()
    pos = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    changed = ctypes.c_int(7)
    assert L.gint_update_positions(None, pos, None, 1, ctypes.byref(changed)) == 1
    assert changed.value == 7
    assert L.gint_select_bricks(None, 0, None) == 1
    assert L.gint_brick_loads(None, None) == 1
    assert L.gint_set_wait_limit(None, 0) == 1
    assert L.gint_debug_fail_alloc(-1) == 1
    assert L.gint_debug_fail_alloc(0) == 0
