"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/fio.h, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fio_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_0809_0719_gb300 import fio

    return fio.lib()


def test_header_declares_the_api():
    names = header_functions()
    # the boundary's calls: plan, apply, adjoint, destroy, errors, the batch of uneven plans
    # with one pointer per plan, and the workspace size
    for n in ("fio_plan", "fio_apply", "fio_apply_adjoint", "fio_destroy", "fio_last_error", "fio_apply_batch",
              "fio_apply_batch_adjoint", "fio_workspace_bytes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in header_functions():
        assert hasattr(lib, n), n


def test_plan_rejects_bad_arguments_without_a_gpu(lib):
    h = ctypes.c_void_p()
    prm = (ctypes.c_double * 4)(2, 1, 16, 1)
    cases = [
        (48, 5, 1, 4, 1, 1, -1, -1),    # N not a power of two
        (2, 5, 1, 4, 1, 1, -1, -1),     # N too small
        (64, 1, 1, 4, 1, 1, -1, -1),    # q < 2
        (64, 4, 1, 4, 1, 1, -1, -1),    # q not compiled
        (64, 5, 9, 4, 1, 1, -1, -1),    # unknown phase
        (64, 5, 1, 3, 1, 1, -1, -1),    # wrong nparams
        (64, 5, 1, 4, 7, 1, -1, -1),    # unknown precision
        (64, 5, 1, 4, 1, 0, -1, -1),    # nrhs_max < 1
        (64, 5, 1, 4, 1, 1, -1, 9),     # e too large
    ]
    for N, q, ph, npar, prec, nr, s, e in cases:
        rc = lib.fio_plan(ctypes.byref(h), N, q, ph, prm, npar, prec, nr, s, e)
        assert rc == -1, (N, q, ph, npar, prec, nr, s, e, rc)
        assert len(lib.fio_last_error()) > 0


def test_batch_and_workspace_reject_bad_arguments_without_a_gpu(lib):
    vp = ctypes.c_void_p
    plans = (vp * 1)(None)
    ptrs = (vp * 1)(None)
    nr = (ctypes.c_int * 1)(1)
    assert lib.fio_apply_batch(plans, 1, ptrs, ptrs, nr, None) == -1
    assert lib.fio_apply_batch(None, 1, ptrs, ptrs, nr, None) == -1
    assert lib.fio_apply_batch_adjoint(plans, 0, ptrs, ptrs, nr, None) == -1
    assert lib.fio_workspace_bytes(None, 1) == 0


def test_calls_on_null_plan_fail_cleanly(lib):
    assert lib.fio_apply(None, None, None, 1, None) == -1
    assert lib.fio_apply_adjoint(None, None, None, 1, None) == -1
    assert lib.fio_destroy(None) == 0
    for impl in (0, 1, 2, 3):  # every switch kernel id, including the tensor-memory one
        assert lib.fio_plan_set_switch(None, impl) == -1
    assert lib.fio_plan_set_tuning(None, 3, -1, -1, -1) == -1
    assert lib.fio_apply_wave(None, None, None, None, 1, ctypes.c_double(0.5), ctypes.c_double(0.5), 0, None) == -1


def test_binding_has_no_cpu_path():
    # the binding's compute calls go through the library only
    src = open(os.path.join(ROOT, "paper_0809_0719_gb300", "fio.py")).read()
    assert "oracle" not in src and "numpy" not in src


def test_batch_calls_reject_bad_arguments_without_a_gpu(lib):
    h = ctypes.c_void_p()
    nr = (ctypes.c_int * 1)(1)
    plans = (ctypes.c_void_p * 1)(None)
    assert lib.fio_batch_create(None, 1, plans, nr, 0) == -1
    assert lib.fio_batch_create(ctypes.byref(h), 0, plans, nr, 0) == -1      # no plans
    assert lib.fio_batch_create(ctypes.byref(h), 5000, plans, nr, 0) == -1   # too many
    assert lib.fio_batch_create(ctypes.byref(h), 1, None, nr, 0) == -1
    assert lib.fio_batch_create(ctypes.byref(h), 1, plans, None, 0) == -1
    assert lib.fio_batch_create(ctypes.byref(h), 1, plans, nr, 8) == -1      # unknown flag
    assert len(lib.fio_last_error()) > 0
    assert lib.fio_batch_apply(None, None, None, 0, None) == -1
    assert lib.fio_batch_offsets(None, None) == -1
    assert lib.fio_batch_info(None, None) == -1
    assert lib.fio_batch_destroy(None) == 0


def test_auto_and_direct_reject_bad_arguments_without_a_gpu(lib):
    h = ctypes.c_void_p()
    q = ctypes.c_int()
    err = ctypes.c_double()
    prm = (ctypes.c_double * 4)(2, 1, 16, 1)
    assert lib.fio_plan_auto(None, 64, 1, prm, 4, 1, 1, -1, -1, 1e-3, 16, 0, ctypes.byref(q), ctypes.byref(err)) == -1
    assert lib.fio_plan_auto(ctypes.byref(h), 48, 1, prm, 4, 1, 1, -1, -1, 1e-3, 16, 0, None, None) == -1  # N
    assert lib.fio_plan_auto(ctypes.byref(h), 64, 1, prm, 4, 1, 1, -1, -1, 0.0, 16, 0, None, None) == -1   # target
    assert lib.fio_plan_auto(ctypes.byref(h), 64, 1, prm, 4, 1, 1, -1, -1, 1e-3, 0, 0, None, None) == -1   # nsample
    assert lib.fio_direct(None, None, 1, None, 1, None, None) == -1
    assert lib.fio_plan_set_tuning(None, -1, -1, -1, -1) == -1


def test_amplitude_rejects_bad_arguments_without_a_gpu(lib):
    assert lib.fio_apply_amplitude(None, None, None, None, 1, None, 1, 0, None) == -1
