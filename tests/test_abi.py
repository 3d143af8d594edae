"""The C-ABI library builds, loads and exports every symbol that
include/lb.h declares; argument checks return before touching a device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    return lb.lib()


def test_every_declared_symbol_is_exported(L):
    from paper_2603_18052_gb300 import lb

    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(lb.EXPORTED)


def test_status_strings(L):
    for s in range(9):
        assert L.lb_status_str(s)
    assert L.lb_version() >= 100


def test_null_arguments_are_rejected_without_a_device(L):
    vp = ctypes.c_void_p
    assert L.lb_create(None, 0, 81, 8, 8) == 1  # LB_EINVAL
    assert L.lb_assemble(None, 3, vp(8), 0, None, vp(8), None) == 1
    assert L.lb_expm_pade(None, 9, 1, vp(8), None, None, 0.1, 0, vp(8), None, None) == 1
    assert L.lb_propagate_batch(None, 9, 1, vp(8), 1, 1, vp(8), 0, 0, None) == 1
    assert L.lb_grape_grad(None, 9, 1, vp(8), vp(8), vp(8), 0.1, 1, 1, vp(8), vp(8), vp(8), vp(8), None) == 1
    assert L.lb_grape_grad_batch(None, 9, 2, 1, vp(8), 0, vp(8), vp(8), 0.1, 1, 1, vp(8), vp(8), 0, vp(8), vp(8),
                                 None) == 1
    assert L.lb_sync_status(None, None) == 1
    assert L.lb_selftest_wait_timeout(None, 1000, None) == 1
    assert L.lb_expm_frechet(None, 9, 1, vp(8), vp(8), vp(8), 0.1, vp(8), vp(8), None) == 1
    assert L.lb_control_update(9, 1, None, vp(8), vp(8), vp(8), None) == 1
    assert L.lb_propagate_resident(None, 9, vp(8), 1, vp(8), None) == 1
    assert L.lb_expmv(None, 9, 1, vp(8), None, None, 0.1, 1, vp(8), None, None) == 1
    assert L.lb_expmv_hermitian(None, 9, 1, vp(8), None, None, 0.1, 1, vp(8), None, None) == 1
    assert L.lb_propagate_host(None, 9, vp(8), 1, vp(8), None) == 1
    assert L.lb_propagate_fixed(15, 9, None, 1, 1, vp(8), None) == 1
    assert L.lb_propagate_fixed(16, 9, vp(8), 1, 1, vp(8), None) == 1  # only Q1.15 and Q1.31
    assert L.lb_propagate_fixed(15, 100, vp(8), 1, 1, vp(8), None) == 1  # n above 81
    for probe in (L.lb_probe_dfma, L.lb_probe_ffma, L.lb_probe_dmma, L.lb_probe_bf16_tc):
        assert probe(None, None) == 1
    assert L.lb_propagate_fixed(15, 8, vp(8), 1, 1, vp(8), None) == 1  # n not a square
    assert L.lb_fixed_quantize(15, 4, None, vp(8), None) == 1
    assert L.lb_fixed_dequantize(7, 4, vp(8), vp(8), None) == 1
    assert L.lb_probe_read(None, 16, 0, vp(8), None) == 1
    assert L.lb_probe_launch(0, 0, None, None) == 1
    assert L.lb_probe_alloc(0, 1, None) == 1
    assert L.lb_probe_copy(None, vp(8), 16, 1, 1, None, None) == 1
    assert L.lb_destroy(None) == 0


def test_bad_sizes_are_rejected(L):
    h = ctypes.c_void_p()
    assert L.lb_create(ctypes.byref(h), 0, 730, 8, 8) == 1  # max_n above 729
    assert L.lb_create(ctypes.byref(h), 0, 81, 0, 8) == 1


def test_no_device_gives_enodev(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert L.lb_create(ctypes.byref(h), 0, 81, 8, 8) == 2  # LB_ENODEV
    assert not h.value
