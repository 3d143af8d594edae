"""The allocation-free propagation entry point (lb_propagate_batch_static).

Callers that cannot allocate device memory (their own allocator owns it, or
they cannot risk cudaMalloc's synchronisation) use this entry point instead
of lb_propagate_batch.  These tests call it through the C ABI and check two
calls in a row against the oracle's chain and against the context-based
entry point, within the 1e-12 relative tolerance of the FP64 path.  The file
is named so that pytest collects it last."""

import ctypes

import numpy as np
import pytest

import oracle as O
from workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lb


def _props(w):
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    return O.slice_propagators(Lb, Ld, w["u"], w["dt"])


@pytest.mark.parametrize("name,B,S,m", [("d27_chain", 64, 2, 1), ("d9_batch", 50, 2, 3)])
def test_static_entry_matches_context_entry_twice(lbm, name, B, S, m):
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w = make_workload(name, B=B, nslices=S)
    P = torch.from_numpy(_props(w)).to(dev)
    x0 = torch.from_numpy(w["states"]).to(dev)
    ctx = lbm.Context(0, max_n=w["n"], max_batch=B, max_slices=S)
    ctx_out = x0.clone()
    lbm.lb_propagate_batch(ctx, P, ctx_out, steps_per_slice=m)
    lbm.lb_sync_status(ctx)
    ctx_out = ctx_out.cpu().numpy()
    ref = O.propagate_chain(P.cpu().numpy(), w["states"], m)
    L = lbm.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        x = x0.clone()
        st = L.lb_propagate_batch_static(w["n"], S, ctypes.c_void_p(P.data_ptr()), m, B,
                                         ctypes.c_void_p(x.data_ptr()), stream)
        assert st == 0, L.lb_status_str(st)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        for b in range(B):
            err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
            assert err <= 1e-12, (call, b, err)
            err = np.linalg.norm(got[b] - ctx_out[b]) / np.linalg.norm(ctx_out[b])
            assert err <= 1e-12, (call, b, err)
    ctx.close()


def test_static_entry_through_the_binding(lbm):
    """The Python wrapper of the same entry point (argument checks only),
    twice in a row, against the oracle."""
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    w = make_workload("d3_single", B=5, nslices=3)
    Pn = _props(w)
    P = torch.from_numpy(Pn).to(dev)
    ref = O.propagate_chain(Pn, w["states"], 4)
    for _ in range(2):
        x = torch.from_numpy(w["states"]).to(dev)
        lbm.lb_propagate_batch_static(P, x, steps_per_slice=4)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        assert np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)) <= 1e-12


def test_static_entry_rejects_host_memory(lbm):
    """Pointers that are not device memory of the current device are refused
    before any work is queued."""
    n = 9
    P = torch.zeros((1, n, n), dtype=torch.complex128).pin_memory()
    x = torch.zeros((2, n), dtype=torch.complex128, device="cuda:0")
    L = lbm.lib()
    before = lbm.lb_launch_count()
    st = L.lb_propagate_batch_static(n, 1, ctypes.c_void_p(P.data_ptr()), 1, 2, ctypes.c_void_p(x.data_ptr()), None)
    assert st == 1  # LB_EINVAL
    assert lbm.lb_launch_count() == before


def test_static_entry_rejects_sizes_beyond_its_buffer(lbm):
    dev = torch.device("cuda:0")
    n, B = 729, 360  # 360 * 729 = 262440 > 262144
    P = torch.zeros((1, n, n), dtype=torch.complex128, device=dev)
    x = torch.zeros((B, n), dtype=torch.complex128, device=dev)
    L = lbm.lib()
    before = lbm.lb_launch_count()
    st = L.lb_propagate_batch_static(n, 1, ctypes.c_void_p(P.data_ptr()), 1, B, ctypes.c_void_p(x.data_ptr()), None)
    assert st == 8  # LB_EUNSUPPORTED
    assert lbm.lb_launch_count() == before
