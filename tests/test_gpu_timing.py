"""The calls behind the GPU timing models (Eq. 7-9, Sec. 3.4):
lb_propagate_resident (states in host memory) and lb_propagate_host (P and
states in host memory, device buffers allocated per call) give the same
states as the device-resident lb_propagate_batch, bit for bit, and the
oracle's within the FP64 bound; the device probes run and return sane
values."""

import math

import numpy as np
import pytest

import oracle as O
from workloads import transmon_chain

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _propagator(nq):
    m = transmon_chain(nq)
    A = O.slice_generator(O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X), 0.03) * m.dt
    return O.expm_pade13(A)


def _states(n, B, seed):
    rng = np.random.default_rng(seed)
    d = int(round(math.sqrt(n)))
    out = np.empty((B, n), dtype=np.complex128)
    for q in range(B):
        G = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
        rho = G @ G.conj().T
        out[q] = (rho / np.trace(rho)).reshape(-1)
    return out


@pytest.mark.parametrize("nq,B", [(1, 1), (1, 128), (2, 8), (3, 1), (3, 32)])
def test_resident_and_host_calls_match_device_call(lbm, nq, B):
    P = _propagator(nq)
    n = P.shape[0]
    X0 = _states(n, B, 10 * nq + B)
    ctx = lbm.Context(0, max_n=n, max_batch=max(B, 8), max_slices=1)
    Pd = torch.from_numpy(P).cuda()
    # kernel-only form: everything on the device
    Xd = torch.from_numpy(X0).cuda()
    lbm.lb_propagate_batch(ctx, Pd.reshape(1, n, n), Xd, 1, "fp64")
    lbm.lb_sync_status(ctx)
    dev_out = Xd.cpu().numpy()
    # resident P: states in (pageable) host memory
    Xh = torch.from_numpy(X0.copy())
    lbm.lb_propagate_resident(ctx, Pd, Xh)
    assert np.array_equal(Xh.numpy(), dev_out)
    # host-visible: P in host memory too
    Xh2 = torch.from_numpy(X0.copy())
    lbm.lb_propagate_host(ctx, torch.from_numpy(P), Xh2)
    assert np.array_equal(Xh2.numpy(), dev_out)
    lbm.lb_sync_status(ctx)
    ref = O.propagate(P, X0, 1)
    assert np.linalg.norm(dev_out - ref) / np.linalg.norm(ref) <= 1e-12
    ctx.close()


def test_resident_call_rejects_device_states(lbm):
    P = torch.eye(9, dtype=torch.complex128, device="cuda")
    ctx = lbm.Context(0, max_n=9, max_batch=2, max_slices=1)
    with pytest.raises(ValueError):
        lbm.lb_propagate_resident(ctx, P, torch.zeros((2, 9), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError):
        lbm.lb_propagate_host(ctx, P, torch.zeros((2, 9), dtype=torch.complex128))
    with pytest.raises(lbm.LBError):
        lbm.lb_propagate_resident(ctx, P, torch.zeros((3, 9), dtype=torch.complex128))  # B above max_batch
    ctx.close()


def test_probes_run(lbm):
    launch = lbm.lb_probe_launch(200, False)
    launch_sync = lbm.lb_probe_launch(50, True)
    assert 0.0 < launch < 1000.0 and 0.0 < launch_sync < 10000.0
    h = torch.zeros(1 << 16, dtype=torch.float64)
    d = torch.empty(1 << 16, dtype=torch.float64, device="cuda")
    assert lbm.lb_probe_copy(h, d, True, 5) > 0.0
    assert lbm.lb_probe_copy(h, d, False, 5) > 0.0
    assert lbm.lb_probe_alloc(1 << 20, 3) > 0.0
    buf = torch.zeros(1 << 20, dtype=torch.complex128, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    for n in (0, 729):
        lbm.lb_probe_read(buf, n, sink)
    torch.cuda.synchronize()
    assert int(sink.item()) == 0  # the impossible match never fires on zeros
