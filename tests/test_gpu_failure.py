"""Failure detection without a GPU fault.

* A device-side wait that runs out: lb_selftest_wait_timeout queues the
  bounded mbarrier wait the tensor-core kernels use on a barrier that
  nothing completes; the wait gives up after its cycle limit, the error word
  reports LB_ETIMEOUT once, and the context keeps working.
* Guard bands: every output buffer is placed inside a larger allocation
  filled with a sentinel; after each call at ragged sizes (n not a multiple
  of any tile, odd batches) the sentinel around the output is intact, so no
  kernel writes outside what it was given.
"""

import numpy as np
import pytest

import oracle as O
from workloads import make_workload
from workloads.rng import ginibre_states, normal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SENTINEL = complex(1.2345e300, -6.789e-300)
GUARD = 4096


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _guarded(shape, dtype=torch.complex128, fill=None):
    """A tensor of `shape` inside a buffer with GUARD sentinel elements on each
    side; returns (view, buffer)."""
    dev = torch.device("cuda:0")
    count = int(np.prod(shape))
    buf = torch.empty(count + 2 * GUARD, dtype=dtype, device=dev)
    buf.fill_(SENTINEL if dtype.is_complex else 1.2345e30)
    view = buf[GUARD:GUARD + count].view(*shape)
    if fill is not None:
        view.copy_(torch.as_tensor(np.ascontiguousarray(fill), device=dev).to(dtype).view(*shape))
    return view, buf


def _intact(buf, dtype=torch.complex128):
    s = SENTINEL if dtype.is_complex else 1.2345e30
    head, tail = buf[:GUARD].cpu().numpy(), buf[-GUARD:].cpu().numpy()
    return bool(np.all(head == s) and np.all(tail == s))


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _model(d, seed):
    H = _rand_c(seed, (d, d))
    H = 0.5 * (H + H.conj().T) / d
    X = _rand_c(seed + 1, (d, d))
    X = 0.5 * (X + X.conj().T) / d
    jumps = 0.05 * np.stack([_rand_c(seed + 2, (d, d)), _rand_c(seed + 3, (d, d))]) / d
    return H, jumps, X


def test_bounded_wait_times_out_and_context_recovers(lbm):
    dev = torch.device("cuda:0")
    ctx = lbm.Context(0, max_n=9, max_batch=3, max_slices=2)
    lbm.lb_selftest_wait_timeout(ctx, 2_000_000)  # about 1 ms
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_sync_status(ctx)
    assert ei.value.name == "LB_ETIMEOUT"
    lbm.lb_sync_status(ctx)  # the word was cleared
    w = make_workload("d3_single", B=3, nslices=2, steps_per_slice=5)
    Ps = O.slice_propagators(O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"]),
                             np.array([0.05, -0.03]), w["dt"])
    R = torch.from_numpy(w["states"]).to(dev)
    lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).to(dev), R, steps_per_slice=5)
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, w["states"], 5)
    assert np.max(np.abs(R.cpu().numpy() - ref)) <= 1e-12


@pytest.mark.parametrize("d,S,prec", [(2, 3, "fp64"), (5, 2, "fp32"), (5, 2, "bf16x3"), (10, 2, "fp64"),
                                      (10, 2, "bf16x3"), (11, 1, "fp32")])
def test_guard_bands_build_and_propagate(lbm, d, S, prec):
    dev = torch.device("cuda:0")
    n = d * d
    H, jumps, X = _model(d, 0x5EED0300 + d)
    ctx = lbm.Context(0, max_n=n, max_batch=37, max_slices=S)
    Lb, Lbb = _guarded((n, n))
    Ld, Ldb = _guarded((n, n))
    lbm.lb_assemble(ctx, torch.from_numpy(H).to(dev), torch.from_numpy(jumps).to(dev), Lb)
    lbm.lb_assemble(ctx, torch.from_numpy(X).to(dev), None, Ld)
    u = torch.from_numpy(np.linspace(-0.1, 0.1, S)).to(dev)
    P, Pb = _guarded((S, n, n))
    lbm.lb_expm_pade(ctx, Lb, Ld, u, 0.1, P, prec=prec)
    lbm.lb_sync_status(ctx)
    B = 37
    R, Rb = _guarded((B, n), fill=ginibre_states(0x5EED0400 + d, d, B))
    lbm.lb_propagate_batch(ctx, P, R, steps_per_slice=2, prec=prec, renorm_trace=(prec != "fp64"))
    lbm.lb_sync_status(ctx)
    for b in (Lbb, Ldb, Pb, Rb):
        assert _intact(b)
    assert torch.isfinite(torch.view_as_real(R)).all()


def test_guard_bands_instances_and_grape(lbm):
    dev = torch.device("cuda:0")
    from workloads import transmon_chain

    ctx = lbm.Context(0, max_n=81, max_batch=16, max_slices=4)
    bufs, arg = [], []
    for k, (nq, S, B) in enumerate([(1, 3, 5), (2, 2, 9), (1, 4, 1)]):
        m = transmon_chain(nq)
        Lb = torch.from_numpy(O.lindbladian(m.H0, m.jumps)).to(dev)
        Ld = torch.from_numpy(O.drive_generator(m.X)).to(dev)
        st, stb = _guarded((B, m.d * m.d), fill=ginibre_states(0x5EED0500 + k, m.d, B))
        bufs.append(stb)
        arg.append(dict(Lbase=Lb, Ldrv=Ld, u=torch.full((S,), 0.05, dtype=torch.float64, device=dev), states=st))
    lbm.lb_run_instances(ctx, arg, 0.1, prec="fp64")
    lbm.lb_sync_status(ctx)
    for b in bufs:
        assert _intact(b)
    # GRAPE: fidelity (1) and gradient (S) outputs
    m = transmon_chain(1)
    n, S = 9, 4
    Lb = torch.from_numpy(O.lindbladian(m.H0, m.jumps)).to(dev)
    Ld = torch.from_numpy(O.drive_generator(m.X)).to(dev)
    X0 = np.zeros((4, n), dtype=complex)
    for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        X0[b, i * 3 + j] = 1.0
    X0d = torch.from_numpy(X0).to(dev)
    F, Fb = _guarded((1,), dtype=torch.float64)
    g, gb = _guarded((S,), dtype=torch.float64)
    lbm.lb_grape_grad(ctx, Lb, Ld, torch.full((S,), 0.05, dtype=torch.float64, device=dev), m.dt, 2, X0d, X0d,
                      F, g)
    lbm.lb_sync_status(ctx)
    assert _intact(Fb, torch.float64) and _intact(gb, torch.float64)
