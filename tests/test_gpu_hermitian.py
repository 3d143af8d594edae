"""FP64 propagation of density matrices on their real coordinates
(lb_propagate_batch with prec LB_FP64_HERMITIAN) against the oracle's
complex product: within 1e-12 for Hermitian states at n = 1, 4 and 9 (the
one-warp form) and 16 <= n <= 81 (the shared-memory form), the d = 3
single-state workload over 10^4 steps, outputs exactly Hermitian, the
upper-triangle reading of the input, and the complex FP64 path above
n = 81."""

import numpy as np
import pytest

import oracle as O
from workloads import make_workload
from workloads.rng import ginibre_states

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _gen(d, seed, scale):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    H = (H + H.conj().T) / 2
    Ls = np.array([(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) * 0.3 for _ in range(2)])
    X = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    return O.lindbladian(H * scale, Ls * np.sqrt(scale)), O.drive_generator((X + X.conj().T) / 2 * scale)


def _props(d, S, seed=11, scale=0.2):
    Lb, Ld = _gen(d, seed + d, scale)
    return np.array([O.expm_pade13(Lb + u * Ld) for u in np.linspace(-0.3, 0.3, S)])


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("d,B,S,m", [(1, 3, 2, 5), (2, 1, 3, 50), (2, 40, 2, 7), (3, 1, 1, 200), (3, 5, 3, 4),
                                     (3, 300, 2, 3)])
def test_hermitian_form_matches_oracle(lbm, d, B, S, m):
    n = d * d
    Ps = _props(d, S)
    X0 = ginibre_states(500 + d, d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=S)
    R = torch.from_numpy(X0).cuda()
    lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).cuda(), R, steps_per_slice=m, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, X0, m)
    got = R.cpu().numpy()
    for b in range(B):
        assert _rel(got[b], ref[b]) <= 1e-12, b
    rho = got.reshape(B, d, d)
    assert np.array_equal(rho, np.conj(np.transpose(rho, (0, 2, 1))))  # exactly Hermitian
    ctx.close()


def test_d3_single_state_workload(lbm):
    w = make_workload("d3_single")
    Lb, Ld = O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"])
    Ps = np.array([O.expm_pade13(O.slice_generator(Lb, Ld, u) * w["dt"]) for u in w["u"]])
    ctx = lbm.Context(0, max_n=9, max_batch=1, max_slices=1)
    R = torch.from_numpy(w["states"]).cuda()
    lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).cuda(), R, steps_per_slice=w["steps_per_slice"],
                           prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, w["states"], w["steps_per_slice"])
    assert _rel(R.cpu().numpy(), ref) <= 1e-12
    ctx.close()


def test_reads_the_upper_triangle(lbm):
    # the lower triangle is not read: a state whose lower triangle is
    # garbage propagates like the Hermitian matrix of its upper triangle
    d, B = 3, 4
    Ps = _props(d, 2)
    X0 = ginibre_states(77, d, B).reshape(B, d, d)
    herm = X0.copy()
    junk = X0.copy()
    iu = np.tril_indices(d, -1)
    junk[:, iu[0], iu[1]] = 5.0 - 7.0j
    junk[:, range(d), range(d)] += 3.0j  # imaginary diagonal parts are not read either
    ctx = lbm.Context(0, max_n=9, max_batch=B, max_slices=2)
    R = torch.from_numpy(junk.reshape(B, 9)).cuda()
    lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).cuda(), R, steps_per_slice=3, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, herm.reshape(B, 9), 3)
    assert _rel(R.cpu().numpy(), ref) <= 1e-12
    ctx.close()


@pytest.mark.parametrize("d,B,S,m", [(4, 3, 2, 5), (5, 2, 1, 20), (9, 1, 2, 3), (9, 200, 1, 50), (9, 1030, 1, 4)])
def test_shared_memory_form_matches_oracle(lbm, d, B, S, m):
    """9 < n <= 81: R and the states in shared memory, one thread per
    output coordinate; B = 1030 leaves a ragged last CTA."""
    n = d * d
    Ps = _props(d, S, scale=0.05)
    X0 = ginibre_states(700 + d + B, d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=S)
    R = torch.from_numpy(X0).cuda()
    lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).cuda(), R, steps_per_slice=m, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, X0, m)
    got = R.cpu().numpy()
    for b in range(B):
        assert _rel(got[b], ref[b]) <= 1e-12, b
    rho = got.reshape(B, d, d)
    assert np.array_equal(rho, np.conj(np.transpose(rho, (0, 2, 1))))
    ctx.close()


@pytest.mark.parametrize("d,B", [(11, 3), (11, 40)])
def test_above_n81_runs_the_real_product(lbm, d, B):
    """n = 121: one real product per step on the real coordinates (the
    few-state form for B <= 8, the real GEMM above); equal to the complex
    FP64 path within 1e-12 relative and exactly Hermitian."""
    n = d * d
    Ps = _props(d, 2, scale=0.05)
    X0 = ginibre_states(600 + d, d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=2)
    outs = {}
    for prec in ("fp64", "fp64_hermitian"):
        R = torch.from_numpy(X0).cuda()
        lbm.lb_propagate_batch(ctx, torch.from_numpy(Ps).cuda(), R, steps_per_slice=4, prec=prec)
        lbm.lb_sync_status(ctx)
        outs[prec] = R.cpu().numpy()
    for b in range(B):
        assert _rel(outs["fp64_hermitian"][b], outs["fp64"][b]) <= 1e-12
    rho = outs["fp64_hermitian"].reshape(B, d, d)
    assert np.array_equal(rho, np.conj(np.transpose(rho, (0, 2, 1))))
    ctx.close()


def test_unknown_precision_is_rejected(lbm):
    ctx = lbm.Context(0, max_n=9, max_batch=2, max_slices=1)
    L = torch.zeros((1, 9, 9), dtype=torch.complex128, device="cuda")
    P = torch.empty((1, 9, 9), dtype=torch.complex128, device="cuda")
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_expm_pade(ctx, L, None, None, 0.1, P, prec=7)
    assert ei.value.name == "LB_EINVAL"
    ctx.close()
