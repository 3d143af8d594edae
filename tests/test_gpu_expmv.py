"""The action of the slice propagators without forming them (lb_expmv):
the same (m, s) as the oracle's rule, states within 1e-12 of the oracle's
Taylor route and of the dense Pade route, for few states (warp-per-row
products) and many (tiled GEMM), with and without a drive, through several
slices and across slice chunks."""

import numpy as np
import pytest

import oracle as O
from oracle import expmv as E
from workloads import transmon_chain
from workloads.rng import ginibre_states
from workloads.transmon import paper_grape_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("model,B,S,max_slices", [
    ("chain1", 1, 3, 8), ("chain1", 8, 2, 8), ("chain1", 20, 2, 8),
    ("chain2", 1, 2, 8), ("chain2", 5, 3, 2), ("chain2", 64, 2, 8),
    ("paper3", 2, 4, 8), ("chain3", 1, 1, 2), ("chain3", 12, 1, 2),
])
def test_expmv_matches_oracle(lbm, model, B, S, max_slices):
    if model.startswith("chain"):
        m = transmon_chain(int(model[-1]))
    else:
        m = paper_grape_model(int(model[-1]))
    Lb, Ld = O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)
    n = Lb.shape[0]
    u = np.linspace(-0.08, 0.1, S)
    X = ginibre_states(70 + B, m.d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=max(B, 8), max_slices=max_slices)
    Xd = _t(X)
    ms = lbm.lb_expmv(ctx, _t(Lb), _t(Ld), _t(u), m.dt, Xd)
    lbm.lb_sync_status(ctx)
    ref, ms_ref = E.expmv_chain(Lb, Ld, u, m.dt, X)
    assert ms == ms_ref
    got = Xd.cpu().numpy()
    assert _rel(got, ref) <= 1e-12
    if n <= 81:  # the dense route agrees too
        R = X.copy()
        for us in u:
            R = R @ O.expm_pade13((Lb + us * Ld) * m.dt).T
        assert _rel(got, R) <= 1e-12
    ctx.close()


def test_expmv_per_slice_generators_and_large_norm(lbm):
    # Ldrv = None: one generator per slice; dt large enough for many sub-steps
    m = transmon_chain(1)
    Lb, Ld = O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)
    gens = np.array([Lb + us * Ld for us in (0.05, -0.02, 0.11)])
    dt = 400.0 * m.dt  # ||A||_1 near 67: several sub-steps
    X = ginibre_states(5, m.d, 3)
    ctx = lbm.Context(0, max_n=9, max_batch=8, max_slices=2)
    Xd = _t(X)
    ms = lbm.lb_expmv(ctx, _t(gens), None, None, dt, Xd)
    a = max(E.onenorm(G * dt) for G in gens)
    assert ms == E.parameters(a) and ms[1] > 1
    R = X.copy()
    for G in gens:
        R = E.expmv(G * dt, R, ms)
    assert _rel(Xd.cpu().numpy(), R) <= 1e-12
    ctx.close()


def test_expmv_errors(lbm):
    ctx = lbm.Context(0, max_n=9, max_batch=2, max_slices=1)
    L = torch.zeros((9, 9), dtype=torch.complex128, device="cuda")
    L[0, 0] = float("nan")
    X = torch.zeros((1, 9), dtype=torch.complex128, device="cuda")
    with pytest.raises(lbm.LBError) as e:
        lbm.lb_expmv(ctx, L.reshape(1, 9, 9), None, None, 0.1, X)
    assert e.value.name == "LB_ENONFINITE"
    # zero generator: (m, s) = (1, 1) and the states stay
    X = torch.ones((2, 9), dtype=torch.complex128, device="cuda")
    assert lbm.lb_expmv(ctx, torch.zeros((1, 9, 9), dtype=torch.complex128, device="cuda"), None, None, 0.1, X) == (1, 1)
    assert torch.equal(X.cpu(), torch.ones((2, 9), dtype=torch.complex128))
    ctx.close()


@pytest.mark.parametrize("model,B,S", [("chain1", 1, 3), ("chain1", 8, 2), ("chain2", 3, 2), ("paper3", 2, 4),
                                       ("chain3", 1, 2), ("chain3", 5, 1)])
def test_expmv_hermitian_matches_oracle(lbm, model, B, S):
    """Density matrices on their real coordinates: within 1e-12 of the
    oracle's complex Taylor route, exactly Hermitian."""
    if model.startswith("chain"):
        m = transmon_chain(int(model[-1]))
    else:
        m = paper_grape_model(int(model[-1]))
    Lb, Ld = O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)
    n = Lb.shape[0]
    u = np.linspace(-0.08, 0.1, S)
    X = ginibre_states(90 + B, m.d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=max(B, 8), max_slices=S)
    Xd = _t(X)
    lbm.lb_expmv(ctx, _t(Lb), _t(Ld), _t(u), m.dt, Xd, hermitian=True)
    lbm.lb_sync_status(ctx)
    ref, _ = E.expmv_chain(Lb, Ld, u, m.dt, X)
    got = Xd.cpu().numpy()
    assert _rel(got, ref) <= 1e-12
    rho = got.reshape(B, m.d, m.d)
    assert np.array_equal(rho, np.conj(np.transpose(rho, (0, 2, 1))))
    ctx.close()


def test_expmv_hermitian_large_batch_is_the_complex_route(lbm):
    m = transmon_chain(1)
    Lb, Ld = O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)
    u = np.array([0.03, -0.05])
    X = ginibre_states(123, m.d, 12)
    ctx = lbm.Context(0, max_n=9, max_batch=12, max_slices=2)
    outs = []
    for herm in (False, True):
        Xd = _t(X)
        lbm.lb_expmv(ctx, _t(Lb), _t(Ld), _t(u), m.dt, Xd, hermitian=herm)
        lbm.lb_sync_status(ctx)
        outs.append(Xd.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    ctx.close()
