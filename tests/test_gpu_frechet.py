"""Propagators and their control derivatives (lb_expm_frechet) and the
first-order reuse of P for nearby controls (lb_control_update), against the
oracle: P by Algorithm 1, dP/du by Van Loan's block-triangular exponential
(an independent route), and the reuse error against a rebuild."""

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


def _relf(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _setup(lbm, nq, u):
    dev = torch.device("cuda:0")
    m = transmon_chain(nq)
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    n = Lb.shape[0]
    S = len(u)
    ctx = lbm.Context(0, max_n=n, max_batch=4, max_slices=S)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    dP = torch.empty_like(P)
    lbm.lb_expm_frechet(ctx, t(Lb), t(Ld), t(np.asarray(u, dtype=np.float64)), m.dt, P, dP)
    lbm.lb_sync_status(ctx)
    return m, Lb, Ld, P.cpu().numpy(), dP.cpu().numpy(), t


@pytest.mark.parametrize("nq", [1, 2])
def test_expm_frechet_matches_oracle(lbm, nq):
    u = [0.05, -0.08, 0.1]
    m, Lb, Ld, P, dP, _ = _setup(lbm, nq, u)
    for s, us in enumerate(u):
        A = O.slice_generator(Lb, Ld, us) * m.dt
        assert _relf(P[s], O.expm_pade13(A)) <= 1e-12
        assert _relf(dP[s], O.frechet_expm(A, Ld * m.dt)) <= 1e-10, (s, _relf(dP[s], O.frechet_expm(A, Ld * m.dt)))


def test_control_update_is_second_order(lbm):
    u = np.array([0.05, -0.03, 0.07, 0.0])
    m, Lb, Ld, P, dP, t = _setup(lbm, 2, u)
    errs = []
    for delta in (1e-1, 1e-2, 1e-3):
        dl = np.full(len(u), delta)
        out = torch.empty((len(u),) + P.shape[1:], dtype=torch.complex128, device="cuda:0")
        lbm.lb_control_update(t(P), t(dP), t(dl), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        exact = O.slice_propagators(Lb, Ld, u + delta, m.dt)
        errs.append(max(_relf(got[s], exact[s]) for s in range(len(u))))
        # the update is exactly P + delta dP
        assert np.allclose(got, P + delta * dP, rtol=0, atol=1e-15)
    # second order: the error falls by about 100 per decade of delta
    assert errs[1] / errs[0] < 0.02 and errs[2] / errs[1] < 0.02, errs
    assert errs[2] <= 1e-6, errs
