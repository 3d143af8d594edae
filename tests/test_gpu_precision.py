"""The reduced-precision forms against the oracle's rounding emulator: after
1000 steps the GPU's error in each form is of the order the emulated
arithmetic predicts (between a tenth of and ten times the emulator's error,
so a form that silently ran at a higher precision fails too), besides being
within the stated bounds (FP32 1e-5, split-BF16 1e-4)."""

import numpy as np
import pytest

import oracle as O
from oracle import precision as Q
from workloads import transmon_chain
from workloads.rng import ginibre_states

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


@pytest.mark.parametrize("nq", [1, 2])
@pytest.mark.parametrize("prec,bound,emulate", [("fp32", 1e-5, Q.propagate_fp32),
                                                ("bf16x3", 1e-4, Q.propagate_bf16x3)])
def test_error_of_the_predicted_order(lbm, nq, prec, bound, emulate):
    m = transmon_chain(nq)
    P = O.expm_pade13(O.slice_generator(O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X), 0.05) * m.dt)
    B, N = 16, 1000
    X = ginibre_states(31, m.d, B)
    ref = O.propagate(P, X, N)
    predicted = np.max(np.linalg.norm(emulate(P, X, N) - ref, axis=1))
    ctx = lbm.Context(0, max_n=m.d * m.d, max_batch=B, max_slices=1)
    R = torch.from_numpy(X).cuda()
    lbm.lb_propagate_batch(ctx, torch.from_numpy(P[None]).cuda(), R, steps_per_slice=N, prec=prec, renorm_trace=True)
    lbm.lb_sync_status(ctx)
    err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
    assert err <= bound, (prec, err)
    assert err <= 10.0 * predicted, (prec, err, predicted)
    assert err >= 0.1 * predicted, (prec, err, predicted)
    ctx.close()
