"""Fixed-point propagation on the GPU (lb_fixed_quantize, lb_propagate_fixed,
lb_fixed_dequantize) against the integer oracle of Algorithm alg:fpga:
bit-exact codes for Q1.15 and Q1.31, on the board's d = 3 drift study, on
random codes over the whole range, at the largest supported n, and on the
saturation and floor cases worked out by hand in the oracle tests."""

import json
import os

import numpy as np
import pytest

import oracle as O
from oracle import fixed as F
from workloads.transmon import paper_grape_model

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fpga_drift.json")
CODE = {15: torch.int16, 31: torch.int32}


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _codes(re, im, f):
    a = np.stack([np.asarray(re, dtype=np.int64), np.asarray(im, dtype=np.int64)], axis=-1)
    return torch.from_numpy(a.astype(np.int16 if f == 15 else np.int32)).cuda()


def _split(t):
    a = t.cpu().numpy().astype(np.int64)
    return a[..., 0], a[..., 1]


def _d3(driven):
    m = paper_grape_model(3)
    sx = np.zeros((3, 3), dtype=np.complex128)
    sx[0, 1] = sx[1, 0] = 1.0
    H = m.H0 + (0.05 * sx if driven else 0.0)
    return O.expm_pade13(O.lindbladian(H, m.jumps) * m.dt)


@pytest.mark.parametrize("f", [15, 31])
@pytest.mark.parametrize("driven", [False, True])
def test_board_drift_bit_exact(lbm, f, driven):
    # the d = 3 drift study of Table tab:fpga_drift_hw: quantise P and
    # |0><0| on the GPU, run 1, 10, 100, 1000, 10000 steps, compare every code
    P = _d3(driven)
    Pq = torch.empty((9, 9, 2), dtype=CODE[f], device="cuda")
    lbm.lb_fixed_quantize(torch.from_numpy(P).cuda(), Pq, f)
    Pr, Pi = F.quantize(P, f)
    gr, gi = _split(Pq)
    assert np.array_equal(gr, Pr) and np.array_equal(gi, Pi)
    r0 = np.zeros((1, 9), dtype=np.complex128)
    r0[0, 0] = 1.0
    X = torch.empty((1, 9, 2), dtype=CODE[f], device="cuda")
    lbm.lb_fixed_quantize(torch.from_numpy(r0).cuda(), X, f)
    Rr, Ri = F.quantize(r0, f)
    done = 0
    rows = {r["steps"]: r for r in json.load(open(GOLDEN))["rows"] if r["case"] == ("driven" if driven else "undriven")}
    ref = r0[0].copy()
    for N in (1, 10, 100, 1000, 10000):
        lbm.lb_propagate_fixed(Pq, X, N - done, f)
        Rr, Ri = F.fixed_propagate_batch(Pr, Pi, Rr, Ri, N - done, f)
        for _ in range(N - done):
            ref = P @ ref
        done = N
        gr, gi = _split(X)
        assert np.array_equal(gr, Rr) and np.array_equal(gi, Ri), N
        if f == 15:
            # the printed population error of the board, from the GPU's codes
            x = torch.empty((1, 9), dtype=torch.complex128, device="cuda")
            lbm.lb_fixed_dequantize(X, x, f)
            q = x.cpu().numpy()[0].reshape(3, 3)
            assert "%.2e" % abs(q[1, 1].real - ref.reshape(3, 3)[1, 1].real) == rows[N]["delta_p1"]


@pytest.mark.parametrize("f,n,B,steps", [
    (15, 9, 1, 3), (15, 9, 300, 25), (15, 81, 1000, 12), (15, 4, 7, 5), (15, 1, 33, 40),
    (15, 16, 40, 9), (15, 25, 7, 5), (15, 9, 5000, 3),
    (31, 9, 300, 10), (31, 81, 3, 4), (31, 4, 5, 6), (31, 1, 2, 30), (31, 16, 3, 4),
])
def test_random_codes_bit_exact(lbm, f, n, B, steps):
    # codes over the whole range (P scaled so sums wander but also saturate),
    # several CTAs with a ragged last one, the largest n (P in shared memory)
    rng = np.random.default_rng(1000 * f + 10 * n + B)
    lo, hi = F.code_range(f)
    Pr = rng.integers(lo // n, hi // n + 1, size=(n, n))
    Pi = rng.integers(lo // n, hi // n + 1, size=(n, n))
    Rr = rng.integers(lo, hi + 1, size=(B, n))
    Ri = rng.integers(lo, hi + 1, size=(B, n))
    X = _codes(Rr, Ri, f)
    lbm.lb_propagate_fixed(_codes(Pr, Pi, f), X, steps, f)
    er, ei = F.fixed_propagate_batch(Pr, Pi, Rr, Ri, steps, f)
    gr, gi = _split(X)
    assert np.array_equal(gr, er) and np.array_equal(gi, ei)


@pytest.mark.parametrize("f", [15, 31])
def test_extreme_codes_saturate(lbm, f):
    # every code -2^f: each product is +2^(2f); n = 4 terms of two products
    # give 2^(2f+3), past 64 bits for Q1.31; the write-back saturates high
    lo, hi = F.code_range(f)
    n = 4
    Pr = np.full((n, n), lo)
    Pi = np.full((n, n), lo)
    Rr = np.full((2, n), lo)
    Ri = np.full((2, n), lo)
    X = _codes(Rr, Ri, f)
    lbm.lb_propagate_fixed(_codes(Pr, Pi, f), X, 3, f)
    er, ei = F.fixed_propagate_batch(Pr, Pi, Rr, Ri, 3, f)
    gr, gi = _split(X)
    assert np.array_equal(gr, er) and np.array_equal(gi, ei)
    # first step by hand: re = sum (P_r r_r - P_i r_i) = 0 ; im = 2 n 2^(2f) -> saturates at 2^f - 1
    X = _codes(Rr, Ri, f)
    lbm.lb_propagate_fixed(_codes(Pr, Pi, f), X, 1, f)
    gr, gi = _split(X)
    assert (gr == 0).all() and (gi == hi).all()


def test_hand_cases(lbm):
    def one(P, r, f=15):
        X = _codes([[r.real]], [[r.imag]], f)
        lbm.lb_propagate_fixed(_codes([[P.real]], [[P.imag]], f), X, 1, f)
        gr, gi = _split(X)
        return int(gr[0, 0]), int(gi[0, 0])

    assert one(16384 + 0j, 3 - 3j) == (1, -2)                 # floor(1.5), floor(-1.5)
    assert one(-32768 + 0j, -32768 + 0j) == (32767, 0)        # 2^30 / 2^15 saturates
    assert one(10000 + 20000j, 30000 - 4000j) == (11596, 17089)
    assert one((1 << 30) + 0j, 3 - 3j, 31) == (1, -2)


def test_quantize_matches_oracle_and_edges(lbm):
    rng = np.random.default_rng(5)
    x = (rng.standard_normal(5000) + 1j * rng.standard_normal(5000)) * 0.7
    x[:4] = [1.0, -1.0, 0.5 / 32768 + 1.5j / 32768, 2.5 / 32768 - 2.5j / 32768]  # saturation and ties to even
    for f in (15, 31):
        q = torch.empty((x.size, 2), dtype=CODE[f], device="cuda")
        lbm.lb_fixed_quantize(torch.from_numpy(x).cuda(), q, f)
        er, ei = F.quantize(x, f)
        gr, gi = _split(q)
        assert np.array_equal(gr, er) and np.array_equal(gi, ei)
        back = torch.empty(x.size, dtype=torch.complex128, device="cuda")
        lbm.lb_fixed_dequantize(q, back, f)
        assert np.array_equal(back.cpu().numpy(), F.dequantize(er, ei, f))
    # non-finite values: NaN -> 0, +-Inf saturate
    y = np.array([complex(np.nan, np.inf), complex(-np.inf, 0.25)])
    q = torch.empty((2, 2), dtype=torch.int16, device="cuda")
    lbm.lb_fixed_quantize(torch.from_numpy(y).cuda(), q, 15)
    assert q.cpu().numpy().tolist() == [[0, 32767], [-32768, 8192]]


def test_zero_steps_and_bad_arguments(lbm):
    X = _codes(np.ones((2, 9)), np.zeros((2, 9)), 15)
    before = X.clone()
    lbm.lb_propagate_fixed(_codes(np.eye(9), np.zeros((9, 9)), 15), X, 0, 15)
    torch.cuda.synchronize()
    assert torch.equal(X, before)
    with pytest.raises(ValueError):
        lbm.lb_propagate_fixed(X, X, 1, 31)  # int16 codes passed as Q1.31
