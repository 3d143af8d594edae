"""Pins of the rounding emulator of the reduced-precision forms: BF16
rounding worked out by hand from the format (7 stored fraction bits, ties
to even), the piece splits against their error bounds, the reduction to the
exact case, and the stated accuracy of the forms after 1000 steps."""

import numpy as np
import pytest

import oracle as O
from oracle import precision as Q
from workloads import transmon_chain
from workloads.rng import ginibre_states


def test_bf16_rounding_by_hand():
    # spacing of BF16 at 1.0 is 2^-7
    cases = [
        (1.0, 1.0),
        (1.0 + 2.0 ** -8, 1.0),                           # tie -> even (1.0)
        (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),           # tie between 1+2^-7 (odd) and 1+2^-6 (even)
        (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),  # just above the tie
        (-2.5, -2.5),
        (3.14159265358979, 3.140625),                     # 1.1001001|0000111... x 2^1, rounded down
        (0.1, 0.10009765625),                             # 1.1001100|1100... x 2^-4, rounded up
        (2.0 ** -130, 2.0 ** -130),                       # float32 subnormal with one bit
    ]
    for x, want in cases:
        assert float(Q.round_bf16(np.array([x]))[0]) == want, x
    assert np.isnan(Q.round_bf16(np.array([np.nan]))[0])
    assert Q.round_bf16(np.array([np.inf]))[0] == np.inf


def test_split_error_bounds():
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    for pieces, bits in ((1, 8), (2, 16), (3, 24)):
        p = Q.split_bf16(x, pieces)
        rest = x.astype(np.float64) - sum(q.astype(np.float64) for q in p)
        assert np.all(np.abs(rest) <= 2.0 ** -bits * np.abs(x.astype(np.float64)) * (1 + 1e-12)), pieces
        for q in p:  # every piece is a BF16 value
            assert np.array_equal(Q.round_bf16(q), q)
    # a float32 value is exactly the sum of its three pieces
    p = Q.split_bf16(x, 3)
    assert np.array_equal(sum(q.astype(np.float64) for q in p), x.astype(np.float64))


def _model():
    m = transmon_chain(1)
    P = O.expm_pade13(O.slice_generator(O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X), 0.05) * m.dt)
    return P, ginibre_states(31, m.d, 6)


def test_exact_case():
    # P = I: the D-form step adds nothing, states stay (already unit trace)
    _, X = _model()
    X32 = X.astype(np.complex64).astype(np.complex128)
    for f in (Q.propagate_fp32, Q.propagate_bf16x3):
        out = f(np.eye(9), X, 5)
        assert np.max(np.abs(out - X32)) <= 2e-7


def test_stated_accuracy_after_1000_steps():
    # FP32 <= 1e-5 and split-BF16 <= 1e-4 in Frobenius norm per state, and
    # both visibly rounded (not the FP64 result)
    P, X = _model()
    ref = O.propagate(P, X, 1000)
    e32 = np.max(np.linalg.norm(Q.propagate_fp32(P, X, 1000) - ref, axis=1))
    e16 = np.max(np.linalg.norm(Q.propagate_bf16x3(P, X, 1000) - ref, axis=1))
    assert 1e-9 < e32 <= 1e-5, e32
    assert 1e-9 < e16 <= 1e-4, e16
