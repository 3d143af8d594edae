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


def _one(z):
    return np.array([[z]], dtype=np.complex128)


def test_fp32_steps_by_hand():
    """d = 1 (a 1 x 1 propagator p, a state x), worked out by hand in binary32.
    (a) p = 1 + 2^-30, x = 1 + 2^-23: the increment (p - 1) x = 2^-30 + 2^-53
    is below half an ulp of x (2^-24), so two FP32 steps leave x exactly as
    it was (accumulating in FP64 would not).  (b) p = 1 + i 2^-10, x = 1:
    x1 = 1 + i 2^-10, x2 = (1 - 2^-20) + i 2^-9, all exact (the sign of the
    Im x Im term).  (c) with the trace division a 1 x 1 state becomes 1."""
    out = Q.propagate_fp32(_one(1 + 2.0 ** -30), _one(1 + 2.0 ** -23), 2, renorm=False)
    assert out[0, 0] == 1 + 2.0 ** -23
    out = Q.propagate_fp32(_one(1 + 1j * 2.0 ** -10), _one(1.0), 2, renorm=False)
    assert out[0, 0] == (1 - 2.0 ** -20) + 1j * 2.0 ** -9
    out = Q.propagate_fp32(_one(1 + 1j * 2.0 ** -10), _one(1.0), 2, renorm=True)
    assert abs(out[0, 0] - 1.0) <= 2.0 ** -22


def test_bf16x3_step_by_hand():
    """One split-BF16 step at d = 1, worked out by hand.  x = (1 + 2^-9)(1 + i)
    splits into x0 = 1, x1 = 2^-9 (both parts); D = p - 1 with
    Re D = 16 (1 + 2^-9 + 2^-18) -> pieces 16, 2^-5, 2^-14 and
    Im D = 16 (1 + 2^-9) -> pieces 16, 2^-5, 0.  With the five products
    x_i d_j, i + j <= 2, Re y = sum (xr_i dr_j - xi_i di_j) = 2^-14 and
    Im y = 32 + 2^-3 + 3 2^-14, so x + y = (1 + 2^-9 + 2^-14)
    + i (33 + 2^-3 + 2^-9 + 3 2^-14), exact in binary32.  The sixth product
    x1 d2 would add 2^-23 to the real part."""
    D = 16 * (1 + 2.0 ** -9 + 2.0 ** -18) + 16j * (1 + 2.0 ** -9)
    x = (1 + 2.0 ** -9) * (1 + 1j)
    out = Q.propagate_bf16x3(_one(1 + D), _one(x), 1, renorm=False)
    assert out[0, 0].real == 1 + 2.0 ** -9 + 2.0 ** -14
    assert out[0, 0].imag == 33 + 2.0 ** -3 + 2.0 ** -9 + 3 * 2.0 ** -14
    out = Q.propagate_bf16x3(_one(1 + 1j * 2.0 ** -10), _one(1.0), 2, renorm=True)
    assert abs(out[0, 0] - 1.0) <= 2.0 ** -22
