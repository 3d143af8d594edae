"""Pins of the fixed-point oracle (Algorithm alg:fpga, Sec. 3.5).

Values come from the paper's board table (Table tab:fpga_drift_hw) and
figure caption (Figure fig:fixed_point_drift), from its cycle model
(Eq. eq:cost_fpga, Table tab:fpga_summary), and from small integer cases
worked out by hand below.
"""

import json
import os

import numpy as np
import pytest

from oracle import fixed as F
from oracle import lindblad as O
from workloads.transmon import paper_grape_model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fpga_drift.json")


def _drift_rows(case):
    g = json.load(open(GOLDEN))
    return g, [r for r in g["rows"] if r["case"] == case]


def _d3_propagator(driven):
    """The d = 3 model of the drift study: the GRAPE landscape model of
    Sec. 2.5 (H0 = diag(0, 1, 2), T1 = 50, T2 = 30, dt = 0.5) with the
    drive 0.05 sigma_x, sigma_x read as |0><1| + |1><0|."""
    m = paper_grape_model(3)
    sx = np.zeros((3, 3), dtype=np.complex128)
    sx[0, 1] = sx[1, 0] = 1.0
    H = m.H0 + (0.05 * sx if driven else 0.0)
    return O.expm_pade13(O.lindbladian(H, m.jumps) * m.dt)


def _drift(P, f, steps):
    """Q1.f and FP64 trajectories from |0><0|; yields (N, trace distance,
    |Tr rho - 1|, |delta p1|) at each N in steps."""
    Pr, Pi = F.quantize(P, f)
    r0 = np.zeros(9, dtype=np.complex128)
    r0[0] = 1.0
    rr, ri = F.quantize(r0, f)
    Rr, Ri = rr[None], ri[None]
    ref = r0.copy()
    done = 0
    for N in steps:
        Rr, Ri = F.fixed_propagate_batch(Pr, Pi, Rr, Ri, N - done, f)
        for _ in range(N - done):
            ref = P @ ref
        done = N
        q = F.dequantize(Rr[0], Ri[0], f).reshape(3, 3)
        r = ref.reshape(3, 3)
        td = 0.5 * np.linalg.svd(q - r, compute_uv=False).sum()
        yield N, td, abs(np.trace(q) - 1.0), abs(q[1, 1].real - r[1, 1].real)


def _fmt(x):
    return "%.2e" % x


def test_undriven_drift_matches_board_table():
    # every printed digit of the undriven rows: 1.0 becomes the largest
    # code, then each floor loses one LSB of the |0><0| population
    g, rows = _drift_rows("undriven")
    P = _d3_propagator(False)
    got = {N: (td, tl, dp) for N, td, tl, dp in _drift(P, 15, [r["steps"] for r in rows])}
    for r in rows:
        td, tl, dp = got[r["steps"]]
        assert _fmt(td) == r["trace_distance"], r
        assert _fmt(tl) == r["trace_loss"], r
        assert dp == 0.0, r


def test_driven_population_error_matches_board_table():
    # the |delta p1| column of the driven rows, and the trace loss of the
    # first step; the printed trace-distance and trace-loss entries after
    # step 1 repeat the undriven values and are not pinned
    g, rows = _drift_rows("driven")
    P = _d3_propagator(True)
    got = {N: (td, tl, dp) for N, td, tl, dp in _drift(P, 15, [r["steps"] for r in rows])}
    for r in rows:
        td, tl, dp = got[r["steps"]]
        assert _fmt(dp) == r["delta_p1"], r
        if r["steps"] == 1:
            assert _fmt(tl) == r["trace_loss"], r


def test_q131_stays_below_caption_bound():
    # Figure fig:fixed_point_drift: Q1.31 stays below 1e-5 over 1e4 steps
    P = _d3_propagator(False)
    (_, td, tl, dp), = list(_drift(P, 31, [10000]))
    assert tl < 1e-5 and td < 1e-5
    assert tl == pytest.approx(10001 / 2.0 ** 31, rel=1e-12)  # one LSB per step plus the saturated 1.0


def test_writeback_floor_saturation_by_hand():
    # n = 1, f = 15: P = 0.5 (code 16384), rho = 3 - 3i
    #   acc = 16384*3 = 49152 -> floor(1.5) = 1 ; 16384*(-3) = -49152 -> floor(-1.5) = -2
    r, i, _ = F.fixed_propagate([[16384]], [[0]], [3], [-3], 1, 15)
    assert (int(r[0]), int(i[0])) == (1, -2)
    # (-1) * (-1): acc = 2^30 -> 32768 saturates to 32767; (-1) * (32767/32768) is exact
    r, i, _ = F.fixed_propagate([[-32768]], [[0]], [-32768], [0], 1, 15)
    assert (int(r[0]), int(i[0])) == (32767, 0)
    r, i, _ = F.fixed_propagate([[-32768]], [[0]], [32767], [0], 1, 15)
    assert (int(r[0]), int(i[0])) == (-32767, 0)
    # complex product: (10000 + 20000i)(30000 - 4000i)
    #   re = 3e8 + 8e7 = 380000000 -> floor(11596.68) = 11596
    #   im = -4e7 + 6e8 = 560000000 -> floor(17089.84) = 17089
    r, i, _ = F.fixed_propagate([[10000]], [[20000]], [30000], [-4000], 1, 15)
    assert (int(r[0]), int(i[0])) == (11596, 17089)
    # row i of P produces output i: P = [[32767, 0], [16384, 0]], rho = (32767, 0)
    #   out0 = floor(32767^2 / 32768) = 32766 ; out1 = floor(16384*32767 / 32768) = 16383
    r, i, _ = F.fixed_propagate([[32767, 0], [16384, 0]], [[0, 0], [0, 0]], [32767, 0], [0, 0], 1, 15)
    assert list(map(int, r)) == [32766, 16383] and list(map(int, i)) == [0, 0]


def test_q131_wide_accumulator_by_hand():
    # n = 1, f = 31: P = 0.5 (2^30), rho = 3 -> floor(1.5) = 1 ; rho = -3 -> -2
    r, i, _ = F.fixed_propagate([[1 << 30]], [[0]], [3], [-3], 1, 31)
    assert (int(r[0]), int(i[0])) == (1, -2)
    # n = 2, all codes -2^31: the real accumulator is 2 * 2^62 = 2^63, one
    # past the int64 range; floor(2^63 / 2^31) = 2^32 saturates to 2^31 - 1
    m = -(1 << 31)
    r, i, amax = F.fixed_propagate([[m, m], [m, m]], [[0, 0], [0, 0]], [m, m], [0, 0], 1, 31)
    assert list(map(int, r)) == [(1 << 31) - 1] * 2 and amax == 1 << 63
    # the batch form gives the same codes
    Rr, Ri = F.fixed_propagate_batch([[m, m], [m, m]], [[0, 0], [0, 0]], [[m, m]], [[0, 0]], 1, 31)
    assert list(map(int, Rr[0])) == [(1 << 31) - 1] * 2


@pytest.mark.parametrize("f", [15, 31])
def test_batch_form_equals_loops(f):
    # acc = R P^T as integer matrix products against the element loops of
    # Algorithm alg:fpga, on random codes spanning the whole range
    rng = np.random.default_rng(7 + f)
    lo, hi = F.code_range(f)
    n, B, steps = 9, 3, 20
    Pr = rng.integers(lo // 9, hi // 9, size=(n, n))
    Pi = rng.integers(lo // 9, hi // 9, size=(n, n))
    Rr = rng.integers(lo, hi, size=(B, n))
    Ri = rng.integers(lo, hi, size=(B, n))
    br, bi = F.fixed_propagate_batch(Pr, Pi, Rr, Ri, steps, f)
    for q in range(B):
        lr, li, _ = F.fixed_propagate(Pr, Pi, Rr[q], Ri[q], steps, f)
        assert np.array_equal(br[q], lr) and np.array_equal(bi[q], li)


def test_accumulator_width_and_cycle_model():
    # Sec. 3.5: 33 + ceil(log2 n) bits, 37 at n = 9, inside the 42-bit register
    assert F.accumulator_bits(9) == 37 and F.accumulator_bits(9) <= 42
    P = _d3_propagator(True)
    Pr, Pi = F.quantize(P, 15)
    r0 = np.zeros(9, dtype=np.complex128)
    r0[0] = 1.0
    rr, ri = F.quantize(r0, 15)
    _, _, amax = F.fixed_propagate(Pr, Pi, rr, ri, 200, 15)
    assert amax < 2 ** (F.accumulator_bits(9) - 1)
    # Eq. eq:cost_fpga and Table tab:fpga_summary: 94 cycles per step at
    # n = 9, k = 1, 94 N + 1 for a run, 95 cycles = 879.6 ns at 108 MHz
    g = json.load(open(GOLDEN))
    c = g["cycle_model"]
    assert F.fpga_cycles(9, 1, 1) == c["single_step_cycles"]
    for N in (1, 10, 1000):
        assert F.fpga_cycles(9, 1, N) == 94 * N + 1
    assert round(c["single_step_cycles"] / (c["clock_mhz"] * 1e6) * 1e9, 1) == c["single_step_ns"]


def test_quantize_rounds_and_saturates():
    # 1.0 -> 32767 (saturated), -1.0 -> -32768, 0.5/32768 is a tie -> even
    re, im = F.quantize(np.array([1.0 + 0j, -1.0 + 0.0j, 0.5 / 32768 + 1.5j / 32768, -2.0 - 2j]), 15)
    assert list(map(int, re)) == [32767, -32768, 0, -32768]
    assert list(map(int, im)) == [0, 0, 2, -32768]
    x = F.dequantize(np.array([16384]), np.array([-8192]), 15)
    assert x[0] == 0.5 - 0.25j
