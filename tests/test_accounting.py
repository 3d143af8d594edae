"""Pins of the work and traffic accounting that turns timings into roofline
fractions: the per-state-step bytes and arithmetic intensity of Eq. 4
against Table 1 (tab:problem_sizes), and the batched and build counts
against their definitions at small sizes counted by brute force."""

import json
import os

import pytest

from paper_2603_18052_gb300 import accounting as A

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def test_problem_sizes_table():
    rows = json.load(open(GOLDEN))["problem_sizes"]["rows"]
    scale = {"KiB": 1024.0, "thousand KiB": 1024.0 * 1000.0}
    for r in rows:
        n = r["n"]
        assert n == r["d"] ** 2
        ws = A.state_step_bytes_single(n) / scale[r["working_set_unit"]]
        assert round(ws, 1 if r["working_set_value"] < 100 else 0) == r["working_set_value"], r
        assert round(A.arithmetic_intensity_single(n), 2) == r["ai_printed"], r


def test_counts_by_brute_force():
    # one complex multiply-add is 8 real FLOPs; a state-step is n^2 of them
    for n in (1, 4, 9):
        assert A.state_step_flops(n) == 8 * sum(1 for _ in range(n) for _ in range(n))
    # batched bytes: P once per step shared by B states, each state in and out
    n, B = 9, 4
    assert A.state_step_bytes_batched(n, B) * B == pytest.approx(16 * n * n + B * 2 * 16 * n)
    # LU: sum over pivots k of (n-k-1)^2 complex multiply-adds ~ n^3 / 3;
    # the n-RHS forward and back substitutions: n^3 complex multiply-adds
    n = 30
    lu = sum((n - k - 1) ** 2 for k in range(n))
    assert 8 * lu == pytest.approx(8 * n ** 3 / 3, rel=0.11)
    subst = sum(k for k in range(n)) * n * 2  # each of n columns: forward + back, k multiply-adds at row k
    assert 8 * subst == pytest.approx(8 * n ** 3, rel=0.04)
    assert A.build_flops_fp64_solve(n) == pytest.approx(8 * n ** 3 / 3 + 8 * n ** 3)
    assert A.build_flops(n, 2) == pytest.approx(8 * 8 * n ** 3 + A.build_flops_fp64_solve(n))


def test_real_coordinate_counts_by_brute_force():
    """A real multiply-add is 2 FLOPs: the real-coordinate state-step is n^2
    of them, and the real build counts the same multiply-adds as the complex
    one at 2 FLOPs each (a quarter of the complex count)."""
    for n in (1, 4, 9):
        assert A.state_step_flops_real(n) == 2 * sum(1 for _ in range(n) for _ in range(n))
        assert 4 * A.state_step_flops_real(n) == A.state_step_flops(n)
    n = 30
    lu = sum((n - k - 1) ** 2 for k in range(n))
    subst = sum(k for k in range(n)) * n * 2
    assert 2 * (lu + subst) == pytest.approx(A.build_flops_real_solve(n), rel=0.06)
    for s in (0, 1, 6):
        assert 4 * A.build_flops_real(n, s) == pytest.approx(A.build_flops(n, s))
