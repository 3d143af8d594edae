"""Pins of the oracle's propagator build (Algorithm 1)."""

import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from workloads import make_workload, paper_grape_model
from workloads.rng import normal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def test_pade_coefficients_match_higham_integers():
    g = json.load(open(GOLDEN))["pade13_higham_integers"]["b"]
    b = O.pade13_coefficients()
    assert b[0] == 1.0
    for j in range(14):
        assert abs(b[j] - g[j] / g[0]) <= 1e-16 * max(1.0, g[j] / g[0])


def test_scalar_pade_approximant_is_exp():
    """The scalar approximant (sum_j b_j x^j) / (sum_j b_j (-x)^j) agrees
    with exp(x) to rounding on |x| <= theta."""
    b = O.pade13_coefficients()
    for x in np.linspace(-0.25, 0.25, 41):
        p = sum(b[j] * x ** j for j in range(14))
        q = sum(b[j] * (-x) ** j for j in range(14))
        assert abs(p / q - math.exp(x)) <= 4e-16 * math.exp(x)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_unitary_case_matches_eigendecomposition(d):
    """No jump operators: P = U kron conj(U) with U = V diag(e^{-i w dt}) V^+
    from a Hermitian eigensolve."""
    Hr = _rand_c(40 + d, (d, d))
    H = 0.5 * (Hr + Hr.conj().T)
    dt = 0.7
    w, V = np.linalg.eigh(H)
    Uu = V @ np.diag(np.exp(-1j * w * dt)) @ V.conj().T
    P = O.expm_pade13(O.lindbladian(H, []) * dt)
    ref = np.kron(Uu, Uu.conj())
    assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 1e-13


@pytest.mark.parametrize("scale", [0.05, 1.0, 13.0])
def test_general_matrix_matches_independent_expm(scale):
    """Against SciPy's expm (an independent implementation) and against the
    eigenvector route exp(A) = V diag(e^lambda) V^-1."""
    A = _rand_c(7, (12, 12))
    A = A * (scale / O.onenorm(A))
    P = O.expm_pade13(A)
    ref = sl.expm(A)
    assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 1e-13
    lam, V = np.linalg.eig(A)
    ref2 = V @ np.diag(np.exp(lam)) @ np.linalg.inv(V)
    assert np.linalg.norm(P - ref2) / np.linalg.norm(ref2) <= 1e-11


def test_diagonal_and_nilpotent_cases():
    dvals = np.array([0.3 - 2.0j, -1.5 + 0.1j, 4.0j, -7.0])
    P = O.expm_pade13(np.diag(dvals))
    assert np.max(np.abs(P - np.diag(np.exp(dvals)))) <= 2e-15 * np.max(np.abs(np.exp(dvals))) * 8
    N = np.triu(_rand_c(9, (5, 5)), 1)
    ref = np.eye(5, dtype=complex)
    term = np.eye(5, dtype=complex)
    for k in range(1, 5):
        term = term @ N / k
        ref = ref + term
    P = O.expm_pade13(N)
    assert np.linalg.norm(P - ref) / np.linalg.norm(ref) <= 1e-14


def test_semigroup_and_inverse():
    w = make_workload("d9_batch", B=1)
    L = O.lindbladian(w["H0"] + 0.05 * w["X"], w["jumps"])
    P1 = O.expm_pade13(L * 0.1)
    P2 = O.expm_pade13(L * 0.2)
    assert np.linalg.norm(P2 - P1 @ P1) / np.linalg.norm(P2) <= 1e-13
    Lu = O.lindbladian(w["H0"] + 0.05 * w["X"], [])
    Pf, Pb = O.expm_pade13(Lu * 0.3), O.expm_pade13(-Lu * 0.3)
    assert np.linalg.norm(Pf @ Pb - np.eye(81)) <= 1e-13


def test_trace_row_of_propagator():
    """vec(I)^T P = vec(I)^T: the propagator preserves the trace."""
    for name in ("d3_single", "d9_batch"):
        w = make_workload(name, B=1)
        L = O.lindbladian(w["H0"] + w["u"][0] * w["X"], w["jumps"])
        P = O.expm_pade13(L * w["dt"])
        vI = O.vec(np.eye(w["d"]))
        assert np.max(np.abs(vI @ P - vI)) <= 1e-14


def test_paper_model_squaring_counts():
    """s per segment 3 / 5 / 6 at d = 3 / 9 / 27 and ||L dt||_1 about 13 at
    d = 27 for the paper's landscape-point model."""
    g = json.load(open(GOLDEN))["squarings_per_segment"]
    for d in (3, 9, 27):
        m = paper_grape_model(d)
        Lb = O.lindbladian(m.H0, m.jumps)
        Ld = O.drive_generator(m.X)
        for om in (0.0, 0.05, 0.1):
            s, nrm = O.squaring_count(O.slice_generator(Lb, Ld, om) * m.dt)
            assert s == g["s"][str(d)], (d, om, s, nrm)
            if d == 27:
                assert abs(nrm - g["norm1_d27_approx"]) / g["norm1_d27_approx"] < 0.1


def test_lu_gepp_reconstructs_and_solves():
    M = _rand_c(21, (30, 30))
    L, U, perm, nswaps = O.lu_gepp(M)
    assert nswaps > 0  # a random matrix needs row exchanges
    assert np.allclose(L @ U, M[perm], atol=1e-12)
    assert np.allclose(np.tril(L), L) and np.allclose(np.diag(L), 1.0) and np.allclose(np.triu(U), U)
    Bm = _rand_c(22, (30, 7))
    X = O.lu_solve(L, U, perm, Bm)
    assert np.linalg.norm(X - np.linalg.solve(M, Bm)) / np.linalg.norm(X) <= 1e-12


@pytest.mark.parametrize("name,slices", [("d3_single", [0]), ("d9_batch", [0]), ("d27_chain", [0, 57, 199])])
def test_no_row_exchanges_on_workloads(name, slices):
    """At theta = 0.25 the Pade denominator V - U is strictly column
    diagonally dominant, so partial pivoting never exchanges rows and an LU
    without pivot search is the same algorithm."""
    w = make_workload(name, B=1)
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    for s in slices:
        A = O.slice_generator(Lb, Ld, w["u"][s]) * w["dt"]
        _, info = O.expm_pade13(A, return_info=True)
        assert info["nswaps"] == 0
        M = info["V"] - info["U"]
        diag = np.abs(np.diag(M))
        off = np.sum(np.abs(M), axis=0) - diag
        assert np.all(diag > off + 0.5)
