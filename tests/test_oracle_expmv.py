"""Pins of the action-of-the-exponential oracle (the route of Sec. 5 that
removes the LU solve): against SciPy's expm_multiply (Al-Mohy and Higham's
algorithm as a library routine), against the Pade oracle of Algorithm 1,
against closed forms, and the parameter rule against its defining bound."""

import math

import numpy as np
import pytest

import oracle as O
from oracle import expmv as E
from workloads.transmon import paper_grape_model, transmon_chain

scipy_linalg = pytest.importorskip("scipy.sparse.linalg")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_theta_meets_its_bound():
    # at theta_m the remainder bound equals u (checked with the exact
    # factorial, not the log-gamma of the bisection), and grows with m
    prev = 0.0
    for m in (1, 2, 5, 10, 18, 30, 45, 55):
        t = E.theta(m)
        bound = t ** (m + 1) / math.factorial(m + 1) * math.exp(t)
        assert bound == pytest.approx(E.UNIT_ROUNDOFF, rel=1e-9)
        assert t > prev
        prev = t


def test_parameter_rule():
    for a in (0.0, 1e-3, 0.7, 3.0, 13.0, 100.0):
        m, s = E.parameters(a)
        assert 1 <= m <= E.M_MAX and s >= 1
        assert a / s <= E.theta(m)
        # no other (m', s') with fewer products satisfies the constraint
        for m2 in range(1, E.M_MAX + 1):
            s2 = max(1, math.ceil(a / E.theta(m2)))
            assert m2 * s2 >= m * s
    assert E.parameters(0.0) == (1, 1)


@pytest.mark.parametrize("nq,u", [(1, 0.05), (2, -0.08)])
def test_matches_scipy_and_pade(nq, u):
    m = transmon_chain(nq)
    A = O.slice_generator(O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X), u) * m.dt * 7.0
    rng = np.random.default_rng(3 + nq)
    X = rng.standard_normal((3, A.shape[0])) + 1j * rng.standard_normal((3, A.shape[0]))
    Y = E.expmv(A, X)
    ref_scipy = scipy_linalg.expm_multiply(A, X.T).T
    ref_pade = X @ O.expm_pade13(A).T
    assert _rel(Y, ref_scipy) <= 1e-12
    assert _rel(Y, ref_pade) <= 1e-12


def test_paper_model_chain_through_slices():
    # the paper's landscape model at d = 3: the chain through several slices
    # against slice-by-slice Pade propagators
    m = paper_grape_model(3)
    Lb, Ld = O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)
    u = np.array([0.1, -0.05, 0.0, 0.2])
    X = np.zeros((2, 9), dtype=np.complex128)
    X[0, 0] = 1.0
    X[1, 4] = 1.0
    Y, ms = E.expmv_chain(Lb, Ld, u, m.dt, X)
    R = X.copy()
    for us in u:
        R = R @ O.expm_pade13((Lb + us * Ld) * m.dt).T
    assert _rel(Y, R) <= 1e-12
    assert ms == E.parameters(max(E.onenorm((Lb + us * Ld) * m.dt) for us in u))


def test_closed_forms():
    # diagonal: exp(t lambda_i) x_i
    lam = np.array([-3.0, -0.5 + 2j, 1.25, 0.0])
    x = np.array([[1.0, 2.0 - 1j, -0.5, 3.0]])
    assert _rel(E.expmv(np.diag(lam), x), x * np.exp(lam)) <= 1e-14
    # rotation generator: [[0, -w], [w, 0]] -> cos / sin
    w = 4.0
    y = E.expmv(np.array([[0.0, -w], [w, 0.0]]), np.array([[1.0, 0.0]]))
    assert _rel(y, np.array([[math.cos(w), math.sin(w)]])) <= 1e-14
    # nilpotent Jordan block: the series ends at k = n - 1
    n = 6
    N = np.diag(np.full(n - 1, 1.5), 1)
    x = np.arange(1.0, n + 1.0)[None, :]
    ref = sum(np.linalg.matrix_power(N, k) / math.factorial(k) for k in range(n)) @ x[0]
    assert _rel(E.expmv(N, x)[0], ref) <= 1e-14


def test_amplitude_damping_and_trace():
    # one decaying qubit: rho_11(t) = exp(-gamma t) rho_11(0), trace kept
    g, t = 0.3, 2.5
    a = np.array([[0.0, 1.0], [0.0, 0.0]], dtype=np.complex128)
    L = O.lindbladian(np.zeros((2, 2)), np.array([math.sqrt(g) * a]))
    rho = np.array([[0.25, 0.1 - 0.2j], [0.1 + 0.2j, 0.75]])
    out = E.expmv(L * t, O.vec(rho)[None, :])[0].reshape(2, 2)
    assert out[1, 1].real == pytest.approx(0.75 * math.exp(-g * t), rel=1e-14)
    assert np.trace(out).real == pytest.approx(1.0, abs=1e-14)
    assert abs(out[0, 1] - rho[0, 1] * math.exp(-g * t / 2)) <= 1e-14
