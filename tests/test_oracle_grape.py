"""Pins of the oracle's GRAPE fidelity and gradient (Sec. 2.5, Eq. 5)."""

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from workloads import make_workload, transmon_chain
from workloads.rng import normal


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def test_frechet_matches_scipy_and_finite_differences():
    A = _rand_c(3, (9, 9)) * 0.1
    E = _rand_c(4, (9, 9)) * 0.1
    D = O.frechet_expm(A, E)
    _, ref = sl.expm_frechet(A, E)
    assert np.linalg.norm(D - ref) / np.linalg.norm(ref) <= 1e-12
    h = 1e-5
    fd = (O.expm_pade13(A + h * E) - O.expm_pade13(A - h * E)) / (2 * h)
    assert np.linalg.norm(D - fd) / np.linalg.norm(D) <= 1e-8


def _gate_problem(nq, S, seed):
    m = transmon_chain(nq)
    d, n = m.d, m.d * m.d
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    u = 0.1 * normal(seed, S)
    B = 4
    X0 = np.zeros((B, n), dtype=complex)
    Xt = np.zeros((B, n), dtype=complex)
    basis = [(0, 0), (0, 1), (1, 0), (1, 1)]
    Ux = np.eye(d, dtype=complex)
    for b, (i, j) in enumerate(basis):
        E = np.zeros((d, d), dtype=complex)
        E[i, j] = 1.0
        X0[b] = O.vec(E)
        Xt[b] = O.vec(Ux @ E @ Ux.conj().T)
    return Lb, Ld, u, m.dt, X0, Xt


@pytest.mark.parametrize("nq,S,m", [(1, 6, 1), (1, 4, 3), (2, 3, 2)])
def test_grape_gradient_matches_finite_differences(nq, S, m):
    Lb, Ld, u, dt, X0, Xt = _gate_problem(nq, S, 77 + S)
    F, g = O.grape_fidelity_grad(Lb, Ld, u, dt, m, X0, Xt)
    h = 1e-6
    for s in range(S):
        up, um = u.copy(), u.copy()
        up[s] += h
        um[s] -= h
        Fp, _ = O.grape_fidelity_grad(Lb, Ld, up, dt, m, X0, Xt)
        Fm, _ = O.grape_fidelity_grad(Lb, Ld, um, dt, m, X0, Xt)
        fd = (Fp - Fm) / (2 * h)
        assert abs(g[s] - fd) <= 1e-7 * max(1e-3, abs(g[s])) + 1e-9


def test_grape_fidelity_of_identity_channel_is_one():
    """A zero generator gives P = I, so the identity target has F = 1 and a
    zero gradient."""
    n = 9
    Z = np.zeros((n, n), dtype=complex)
    X0 = np.eye(n, dtype=complex)[:4]
    F, g = O.grape_fidelity_grad(Z, Z, np.array([0.3, -0.2]), 0.1, 1, X0, X0)
    assert abs(F - 1.0) <= 1e-15
    assert np.max(np.abs(g)) <= 1e-15
