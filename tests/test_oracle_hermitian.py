"""Pins of the oracle's real coordinates of Hermitian matrices and of the
real form of a Hermiticity-preserving superoperator (oracle/hermitian.py),
which define what the library's real-coordinate build and propagation
compute.  The pins are mathematical facts the definition must satisfy, not
restatements of it: closed forms for a precessing and a decaying qubit, the
trace functional, multiplicativity, and the exponential through SciPy."""

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from oracle import hermitian as H
from workloads import make_workload
from workloads.rng import normal


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _random_lindbladian(seed, d):
    Hr = _rand_c(seed, (d, d))
    Hm = 0.5 * (Hr + Hr.conj().T)
    jumps = list(0.3 * _rand_c(seed + 1, (2, d, d)))
    return O.lindbladian(Hm, jumps)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_coordinates_round_trip(d):
    Ar = _rand_c(0x77 + d, (d, d))
    rho = Ar + Ar.conj().T  # exactly Hermitian (a real diagonal)
    c = H.coords(rho)
    assert c.shape == (d * d,)
    assert np.array_equal(H.from_coords(c, d), rho)  # exact: the entries are copied


def test_coordinate_order_d3():
    """Diagonal first, then (Re, Im) of (0,1), (0,2), (1,2)."""
    rho = np.array([[1.0, 2 + 3j, 4 + 5j], [2 - 3j, 6.0, 7 + 8j], [4 - 5j, 7 - 8j, 9.0]])
    assert list(H.coords(rho)) == [1.0, 6.0, 9.0, 2.0, 3.0, 4.0, 5.0, 7.0, 8.0]


def test_precession_closed_form():
    """H = (w/2) sigma_z, no jumps: d rho_01 / dt = -i w rho_01, so on
    (rho_00, rho_11, Re rho_01, Im rho_01) the generator is
    Re' = w Im, Im' = -w Re and the diagonal is constant."""
    w = 0.37
    L = O.lindbladian(np.diag([w / 2, -w / 2]).astype(complex), [])
    G = H.real_form(L, 2)
    ref = np.zeros((4, 4))
    ref[2, 3] = w
    ref[3, 2] = -w
    assert np.max(np.abs(G - ref)) <= 1e-16


def test_amplitude_damping_closed_form():
    """L = sqrt(g) |0><1|: rho_11' = -g rho_11, rho_00' = +g rho_11,
    rho_01' = -(g/2) rho_01."""
    g = 0.21
    Lk = np.sqrt(g) * np.array([[0, 1], [0, 0]], dtype=complex)
    G = H.real_form(O.lindbladian(np.zeros((2, 2), dtype=complex), [Lk]), 2)
    ref = np.array([[0, g, 0, 0], [0, -g, 0, 0], [0, 0, -g / 2, 0], [0, 0, 0, -g / 2]])
    assert np.max(np.abs(G - ref)) <= 1e-16


@pytest.mark.parametrize("d", [2, 3, 4])
def test_trace_row_vanishes(d):
    """Tr rho = sum of the diagonal coordinates is conserved by every
    Lindbladian: (1..1, 0..0) G = 0."""
    G = H.real_form(_random_lindbladian(0x100 + d, d), d)
    t = np.zeros(d * d)
    t[:d] = 1.0
    assert np.max(np.abs(t @ G)) <= 1e-13 * np.max(np.abs(G))


@pytest.mark.parametrize("d", [2, 3])
def test_real_form_is_multiplicative(d):
    """real_form(S1 S2) = real_form(S1) real_form(S2) and real_form(I) = I."""
    L1 = _random_lindbladian(0x200 + d, d)
    L2 = _random_lindbladian(0x300 + d, d)
    G12 = H.real_form(L1 @ L2, d)
    assert np.max(np.abs(G12 - H.real_form(L1, d) @ H.real_form(L2, d))) <= 1e-12 * np.max(np.abs(G12))
    assert np.array_equal(H.real_form(np.eye(d * d, dtype=complex), d), np.eye(d * d))


@pytest.mark.parametrize("d", [2, 3])
def test_exponential_commutes_with_real_form(d):
    """exp(real_form(L dt)) = real_form(exp(L dt)), both exponentials by
    SciPy (an independent implementation)."""
    A = 0.8 * _random_lindbladian(0x400 + d, d)
    lhs = sl.expm(H.real_form(A, d))
    rhs = H.real_form(sl.expm(A), d)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13


def test_real_form_acts_on_coordinates():
    """real_form(P) c(rho) = c(P rho) on a Ginibre state of the d = 3
    workload, P its first slice propagator."""
    w = make_workload("d3_single", B=2, nslices=1)
    P = O.slice_propagators(O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"]), w["u"], w["dt"])[0]
    R = H.real_form(P, 3)
    for rho in w["states"]:
        lhs = R @ H.coords(rho.reshape(3, 3))
        rhs = H.coords((P @ rho).reshape(3, 3))
        assert np.max(np.abs(lhs - rhs)) <= 1e-15


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_real_norm_bound(seed):
    """A column of G is c(S Y_b) with Y_b one or two columns' worth of unit
    entries and ||c(Z)||_1 <= ||vec Z||_1 for Hermitian Z (the off-diagonal
    pair counts once with |Re| + |Im| <= sqrt(2) |z| <= 2 |z|), so
    ||G||_1 <= 2 ||L||_1."""
    A = _random_lindbladian(0x500 + seed, 3)
    assert H.real_norm1(A, 3) <= 2.0 * O.onenorm(A)


def test_squaring_count_on_the_workload():
    """On the d = 3 transmon slice generator both coordinates give s = 0
    (||L dt||_1 = 0.145, ||G dt||_1 = 0.159, both below theta = 0.25)."""
    w = make_workload("d3_single", nslices=1)
    A = (O.lindbladian(w["H0"], w["jumps"]) + w["u"][0] * O.drive_generator(w["X"])) * w["dt"]
    s_c, n_c = O.squaring_count(A)
    s_r, n_r = H.squaring_count_real(A, 3)
    assert s_c == s_r == 0
    assert n_r <= 2.0 * n_c
