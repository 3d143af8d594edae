"""Pins of the oracle's propagation (Algorithm 2) against closed forms and
invariants of the Lindblad equation (Eq. 1)."""

import math

import numpy as np

import oracle as O
from workloads import annihilation, make_workload


def _evolve(H, jumps, rho0, dt, nsteps):
    P = O.expm_pade13(O.lindbladian(H, jumps) * dt)
    return O.propagate(P, O.vec(rho0)[None, :], nsteps)[0].reshape(rho0.shape)


def test_amplitude_damping_closed_form():
    """H = 0, L = sqrt(g) a on two levels: rho_11(t) = e^{-g t}, and the
    coherence of |+><+| decays as e^{-g t / 2}."""
    g, dt, N = 0.3, 0.05, 40
    a = annihilation(2)
    rho = np.array([[0, 0], [0, 1]], dtype=complex)
    out = _evolve(np.zeros((2, 2)), [math.sqrt(g) * a], rho, dt, N)
    t = dt * N
    assert abs(out[1, 1] - math.exp(-g * t)) <= 1e-13
    plus = 0.5 * np.ones((2, 2), dtype=complex)
    out = _evolve(np.zeros((2, 2)), [math.sqrt(g) * a], plus, dt, N)
    assert abs(out[0, 1] - 0.5 * math.exp(-g * t / 2)) <= 1e-13


def test_dephasing_closed_form():
    """L = sqrt(gp) a^+ a: rho_jk(t) = rho_jk(0) e^{-gp (j-k)^2 t / 2}."""
    gp, dt, N, d = 0.2, 0.1, 25, 3
    a = annihilation(d)
    n_op = a.conj().T @ a
    rho0 = make_workload("d3_single")["states"][0].reshape(d, d)
    out = _evolve(np.zeros((d, d)), [math.sqrt(gp) * n_op], rho0, dt, N)
    t = dt * N
    j, k = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    ref = rho0 * np.exp(-gp * (j - k) ** 2 * t / 2)
    assert np.max(np.abs(out - ref)) <= 1e-13


def test_rabi_closed_form():
    """d = 2, H = u sigma_x, no jumps, rho0 = |0><0|: rho_11(t) = sin^2(u t)."""
    u, dt = 0.37, 0.1
    sx = np.array([[0, 1], [1, 0]], dtype=complex)
    rho = np.array([[1, 0], [0, 0]], dtype=complex)
    for N in (1, 7, 100):
        out = _evolve(u * sx, [], rho, dt, N)
        assert abs(out[1, 1] - math.sin(u * dt * N) ** 2) <= 1e-13


def test_long_chain_invariants():
    """10^4 steps of the single-transmon workload: trace, Hermiticity and
    positivity are kept, and the result equals exp(L N dt) rho0."""
    w = make_workload("d3_single")
    d = w["d"]
    L = O.lindbladian(w["H0"] + w["u"][0] * w["X"], w["jumps"])
    P = O.expm_pade13(L * w["dt"])
    R = O.propagate(P, w["states"], w["steps_per_slice"])
    rho = R[0].reshape(d, d)
    # rounding bound after N steps: N * n * eps = 1e4 * 9 * 1.1e-16 ~ 1e-11
    tol = w["steps_per_slice"] * w["n"] * 1.2e-16
    assert abs(np.trace(rho) - 1.0) <= tol
    assert np.max(np.abs(rho - rho.conj().T)) <= tol
    assert np.min(np.linalg.eigvalsh(0.5 * (rho + rho.conj().T))) >= -tol
    Pn = O.expm_pade13(L * w["dt"] * w["steps_per_slice"])
    ref = Pn @ w["states"][0]
    assert np.linalg.norm(R[0] - ref) / np.linalg.norm(ref) <= 1e-11


def test_amplitude_damping_steady_state():
    a = annihilation(3)
    rho0 = make_workload("d3_single")["states"][0].reshape(3, 3)
    out = _evolve(np.zeros((3, 3)), [math.sqrt(0.5) * a], rho0, 1.0, 200)
    ref = np.zeros((3, 3))
    ref[0, 0] = 1.0
    assert np.max(np.abs(out - ref)) <= 1e-12


def test_chain_uses_slice_propagators_in_order():
    """Step t uses P[t // steps_per_slice]: two non-commuting slices applied
    in the other order give a different state."""
    w = make_workload("d9_batch", B=2)
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    Ps = O.slice_propagators(Lb, Ld, np.array([0.1, -0.3]), 0.5)
    fwd = O.propagate_chain(Ps, w["states"], 2)
    ref = w["states"]
    for P in (Ps[0], Ps[0], Ps[1], Ps[1]):
        ref = ref @ P.T
    assert np.max(np.abs(fwd - ref)) <= 1e-15
    rev = O.propagate_chain(Ps[::-1], w["states"], 2)
    assert np.max(np.abs(fwd - rev)) > 1e-6
