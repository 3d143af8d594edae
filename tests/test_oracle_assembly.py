"""Pins of the oracle's Lindbladian assembly (Eq. 1-3, Eq. 5).

The assembly uses the Kronecker formula; these tests check it against the
matrix form of Eq. 1 applied directly to random operators, and against
structural invariants that any correct Lindbladian has."""

import json
import os

import numpy as np
import pytest

import oracle as O
from workloads import make_workload, transmon_chain
from workloads.rng import normal, splitmix64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _rhs_eq1(H, jumps, rho):
    """Eq. 1 written with matrix products: -i[H, rho] + sum_k (L rho L^+ - 1/2 {L^+ L, rho})."""
    out = -1j * (H @ rho - rho @ H)
    for L in jumps:
        G = L.conj().T @ L
        out = out + L @ rho @ L.conj().T - 0.5 * (G @ rho + rho @ G)
    return out


@pytest.mark.parametrize("d,K", [(2, 1), (3, 2), (4, 3), (6, 0)])
def test_assembly_matches_eq1_bruteforce(d, K):
    Hr = _rand_c(11 + d, (d, d))
    H = Hr + Hr.conj().T
    jumps = [_rand_c(100 + 7 * k + d, (d, d)) * 0.3 for k in range(K)]
    L = O.lindbladian(H, jumps)
    for t in range(3):
        X = _rand_c(1000 + 13 * t + d, (d, d))  # any matrix, not only states
        lhs = L @ O.vec(X)
        rhs = O.vec(_rhs_eq1(H, jumps, X))
        assert np.max(np.abs(lhs - rhs)) <= 1e-13 * max(1.0, np.max(np.abs(rhs)))


def test_trace_preservation_and_hermiticity_map():
    m = transmon_chain(2)
    L = O.lindbladian(m.H0, m.jumps)
    d = m.d
    vI = O.vec(np.eye(d))
    # d/dt Tr(rho) = vec(I)^T L vec(rho) = 0 for every rho
    assert np.max(np.abs(vI @ L)) <= 1e-13
    # Hermiticity preservation: L[(i,j),(k,l)] = conj(L[(j,i),(l,k)])
    L4 = L.reshape(d, d, d, d)
    assert np.max(np.abs(L4 - np.conj(L4.transpose(1, 0, 3, 2)))) <= 1e-13


def test_decomposed_generator_matches_monolithic():
    """Eq. 5: L(u) = L_base + u L_drv equals the Lindbladian of H0 + u X
    (the paper's own decomposed-vs-monolithic unit test)."""
    m = transmon_chain(2)
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    for u in (-0.1, 0.0, 0.037, 0.1):
        mono = O.lindbladian(m.H0 + u * m.X, m.jumps)
        assert np.max(np.abs(O.slice_generator(Lb, Ld, u) - mono)) <= 1e-14


def test_row_major_vec_identity():
    """vec(A X B) = (A kron B^T) vec(X) for the row-major vec used throughout."""
    A, X, B = _rand_c(1, (3, 3)), _rand_c(2, (3, 3)), _rand_c(3, (3, 3))
    assert np.allclose(np.kron(A, B.T) @ O.vec(X), O.vec(A @ X @ B), atol=1e-13)


def test_splitmix64_reference_vector():
    g = json.load(open(GOLDEN))["splitmix64"]
    assert list(map(int, splitmix64(g["seed"], 5))) == g["out"]


@pytest.mark.parametrize("name", ["d3_single", "d9_batch", "d27_chain"])
def test_workload_states_are_density_matrices(name):
    w = make_workload(name, B=8, nslices=4)
    d = w["d"]
    for v in w["states"]:
        rho = v.reshape(d, d)
        assert abs(np.trace(rho) - 1.0) <= 1e-14
        assert np.max(np.abs(rho - rho.conj().T)) <= 1e-15
        assert np.min(np.linalg.eigvalsh(rho)) >= -1e-14
    assert np.all(np.abs(w["u"]) <= 0.1 + 1e-15)
