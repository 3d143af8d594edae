"""Real coordinates of Hermitian matrices and the real form of a
Hermiticity-preserving superoperator.

TEST INFRASTRUCTURE ONLY (see ``oracle.lindblad``): plain numpy loops that
define what the library's real-coordinate ("Hermitian") forms compute.  The
library never imports this module.

A density matrix is Hermitian, and each term of Eq. 1 maps a Hermitian rho
to a Hermitian matrix, so the Lindbladian L, its exponential P = exp(L dt)
(Algorithm 1) and every product of Algorithm 2 map Hermitian matrices to
Hermitian matrices.  A Hermitian d x d matrix is fixed by n = d^2 real
numbers, its coordinates

    c(rho) = (rho_00, ..., rho_{d-1,d-1},  Re rho_kl, Im rho_kl for k < l)

with the pairs (k, l) in row-major order of the upper triangle.  On them a
Hermiticity-preserving superoperator S acts as the real n x n matrix
real_form(S) with real_form(S) c(rho) = c(S rho).  The correspondence takes
products to products and the identity to the identity, so
exp(real_form(L dt)) = real_form(exp(L dt)).
"""

import numpy as np

from .lindblad import onenorm, squaring_count, unvec, vec


def pairs(d):
    """The upper-triangle pairs (k, l), k < l, in row-major order."""
    return [(k, l) for k in range(d) for l in range(k + 1, d)]


def coords(rho):
    """c(rho): the diagonal, then Re and Im of each upper-triangle entry."""
    rho = np.asarray(rho)
    d = rho.shape[0]
    c = [float(np.real(rho[k, k])) for k in range(d)]
    for k, l in pairs(d):
        c.append(float(np.real(rho[k, l])))
        c.append(float(np.imag(rho[k, l])))
    return np.array(c)


def from_coords(c, d):
    """The Hermitian matrix whose coordinates are c."""
    rho = np.zeros((d, d), dtype=np.complex128)
    for k in range(d):
        rho[k, k] = c[k]
    a = d
    for k, l in pairs(d):
        rho[k, l] = c[a] + 1j * c[a + 1]
        rho[l, k] = c[a] - 1j * c[a + 1]
        a += 2
    return rho


def real_form(S, d):
    """The real n x n matrix of the superoperator S (n x n complex, acting on
    row-major vec) on the coordinates: column b is c(S Y_b), where Y_b is the
    Hermitian matrix whose coordinate vector is the b-th unit vector."""
    n = d * d
    G = np.zeros((n, n))
    for b in range(n):
        e = np.zeros(n)
        e[b] = 1.0
        G[:, b] = coords(unvec(S @ vec(from_coords(e, d)), d))
    return G


def squaring_count_real(A, d):
    """The squaring count of Algorithm 1 taken on the real form of A, as the
    real-coordinate build takes it: s = max(0, ceil(log2(||G||_1 / theta)))
    with G = real_form(A)."""
    return squaring_count(real_form(A, d))


def real_norm1(A, d):
    return onenorm(real_form(A, d))
