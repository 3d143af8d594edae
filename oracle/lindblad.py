"""FP64 CPU oracle for dense small-d Lindblad propagation.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test suite, the smoke check of the
package entry module and the CPU-baseline leg of the benchmark may import it;
the library never does, and the two share no code.

Everything is complex128 numpy.  Each function follows one passage of the
paper (arXiv 2603.18052, "Hardware-Aware Performance Characterization of Small
Dense Lindblad Propagation for Near-Term Quantum Control") and names it.
Library primitives used as single steps: matrix product (``@``), ``kron``,
``argmax``.  No blocking, fusion or reordering beyond what the cited passage
states.

Conventions (readings of the paper, all listed with the design notes):
  * vec is row-major: vec(X)[i*d + j] = X[i, j] (Sec. 3.2 states that the
    row-major d x d array already is the n-vector), hence
    vec(A X B) = (A kron B^T) vec(X).
  * ||.||_1 is the induced 1-norm, the maximum absolute column sum.
  * Pade [13/13] coefficients come from the closed form of the diagonal Pade
    approximant of exp, b_j = (2m-j)! m! / ((2m)! j! (m-j)!), b_0 = 1.
"""

import math
from fractions import Fraction

import numpy as np

THETA = 0.25  # scaling threshold of Algorithm 1 (Sec. 3.1 sets theta = 0.25)
PADE_M = 13


# ---------------------------------------------------------------- assembly --

def vec(X):
    """Row-major vectorisation of a d x d matrix (Sec. 3.2, Algorithm 2)."""
    return np.ascontiguousarray(X).reshape(-1)


def unvec(v, d):
    return np.asarray(v).reshape(d, d)


def lindbladian(H, jumps):
    """Vectorised Lindbladian of Eq. 1 under row-major vec (Eq. 2-3).

    L = -i (H kron I - I kron H^T)
        + sum_k [ L_k kron conj(L_k) - 1/2 (L_k^+ L_k) kron I - 1/2 I kron (L_k^+ L_k)^T ]

    Each term is the row-major image of one term of Eq. 1: H rho -> H kron I,
    rho H -> I kron H^T, L rho L^+ -> L kron (L^+)^T = L kron conj(L).
    """
    H = np.asarray(H, dtype=np.complex128)
    d = H.shape[0]
    eye = np.eye(d, dtype=np.complex128)
    L = -1j * (np.kron(H, eye) - np.kron(eye, H.T))
    for Lk in jumps:
        Lk = np.asarray(Lk, dtype=np.complex128)
        G = Lk.conj().T @ Lk
        L = L + np.kron(Lk, Lk.conj()) - 0.5 * np.kron(G, eye) - 0.5 * np.kron(eye, G.T)
    return L


def drive_generator(X):
    """Coherent drive term of the decomposed generator (Eq. 5): the
    Lindbladian of Hamiltonian X with no jump operators."""
    return lindbladian(X, [])


def slice_generator(L_base, L_drv, u):
    """Segment generator L(u) = L_base + u * L_drv (Eq. 5, with L_0 and
    L_diss folded into L_base)."""
    return L_base + u * L_drv


# ------------------------------------------------------------------- expm --

def pade13_coefficients():
    """b_0 .. b_13 of the [13/13] Pade approximant of exp (Algorithm 1).

    Closed form b_j = (2m-j)! m! / ((2m)! j! (m-j)!), evaluated exactly in
    rationals and rounded once to double."""
    m = PADE_M
    f = math.factorial
    return np.array([float(Fraction(f(2 * m - j) * f(m), f(2 * m) * f(j) * f(m - j)))
                     for j in range(m + 1)])


def onenorm(A):
    """Induced 1-norm: maximum absolute column sum."""
    return float(np.max(np.sum(np.abs(A), axis=0))) if A.size else 0.0


def squaring_count(A, theta=THETA):
    """s = max(0, ceil(log2(||A||_1 / theta))) (Algorithm 1, first line)."""
    nrm = onenorm(A)
    if nrm <= 0.0:
        return 0, nrm
    return max(0, int(math.ceil(math.log2(nrm / theta)))), nrm


def lu_gepp(M):
    """LU with partial pivoting (Algorithm 1, the LU solve of the Padé denominator): P M = L U.

    Gaussian elimination column by column; the pivot is the first entry of
    largest modulus in the column.  Returns (L, U, perm, nswaps) with
    M[perm] = L @ U, L unit lower triangular."""
    A = np.array(M, dtype=np.complex128, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    nswaps = 0
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if p != k:
            A[[k, p], :] = A[[p, k], :]
            perm[[k, p]] = perm[[p, k]]
            nswaps += 1
        piv = A[k, k]
        if piv == 0:
            raise ZeroDivisionError("singular matrix in lu_gepp")
        A[k + 1:, k] = A[k + 1:, k] / piv
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    L = np.tril(A, -1) + np.eye(n, dtype=np.complex128)
    U = np.triu(A)
    return L, U, perm, nswaps


def lu_solve(L, U, perm, B):
    """Solve (L U) X = B[perm] by forward then back substitution, all columns
    of B at once (Algorithm 1, the LU solve of the Padé denominator)."""
    Y = np.array(B[perm], dtype=np.complex128, copy=True)
    n = L.shape[0]
    for i in range(n):
        if i:
            Y[i] -= L[i, :i] @ Y[:i]
    X = np.empty_like(Y)
    for i in range(n - 1, -1, -1):
        acc = Y[i] - (U[i, i + 1:] @ X[i + 1:] if i + 1 < n else 0.0)
        X[i] = acc / U[i, i]
    return X


def expm_pade13(A0, theta=THETA, return_info=False):
    """P = exp(A0) by Algorithm 1: scaling, Pade [13/13] with the three power
    products and three U/V products, an LU solve, and s squarings."""
    A0 = np.asarray(A0, dtype=np.complex128)
    n = A0.shape[0]
    b = pade13_coefficients()
    s, nrm = squaring_count(A0, theta)
    A = A0 / (2.0 ** s)
    I = np.eye(n, dtype=np.complex128)
    A2 = A @ A
    A4 = A2 @ A2
    A6 = A4 @ A2
    V = A6 @ (b[12] * A6 + b[10] * A4 + b[8] * A2) + b[6] * A6 + b[4] * A4 + b[2] * A2 + b[0] * I
    W = A6 @ (b[13] * A6 + b[11] * A4 + b[9] * A2)
    U = A @ (W + b[7] * A6 + b[5] * A4 + b[3] * A2 + b[1] * I)
    L, Uf, perm, nswaps = lu_gepp(V - U)
    P = lu_solve(L, Uf, perm, V + U)
    for _ in range(s):
        P = P @ P
    if return_info:
        return P, dict(s=s, norm1=nrm, nswaps=nswaps, V=V, U=U)
    return P


def slice_propagators(L_base, L_drv, u, dt, return_info=False):
    """P_s = exp((L_base + u_s L_drv) dt) for every control slice (Eq. 5 and
    Algorithm 1, one build per segment)."""
    Ps, infos = [], []
    for us in np.asarray(u, dtype=np.float64):
        P, info = expm_pade13(slice_generator(L_base, L_drv, us) * dt, return_info=True)
        Ps.append(P)
        infos.append(info)
    Ps = np.array(Ps)
    return (Ps, infos) if return_info else Ps


def frechet_expm(A, E):
    """Frechet derivative of exp at A in direction E, taken independently of
    the differentiated Pade route as the top-right block of
    exp([[A, E], [0, A]]) (Van Loan's block-triangular identity)."""
    n = A.shape[0]
    Z = np.zeros((2 * n, 2 * n), dtype=np.complex128)
    Z[:n, :n] = A
    Z[n:, n:] = A
    Z[:n, n:] = E
    return expm_pade13(Z)[:n, n:]


# ------------------------------------------------------------ propagation --

def propagate_step(P, R):
    """One step of Algorithm 2 for every row of R (each row one state):
    out_i = sum_j P_ij rho_j."""
    return R @ P.T


def propagate(P, states, nsteps):
    """nsteps chained applications of Algorithm 2 (batched over states as in
    Algorithm 3; the steps of one state stay sequential)."""
    R = np.array(states, dtype=np.complex128, copy=True)
    for _ in range(nsteps):
        R = propagate_step(P, R)
    return R


def propagate_chain(Ps, states, steps_per_slice=1):
    """Per-slice chain: step t uses P[t // steps_per_slice]."""
    R = np.array(states, dtype=np.complex128, copy=True)
    for P in Ps:
        for _ in range(steps_per_slice):
            R = propagate_step(P, R)
    return R


def trace_of(R, d):
    """Tr(rho) of each row-major state vector: sum of entries i*d + i."""
    return np.sum(R[:, :: d + 1], axis=1)


# ------------------------------------------------------------------ GRAPE --

def grape_fidelity_grad(L_base, L_drv, u, dt, steps_per_slice, X0, Xt):
    """Fidelity and gradient of a piecewise-constant control (Sec. 2.5,
    Eq. 5: one propagator per segment, applied steps_per_slice times).

    F = Re sum_b <Xt_b, X_T,b> / B with X_T = P_S^m ... P_1^m X0 and
    <a, b> = sum_i conj(a_i) b_i.
    dF/du_s = sum over the steps t of slice s of Re <Lam_t, dP_s X_{t-1}> / B,
    with the adjoint chain Lam_T = Xt, Lam_{t-1} = P^+ Lam_t and
    dP_s = Frechet derivative of exp at (L_base + u_s L_drv) dt in the
    direction L_drv dt.
    """
    u = np.asarray(u, dtype=np.float64)
    B = X0.shape[0]
    S = len(u)
    m = steps_per_slice
    E = L_drv * dt
    Ps, dPs = [], []
    for us in u:
        A = slice_generator(L_base, L_drv, us) * dt
        Ps.append(expm_pade13(A))
        dPs.append(frechet_expm(A, E))
    X = [np.array(X0, dtype=np.complex128, copy=True)]
    for t in range(S * m):
        X.append(propagate_step(Ps[t // m], X[-1]))
    F = float(np.real(np.sum(np.conj(Xt) * X[-1]))) / B
    grad = np.zeros(S)
    lam = np.array(Xt, dtype=np.complex128, copy=True)
    for t in range(S * m - 1, -1, -1):
        s = t // m
        grad[s] += float(np.real(np.sum(np.conj(lam) * propagate_step(dPs[s], X[t])))) / B
        lam = lam @ np.conj(Ps[s])
    return F, grad
