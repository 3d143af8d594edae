"""Action of the slice propagator on the states without forming it.

TEST INFRASTRUCTURE ONLY.  Like ``oracle.lindblad`` this module is the slow,
plain reference that the CUDA path is checked against; only the test suite,
the smoke check of the package entry module and the CPU-baseline leg of the
benchmark may import it, and it shares no code with the library.

The paper's discussion (Sec. 5) names this route as the one that removes the
LU solve: apply exp(L dt) to the states directly, as in the action-of-the-
exponential methods it cites (Al-Mohy and Higham 2011; EXPOKIT), at the
price of leaving the fixed-propagator regime.  The paper gives the route, not
its parameters; the method here is the truncated Taylor series with scaling
of Al-Mohy and Higham, with an a priori parameter choice of our own (a
reading, listed with the design notes):

  * for A = L dt and a batch of states x (rows of X), s sub-steps of
        y <- y + sum_{k=1..m} (A/s)^k / k! y ;
  * theta_m is the largest theta with theta^(m+1) / (m+1)! * e^theta <= u,
    u = 2^-53: when ||A/s||_1 <= theta_m this bounds the remainder of the
    degree-m Taylor polynomial of exp(A/s) applied to a vector by u times
    the vector's norm;
  * (m, s) minimises the number of products m * s subject to
    ||A||_1 / s <= theta_m, 1 <= m <= 55, the smaller m on ties;
  * a call over several control slices uses one (m, s), chosen from the
    largest ||A_s||_1 of the call.
"""

import math

import numpy as np

UNIT_ROUNDOFF = 2.0 ** -53
M_MAX = 55


def theta(m, u=UNIT_ROUNDOFF):
    """Largest theta with theta^(m+1)/(m+1)! e^theta <= u, by bisection on
    the logarithm (increasing in theta)."""
    lg = math.lgamma(m + 2.0)
    lu = math.log(u)

    def g(t):
        return (m + 1) * math.log(t) + t - lg - lu

    lo, hi = 1e-300, 64.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) <= 0.0:
            lo = mid
        else:
            hi = mid
    return lo


def parameters(a):
    """(m, s) for ||A||_1 = a: fewest products m * s with a / s <= theta_m."""
    best = None
    for m in range(1, M_MAX + 1):
        s = max(1, int(math.ceil(a / theta(m))))
        if best is None or m * s < best[0] * best[1]:
            best = (m, s)
    return best


def onenorm(A):
    """Induced 1-norm: the largest absolute column sum."""
    return float(np.abs(np.asarray(A)).sum(axis=0).max())


def expmv(A, X, ms=None):
    """Rows of X advanced by exp(A): X_out[b] = exp(A) X[b].  ms = (m, s)
    overrides the parameter choice."""
    A = np.asarray(A, dtype=np.complex128)
    Y = np.array(X, dtype=np.complex128, copy=True)
    m, s = parameters(onenorm(A)) if ms is None else ms
    for _ in range(s):
        V = Y.copy()
        for k in range(1, m + 1):
            V = (V @ A.T) / (s * k)  # the k-th Taylor term of exp(A/s) applied to y
            Y = Y + V
    return Y


def expmv_chain(L_base, L_drv, u, dt, X):
    """The states through the control slices: X <- exp((L_base + u_s L_drv)
    dt) X for s = 0, 1, ..., with one (m, s) for the whole call, chosen from
    the largest ||(L_base + u_s L_drv) dt||_1.  Returns (X, (m, s))."""
    L_base = np.asarray(L_base)
    L_drv = np.asarray(L_drv)

    def gen(us):
        return (L_base + us * L_drv) * dt

    # two passes (norms, then the products) so that only one generator is
    # held at a time
    a = max((onenorm(gen(us)) for us in u), default=0.0)
    ms = parameters(a)
    Y = np.array(X, dtype=np.complex128, copy=True)
    for us in u:
        Y = expmv(gen(us), Y, ms)
    return Y, ms
