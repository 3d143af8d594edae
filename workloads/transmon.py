"""Model operators for the synthetic transmon workloads.

Units are ns and rad/ns.  A chain of ``nq`` transmons truncated to ``levels``
levels has Hilbert dimension d = levels**nq; transmon 0 is the most significant
index of the Kronecker order.  These are inputs to the method (H, the jump
operators L_k and the drive operator X), not part of it.
"""

from dataclasses import dataclass, field
import math

import numpy as np


def annihilation(levels):
    """Truncated annihilation operator: a[k-1, k] = sqrt(k)."""
    a = np.zeros((levels, levels), dtype=np.complex128)
    for k in range(1, levels):
        a[k - 1, k] = math.sqrt(k)
    return a


def _embed(op, site, nq, levels):
    out = np.ones((1, 1), dtype=np.complex128)
    eye = np.eye(levels, dtype=np.complex128)
    for q in range(nq):
        out = np.kron(out, op if q == site else eye)
    return out


@dataclass
class TransmonModel:
    """H(u) = H0 + u * X, with jump operators ``jumps`` (K x d x d)."""

    d: int
    H0: np.ndarray
    X: np.ndarray
    jumps: np.ndarray
    dt: float
    meta: dict = field(default_factory=dict)


def transmon_chain(nq, levels=3, alpha=-2.0 * math.pi * 0.2, g=2.0 * math.pi * 0.005,
                   gamma1=1e-3, gamma_phi=5e-4, dt=0.1):
    """Chain of ``nq`` anharmonic transmons in the frame rotating with the
    (degenerate) qubit frequency.

    H0 = sum_i (alpha/2) a_i^+ a_i^+ a_i a_i + g sum_i (a_i^+ a_{i+1} + a_i a_{i+1}^+),
    drive X = a_0 + a_0^+, jumps sqrt(gamma1) a_i and sqrt(gamma_phi) a_i^+ a_i
    for every transmon i.
    """
    a = annihilation(levels)
    ad = a.conj().T
    d = levels ** nq
    H0 = np.zeros((d, d), dtype=np.complex128)
    jumps = []
    for q in range(nq):
        aq = _embed(a, q, nq, levels)
        aqd = aq.conj().T
        H0 += 0.5 * alpha * (aqd @ aqd @ aq @ aq)
        jumps.append(math.sqrt(gamma1) * aq)
        jumps.append(math.sqrt(gamma_phi) * (aqd @ aq))
    for q in range(nq - 1):
        aq = _embed(a, q, nq, levels)
        ar = _embed(a, q + 1, nq, levels)
        H0 += g * (aq.conj().T @ ar + aq @ ar.conj().T)
    a0 = _embed(a, 0, nq, levels)
    X = a0 + a0.conj().T
    del ad
    return TransmonModel(d=d, H0=H0, X=X, jumps=np.ascontiguousarray(np.array(jumps)), dt=dt,
                         meta=dict(nq=nq, levels=levels, alpha=alpha, g=g, gamma1=gamma1,
                                   gamma_phi=gamma_phi))


def paper_grape_model(d, T1=50.0, T2=30.0, dt=0.5):
    """The paper's landscape-point model (its protocol section): a single
    d-level system with H0 = diag(0, ..., d-1), the truncated sigma_x drive
    read as a + a^+, amplitude damping sqrt(1/T1) a and pure dephasing
    sqrt(gamma_phi) a^+ a with gamma_phi = 1/T2 - 1/(2 T1)."""
    a = annihilation(d)
    H0 = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128)
    gphi = 1.0 / T2 - 1.0 / (2.0 * T1)
    jumps = np.array([math.sqrt(1.0 / T1) * a, math.sqrt(gphi) * (a.conj().T @ a)])
    return TransmonModel(d=d, H0=H0, X=a + a.conj().T, jumps=jumps, dt=dt,
                         meta=dict(T1=T1, T2=T2, gamma_phi=gphi))
