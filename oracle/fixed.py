"""Integer oracle of the element-serial fixed-point propagation step.

TEST INFRASTRUCTURE ONLY.  Like ``oracle.lindblad`` this module is the slow,
plain reference that the CUDA path is checked against; only the test suite,
the smoke check of the package entry module and the CPU-baseline leg of the
benchmark may import it, and it shares no code with the library.

It follows Algorithm alg:fpga (Sec. 3.5) and the fixed-point formats of
Sec. 2.2: a Q1.f number is a two's-complement integer code c of 1 + f bits
standing for c / 2^f (f = 15: 16-bit Q1.15, the format of the board; f = 31:
32-bit Q1.31, the wider format of Figure fig:fixed_point_drift).  One step of
the algorithm, for every output row i of the n x n complex propagator P:

  * acc_i = sum_j P_ij rho_j, each complex product formed from four exact
    integer products of codes (re = Pr rr - Pi ri, im = Pr ri + Pi rr), summed
    exactly (the board's accumulator has 33 + ceil(log2 n) bits, Sec. 3.5, so
    nothing is lost);
  * rho_i = sat(floor(acc_i / 2^f)), floor being the rounding towards minus
    infinity of the exact quotient and sat the clamp to the code range
    [-2^f, 2^f - 1].

Readings (the paper does not print them):
  * the real propagator and the double-precision state become codes by
    rounding x * 2^f to the nearest integer, ties to even, then saturating;
    so 1.0 becomes the largest code 2^f - 1;
  * codes are kept as exact Python integers here (numpy int64 for the Q1.15
    products, whose sums stay below 2^40; Python integers for Q1.31, whose
    sums need up to 71 bits).
"""

import math

import numpy as np

FORMATS = (15, 31)


def code_range(f):
    """Smallest and largest code of Q1.f (Sec. 2.2: one sign bit and f
    fractional bits, two's complement)."""
    return -(1 << f), (1 << f) - 1


def accumulator_bits(n):
    """Width of the board's accumulator for an n-element row: 33 bits plus
    ceil(log2 n) (Sec. 3.5; 37 bits at n = 9, within the 42-bit register of
    Algorithm alg:fpga)."""
    return 33 + int(math.ceil(math.log2(n))) if n > 1 else 33


def quantize(x, f):
    """Complex array -> (re codes, im codes) as int64 arrays: round x * 2^f to
    the nearest integer (ties to even), then saturate (reading above)."""
    lo, hi = code_range(f)
    x = np.asarray(x, dtype=np.complex128)
    scale = float(1 << f)
    re = np.clip(np.rint(x.real * scale), lo, hi).astype(np.int64)
    im = np.clip(np.rint(x.imag * scale), lo, hi).astype(np.int64)
    return re, im


def dequantize(re, im, f):
    """Codes -> complex128 values c / 2^f (exact in double for f <= 31)."""
    scale = float(1 << f)
    return np.asarray(re, dtype=np.float64) / scale + 1j * (np.asarray(im, dtype=np.float64) / scale)


def _floor_sat(acc, f):
    """sat(floor(acc / 2^f)) of an exact integer (Algorithm alg:fpga write-back)."""
    lo, hi = code_range(f)
    q = acc >> f  # Python's shift of a negative integer rounds towards -infinity
    return lo if q < lo else hi if q > hi else q


def fixed_step(Pr, Pi, rr, ri, f):
    """One step of Algorithm alg:fpga on one state.

    Pr, Pi: n x n integer codes of the propagator (row i = output i).
    rr, ri: n integer codes of the state vector.
    Returns the new (rr, ri) as lists of Python integers, together with the
    largest |accumulator| seen (for the accumulator-width check).
    """
    n = len(rr)
    out_r, out_i = [0] * n, [0] * n
    amax = 0
    for i in range(n):
        acc_r = 0
        acc_i = 0
        for j in range(n):  # row-major (i, j) order; exact integer products
            a, b = int(Pr[i][j]), int(Pi[i][j])
            c, d = int(rr[j]), int(ri[j])
            acc_r += a * c - b * d
            acc_i += a * d + b * c
        amax = max(amax, abs(acc_r), abs(acc_i))
        out_r[i] = _floor_sat(acc_r, f)
        out_i[i] = _floor_sat(acc_i, f)
    return out_r, out_i, amax


def fixed_propagate(Pr, Pi, rr, ri, nsteps, f):
    """nsteps chained steps of Algorithm alg:fpga on one state (pure Python,
    for small cases).  Returns (rr, ri, largest |accumulator|)."""
    Pr = [[int(v) for v in row] for row in np.asarray(Pr)]
    Pi = [[int(v) for v in row] for row in np.asarray(Pi)]
    rr = [int(v) for v in np.asarray(rr)]
    ri = [int(v) for v in np.asarray(ri)]
    amax = 0
    for _ in range(nsteps):
        rr, ri, a = fixed_step(Pr, Pi, rr, ri, f)
        amax = max(amax, a)
    return np.array(rr, dtype=np.int64), np.array(ri, dtype=np.int64), amax


def fixed_propagate_batch(Pr, Pi, Rr, Ri, nsteps, f):
    """The same steps for B states at once (rows of Rr, Ri: B x n codes).

    Each step forms the exact accumulators acc = R P^T as integer matrix
    products (numpy int64 for Q1.15, whose sums stay below 2^(33 + log2 n);
    Python integers through object arrays for Q1.31), then the floor and
    saturation of the write-back.  Returns the new (Rr, Ri) as int64 arrays.
    """
    lo, hi = code_range(f)
    if f <= 15:
        Pr = np.asarray(Pr, dtype=np.int64)
        Pi = np.asarray(Pi, dtype=np.int64)
        Rr = np.asarray(Rr, dtype=np.int64).copy()
        Ri = np.asarray(Ri, dtype=np.int64).copy()
        for _ in range(nsteps):
            acc_r = Rr @ Pr.T - Ri @ Pi.T
            acc_i = Ri @ Pr.T + Rr @ Pi.T
            Rr = np.clip(acc_r >> f, lo, hi)  # numpy's >> on int64 is arithmetic: floor
            Ri = np.clip(acc_i >> f, lo, hi)
        return Rr, Ri
    Pr = np.asarray(Pr, dtype=np.int64).astype(object)
    Pi = np.asarray(Pi, dtype=np.int64).astype(object)
    Rr = np.asarray(Rr, dtype=np.int64).astype(object)
    Ri = np.asarray(Ri, dtype=np.int64).astype(object)
    for _ in range(nsteps):
        acc_r = Rr.dot(Pr.T) - Ri.dot(Pi.T)
        acc_i = Ri.dot(Pr.T) + Rr.dot(Pi.T)
        Rr = np.vectorize(lambda v: _floor_sat(int(v), f), otypes=[object])(acc_r)
        Ri = np.vectorize(lambda v: _floor_sat(int(v), f), otypes=[object])(acc_i)
    return Rr.astype(np.int64), Ri.astype(np.int64)


def fpga_cycles(n, k=1, nsteps=1):
    """Cycle count of Algorithm alg:fpga (Eq. eq:cost_fpga): n^2/k + n + 4
    cycles per step, N steps plus one start cycle."""
    return nsteps * (n * n // k + n + 4) + 1
