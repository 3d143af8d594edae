"""Rounding emulator for the reduced-precision propagation forms.

TEST INFRASTRUCTURE ONLY.  Like ``oracle.lindblad`` this module is the slow,
plain reference the CUDA path is checked against; only the test suite, the
smoke check of the package entry module and the CPU-baseline leg of the
benchmark may import it, and it shares no code with the library.

It predicts, on the CPU, the error that the FP32 and split-BF16 forms of the
propagation step should show against FP64, so that the GPU's error can be
judged against an expectation and not only against the stated bound.  It
emulates the arithmetic the forms are defined by, not the kernels' order of
operations:

  * the step in the reduced forms is rho <- rho + D rho with D = P - I
    (the D-form, read from the paper's Sec. 3.2 step as the design notes
    state), optionally followed by division by the trace;
  * FP32: D and the states rounded to float32, products and sums in float32;
  * split-BF16: x ~ x0 + x1 (two BF16 pieces of the float32 state) and
    D ~ d0 + d1 + d2 (three BF16 pieces), the five products x_i d_j with
    i + j <= 2 summed in float32, then the residual and the trace factor in
    float32.

BF16 is the upper half of an IEEE binary32: 1 sign bit, 8 exponent bits and
7 stored fraction bits; rounding to it is to the nearest value, ties to the
even last bit (written out here from that definition, on the float32 bit
pattern).
"""

import numpy as np


def round_bf16(x):
    """Real array -> nearest BF16 values (ties to even), as float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16 << 16  # add half an ulp (and the tie bit), drop 16 bits
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isfinite(f), out, f)


def split_bf16(x, pieces):
    """Real float32 array -> list of BF16 pieces (float32 arrays) with
    x ~ sum of the pieces: each piece is the BF16 rounding of what the
    previous ones leave, the remainders formed exactly in float64."""
    rest = np.asarray(x, dtype=np.float64)
    out = []
    for _ in range(pieces):
        p = round_bf16(rest)
        out.append(p)
        rest = rest - p.astype(np.float64)
    return out


def _c32(z):
    z = np.asarray(z)
    return z.real.astype(np.float32), z.imag.astype(np.float32)


def _trace_div(Rr, Ri, d):
    """Divide each row (a d x d state) by its trace, in float32."""
    idx = [k * (d + 1) for k in range(d)]
    tr = Rr[:, idx].sum(axis=1, dtype=np.float32)
    ti = Ri[:, idx].sum(axis=1, dtype=np.float32)
    m2 = tr * tr + ti * ti
    cr, ci = (tr / m2)[:, None], (-ti / m2)[:, None]
    return Rr * cr - Ri * ci, Rr * ci + Ri * cr


def propagate_fp32(P, states, nsteps, renorm=True):
    """nsteps FP32 D-form steps of the rows of `states` (B x n complex):
    rho <- rho + D rho in float32, then the trace division."""
    P = np.asarray(P)
    n = P.shape[0]
    d = int(round(np.sqrt(n)))
    Dr, Di = _c32(P - np.eye(n))
    Rr, Ri = _c32(states)
    for _ in range(nsteps):
        # (R D^T): real and imaginary parts of the complex product in float32
        yr = Rr @ Dr.T - Ri @ Di.T
        yi = Rr @ Di.T + Ri @ Dr.T
        Rr, Ri = Rr + yr, Ri + yi
        if renorm:
            Rr, Ri = _trace_div(Rr, Ri, d)
    return Rr.astype(np.float64) + 1j * Ri.astype(np.float64)


def propagate_bf16x3(P, states, nsteps, renorm=True):
    """nsteps split-BF16 D-form steps: D in three BF16 pieces, the float32
    states in two, the five products x_i d_j (i + j <= 2) summed in float32,
    then the residual and the trace division in float32."""
    P = np.asarray(P)
    n = P.shape[0]
    d = int(round(np.sqrt(n)))
    Dr, Di = _c32(P - np.eye(n))
    dr = split_bf16(Dr, 3)
    di = split_bf16(Di, 3)
    Rr, Ri = _c32(states)
    for _ in range(nsteps):
        xr = split_bf16(Rr, 2)
        xi = split_bf16(Ri, 2)
        yr = np.zeros_like(Rr)
        yi = np.zeros_like(Ri)
        for i in range(2):
            for j in range(3):
                if i + j <= 2:
                    yr += xr[i] @ dr[j].T - xi[i] @ di[j].T
                    yi += xr[i] @ di[j].T + xi[i] @ dr[j].T
        Rr, Ri = Rr + yr, Ri + yi
        if renorm:
            Rr, Ri = _trace_div(Rr, Ri, d)
    return Rr.astype(np.float64) + 1j * Ri.astype(np.float64)
