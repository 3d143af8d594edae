"""Work and traffic accounting used to turn timings into roofline fractions.

Eq. 4 of the paper counts one state-step (one matvec P rho, n = d^2) as
8 n^2 real FLOPs (a complex multiply-add = 8 FLOPs) and
16 (n^2 + 2n) bytes for one state with P, rho_in and rho_out in FP64.
For a batch of B states sharing one P per step, P is read once per step, so
the compulsory bytes per state-step are 16 n^2 / B + 32 n (FP64).

The dense Pade build of one n x n propagator with s squarings counts (as
real FLOPs of dense complex arithmetic): six products and s squarings at
8 n^3 each, the LU at 8 n^3 / 3 and the n-right-hand-side solve at 8 n^3.
"""


def state_step_flops(n):
    return 8 * n * n


def state_step_bytes_single(n):
    """Eq. 4: one P, one input and one output state in FP64."""
    return 16 * (n * n + 2 * n)


def arithmetic_intensity_single(n):
    return state_step_flops(n) / state_step_bytes_single(n)


def state_step_bytes_batched(n, B, elem_bytes=16):
    """P read once per step and shared by B states; each state read and
    written once."""
    return elem_bytes * n * n / B + 2 * elem_bytes * n


def build_flops(n, s):
    """Dense FLOPs of one Pade-13 build with s squarings."""
    return (6 + s) * 8 * n ** 3 + 8 * n ** 3 / 3 + 8 * n ** 3


def build_flops_fp64_solve(n):
    """The FP64 LU factorisation and n-RHS solve of one build."""
    return 8 * n ** 3 / 3 + 8 * n ** 3


def gauss_fp64_instr_fraction():
    """The GPU's FP64 complex products use Gauss's three real products per
    complex multiply-add: the FP64 pipe executes 3/4 of the FMAs counted
    above."""
    return 0.75


# Real-coordinate ("Hermitian") forms: every matrix is a real n x n matrix
# (the action of the superoperator on the n = d^2 real coordinates of a
# Hermitian matrix), so a multiply-add is 2 real FLOPs.

def state_step_flops_real(n):
    return 2 * n * n


def build_flops_real(n, s):
    """Dense real FLOPs of one Pade-13 build on the real coordinates with s
    squarings: six products and s squarings at 2 n^3, the LU at 2 n^3 / 3
    and the n-right-hand-side solve at 2 n^3."""
    return (6 + s) * 2 * n ** 3 + 2 * n ** 3 / 3 + 2 * n ** 3


def build_flops_real_solve(n):
    return 2 * n ** 3 / 3 + 2 * n ** 3
