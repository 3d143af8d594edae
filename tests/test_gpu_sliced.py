"""The sliced FP64 product (lb_gemm_f64_sliced: FP64 operands written as
exact BF16 digit slices, products of equal weight summed exactly on the
tensor cores) and the LB_FP64_SLICED form built on it.

The product's stated error is |C - A B| <= K 2^(e_r + f_c) 2^-54 (13/4) per
element (2^e_r above row r of A, 2^f_c above column c of B) plus the final
rounding to FP64.  Pins:
  * integer operands whose digits all fall inside the kept pairs: the result
    is the exact product, bit for bit;
  * operands whose digits sit near their maxima, so that the group sums
    reach 86 % of 2^24 at K = 1488: the result is the kept pairs' exact sum
    rounded once (this checks that the FP32 accumulation on the tensor
    cores is exact up to the stated K);
  * random operands with rows and columns of very different magnitudes,
    against an extended-precision product, within the stated bound;
  * alpha, beta, aliasing of C with an operand, ragged and degenerate
    sizes, the K limit.
The form: the build at d = 2 .. 27 against the oracle's Pade build (1e-12
relative Frobenius per slice, as for every FP64 form) and the d = 27
propagation against the oracle's chain (1e-12 relative per state)."""

import numpy as np
import pytest

import oracle as O
from oracle import hermitian as OH
from workloads import make_workload
from workloads.rng import normal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lb


@pytest.fixture(scope="module")
def ctx(lbm):
    c = lbm.Context(0, max_n=729, max_batch=256, max_slices=4)
    yield c
    c.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _relf(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _gemm(lbm, ctx, A, B, C0=None, alpha=1.0, beta=0.0):
    nb, M, _ = A.shape
    N = B.shape[2]
    C = _t(C0) if C0 is not None else torch.zeros((nb, M, N), dtype=torch.float64, device="cuda")
    lbm.lb_gemm_f64_sliced(ctx, _t(A), _t(B), C, alpha=alpha, beta=beta)
    lbm.lb_sync_status(ctx)
    return C.cpu().numpy()


@pytest.mark.parametrize("M,N,K,batch", [(300, 100, 729, 2), (129, 33, 1488, 1), (1, 1, 1, 1), (5, 200, 17, 3)])
def test_integer_operands_exact(lbm, ctx, M, N, K, batch):
    """Integers below 2^20: every digit past the fourth is zero, so all
    digit products are kept and the result is the exact integer product
    (below 2^53, exact in FP64 on the CPU too)."""
    rng = np.random.default_rng(7 + M + K)
    A = rng.integers(-(2**20) + 1, 2**20, size=(batch, M, K)).astype(np.float64)
    B = rng.integers(-(2**20) + 1, 2**20, size=(batch, K, N)).astype(np.float64)
    got = _gemm(lbm, ctx, A, B)
    assert np.array_equal(got, A @ B)


def test_group_sums_near_their_bound_exact(lbm, ctx):
    """Operands whose digits are (63, 31, 31, 31, 31, 31, 31, 31) in every
    entry at K = 1488: the group sums reach up to 9672 K = 1.44e7 of the
    2^24 = 1.68e7 that FP32 holds exactly.  The result must be the kept
    pairs' sum rounded once to FP64, computed here in exact rational
    arithmetic, bit for bit."""
    from fractions import Fraction

    K = 1488
    digits = [63] + [31] * 7
    x = sum(Fraction(dg, 64 ** (i + 1)) for i, dg in enumerate(digits))
    xf = float(x)
    assert Fraction(xf) == x
    A = np.full((1, 130, K), xf)
    B = np.full((1, K, 40), -xf)
    got = _gemm(lbm, ctx, A, B)
    kept = sum(Fraction(digits[i] * digits[j], 64 ** (i + j + 2)) for i in range(8) for j in range(8) if i + j + 2 <= 10)
    want = float(-K * kept)
    assert np.all(got == want), (got[0, 0, 0], want)


def test_random_within_stated_bound(lbm, ctx):
    """Normal entries with rows of A and columns of B scaled over 2^-40 ..
    2^40: error per element within K 2^(e_r + f_c) 2^-54 (13/4) plus one
    rounding, against a long-double product."""
    M, N, K, batch = 200, 150, 729, 2
    A = normal(11, batch * M * K).reshape(batch, M, K)
    B = normal(12, batch * K * N).reshape(batch, K, N)
    rs = 2.0 ** np.round(np.linspace(-40, 40, M))
    cs = 2.0 ** np.round(np.linspace(40, -40, N))
    A = A * rs[None, :, None]
    B = B * cs[None, None, :]
    got = _gemm(lbm, ctx, A, B)
    ref = np.matmul(A.astype(np.longdouble), B.astype(np.longdouble))
    er = np.frexp(np.max(np.abs(A), axis=2))[1]          # 2^er > row max
    fc = np.frexp(np.max(np.abs(B), axis=1))[1]          # 2^fc > column max
    bound = K * 3.25 * np.ldexp(1.0, er[:, :, None] + fc[:, None, :] - 54) + np.abs(got) * 2.0**-53
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= bound), float(np.max(err / bound))
    # and close to an FP64 product's accuracy in the relative sense too
    assert _relf(got, (A @ B)) <= 1e-14


def test_alpha_beta_and_alias(lbm, ctx):
    M, K = 97, 97
    A = normal(21, M * K).reshape(1, M, K)
    C0 = normal(22, M * K).reshape(1, M, K)
    got = _gemm(lbm, ctx, A, A, C0=C0, alpha=-1.0, beta=0.5)
    assert _relf(got, 0.5 * C0 - A @ A) <= 1e-14
    # C aliases both operands: X <- X X
    X = _t(A)
    lbm.lb_gemm_f64_sliced(ctx, X, X, X)
    lbm.lb_sync_status(ctx)
    assert _relf(X.cpu().numpy(), A @ A) <= 1e-14


def test_zero_rows_and_k_limit(lbm, ctx):
    A = np.zeros((1, 40, 64))
    A[0, 3, :] = normal(31, 64)
    B = normal(32, 64 * 20).reshape(1, 64, 20)
    got = _gemm(lbm, ctx, A, B)
    assert np.count_nonzero(got[0, np.arange(40) != 3]) == 0
    assert _relf(got, A @ B) <= 1e-14
    with pytest.raises(lbm.LBError):
        Z = torch.zeros((1, 4, 1489), dtype=torch.float64, device="cuda")
        W = torch.zeros((1, 1489, 4), dtype=torch.float64, device="cuda")
        lbm.lb_gemm_f64_sliced(ctx, Z, W, torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda"))


def _gen_pair(d, seed, scale):
    Hr = _rand_c(seed, (d, d))
    H = 0.5 * (Hr + Hr.conj().T)
    jumps = list(_rand_c(seed + 1, (2, d, d)) * 0.3)
    Xr = _rand_c(seed + 2, (d, d))
    X = 0.5 * (Xr + Xr.conj().T)
    Lb = O.lindbladian(H, jumps)
    Ld = O.drive_generator(X)
    f = scale / O.onenorm(Lb)
    return Lb * f, Ld * f


@pytest.mark.parametrize("d,S,scale", [(2, 3, 0.2), (3, 3, 3.0), (6, 2, 13.0), (9, 3, 1.7), (11, 2, 0.6),
                                       (16, 2, 0.9), (17, 2, 2.0)])
def test_build_sliced_matches_oracle(lbm, d, S, scale):
    """Squaring counts 0 to 7: every squaring a sliced product.  n = 256 and
    289 take the 128-wide LU blocks (two 64-wide halves; 289 ends in a
    33-wide block with no second half)."""
    n = d * d
    Lb, Ld = _gen_pair(d, 2500 + d, scale)
    u = np.linspace(-0.3, 0.4, S)
    c = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device="cuda")
    s_out = torch.empty(S, dtype=torch.int32, device="cuda")
    lbm.lb_expm_pade(c, _t(Lb), _t(Ld), _t(u), 1.0, P, prec="fp64_sliced", s_out=s_out)
    lbm.lb_sync_status(c)
    Pg, sg = P.cpu().numpy(), s_out.cpu().numpy()
    for s in range(S):
        A = Lb + u[s] * Ld
        assert sg[s] == OH.squaring_count_real(A, d)[0], s
        assert _relf(Pg[s], O.expm_pade13(A)) <= 1e-12, (s, _relf(Pg[s], O.expm_pade13(A)))
    c.close()


@pytest.mark.parametrize("name,S", [("d9_batch", 3), ("d27_chain", 2)])
def test_build_sliced_workloads(lbm, ctx, name, S):
    w = make_workload(name, nslices=S)
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    n = w["n"]
    P = torch.empty((S, n, n), dtype=torch.complex128, device="cuda")
    lbm.lb_expm_pade(ctx, _t(Lb), _t(Ld), _t(w["u"]), w["dt"], P, prec="fp64_sliced")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    for s in range(S):
        assert _relf(P.cpu().numpy()[s], ref[s]) <= 1e-12, s


@pytest.mark.parametrize("B,S,m", [(256, 2, 2), (37, 3, 1)])
def test_propagate_sliced_d27(lbm, ctx, B, S, m):
    w = make_workload("d27_chain", B=B, nslices=S)
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    Ps = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    ref = O.propagate_chain(Ps, w["states"], m)
    R = _t(w["states"])
    lbm.lb_propagate_batch(ctx, _t(Ps), R, steps_per_slice=m, prec="fp64_sliced")
    lbm.lb_sync_status(ctx)
    got = R.cpu().numpy()
    for b in range(B):
        assert _relf(got[b], ref[b]) <= 1e-12, b
