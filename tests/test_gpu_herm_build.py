"""GPU parity of the real-coordinate ("Hermitian") propagator build and of
the real-coordinate propagation for n > 81, against the oracle.

lb_expm_pade with prec "fp64_hermitian" runs Algorithm 1 on the real form
G of each slice generator (oracle/hermitian.py defines it) and rebuilds the
complex P at the end; the result is exp(L dt) like the complex build, so it
is compared with the oracle's complex Pade build: 1e-12 relative Frobenius
per slice, as for the complex FP64 form.  The squaring count is the one of
||G||_1 (oracle.hermitian.squaring_count_real).  "fp32_hermitian" runs the
six Pade products and the near-I squarings in FP32: like the complex FP32
form, P is within 1e-6 relative.  Propagation with "fp64_hermitian" at
n > 81 is compared with the oracle's complex chain at 1e-12 per state."""

import numpy as np
import pytest

import oracle as O
from oracle import hermitian as OH
from workloads import make_workload, paper_grape_model
from workloads.rng import ginibre_states, normal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return lb


@pytest.fixture(scope="module")
def dev():
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _relf(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _gen_pair(d, seed, scale):
    """Random Lindblad generators (a base with jumps and a Hermitian drive)."""
    Hr = _rand_c(seed, (d, d))
    H = 0.5 * (Hr + Hr.conj().T)
    jumps = list(_rand_c(seed + 1, (2, d, d)) * 0.3)
    Xr = _rand_c(seed + 2, (d, d))
    X = 0.5 * (Xr + Xr.conj().T)
    Lb = O.lindbladian(H, jumps)
    Ld = O.drive_generator(X)
    f = scale / O.onenorm(Lb)
    return Lb * f, Ld * f


def test_expm_herm_d1(lbm, dev):
    """d = 1: a Hermiticity-preserving generator is a real number (every
    Lindbladian of one level is 0); exp of the 1 x 1 real forms, within a
    few ulps (2.5 x 0.7 takes three squarings, each doubling the relative
    rounding error of the approximant)."""
    gens = np.array([[[-0.3]], [[2.5]], [[0.0]]], dtype=np.complex128)
    ctx = lbm.Context(0, max_n=1, max_batch=1, max_slices=3)
    P = torch.empty((3, 1, 1), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(gens, dev), None, None, 0.7, P, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    for s in range(3):
        ref = np.exp(0.7 * gens[s, 0, 0].real)
        assert abs(P.cpu().numpy()[s, 0, 0] - ref) <= 1e-14 * ref


@pytest.mark.parametrize("d,S,scale", [(2, 5, 0.2), (3, 4, 3.0), (5, 3, 0.9), (6, 2, 1.3),
                                       (7, 2, 13.0), (9, 3, 1.7), (11, 2, 0.6)])
def test_expm_herm_fp64_matches_oracle(lbm, dev, d, S, scale):
    """n = 4 .. 121: one to four LU blocks with a ragged last one, 16 x 16
    and 32 x 32 GEMM tiles with ragged edges, squaring counts 0 to 7."""
    n = d * d
    Lb, Ld = _gen_pair(d, 1500 + d, scale)
    u = np.linspace(-0.3, 0.4, S)
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    s_out = torch.empty(S, dtype=torch.int32, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), 1.0, P, prec="fp64_hermitian", s_out=s_out)
    lbm.lb_sync_status(ctx)
    Pg = P.cpu().numpy()
    sg = s_out.cpu().numpy()
    for s in range(S):
        A = Lb + u[s] * Ld
        assert sg[s] == OH.squaring_count_real(A, d)[0], s
        assert _relf(Pg[s], O.expm_pade13(A)) <= 1e-12, (s, _relf(Pg[s], O.expm_pade13(A)))


def test_expm_herm_per_slice_generators_and_chunking(lbm, dev):
    """Ldrv = NULL (one generator per slice) and more slices than the context
    holds at once."""
    d, S = 4, 7
    n = d * d
    gens = np.array([_gen_pair(d, 1600 + 3 * s, 0.2 + 0.5 * s)[0] for s in range(S)])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=3)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(gens, dev), None, None, 0.5, P, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    Pg = P.cpu().numpy()
    for s in range(S):
        assert _relf(Pg[s], O.expm_pade13(gens[s] * 0.5)) <= 1e-12


@pytest.mark.parametrize("prec,tol", [("fp64_hermitian", 1e-12), ("fp32_hermitian", 1e-6), ("fp64_sliced", 1e-12)])
def test_expm_herm_sparse_and_dense_slices(lbm, dev, prec, tol):
    """Slices whose powers of A are sparse (a dephasing generator: the real
    form is 2 x 2 block diagonal, so A and A^2 take the zero-skipping
    products) alternate with dense random generators in one call; every
    slice against the oracle.  In the sliced form (one generator per slice,
    no drive) A^2 is the per-slice zero-skipping product and the rest sliced."""
    d, S = 4, 6
    n = d * d
    rng_h = _rand_c(1800, (d, d))
    Hd = np.diag(np.real(np.diag(rng_h)))  # diagonal Hamiltonian
    num = np.diag(np.arange(d, dtype=float)).astype(complex)
    sparse_gen = O.lindbladian(Hd, [0.3 * num])
    gens = []
    for s in range(S):
        if s % 2 == 0:
            gens.append(sparse_gen * (0.5 + 0.3 * s))
        else:
            gens.append(_gen_pair(d, 1900 + s, 0.4 + 0.7 * s)[0])
    gens = np.array(gens)
    assert np.count_nonzero(OH.real_form(gens[0], d)) <= 0.15 * n * n
    assert np.count_nonzero(OH.real_form(gens[1], d)) > 0.15 * n * n
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(gens, dev), None, None, 1.0, P, prec=prec)
    lbm.lb_sync_status(ctx)
    for s in range(S):
        ref = O.expm_pade13(gens[s])
        assert _relf(P.cpu().numpy()[s], ref) <= tol, (s, _relf(P.cpu().numpy()[s], ref))


@pytest.mark.parametrize("name,S", [("d9_batch", 3), ("d27_chain", 2)])
def test_expm_herm_workloads(lbm, dev, name, S):
    w = make_workload(name, nslices=S)
    n = w["n"]
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    Lbg = torch.empty((n, n), dtype=torch.complex128, device=dev)
    Ldg = torch.empty_like(Lbg)
    lbm.lb_assemble(ctx, _t(w["H0"], dev), _t(w["jumps"], dev), Lbg)
    lbm.lb_assemble(ctx, _t(w["X"], dev), None, Ldg)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, Lbg, Ldg, _t(w["u"], dev), w["dt"], P, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    Pg = P.cpu().numpy()
    for s in range(S):
        assert _relf(Pg[s], ref[s]) <= 1e-12, (s, _relf(Pg[s], ref[s]))


@pytest.mark.parametrize("name,S", [("d9_batch", 3), ("d27_chain", 2)])
def test_expm_herm_fp32(lbm, dev, name, S):
    """FP32 Pade products on the real coordinates: each product of
    ||A||_1 <= 0.25 matrices is off by ~n 2^-24 relative on terms that enter
    V and U scaled by b_j ||A||^j <= 0.03 (b_1 A is added in FP64), so P is
    off by ~1e-7 relative; the test allows 1e-6, as for the complex FP32
    form."""
    w = make_workload(name, nslices=S)
    n = w["n"]
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P, prec="fp32_hermitian")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(S))
    assert err <= 1e-6, err


def test_expm_herm_fp32_paper_model_squarings(lbm, dev):
    """The paper's d = 9 model (s = 5): the leading squarings on D = R - I in
    FP32, the last in FP64; the FP32 error of the scaled approximant grows by
    about 2^s; the test allows 1e-6 relative."""
    m = paper_grape_model(9)
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    u = np.array([0.0, 0.05, -0.1])
    ctx = lbm.Context(0, max_n=81, max_batch=1, max_slices=3)
    P = torch.empty((3, 81, 81), dtype=torch.complex128, device=dev)
    s_out = torch.empty(3, dtype=torch.int32, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), m.dt, P, prec="fp32_hermitian", s_out=s_out)
    lbm.lb_sync_status(ctx)
    for s in range(3):
        assert s_out.cpu().numpy()[s] == OH.squaring_count_real((Lb + u[s] * Ld) * m.dt, 9)[0]
    ref = O.slice_propagators(Lb, Ld, u, m.dt)
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(3))
    assert err <= 1e-6, err


def test_expm_herm_output_maps_hermitian_to_hermitian(lbm, dev):
    """The rebuilt P maps every Hermitian matrix to an exactly representable
    Hermitian one up to rounding: P(rho)^+ = P(rho) within 1e-15 relative."""
    d, S = 5, 2
    n = d * d
    Lb, Ld = _gen_pair(d, 1700, 0.8)
    u = np.array([0.1, -0.2])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), 1.0, P, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    rho = ginibre_states(0x1701, d, 1)[0]
    for s in range(S):
        out = (P.cpu().numpy()[s] @ rho).reshape(d, d)
        assert np.max(np.abs(out - out.conj().T)) <= 1e-15 * np.max(np.abs(out))


def test_expm_herm_rejects_non_square(lbm, dev):
    ctx = lbm.Context(0, max_n=10, max_batch=1, max_slices=1)
    z = torch.zeros((1, 10, 10), dtype=torch.complex128, device=dev)
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_expm_pade(ctx, z, None, None, 0.1, z.clone(), prec="fp64_hermitian")
    assert ei.value.name == "LB_EINVAL"


def _random_model(seed, d):
    H = _rand_c(seed, (d, d))
    H = 0.5 * (H + H.conj().T) / d
    X = _rand_c(seed + 1, (d, d))
    X = 0.5 * (X + X.conj().T) / d
    jumps = 0.05 * np.stack([_rand_c(seed + 2, (d, d)), _rand_c(seed + 3, (d, d))]) / d
    return O.lindbladian(H, jumps), O.drive_generator(X)


@pytest.mark.parametrize("d,B,S,m", [(27, 256, 2, 1), (27, 37, 2, 2), (27, 8, 2, 3), (27, 1, 1, 2),
                                     (27, 9, 1, 1), (10, 70, 3, 2), (11, 5, 2, 3), (11, 200, 1, 2)])
def test_propagate_herm_large_n(lbm, dev, d, B, S, m):
    """n = 100, 121, 729 on the real coordinates: the few-state product for
    B <= 8, the real GEMM above; against the oracle's complex chain, 1e-12
    relative per state, and the states come back exactly Hermitian."""
    n = d * d
    if d == 27:
        w = make_workload("d27_chain", B=B, nslices=S)
        Ps = O.slice_propagators(O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"]), w["u"], w["dt"])
        X0 = w["states"]
    else:
        Lb, Ld = _random_model(0x5EED0300 + d, d)
        Ps = O.slice_propagators(Lb, Ld, np.linspace(-0.1, 0.1, S), 0.1)
        X0 = ginibre_states(0x5EED0400 + d, d, B)
    ref = O.propagate_chain(Ps, X0, m)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=S)
    R = _t(X0, dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m, prec="fp64_hermitian")
    lbm.lb_sync_status(ctx)
    Rg = R.cpu().numpy()
    for b in range(B):
        assert _relf(Rg[b], ref[b]) <= 1e-12, (b, _relf(Rg[b], ref[b]))
        M = Rg[b].reshape(d, d)
        assert np.array_equal(M, M.conj().T)


def test_herm_chain_matches_complex_chain_d27(lbm, dev):
    """The whole d = 27 step in the Hermitian FP64 form (build and
    propagation on the real coordinates) against the same step in the
    complex FP64 form, on 4 slices and 16 states: 1e-12 relative."""
    w = make_workload("d27_chain", B=16, nslices=4)
    n = w["n"]
    ctx = lbm.Context(0, max_n=n, max_batch=16, max_slices=4)
    Lbg = torch.empty((n, n), dtype=torch.complex128, device=dev)
    Ldg = torch.empty_like(Lbg)
    lbm.lb_assemble(ctx, _t(w["H0"], dev), _t(w["jumps"], dev), Lbg)
    lbm.lb_assemble(ctx, _t(w["X"], dev), None, Ldg)
    out = {}
    for prec in ("fp64", "fp64_hermitian"):
        P = torch.empty((4, n, n), dtype=torch.complex128, device=dev)
        lbm.lb_expm_pade(ctx, Lbg, Ldg, _t(w["u"], dev), w["dt"], P, prec=prec)
        R = _t(w["states"], dev)
        lbm.lb_propagate_batch(ctx, P, R, steps_per_slice=1, prec=prec)
        lbm.lb_sync_status(ctx)
        out[prec] = R.cpu().numpy()
    for b in range(16):
        assert _relf(out["fp64_hermitian"][b], out["fp64"][b]) <= 1e-12
