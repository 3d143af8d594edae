"""GPU vs oracle parity of assembly, propagator build and propagation.

Every call goes through the C ABI (ctypes binding).  Tolerances: FP64 paths
1e-12 relative Frobenius per result; FP32 propagation 1e-5 absolute Frobenius
per state after 1000 steps; FP32 Pade products 1e-6 relative on P (see the
comment at that test for the derivation)."""

import numpy as np
import pytest

import oracle as O
from workloads import make_workload, transmon_chain
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
def dev():
    return torch.device("cuda:0")


def _t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def _rand_c(seed, shape):
    z = normal(seed, 2 * int(np.prod(shape))).reshape(*shape, 2)
    return z[..., 0] + 1j * z[..., 1]


def _relf(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ assembly

@pytest.mark.parametrize("d,K", [(1, 0), (2, 1), (3, 2), (5, 3), (9, 4), (27, 6)])
def test_assemble_matches_oracle(lbm, dev, d, K):
    ctx = lbm.Context(0, max_n=d * d, max_batch=1, max_slices=1)
    Hr = _rand_c(300 + d, (d, d))
    H = Hr + Hr.conj().T
    Ls = _rand_c(400 + d, (K, d, d)) * 0.2 if K else None
    out = torch.empty((d * d, d * d), dtype=torch.complex128, device=dev)
    lbm.lb_assemble(ctx, _t(H, dev), _t(Ls, dev) if K else None, out)
    lbm.lb_sync_status(ctx)
    ref = O.lindbladian(H, [] if Ls is None else list(Ls))
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


# ------------------------------------------------------------------- build

def _gen_pair(d, seed, scale):
    """Random Lindblad generators (a base with jumps and a drive term)."""
    Hr = _rand_c(seed, (d, d))
    H = 0.5 * (Hr + Hr.conj().T)
    jumps = list(_rand_c(seed + 1, (2, d, d)) * 0.3)
    Xr = _rand_c(seed + 2, (d, d))
    X = 0.5 * (Xr + Xr.conj().T)
    Lb = O.lindbladian(H, jumps)
    Ld = O.drive_generator(X)
    f = scale / O.onenorm(Lb)
    return Lb * f, Ld * f


@pytest.mark.parametrize("d,S,scale", [(1, 3, 0.1), (2, 5, 0.2), (3, 4, 3.0), (5, 3, 0.9), (7, 2, 13.0),
                                       (9, 3, 1.7)])
def test_expm_fp64_matches_oracle(lbm, dev, d, S, scale):
    """Sizes n = 1..81 cover the ragged LU blocks (n not a multiple of 32)
    and squaring counts from 0 to 6."""
    n = d * d
    Lb, Ld = _gen_pair(d, 500 + d, scale)
    u = np.linspace(-0.3, 0.4, S)
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    s_out = torch.empty(S, dtype=torch.int32, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), 1.0, P, s_out=s_out)
    lbm.lb_sync_status(ctx)
    Pg = P.cpu().numpy()
    sg = s_out.cpu().numpy()
    for s in range(S):
        ref, info = O.expm_pade13(Lb + u[s] * Ld, return_info=True)
        assert sg[s] == info["s"]
        assert _relf(Pg[s], ref) <= 1e-12, (s, _relf(Pg[s], ref))


def test_expm_fp64_per_slice_generators_and_chunking(lbm, dev):
    """Ldrv = NULL (one generator per slice) and more slices than the
    context holds at once (processed in chunks)."""
    d, S = 4, 7
    n = d * d
    gens = []
    for s in range(S):
        Lb, _ = _gen_pair(d, 600 + 3 * s, 0.2 + 0.5 * s)
        gens.append(Lb)
    gens = np.array(gens)
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=3)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(gens, dev), None, None, 0.5, P)
    lbm.lb_sync_status(ctx)
    Pg = P.cpu().numpy()
    for s in range(S):
        assert _relf(Pg[s], O.expm_pade13(gens[s] * 0.5)) <= 1e-12


@pytest.mark.parametrize("name,S", [("d9_batch", 2), ("d27_chain", 2)])
def test_expm_fp64_workloads(lbm, dev, name, S):
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
    lbm.lb_expm_pade(ctx, Lbg, Ldg, _t(w["u"], dev), w["dt"], P)
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    Pg = P.cpu().numpy()
    for s in range(S):
        assert _relf(Pg[s], ref[s]) <= 1e-12


def test_expm_fp32_products(lbm, dev):
    """FP32 Pade products, FP64 LU/solve/squarings.  Each product of
    ||A||_1 <= 0.25 matrices carries a relative error of about
    n * 2^-24 ~ 5e-6 on terms that enter V and U scaled by b_j ||A||^j <= 0.03,
    so P is off by about 1e-7 relative; the test allows 1e-6."""
    w = make_workload("d9_batch", nslices=3)
    w["u"] = np.array([0.05, -0.08, 0.1])
    n = w["n"]
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=3)
    P = torch.empty((3, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P, prec="fp32")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(3))
    assert err <= 1e-6, err


@pytest.mark.parametrize("prec", ["fp64", "fp64_hermitian", "fp64_sliced"])
def test_expm_nonfinite_input_is_reported(lbm, dev, prec):
    n = 9
    Lb = np.zeros((n, n), dtype=complex)
    Lb[2, 3] = np.nan
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=1)
    P = torch.empty((1, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb[None], dev), None, None, 0.1, P, prec=prec)
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_sync_status(ctx)
    assert ei.value.name == "LB_ENONFINITE"
    lbm.lb_sync_status(ctx)  # the word was cleared


# ------------------------------------------------------------- propagation

def _slice_props(w, u):
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    return O.slice_propagators(Lb, Ld, u, w["dt"])


@pytest.mark.parametrize("name,B,S,m", [("d3_single", 1, 1, 200), ("d3_single", 5, 3, 4),
                                        ("d9_batch", 37, 2, 3), ("d9_batch", 300, 1, 5),
                                        ("d9_batch", 1, 2, 50), ("d9_batch", 4, 1, 7), ("d9_batch", 5, 1, 3)])
def test_propagate_fp64_resident(lbm, dev, name, B, S, m):
    w = make_workload(name, B=B)
    u = np.linspace(-0.1, 0.1, S)
    Ps = _slice_props(w, u)
    ctx = lbm.Context(0, max_n=w["n"], max_batch=B, max_slices=S)
    R = _t(w["states"], dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m)
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, w["states"], m)
    Rg = R.cpu().numpy()
    for b in range(B):
        assert _relf(Rg[b], ref[b]) <= 1e-12


@pytest.mark.parametrize("B,S,m", [(256, 2, 1), (37, 1, 2), (1, 2, 3), (3, 1, 2), (8, 2, 1), (9, 1, 1)])
def test_propagate_fp64_d27(lbm, dev, B, S, m):
    """B <= 8 states take the warp-per-row product (k_gemv.cu), more the
    tiled GEMM."""
    w = make_workload("d27_chain", B=B, nslices=S)
    Ps = _slice_props(w, w["u"])
    ctx = lbm.Context(0, max_n=w["n"], max_batch=B, max_slices=S)
    R = _t(w["states"], dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m)
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, w["states"], m)
    Rg = R.cpu().numpy()
    for b in range(B):
        assert _relf(Rg[b], ref[b]) <= 1e-12


def test_propagate_fp32_d9_1000_steps(lbm, dev):
    """The d = 9 batch: 1024 states, 1000 steps, FP32 with the per-step trace
    renormalisation; max over states of ||rho - rho_ref||_F <= 1e-5."""
    w = make_workload("d9_batch")
    Ps = _slice_props(w, w["u"])
    ref = O.propagate(Ps[0], w["states"], w["steps_per_slice"])
    ctx = lbm.Context(0, max_n=w["n"], max_batch=w["B"], max_slices=1)
    for renorm in (True, False):
        R = _t(w["states"], dev)
        lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=w["steps_per_slice"], prec="fp32",
                               renorm_trace=renorm)
        lbm.lb_sync_status(ctx)
        err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
        assert err <= 1e-5, (renorm, err)


def test_propagate_fp32_d27(lbm, dev):
    w = make_workload("d27_chain", B=64, nslices=3)
    Ps = _slice_props(w, w["u"])
    ref = O.propagate_chain(Ps, w["states"], 1)
    ctx = lbm.Context(0, max_n=w["n"], max_batch=64, max_slices=3)
    R = _t(w["states"], dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=1, prec="fp32", renorm_trace=True)
    lbm.lb_sync_status(ctx)
    err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
    assert err <= 1e-6, err


def _random_model(seed, d):
    """A random open system of dimension d: Hermitian H and drive X, two jump
    operators, scaled like the transmon generators (||L dt|| well below 1)."""
    H = _rand_c(seed, (d, d))
    H = 0.5 * (H + H.conj().T) / d
    X = _rand_c(seed + 1, (d, d))
    X = 0.5 * (X + X.conj().T) / d
    jumps = 0.05 * np.stack([_rand_c(seed + 2, (d, d)), _rand_c(seed + 3, (d, d))]) / d
    return O.lindbladian(H, jumps), O.drive_generator(X)


@pytest.mark.parametrize("d,B,S,m,renorm", [
    (27, 256, 2, 1, True),    # 4 x 12 tiles, K split in 3
    (27, 37, 2, 2, False),    # ragged batch, K split in 8
    (27, 37, 1, 3, True),
    (10, 70, 3, 1, True),     # n = 100: ragged K and N, no split
    (11, 200, 2, 2, False),   # n = 121, 4 x 2 tiles
])
def test_propagate_fp32_chain_shapes(lbm, dev, d, B, S, m, renorm):
    """FP32 chain kernel for n > 81 (split-K, padding, deferred trace
    renormalisation) against the oracle chain; 1e-6 absolute Frobenius per
    state for these short chains."""
    from workloads.rng import ginibre_states

    n = d * d
    if d == 27:
        w = make_workload("d27_chain", B=B, nslices=S)
        Ps = _slice_props(w, w["u"])
        X0 = w["states"]
    else:
        Lb, Ld = _random_model(0x5EED0100 + d, d)
        u = np.linspace(-0.1, 0.1, S)
        Ps = O.slice_propagators(Lb, Ld, u, 0.1)
        X0 = ginibre_states(0x5EED0200 + d, d, B)
    ref = O.propagate_chain(Ps, X0, m)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=S)
    R = _t(X0, dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m, prec="fp32", renorm_trace=renorm)
    lbm.lb_sync_status(ctx)
    err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
    assert err <= 1e-6, err


def test_propagate_fp32_d27_200_steps(lbm, dev):
    """Long FP32 chain at d = 27 (200 steps, the length of the 200-slice
    workload), renormalised: <= 1e-5 absolute Frobenius per state; run twice
    to check that the split-K tickets are reset between launches."""
    w = make_workload("d27_chain", B=16, nslices=2)
    Ps = _slice_props(w, w["u"])
    ref = O.propagate_chain(Ps, w["states"], 100)
    ctx = lbm.Context(0, max_n=729, max_batch=16, max_slices=2)
    out = []
    for _ in range(2):
        R = _t(w["states"], dev)
        lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=100, prec="fp32", renorm_trace=True)
        lbm.lb_sync_status(ctx)
        out.append(R.cpu().numpy())
        err = np.max(np.linalg.norm(out[-1] - ref, axis=1))
        assert err <= 1e-5, err
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("B,renorm", [(64, True), (37, False)])
def test_propagate_fp32_d27_persistent(lbm, dev, B, renorm):
    """The d = 27 FP32 chain with many steps runs as one persistent launch
    (grid barrier between steps) rather than one launch per step: 60 steps
    over 3 slices take at most a handful of launches, match the oracle chain
    (1e-5 absolute Frobenius per state) and repeat bit for bit (the barrier
    counter is reset per launch)."""
    w = make_workload("d27_chain", B=B, nslices=3)
    Ps = _slice_props(w, w["u"])
    ref = O.propagate_chain(Ps, w["states"], 20)
    ctx = lbm.Context(0, max_n=729, max_batch=B, max_slices=3)
    out = []
    for _ in range(2):
        R = _t(w["states"], dev)
        n0 = lbm.lb_launch_count()
        lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=20, prec="fp32", renorm_trace=renorm)
        lbm.lb_sync_status(ctx)
        launches = lbm.lb_launch_count() - n0
        assert launches <= 8, launches
        out.append(R.cpu().numpy())
        err = np.max(np.linalg.norm(out[-1] - ref, axis=1))
        assert err <= 1e-5, err
    assert np.array_equal(out[0], out[1])


def test_zero_steps_and_slices_leave_states(lbm, dev):
    w = make_workload("d3_single", B=3)
    Ps = _slice_props(w, np.array([0.05]))
    ctx = lbm.Context(0, max_n=9, max_batch=3, max_slices=1)
    R = _t(w["states"], dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=0)
    lbm.lb_sync_status(ctx)
    assert np.array_equal(R.cpu().numpy(), w["states"])


# -------------------------------------------------------------------- GRAPE

def _gate_problem(nq, S, seed, B=4):
    m = transmon_chain(nq)
    d, n = m.d, m.d * m.d
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    u = 0.3 * normal(seed, S)
    X0 = np.zeros((B, n), dtype=complex)
    Xt = np.zeros((B, n), dtype=complex)
    basis = [(0, 0), (0, 1), (1, 0), (1, 1)][:B]
    th = 0.7
    Ux = np.eye(d, dtype=complex)
    Ux[:2, :2] = [[np.cos(th / 2), -1j * np.sin(th / 2)], [-1j * np.sin(th / 2), np.cos(th / 2)]]
    for b, (i, j) in enumerate(basis):
        E = np.zeros((d, d), dtype=complex)
        E[i, j] = 1.0
        X0[b] = O.vec(E)
        Xt[b] = O.vec(Ux @ E @ Ux.conj().T)
    return Lb, Ld, u, m.dt, X0, Xt


@pytest.mark.parametrize("nq,S,m,dtscale", [(1, 7, 1, 1.0), (1, 4, 3, 20.0), (2, 5, 2, 1.0), (2, 3, 1, 30.0)])
def test_grape_matches_oracle(lbm, dev, nq, S, m, dtscale):
    """F and dF/du against the oracle (Van Loan block Frechet derivative);
    dtscale > 1 forces several squarings.  Both sides are exact to rounding
    plus the Pade truncation (~1e-13 relative): F within 1e-12, gradient
    within 1e-9 of max |g|."""
    Lb, Ld, u, dt, X0, Xt = _gate_problem(nq, S, 900 + S)
    dt = dt * dtscale
    F_ref, g_ref = O.grape_fidelity_grad(Lb, Ld, u, dt, m, X0, Xt)
    n = Lb.shape[0]
    ctx = lbm.Context(0, max_n=n, max_batch=4, max_slices=S)
    Fo = torch.zeros(1, dtype=torch.float64, device=dev)
    go = torch.zeros(S, dtype=torch.float64, device=dev)
    lbm.lb_grape_grad(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), dt, m, _t(X0, dev), _t(Xt, dev), Fo, go)
    lbm.lb_sync_status(ctx)
    F = float(Fo.item())
    g = go.cpu().numpy()
    assert abs(F - F_ref) <= 1e-12 * max(1.0, abs(F_ref)), (F, F_ref)
    assert np.max(np.abs(g - g_ref)) <= 1e-9 * max(1e-6, np.max(np.abs(g_ref))), (g, g_ref)


@pytest.mark.parametrize("nq,K,S,m,prec,tol", [(1, 5, 7, 1, "fp64", 1e-9), (1, 3, 4, 3, "fp64", 1e-9),
                                                (2, 3, 5, 2, "fp64", 1e-9), (1, 4, 6, 1, "fp32", 1e-5),
                                                (2, 2, 3, 1, "fp32", 1e-5)])
def test_grape_batch_matches_oracle(lbm, dev, nq, K, S, m, prec, tol):
    """K problems with their own base generators (jump rates), controls and
    targets in one call, each against the oracle's F and gradient (Van Loan
    block Frechet derivative): FP64 as lb_grape_grad (F within 1e-12,
    gradient within 1e-9 of max |g|); FP32 products: within 1e-5 of max |g|
    (products of operands rounded to 2^-24 relative, n terms each)."""
    from workloads import transmon_chain

    models = [transmon_chain(nq, gamma1=1e-3 * (k + 1), gamma_phi=5e-4 / (k + 1)) for k in range(K)]
    Lbs = np.array([O.lindbladian(mm.H0, mm.jumps) for mm in models])
    Ld = O.drive_generator(models[0].X)
    n = Lbs.shape[1]
    us, X0s, Xts, refs = [], [], [], []
    for k in range(K):
        _, _, u, dt, X0, Xt = _gate_problem(nq, S, 1000 + 17 * k)
        us.append(u)
        X0s.append(X0)
        Xts.append(np.roll(Xt, k, axis=0))  # a different target per problem
        refs.append(O.grape_fidelity_grad(Lbs[k], Ld, u, dt, m, X0s[-1], Xts[-1]))
    ctx = lbm.Context(0, max_n=n, max_batch=4 * K, max_slices=K * S)
    Fo = torch.zeros(K, dtype=torch.float64, device=dev)
    go = torch.zeros((K, S), dtype=torch.float64, device=dev)
    lbm.lb_grape_grad_batch(ctx, _t(Lbs, dev), _t(Ld, dev), _t(np.array(us), dev), dt, m, _t(np.array(X0s), dev),
                            _t(np.array(Xts), dev), Fo, go, prec=prec)
    lbm.lb_sync_status(ctx)
    F, g = Fo.cpu().numpy(), go.cpu().numpy()
    for k in range(K):
        F_ref, g_ref = refs[k]
        assert abs(F[k] - F_ref) <= max(tol, 1e-12) * max(1.0, abs(F_ref)), (k, F[k], F_ref)
        assert np.max(np.abs(g[k] - g_ref)) <= tol * max(1e-6, np.max(np.abs(g_ref))), (k, g[k], g_ref)


def test_grape_batch_shared_base_equals_single_calls(lbm, dev):
    """A shared base generator (stride 0): every problem equals its own
    lb_grape_grad call to rounding."""
    K, S = 4, 6
    Lb, Ld, _, dt, X0, Xt = _gate_problem(1, S, 1200)
    n = Lb.shape[0]
    us = np.array([0.3 * normal(1300 + k, S) for k in range(K)])
    ctx = lbm.Context(0, max_n=n, max_batch=4 * K, max_slices=K * S)
    Fo = torch.zeros(K, dtype=torch.float64, device=dev)
    go = torch.zeros((K, S), dtype=torch.float64, device=dev)
    X0b = np.repeat(X0[None], K, axis=0)
    Xtb = np.repeat(Xt[None], K, axis=0)
    lbm.lb_grape_grad_batch(ctx, _t(Lb, dev), _t(Ld, dev), _t(us, dev), dt, 1, _t(X0b, dev), _t(Xtb, dev), Fo, go)
    lbm.lb_sync_status(ctx)
    for k in range(K):
        F1 = torch.zeros(1, dtype=torch.float64, device=dev)
        g1 = torch.zeros(S, dtype=torch.float64, device=dev)
        lbm.lb_grape_grad(ctx, _t(Lb, dev), _t(Ld, dev), _t(us[k], dev), dt, 1, _t(X0, dev), _t(Xt, dev), F1, g1)
        lbm.lb_sync_status(ctx)
        assert abs(Fo[k].item() - F1.item()) <= 1e-13
        assert np.max(np.abs(go[k].cpu().numpy() - g1.cpu().numpy())) <= 1e-12 * max(1e-6, g1.abs().max().item())


def test_grape_rejects_large_contexts(lbm, dev):
    ctx = lbm.Context(0, max_n=729, max_batch=4, max_slices=2)
    z = torch.zeros((9, 9), dtype=torch.complex128, device=dev)
    x = torch.zeros((1, 9), dtype=torch.complex128, device=dev)
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_grape_grad(ctx, z, z, torch.zeros(2, dtype=torch.float64, device=dev), 0.1, 1, x, x,
                          torch.zeros(1, dtype=torch.float64, device=dev),
                          torch.zeros(2, dtype=torch.float64, device=dev))
    assert ei.value.name == "LB_EUNSUPPORTED"


def test_expm_fp32_mixed_squarings_paper_model(lbm, dev):
    """Mixed build on the paper's d = 9 model (||L dt||_1 ~ 4, s = 5): four
    squarings on D = P - I in FP32, the last in FP64.  The FP32 error of the
    scaled approximant (~1e-8) grows by about 2^s through the squarings; the
    test allows 1e-6 relative."""
    from workloads import paper_grape_model

    m = paper_grape_model(9)
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    u = np.array([0.0, 0.05, -0.1])
    n = 81
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=3)
    P = torch.empty((3, n, n), dtype=torch.complex128, device=dev)
    s_out = torch.empty(3, dtype=torch.int32, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), m.dt, P, prec="fp32", s_out=s_out)
    lbm.lb_sync_status(ctx)
    assert list(s_out.cpu().numpy()) == [5, 5, 5]
    ref = O.slice_propagators(Lb, Ld, u, m.dt)
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(3))
    assert err <= 1e-6, err


def test_expm_fp32_d27(lbm, dev):
    w = make_workload("d27_chain", nslices=2)
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=729, max_batch=1, max_slices=2)
    P = torch.empty((2, 729, 729), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P, prec="fp32")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(2))
    assert err <= 1e-6, err


@pytest.mark.parametrize("name,S,tol", [("d9_batch", 3, 1e-6), ("d27_chain", 2, 1e-6)])
def test_expm_bf16x3_products(lbm, dev, name, S, tol):
    """Split-BF16 x3 Pade products on the tensor cores.  Each operand keeps
    about 16 significant bits (relative rounding 2^-17), so A^2 is off by
    ~1e-6 relative; it enters P through b_2 A^2 (b_2 = 0.12, ||A^2|| <= 0.06)
    and U is formed as A (W' - b_1 I) + b_1 A so that only its O(A^3) part is
    rounded: P is off by ~1e-7; the test allows `tol`."""
    w = make_workload(name, nslices=S)
    n = w["n"]
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P, prec="bf16x3")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(S))
    assert err <= tol, err


def test_expm_bf16x3_paper_model_squarings(lbm, dev):
    """s = 5 (four FP32 D-form squarings and one FP64): the ~1e-7 error of
    the scaled approximant grows by about 2^s; the test allows 1e-5."""
    from workloads import paper_grape_model

    m = paper_grape_model(9)
    Lb = O.lindbladian(m.H0, m.jumps)
    Ld = O.drive_generator(m.X)
    u = np.array([0.0, 0.05, -0.1])
    ctx = lbm.Context(0, max_n=81, max_batch=1, max_slices=3)
    P = torch.empty((3, 81, 81), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), m.dt, P, prec="bf16x3")
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, u, m.dt)
    err = max(_relf(P.cpu().numpy()[s], ref[s]) for s in range(3))
    assert err <= 1e-5, err


@pytest.mark.parametrize("d,S,scale", [(2, 3, 0.2), (5, 2, 0.9), (7, 2, 3.0)])
def test_expm_bf16x3_ragged_sizes(lbm, dev, d, S, scale):
    """n = 4, 25, 49: tiles far from full (M, N, K < 128) exercise the
    zero-filled TMA boxes."""
    n = d * d
    Lb, Ld = _gen_pair(d, 700 + d, scale)
    u = np.linspace(-0.2, 0.3, S)
    ctx = lbm.Context(0, max_n=n, max_batch=1, max_slices=S)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(u, dev), 1.0, P, prec="bf16x3")
    lbm.lb_sync_status(ctx)
    for s in range(S):
        ref = O.expm_pade13(Lb + u[s] * Ld)
        assert _relf(P.cpu().numpy()[s], ref) <= 1e-5


def test_propagate_bf16x3_d9_1000_steps(lbm, dev):
    """The d = 9 batch in split-BF16 x3 on the tensor cores: max over states
    of ||rho - rho_ref||_F after 1000 steps <= 1e-4 (with and without the
    trace renormalisation)."""
    w = make_workload("d9_batch")
    Ps = _slice_props(w, w["u"])
    ref = O.propagate(Ps[0], w["states"], w["steps_per_slice"])
    ctx = lbm.Context(0, max_n=w["n"], max_batch=w["B"], max_slices=1)
    for renorm in (True, False):
        R = _t(w["states"], dev)
        lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=w["steps_per_slice"], prec="bf16x3",
                               renorm_trace=renorm)
        lbm.lb_sync_status(ctx)
        err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
        assert err <= 1e-4, (renorm, err)


@pytest.mark.parametrize("B,S,m", [(256, 3, 1), (37, 2, 2)])
def test_propagate_bf16x3_d27(lbm, dev, B, S, m):
    w = make_workload("d27_chain", B=B, nslices=S)
    Ps = _slice_props(w, w["u"])
    ref = O.propagate_chain(Ps, w["states"], m)
    ctx = lbm.Context(0, max_n=729, max_batch=B, max_slices=S)
    R = _t(w["states"], dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m, prec="bf16x3", renorm_trace=True)
    lbm.lb_sync_status(ctx)
    err = np.max(np.linalg.norm(R.cpu().numpy() - ref, axis=1))
    assert err <= 1e-5, err


# --------------------------------------------------------- many instances

def _instance_set(seed, spec):
    """spec: list of (nq, nslices, B, steps_per_slice)."""
    from workloads.rng import uniform01, stream_seed, ginibre_states

    out = []
    for k, (nq, S, B, m) in enumerate(spec):
        mdl = transmon_chain(nq)
        u = (2.0 * uniform01(stream_seed(seed, "u%d" % k), S) - 1.0) * 0.1
        st = ginibre_states(stream_seed(seed, "s%d" % k), mdl.d, B)
        out.append(dict(model=mdl, u=u, states=st, steps=m))
    return out


@pytest.mark.parametrize("prec,tol,kind", [("fp64", 1e-12, "rel"), ("fp32", 2e-6, "rel"), ("bf16x3", 1e-4, "abs"),
                                           ("fp64_hermitian", 1e-12, "rel"), ("fp32_hermitian", 2e-6, "rel"),
                                           ("fp64_sliced", 1e-12, "rel")])
def test_run_instances_matches_oracle(lbm, dev, prec, tol, kind):
    """Mixed d = 3 / 9 / 27 instances in one call, with chunks that hold
    several whole instances (max_slices = 6), 1 to 64 states per instance
    (d = 27 with 1, 5 and 64) and several steps per slice.  FP64 and FP32:
    relative Frobenius per state; split-BF16 (the form the bench times): the
    stated bound, 1e-4 absolute Frobenius per state."""
    spec = [(1, 3, 1, 2), (2, 2, 11, 1), (1, 5, 9, 3), (3, 2, 5, 1), (2, 4, 3, 2), (1, 1, 20, 1), (2, 6, 2, 1),
            (3, 1, 64, 2), (3, 2, 1, 1), (1, 2, 64, 1)]
    inst = _instance_set(0x5EED0003, spec)
    ctx = lbm.Context(0, max_n=729, max_batch=64, max_slices=6)
    keep, arg = [], []
    for x in inst:
        m = x["model"]
        Lb = O.lindbladian(m.H0, m.jumps)
        Ld = O.drive_generator(m.X)
        t = dict(Lbase=_t(Lb, dev), Ldrv=_t(Ld, dev), u=_t(x["u"], dev), states=_t(x["states"], dev),
                 steps_per_slice=x["steps"])
        keep.append((Lb, Ld, t))
        arg.append(t)
    lbm.lb_run_instances(ctx, arg, 0.1, prec=prec, renorm_trace=not prec.startswith("fp64"))
    lbm.lb_sync_status(ctx)
    for x, (Lb, Ld, t) in zip(inst, keep):
        Ps = O.slice_propagators(Lb, Ld, x["u"], 0.1)
        ref = O.propagate_chain(Ps, x["states"], x["steps"])
        got = t["states"].cpu().numpy()
        if kind == "rel":
            err = np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1))
        else:
            err = np.max(np.linalg.norm(got - ref, axis=1))
        assert err <= tol, (x["model"].d, err)


@pytest.mark.parametrize("d,B,S,m", [(1, 3, 2, 5), (2, 1, 3, 50), (3, 7, 2, 10), (3, 1, 1, 400), (4, 33, 2, 4),
                                     (3, 300, 2, 3), (4, 200, 1, 5), (5, 2, 1, 6), (7, 4, 2, 3), (6, 5, 1, 2)])
def test_propagate_fp64_small_n_forms(lbm, dev, d, B, S, m):
    """n = 1, 4, 9, 16 with at most one state per SM take the four-warp
    latency kernel (one CTA per state), with more states the one-warp-per-
    state kernel; 16 < n <= 81 the warp-per-row product for at most four
    states, else the shared memory kernel."""
    from workloads.rng import ginibre_states

    n = d * d
    Lb, Ld = _gen_pair(d, 800 + d, 0.3)
    u = np.linspace(-0.2, 0.2, S)
    Ps = np.array([O.expm_pade13(Lb + us * Ld) for us in u])
    states = ginibre_states(900 + d, d, B)
    ctx = lbm.Context(0, max_n=n, max_batch=B, max_slices=S)
    R = _t(states, dev)
    lbm.lb_propagate_batch(ctx, _t(Ps, dev), R, steps_per_slice=m)
    lbm.lb_sync_status(ctx)
    ref = O.propagate_chain(Ps, states, m)
    Rg = R.cpu().numpy()
    for b in range(B):
        assert _relf(Rg[b], ref[b]) <= 1e-12


def test_autotune_keeps_results(lbm, dev):
    """Tile choices change only the work split: the FP64 build is equal to
    rounding before and after tuning, and matches the oracle."""
    w = make_workload("d9_batch", nslices=4)
    n = w["n"]
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    ctx = lbm.Context(0, max_n=n, max_batch=8, max_slices=4)
    P1 = torch.empty((4, n, n), dtype=torch.complex128, device=dev)
    P2 = torch.empty_like(P1)
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P1)
    shapes = lbm.lb_autotune(ctx, n, 4, 8)
    assert shapes > 0
    lbm.lb_expm_pade(ctx, _t(Lb, dev), _t(Ld, dev), _t(w["u"], dev), w["dt"], P2)
    lbm.lb_sync_status(ctx)
    ref = O.slice_propagators(Lb, Ld, w["u"], w["dt"])
    for s in range(4):
        assert _relf(P2.cpu().numpy()[s], ref[s]) <= 1e-12
        assert _relf(P2.cpu().numpy()[s], P1.cpu().numpy()[s]) <= 1e-13
