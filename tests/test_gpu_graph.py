"""CUDA-graph capture of the build and the propagation (fixed squaring
bound, no host waits): a replayed graph gives the same states as the
uncaptured calls; without a bound the calls refuse to be captured; a slice
that needs more squarings than the bound is reported."""

import numpy as np
import pytest

import oracle as O
from workloads import make_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _setup(lbm, prec):
    dev = torch.device("cuda:0")
    w = make_workload("d9_batch", B=16, nslices=3, steps_per_slice=4)
    w["u"] = np.array([0.05, -0.07, 0.09])
    n = w["n"]
    ctx = lbm.Context(0, max_n=n, max_batch=16, max_slices=3)
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    Lb = put(O.lindbladian(w["H0"], w["jumps"]))
    Ld = put(O.drive_generator(w["X"]))
    u = put(w["u"])
    P = torch.empty((3, n, n), dtype=torch.complex128, device=dev)
    s0 = put(w["states"])
    return ctx, w, Lb, Ld, u, P, s0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x3"])
def test_captured_build_and_propagation_replay(lbm, prec):
    ctx, w, Lb, Ld, u, P, s0 = _setup(lbm, prec)
    lbm.lb_set_max_squarings(ctx, 4)

    def step(R):
        lbm.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P, prec=prec)
        lbm.lb_propagate_batch(ctx, P, R, steps_per_slice=4, prec=prec, renorm_trace=(prec != "fp64"))

    ref = s0.clone()
    step(ref)  # uncaptured (also initialises the library's lazy state)
    lbm.lb_sync_status(ctx)
    R = s0.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step(R)
    for _ in range(2):
        R.copy_(s0)
        g.replay()
        torch.cuda.synchronize()
        lbm.lb_sync_status(ctx)
        assert torch.equal(R, ref)
    Ps = O.slice_propagators(O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"]), w["u"], w["dt"])
    exact = O.propagate_chain(Ps, w["states"], 4)
    err = np.max(np.linalg.norm(R.cpu().numpy() - exact, axis=1))
    assert err <= (1e-12 if prec == "fp64" else 1e-5)


def test_capture_without_bound_is_refused(lbm):
    ctx, w, Lb, Ld, u, P, s0 = _setup(lbm, "fp64")
    lbm.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P)  # initialise outside the capture
    lbm.lb_sync_status(ctx)
    g = torch.cuda.CUDAGraph()
    with pytest.raises(lbm.LBError) as ei:
        with torch.cuda.graph(g):
            lbm.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P)
    assert ei.value.name == "LB_EUNSUPPORTED"


def test_squaring_bound_exceeded_is_reported(lbm):
    ctx, w, Lb, Ld, u, P, s0 = _setup(lbm, "fp64")
    lbm.lb_set_max_squarings(ctx, 0)  # the d = 9 slices need one squaring
    lbm.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P)
    with pytest.raises(lbm.LBError) as ei:
        lbm.lb_sync_status(ctx)
    assert ei.value.name == "LB_EUNSUPPORTED"


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "fp32_hermitian", "fp64_sliced"])
def test_captured_mixed_instances_replay(lbm, prec):
    """24 instances of the mixed-size batch (d = 3 / 9 / 27, 50 slices,
    1..64 states) captured in one graph: the replay equals the uncaptured
    call bit for bit, and every instance's final states match the oracle
    (its Taylor route through the 50 slices): 1e-12 relative per state in
    FP64, the stated bounds (split-BF16 1e-4, FP32 1e-5) absolute per state
    in the reduced forms; fp64_sliced is the form the bench captures)."""
    from oracle import expmv as E

    dev = torch.device("cuda:0")
    from workloads.configs import make_instances

    inst, models = make_instances(24)
    assert {x["d"] for x in inst} == {3, 9, 27}
    put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ctx = lbm.Context(0, max_n=729, max_batch=64, max_slices=100)
    lbm.lb_set_max_squarings(ctx, 3)
    gens_h = {q: (O.lindbladian(m.H0, m.jumps), O.drive_generator(m.X)) for q, m in models.items()}
    gens = {q: (put(a), put(b)) for q, (a, b) in gens_h.items()}
    s0 = [put(x["states"]) for x in inst]
    arg = [dict(Lbase=gens[x["nq"]][0], Ldrv=gens[x["nq"]][1], u=put(x["u"]), states=s0[i].clone())
           for i, x in enumerate(inst)]
    renorm = not prec.startswith("fp64")
    lbm.lb_run_instances(ctx, arg, 0.1, prec=prec, renorm_trace=renorm)
    lbm.lb_sync_status(ctx)
    ref = [a["states"].clone() for a in arg]
    for a, s in zip(arg, s0):
        a["states"].copy_(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lbm.lb_run_instances(ctx, arg, 0.1, prec=prec, renorm_trace=renorm)
    for a, s in zip(arg, s0):
        a["states"].copy_(s)
    g.replay()
    torch.cuda.synchronize()
    lbm.lb_sync_status(ctx)
    for a, r in zip(arg, ref):
        assert torch.equal(a["states"], r)
    for x, a in zip(inst, arg):
        Lb, Ld = gens_h[x["nq"]]
        exact, _ = E.expmv_chain(Lb, Ld, x["u"], 0.1, x["states"])
        got = a["states"].cpu().numpy()
        if prec in ("fp64", "fp64_sliced"):
            err = np.max(np.linalg.norm(got - exact, axis=1) / np.linalg.norm(exact, axis=1))
            assert err <= 1e-12, (x["d"], err)
        else:  # the stated bounds: split-BF16 1e-4, FP32 1e-5 (absolute per state)
            err = np.max(np.linalg.norm(got - exact, axis=1))
            assert err <= (1e-4 if prec == "bf16x3" else 1e-5), (x["d"], err)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_captured_chain_replay_d27(lbm, prec):
    """n = 729 chain steps (launched back to back with programmatic
    dependent launch) captured in a graph: replays equal the uncaptured run
    bit for bit and stay within the form's tolerance of the oracle."""
    dev = torch.device("cuda:0")
    w = make_workload("d27_chain", B=16, nslices=3)
    Ps = O.slice_propagators(O.lindbladian(w["H0"], w["jumps"]), O.drive_generator(w["X"]), w["u"], w["dt"])
    ctx = lbm.Context(0, max_n=729, max_batch=16, max_slices=3)
    P = torch.from_numpy(Ps).to(dev)
    s0 = torch.from_numpy(w["states"]).to(dev)

    def run(R):
        lbm.lb_propagate_batch(ctx, P, R, steps_per_slice=2, prec=prec, renorm_trace=True)

    ref = s0.clone()
    run(ref)
    lbm.lb_sync_status(ctx)
    R = s0.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run(R)
    for _ in range(2):
        R.copy_(s0)
        g.replay()
        torch.cuda.synchronize()
        lbm.lb_sync_status(ctx)
        assert torch.equal(R, ref)
    exact = O.propagate_chain(Ps, w["states"], 2)
    err = np.max(np.linalg.norm(R.cpu().numpy() - exact, axis=1))
    assert err <= 1e-5, err
