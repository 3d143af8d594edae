"""What the trained warm-start network gains over plain GRAPE: on held-out
single-transmon gates (d = 3, 100 slices), GRAPE from the network's proposal
reaches average gate fidelity 0.999 in fewer iterations than from a random
start.  The network is trained by the library's own kernels on GRAPE
solutions the library generates (a reduced set: 32 problems)."""

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_warm_start_needs_fewer_grape_iterations():
    from paper_2603_18052_gb300 import _build, warmstart

    _build.build()
    res = warmstart.experiment(nq=1, n_train=32, n_test=4, max_iter=300, epochs=200, log=lambda *a: None)
    assert res["warm_reached"] >= res["random_reached"]
    assert res["median_warm_iters"] < res["median_random_iters"]


def test_batched_warm_start_d3_and_d9():
    """The batched pipeline at reduced scale, both sizes: GRAPE solutions
    generated with lb_grape_grad_batch (FP32 products at d = 9), one network
    for both sizes, then held-out problems from the network's proposal and
    from a random start to thresholds fixed beforehand (d = 3: F_avg 0.999;
    d = 9: 0.96, below the ceiling that one drive on transmon 0 reaches in
    10 ns against the exchange coupling)."""
    from paper_2603_18052_gb300 import _build, warmstart

    _build.build()
    res = warmstart.experiment_batched(n_train=(128, 64), n_test=8, max_iter=300, targets=(0.999, 0.96),
                                       batch=(128, 64), precs=("fp64", "fp32"), epochs=150, train_batch=32,
                                       log=lambda *a: None)
    for key in ("d3", "d9"):
        r = res["sizes"][key]
        assert r["dataset_reached"] >= 0.5 * r["n_train"], (key, r)
        assert r["warm_reached"] >= r["random_reached"], (key, r)
        assert r["median_warm_iters"] < r["median_random_iters"], (key, r)
