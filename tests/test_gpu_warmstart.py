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
