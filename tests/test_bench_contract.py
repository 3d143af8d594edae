"""The bench's command-line contract (no GPU needed): with no flags it runs
one GPU with at least three warm-up steps, the reference arm is selectable,
and the reported metric is the one the workload is quoted on."""

import sys

import pytest


@pytest.fixture()
def bench(monkeypatch):
    import bench as b

    return b


def test_defaults(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "ours"
    assert a.trials is None and not a.headline_only


def test_reference_arm_and_flags(bench, monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "4",
                                      "--warmup", "3", "--trials", "t.jsonl"])
    a = bench.parse()
    assert (a.impl, a.gpus, a.steps, a.warmup, a.trials) == ("reference", 2, 4, 3, "t.jsonl")


def test_metric_names_the_workload(bench):
    assert "state-steps/s" in bench.METRIC and "d=27" in bench.METRIC
    assert bench.WORKLOAD == "d27_chain"


def test_headline_form_is_fp64(bench):
    """The recorded value is an FP64 form (FP64 operands and results, the
    dense products as exact slices on the tensor cores), the FP64-pipe form
    is reported beside it, and the reduced-precision forms under "mixed"."""
    assert bench.HEADLINE in bench.FORMS and bench.DTYPES[bench.HEADLINE] == "f64"
    assert bench.FORMS[bench.HEADLINE][:2] == ("fp64_sliced", "fp64_sliced")
    assert bench.FORMS[bench.FP64_NATIVE][:2] == ("fp64_hermitian", "fp64_hermitian")
    assert bench.DTYPES[bench.FP64_NATIVE] == "f64"
    for f in bench.MIXED_FORMS:
        assert f in bench.FORMS and bench.DTYPES[f] != "f64"
