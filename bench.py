#!/usr/bin/env python
"""Throughput of the d = 27 propagator-build + propagation chain on GB300.

One step = one pass of the whole hot path over the d = 27 three-transmon
chain workload: assemble the base and drive Lindbladians (729 x 729), build
the 200 slice propagators by Pade-13 scaling and squaring with the FP64 LU
solve, and propagate 256 density matrices through the 200-slice chain (one
step per slice).  Five forms are timed:

  fp64_sliced     (headline) the real-coordinate form below with every dense
                  FP64 product (Pade products after A^2, the LU and solve
                  block products, the squarings, the propagation steps)
                  computed on the BF16 tensor cores through exact digit
                  slices (FP64 operands and results, error of the size of an
                  FP64 product's rounding)
  fp64_hermitian  all FP64 on the FP64 pipe, every product, the LU and the
                  solve on the real coordinates of Hermitian matrices (real
                  n x n matrices: one FMA per multiply-add instead of four)
  fp64            all FP64 on the complex superoperators, as the paper states
                  the method
  fp32_hermitian  real-coordinate build with FP32 Pade products and near-I
                  squarings, FP64 LU and solve; FP32 propagation
  bf16x3          split-BF16 on the tcgen05 tensor cores, FP64 LU and solve
  fp32            FP32 products and propagation, FP64 LU and solve

Prints ONE JSON line.  `value` is state-steps/s of the whole step in the
FP64 form (256 x 200 state-steps per step, builds included); `builds_per_s`
is propagator builds/s (200 per step); `mixed` holds the fastest
reduced-precision form with every mixed form's numbers and errors.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--headline-only] [--trials PATH]

Besides the headline, the line carries the arithmetic peaks measured by the
library's probes in this run, the roofline of the dominant kernel, each
form's propagation roofline and its accuracy against the oracle, the
end-to-end run with host buffers, the clocks seen during the timed region,
the CPU oracle baseline, and "other_workloads": the d = 3 and d = 9
configurations, a GRAPE landscape point, the mixed-size batch, the reuse of
P for nearby controls, the action of the exponential, the fixed-point step,
and the GPU timing models of the paper's Sec. 3.4.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "d27_chain"
METRIC = "state-steps/s and propagator builds/s at d=27, mixed-precision vs FP64, one GB300"
WORKLOAD_DESC = ("d=27 three-transmon chain: 200 control slices u~U(-0.1,0.1), 200 Pade-13 builds of "
                 "729x729 complex propagators (FP64 LU), B=256 Ginibre states propagated through the "
                 "200-slice chain, 1 step per slice")
SM_COUNT = 152
# fallbacks from unit counts, used only where a probe of this run failed
FP64_PEAK = SM_COUNT * 2 * 2 * 2.07e9   # 2 DFMA/clk/SM x 2 FLOP x 2.07 GHz max clock = 1.259 TFLOP/s
FP32_PEAK = SM_COUNT * 128 * 2 * 2.07e9  # 128 FFMA/clk/SM = 80.5 TFLOP/s
INT_MAC_PEAK = SM_COUNT * 64 * 2.07e9    # 32-bit integer multiply-add: 64 lanes/clk/SM = 20.1 T/s


def _measured_bf16_peak():
    try:
        return 1e12 * float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1.9e15  # fallback of the profiling recipe


BF16_PEAK = _measured_bf16_peak()
# form: (build precision, propagation precision, per-step trace renormalisation)
FORMS = {"fp64_sliced": ("fp64_sliced", "fp64_sliced", False),
         "fp64_hermitian": ("fp64_hermitian", "fp64_hermitian", False), "fp64": ("fp64", "fp64", False),
         "fp32_hermitian": ("fp32_hermitian", "fp32", True), "bf16x3": ("bf16x3", "bf16x3", True),
         "fp32": ("fp32", "fp32", True)}
HEADLINE = "fp64_sliced"
FP64_NATIVE = "fp64_hermitian"
OZ_KERNEL_VERSION = "persistent-320t-4stage-xo"  # the sliced-product kernel a traffic capture describes
MIXED_FORMS = ("fp32_hermitian", "bf16x3", "fp32")
DTYPES = {"fp64_sliced": "f64", "fp64_hermitian": "f64", "fp64": "f64", "fp32_hermitian": "f32+f64",
          "bf16x3": "bf16 split (x3 build, x5 propagation) + f64", "fp32": "f32+f64"}
PRECISION_DESC = {
    "fp64_sliced": "FP64 operands and results on the real coordinates; every dense product (A^4, A^6, A^6 Z1, "
                   "A^6 Z2, the LU and solve block products, the squarings, the propagation steps) as an exact "
                   "sliced product on the BF16 tensor cores: each row / column written as nine signed base-64 "
                   "digits against its power-of-two exponent, the 45 digit products of equal weight summed exactly "
                   "in FP32 in TMEM, combined in integer arithmetic and rounded once to FP64 (error <= "
                   "K 2^-54 13/4 of the row and column maxima, the size of an FP64 product's rounding); A^2 and "
                   "A W skip A's zeros in FP64; the 64 x 64 diagonal LU blocks and their inverses in FP64",
    "fp64_hermitian": "all FP64 on the real coordinates of Hermitian matrices (diagonal, Re and Im of the upper "
                      "triangle): the real form of each slice generator, Pade products, LU, solve and squarings "
                      "as real 729x729 FP64 matrices, P rebuilt from its real form; propagation on the states' "
                      "real coordinates; same result as the complex FP64 form to 1e-12",
    "fp64": "all FP64 on the complex superoperators",
    "fp32_hermitian": "real-coordinate build with FP32 Pade products (FP32 accumulation) and FP32 D-form "
                      "squarings, FP64 generator, norm, LU and solve; FP32 propagation (D = P - I, per-step trace "
                      "renormalisation)",
    "bf16x3": "split-BF16 on tcgen05 tensor cores with FP32 accumulation: Pade products as hi+lo pieces "
              "(3 products per real product), propagation with D = P - I in three pieces and states in two "
              "(5 products), FP32 states and per-step trace renormalisation; FP32 D-form squarings; FP64 norm, "
              "LU and solve",
    "fp32": "FP32 Pade products, FP32 D-form squarings and FP32 propagation (D = P - I, per-step trace "
            "renormalisation); FP64 norm, LU and solve",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline-only", action="store_true",
                    help="time only the split-BF16 form and print its launch count per step (for a "
                         "profiler's launch list); no other forms, end-to-end run or side workloads")
    ap.add_argument("--trials", default=None, metavar="PATH",
                    help="also write the raw timings (every timed step of each form, every trial of the "
                         "GPU timing models) to PATH as JSON lines")
    ap.add_argument("--form", default=None, choices=sorted(FORMS),
                    help="with --headline-only: the form to time (default: the headline form)")
    ap.add_argument("--instances", type=int, default=4096,
                    help="instances of the mixed-size batch (default: the whole 4096 of the workload)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the tile autotuner (profiler runs: its launches would precede the step)")
    ap.add_argument("--profile-size", action="store_true",
                    help="with --headline-only: the d = 27 chain cut to 8 slices and 16 states (a few GB on the "
                         "device), for profiler captures of single launches")
    return ap.parse_args()


def dist_env():
    from paper_2603_18052_gb300 import ranks

    return ranks.dist_env()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower() in ("active", "0x1") or r[key].startswith("Active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(rows), "power_w_max": max(r["power"] for r in rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------- reference arm --

def oracle_sample(w, nslices):
    """The FP64 oracle on the first ``nslices`` slices: build each propagator
    and propagate all B states through them.  Returns seconds."""
    import numpy as np

    import oracle as O

    t0 = time.perf_counter()
    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    Ps = O.slice_propagators(Lb, Ld, w["u"][:nslices], w["dt"])
    R = O.propagate_chain(Ps, w["states"], 1)
    t1 = time.perf_counter()
    assert np.isfinite(R).all()
    return t1 - t0


def oracle_single_thread(nslices=1):
    """The same oracle sample in a child process whose BLAS and OpenMP pools
    have one thread (their size is fixed when numpy loads).  Seconds, or None
    if the child fails."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1")
    code = ("import json, bench; from workloads import make_workload; "
            "print(json.dumps(bench.oracle_sample(make_workload(bench.WORKLOAD), %d)))" % nslices)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                           timeout=900)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def cpu_baseline(w, nslices):
    t = oracle_sample(w, nslices)
    B = w["B"]
    out = {"value": B * nslices / t, "unit": "state-steps/s", "builds_per_s": nslices / t, "cores": host_cores(),
           "kind": "oracle",
           "sample": "%d of the 200 slices: %d Pade-13 builds (729x729, numpy FP64 with its BLAS threads) and "
                     "%d states x %d steps, %.1f s" % (nslices, nslices, B, nslices, t)}
    t1 = oracle_single_thread(1)
    if t1 is not None:
        out["single_thread"] = {"value": B / t1, "unit": "state-steps/s", "builds_per_s": 1.0 / t1, "cores": 1,
                                "sample": "1 slice (one build and 256 state-steps), one BLAS / OpenMP thread, "
                                          "%.1f s" % t1}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from workloads import make_workload

    w = make_workload(WORKLOAD)
    per_step = 2
    for _ in range(args.warmup):
        oracle_sample(w, per_step)
    ts = [oracle_sample(w, per_step) for _ in range(args.steps)]
    t = sum(ts) / len(ts)
    v = w["B"] * per_step / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "state-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "arithmetic": "FP64 inputs and results; the dense FP64 products run on the BF16 tensor cores as exact "
                      "digit slices (Ozaki scheme) with FP64-size rounding error; the FP64-pipe form is under "
                      "fp64_native",
            "builds_per_s": per_step / t,
            "config": {"workload": WORKLOAD_DESC,
                       "sample_per_step": "%d of the 200 slices per step (%d Pade builds + 256 states x %d steps); the "
                                          "rate is per state-step and per build, so a full 200-slice step would take "
                                          "%d times as long (linear extrapolation, not run)" % (per_step, per_step,
                                                                                                per_step,
                                                                                                200 // per_step)},
            "cpu_baseline": {"value": v, "unit": "state-steps/s", "cores": host_cores(), "kind": "oracle",
                             "sample": "%d slices per step of the d=27 chain, FP64 numpy oracle" % per_step},
            "e2e": {"value": v, "unit": "state-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ours ---

def mixed_instances(lb, ctx_big, dev, stream, count, trials):
    """The mixed-size batch (d = 3 / 9 / 27 in ratio 8:4:1, 50 slices and
    1..64 states each, `count` instances): every instance in one CUDA graph
    (lb_run_instances for the d <= 9 instances on a context sized for large
    chunks, then for the d = 27 instances on the chain's context, both with a
    fixed squaring bound so that nothing waits on the host), replayed
    `trials` times in the fastest mixed form; then the FP64 forms against
    per-instance FP64 launches (lb_expm_pade + lb_propagate_batch per
    instance), each on a stated sample, extrapolated by instance counts."""
    import collections

    import numpy as np
    import torch

    from paper_2603_18052_gb300 import ranks
    from workloads.configs import make_instances

    inst, models = make_instances(count)
    rank, world, _ = ranks.dist_env()
    if world > 1:  # this rank's share of the independent problems
        costs = [ranks.instance_cost(x["d"], len(x["u"]), x["states"].shape[0]) for x in inst]
        inst = [inst[i] for i in ranks.partition(costs, world)[rank]]

    def dput(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    ctx_small = lb.Context(dev.index or 0, max_n=81, max_batch=64, max_slices=4096)
    for c in (ctx_small, ctx_big):
        lb.lb_set_max_squarings(c, 2)
    gens = {}
    for q, m in models.items():
        n = m.d * m.d
        Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
        Ld = torch.empty_like(Lb)
        lb.lb_assemble(ctx_big, dput(m.H0), dput(m.jumps), Lb)
        lb.lb_assemble(ctx_big, dput(m.X), None, Ld)
        gens[q] = (Lb, Ld)
    dt = models[1].dt
    us = [dput(x["u"]) for x in inst]
    s0 = [dput(x["states"]) for x in inst]
    st = [x.clone() for x in s0]
    arg = [dict(Lbase=gens[x["nq"]][0], Ldrv=gens[x["nq"]][1], u=us[i], states=st[i]) for i, x in enumerate(inst)]
    small = [i for i, x in enumerate(inst) if x["d"] <= 9]
    big = [i for i, x in enumerate(inst) if x["d"] > 9]
    counts = collections.Counter(x["d"] for x in inst)

    def reset(idx):
        for i in idx:
            st[i].copy_(s0[i])

    def ev_ms(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    def run_all(prec, idx_small, idx_big):
        renorm = prec not in ("fp64", "fp64_hermitian", "fp64_sliced")
        if idx_small:
            lb.lb_run_instances(ctx_small, [arg[i] for i in idx_small], dt, prec=prec, renorm_trace=renorm)
        if idx_big:
            lb.lb_run_instances(ctx_big, [arg[i] for i in idx_big], dt, prec=prec, renorm_trace=renorm)

    builds = sum(len(x["u"]) for x in inst)
    ssteps = sum(len(x["u"]) * x["states"].shape[0] for x in inst)
    res = {"workload": "%d instances (d=3/9/27: %d/%d/%d), 50 slices each, B~U{1..64}; %d builds, %d state-steps"
                       % (len(inst), counts[3], counts[9], counts[27], builds, ssteps)
                       + ("" if world == 1 else " (this rank's share of %d, split by cost)" % count)}

    # the whole batch in one captured graph, in the fastest form (FP64 via
    # exact slices)
    form = "fp64_sliced"
    reset(range(len(inst)))
    run_all(form, small, big)  # warm-up (tables, kernels)
    torch.cuda.synchronize()
    lb.lb_sync_status(ctx_small)
    lb.lb_sync_status(ctx_big)
    g = torch.cuda.CUDAGraph()
    n0 = lb.lb_launch_count()
    with torch.cuda.graph(g):
        run_all(form, small, big)
    launches = lb.lb_launch_count() - n0
    ts = []
    for _ in range(max(1, trials)):
        reset(range(len(inst)))
        ts.append(ev_ms(g.replay))
    lb.lb_sync_status(ctx_small)
    lb.lb_sync_status(ctx_big)
    ms = statistics.median(ts)
    res["captured_" + form] = {"captured": True, "ms": ms, "trial_ms": ts, "builds_per_s": builds / (ms / 1e3),
                               "state_steps_per_s": ssteps / (ms / 1e3),
                               "kernel_nodes": launches,
                               "note": "one CUDA graph holding lb_run_instances for the d<=9 instances (context "
                                       "with 4096-slice chunks) and for the d=27 instances (200-slice chunks); "
                                       "median of the replays"}
    del g
    for c in (ctx_small, ctx_big):  # the FP64 arms run uncaptured, as a caller would
        lb.lb_set_max_squarings(c, -1)

    # FP64: batched (lb_run_instances) against per-instance launches, per
    # d class on a stated sample, extrapolated by the class's instance count
    samp = {3: 64, 9: 32, 27: 2}
    by_d = collections.defaultdict(list)
    for i, x in enumerate(inst):
        by_d[x["d"]].append(i)

    def per_instance(idx, prec):
        for i in idx:
            x = inst[i]
            S = len(x["u"])
            n = x["d"] * x["d"]
            ctx = ctx_small if n <= 81 else ctx_big
            P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
            lb.lb_expm_pade(ctx, arg[i]["Lbase"], arg[i]["Ldrv"], us[i], dt, P, prec=prec)
            lb.lb_propagate_batch(ctx, P, st[i], steps_per_slice=1, prec=prec)

    fp = {}
    for prec in ("fp64_sliced", "fp64_hermitian", "fp64"):
        tot_batched, tot_loop, classes = 0.0, 0.0, {}
        for d, idx in sorted(by_d.items()):
            k = min(samp[d], len(idx))
            sample = idx[:k]
            scale = len(idx) / k
            # batched: the whole class for d <= 9 (cheap), the sample at d = 27
            bidx = idx if d <= 9 else sample
            bscale = 1.0 if d <= 9 else scale
            reset(bidx)
            run_all(prec, bidx if d <= 9 else [], [] if d <= 9 else bidx)  # warm-up
            tb = []
            for _ in range(3):
                reset(bidx)
                tb.append(ev_ms(lambda: run_all(prec, bidx if d <= 9 else [], [] if d <= 9 else bidx)))
            tb = statistics.median(tb) * bscale
            reset(sample)
            per_instance(sample[:1], prec)  # warm-up
            reset(sample)
            t0 = time.perf_counter()
            per_instance(sample, prec)
            torch.cuda.synchronize()
            tl = (time.perf_counter() - t0) * 1e3 * scale
            classes["d%d" % d] = {"instances": len(idx), "batched_ms": tb, "per_instance_ms": tl,
                                  "speedup": tl / tb,
                                  "sample": ("all %d" % len(idx) if d <= 9 else "%d of %d, x%.1f" % (k, len(idx), scale))
                                  + " batched; %d of %d per instance, x%.1f" % (k, len(idx), scale)}
            tot_batched += tb
            tot_loop += tl
        fp[prec] = {"batched_ms": tot_batched, "per_instance_ms": tot_loop, "speedup": tot_loop / tot_batched,
                    "classes": classes}
    lb.lb_sync_status(ctx_small)
    lb.lb_sync_status(ctx_big)
    res["fp64_forms"] = fp
    res["speedup_fp64_hermitian_batched_vs_per_instance_fp64"] = (fp["fp64"]["per_instance_ms"]
                                                                 / fp["fp64_hermitian"]["batched_ms"])
    res["speedup_fp64_sliced_batched_vs_per_instance_fp64"] = (fp["fp64"]["per_instance_ms"]
                                                              / fp["fp64_sliced"]["batched_ms"])
    res["speedup_captured_%s_vs_per_instance_fp64" % form] = fp["fp64"]["per_instance_ms"] / ms
    res["note"] = ("per-instance arms: one lb_expm_pade + lb_propagate_batch call pair per instance through the "
                   "Python binding, timed with the host clock on a sample per d class and scaled by the class's "
                   "instance count; batched FP64 at d=27 likewise on a sample (every d=27 build is LU-bound, "
                   "so its time is linear in the count)")
    ctx_small.close()
    return res


def other_workloads(lb, accounting, dev, stream, reps=5, fp64_peak=None, fp32_peak=None, bf16_peak=None):
    """Secondary measurements on the smaller workloads: the d = 3 single-state
    chain (latency per step), the d = 9 batch (FP64 and FP32 throughput), and
    one d = 9 GRAPE landscape point (100 slices, 4 basis operators)."""
    import numpy as np
    import torch

    from workloads import make_workload, transmon_chain

    def dput(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def time_ms(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {}
    ctx = lb.Context(dev.index or 0, max_n=81, max_batch=1024, max_slices=100)

    def props(w):
        n = w["n"]
        Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
        Ld = torch.empty_like(Lb)
        lb.lb_assemble(ctx, dput(w["H0"]), dput(w["jumps"]), Lb)
        lb.lb_assemble(ctx, dput(w["X"]), None, Ld)
        P = torch.empty((w["nslices"], n, n), dtype=torch.complex128, device=dev)
        lb.lb_expm_pade(ctx, Lb, Ld, dput(w["u"]), w["dt"], P)
        return Lb, Ld, P

    # d = 3, one state, 10^4 steps, FP64 (Algorithm 2 latency)
    w = make_workload("d3_single")
    _, _, P = props(w)
    R = dput(w["states"])
    N = w["steps_per_slice"]
    ms = time_ms(lambda: lb.lb_propagate_batch(ctx, P, R, steps_per_slice=N))
    out["d3_single"] = {"workload": "d=3, 1 state, 10^4 chained FP64 steps", "ns_per_step": 1e6 * ms / N,
                        "state_steps_per_s": N / (ms / 1e3), "paper_context_ns_per_step": 309.5}
    # the same chain on the density matrix's 9 real coordinates (FP64)
    R = dput(w["states"])
    ms = time_ms(lambda: lb.lb_propagate_batch(ctx, P, R, steps_per_slice=N, prec="fp64_hermitian"))
    out["d3_single_hermitian"] = {"workload": "d=3, 1 state, 10^4 chained FP64 steps on the real coordinates "
                                              "of the density matrix (lb_propagate_batch, fp64_hermitian)",
                                  "ns_per_step": 1e6 * ms / N, "state_steps_per_s": N / (ms / 1e3),
                                  "paper_context_ns_per_step": 309.5}
    # d = 9, 1024 states, 1000 steps
    w = make_workload("d9_batch")
    _, _, P = props(w)
    N, B, n = w["steps_per_slice"], w["B"], w["n"]
    for prec, renorm in (("fp64", False), ("fp32", True), ("bf16x3", True), ("fp64_hermitian", False)):
        R = dput(w["states"])
        ms = time_ms(lambda: lb.lb_propagate_batch(ctx, P, R, steps_per_slice=N, prec=prec, renorm_trace=renorm))
        # the Hermitian form does n^2 real multiply-adds per state-step
        per = 2.0 * n * n if prec == "fp64_hermitian" else accounting.state_step_flops(n)
        fl = B * N * per / (ms / 1e3)
        p64, p32, p16 = fp64_peak or FP64_PEAK, fp32_peak or FP32_PEAK, bf16_peak or BF16_PEAK
        peak = {"fp64": p64, "fp32": p32, "bf16x3": p16 / 5, "fp64_hermitian": p64}[prec]
        out["d9_batch_" + prec] = {"workload": "d=9, 1024 states, 1000 steps, %s" % prec, "ms": ms,
                                   "state_steps_per_s": B * N / (ms / 1e3),
                                   "roofline": {"bound": "tensor" if prec == "bf16x3" else "alu",
                                                "achieved": fl / 1e12, "peak": peak / 1e12,
                                                "unit": "TFLOP/s", "frac": fl / peak}}
    # one GRAPE landscape point at d = 9
    m = transmon_chain(2)
    S, Bg, n = 100, 4, 81
    wl = {"H0": m.H0, "jumps": m.jumps, "X": m.X, "u": 0.05 * np.sin(np.arange(S) * 0.3), "dt": m.dt,
          "nslices": S, "n": n}
    Lb, Ld, _ = props(wl)
    X0 = np.zeros((Bg, n), dtype=complex)
    for b, (i, j) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        X0[b, i * 9 + j] = 1.0
    X0d = dput(X0)
    Fo = torch.zeros(1, dtype=torch.float64, device=dev)
    go = torch.zeros(S, dtype=torch.float64, device=dev)
    ud = dput(wl["u"])
    ms = time_ms(lambda: lb.lb_grape_grad(ctx, Lb, Ld, ud, m.dt, 1, X0d, X0d, Fo, go))
    out["d9_grape"] = {"workload": "d=9 GRAPE landscape point: 100 slices, 100 Pade builds + Frechet "
                                   "derivatives, forward/adjoint chains of 4 basis operators", "ms": ms}
    ctx.close()
    out["paper_model_build_breakdown"] = paper_model_breakdown(lb, dev)
    out["control_reuse_d9"] = control_reuse(lb, dev, time_ms)
    out["fixed_point"] = fixed_point(lb, dev, stream)
    out["action_of_exponential_d27"] = action_of_exponential(lb, dev, stream, fp64_peak=fp64_peak)
    out["gpu_timing_models"] = gpu_timing_models(lb, dev, stream)
    return out


def action_of_exponential(lb, dev, stream, S=10, fp64_peak=None):
    """The d = 27 chain's first S slices without dense propagators
    (lb_expmv: truncated Taylor series, FP64, no LU) against the dense route
    (Pade build of the S propagators, then the chain) in FP64 and in the
    split-BF16 form, for B = 1, 8, 64 states.  The Taylor products count
    8 n^2 B FLOPs each."""
    import numpy as np
    import torch

    from workloads import make_workload

    out = {}
    w = make_workload("d27_chain", B=64, nslices=S)
    n = w["n"]
    ctx = lb.Context(dev.index or 0, max_n=n, max_batch=64, max_slices=S)
    Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
    Ld = torch.empty_like(Lb)
    lb.lb_assemble(ctx, torch.from_numpy(w["H0"]).to(dev), torch.from_numpy(w["jumps"]).to(dev), Lb)
    lb.lb_assemble(ctx, torch.from_numpy(w["X"]).to(dev), None, Ld)
    u = torch.from_numpy(np.ascontiguousarray(w["u"][:S])).to(dev)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    for B in (1, 8, 64):
        X = torch.from_numpy(np.ascontiguousarray(w["states"][:B])).to(dev)
        ms_pair = [None]

        def taylor():
            ms_pair[0] = lb.lb_expmv(ctx, Lb, Ld, u, w["dt"], X)

        def dense():
            lb.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P)
            lb.lb_propagate_batch(ctx, P, X, 1, "fp64")

        def dense_mixed():
            lb.lb_expm_pade(ctx, Lb, Ld, u, w["dt"], P, prec="bf16x3")
            lb.lb_propagate_batch(ctx, P, X, 1, "bf16x3")

        t_taylor = timed(taylor)
        t_dense = timed(dense)
        t_mixed = timed(dense_mixed)
        t_herm = timed(lambda: lb.lb_expmv(ctx, Lb, Ld, u, w["dt"], X, hermitian=True)) if B <= 8 else None
        m, s = ms_pair[0]
        fl = S * s * m * 8.0 * n * n * B
        out["B%d" % B] = {"taylor_ms_per_slice": t_taylor / S, "dense_fp64_ms_per_slice": t_dense / S,
                          "dense_bf16x3_ms_per_slice": t_mixed / S,
                          "speedup_vs_dense_fp64": t_dense / t_taylor, "speedup_vs_dense_bf16x3": t_mixed / t_taylor,
                          "taylor_hermitian_ms_per_slice": t_herm / S if t_herm else None,
                          "m": m, "s": s,
                          "taylor_roofline": {"bound": "alu", "achieved": fl / (t_taylor / 1e3) / 1e12,
                                              "peak": (fp64_peak or FP64_PEAK) / 1e12, "unit": "TFLOP/s",
                                              "frac": fl / (t_taylor / 1e3) / (fp64_peak or FP64_PEAK)}}
    lb.lb_sync_status(ctx)
    ctx.close()
    return out


def fixed_point(lb, dev, stream):
    """The Q1.15 fixed-point step of Algorithm alg:fpga on the GPU: the d = 3
    single-state chain (per-step latency and its spread, beside the board's
    94 cycles at 108 MHz) and batched throughput at d = 3 and d = 9, counted
    in exact integer products (4 n^2 per state-step) against the 32-bit
    integer multiply-add rate."""
    import numpy as np
    import torch

    from paper_2603_18052_gb300 import timing
    from workloads import transmon_chain

    def ev_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    out = {}
    ctx = lb.Context(dev.index or 0, max_n=81, max_batch=8, max_slices=1)
    for nq, B, N in ((1, 1, 10000), (1, 1 << 17, 1000), (2, 1 << 14, 200)):
        m = transmon_chain(nq)
        n = m.d * m.d
        Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
        Ld = torch.empty_like(Lb)
        lb.lb_assemble(ctx, torch.from_numpy(m.H0).to(dev), torch.from_numpy(m.jumps).to(dev), Lb)
        lb.lb_assemble(ctx, torch.from_numpy(m.X).to(dev), None, Ld)
        P = torch.empty((1, n, n), dtype=torch.complex128, device=dev)
        lb.lb_expm_pade(ctx, Lb, Ld, torch.tensor([0.05], dtype=torch.float64, device=dev), m.dt, P)
        Pq = torch.empty((n, n, 2), dtype=torch.int16, device=dev)
        lb.lb_fixed_quantize(P[0], Pq, 15)
        x0 = np.zeros((B, n), dtype=np.complex128)
        x0[:, 0] = 1.0
        X = torch.empty((B, n, 2), dtype=torch.int16, device=dev)
        lb.lb_fixed_quantize(torch.from_numpy(x0).to(dev), X, 15)
        ts = ev_ms(lambda: lb.lb_propagate_fixed(Pq, X, N, 15))
        ms = statistics.median(ts)
        key = "d%d_q115_%s" % (m.d, "single" if B == 1 else "batch")
        r = {"workload": "d=%d, %d state%s, %d chained Q1.15 steps" % (m.d, B, "" if B == 1 else "s", N),
             "ms": ms, "state_steps_per_s": B * N / (ms / 1e3)}
        if B == 1:
            r["ns_per_step"] = 1e6 * ms / N
            r["ns_per_step_min_max"] = [1e6 * min(ts) / N, 1e6 * max(ts) / N]
            r["fpga_ns_per_step"] = 1e9 * (timing.fpga_cycles(n, 1, N) - 1) / N / 108e6
        else:
            macs = 4.0 * n * n * B * N / (ms / 1e3)
            r["roofline"] = {"bound": "alu", "achieved": macs / 1e12, "peak": INT_MAC_PEAK / 1e12,
                             "unit": "T int-MAC/s", "frac": macs / INT_MAC_PEAK}
        out[key] = r
    lb.lb_sync_status(ctx)
    ctx.close()
    return out


def gpu_timing_models(lb, dev, stream):
    """The three GPU timing models of Sec. 3.4 (Eq. 7-9) on this GPU, as in
    Table tab:cost_model_gpu: the device probes of Table tab:probes_gpu
    (launch, launch + sync, copy latency and pageable H2D / D2H rates, stream
    and stride-n gather reads of 8.3 MB and 64 MiB), then for d = 3, 9, 27
    and b = 1, 8, 32, 128 the idealized cost from those probes beside the
    measured median of five trials of 50 one-step calls: kernel-only with
    CUDA events (lb_propagate_batch), resident-P and host-visible with the
    host clock around the whole call (lb_propagate_resident,
    lb_propagate_host; the ctypes call is inside the timed region)."""
    import numpy as np
    import torch

    from paper_2603_18052_gb300 import timing
    from workloads import transmon_chain

    med = statistics.median
    launch = med(lb.lb_probe_launch(1000, False) for _ in range(5))
    launch_sync = med(lb.lb_probe_launch(200, True) for _ in range(5))

    def copy_us(nbytes, to_dev, reps):
        h = torch.zeros(nbytes // 8, dtype=torch.float64)  # pageable host memory
        d = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
        return med(lb.lb_probe_copy(h, d, to_dev, reps) for _ in range(5))

    big = 64 << 20
    lat_h2d, lat_d2h = copy_us(16, True, 200), copy_us(16, False, 200)
    h2d = big / (1e3 * (copy_us(big, True, 5) - lat_h2d))
    d2h = big / (1e3 * (copy_us(big, False, 5) - lat_d2h))

    def read_gbs(nbytes, n):
        count = nbytes // 16
        buf = torch.ones(count, dtype=torch.complex128, device=dev)
        sink = torch.zeros(1, dtype=torch.int64, device=dev)
        read = 16 * (count if n == 0 else (count // n) * n)
        ts = []
        lb.lb_probe_read(buf, n, sink)
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(20):
                lb.lb_probe_read(buf, n, sink)
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b) / 20)
        return read / (med(ts) * 1e6)

    ws27 = 16 * (729 * 729 + 2 * 729)  # the d = 27 working set, "8.3 MB"
    reads = {"stream_8p3MB": read_gbs(ws27, 0), "gather_8p3MB": read_gbs(ws27, 729),
             "stream_64MiB": read_gbs(big, 0), "gather_64MiB": read_gbs(big, 729)}
    probes = timing.Probes(launch_us=launch, launch_sync_us=launch_sync, lat_h2d_us=lat_h2d, lat_d2h_us=lat_d2h,
                           h2d_gbs=h2d, d2h_gbs=d2h, stream_gbs=max(reads["stream_8p3MB"], reads["stream_64MiB"]),
                           alloc_calls=4, alloc_us_each=3.0)
    # the allocation term measured (a cudaMalloc + cudaFree pair of the d = 27
    # propagator's size), beside the paper's stated 3 us per call
    alloc_pair_us = med(lb.lb_probe_alloc(16 * 729 * 729, 10) for _ in range(5))
    probes_measured_alloc = timing.Probes(**{**probes.__dict__, "alloc_calls": 2, "alloc_us_each": alloc_pair_us})
    out = {"probes": {"launch_us": launch, "launch_sync_us": launch_sync, "copy_latency_h2d_us": lat_h2d,
                      "copy_latency_d2h_us": lat_d2h, "h2d_gbs": h2d, "d2h_gbs": d2h, **{k + "_gbs": v for k, v in reads.items()},
                      "alloc": "4 calls (2 cudaMalloc + 2 cudaFree) at the paper's stated 3 us each",
                      "alloc_pair_measured_us": alloc_pair_us},
           "rows": []}
    ctx = lb.Context(dev.index or 0, max_n=729, max_batch=128, max_slices=1)
    for nq in (1, 2, 3):
        m = transmon_chain(nq)
        n = m.d * m.d
        Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
        Ld = torch.empty_like(Lb)
        lb.lb_assemble(ctx, torch.from_numpy(m.H0).to(dev), torch.from_numpy(m.jumps).to(dev), Lb)
        lb.lb_assemble(ctx, torch.from_numpy(m.X).to(dev), None, Ld)
        P = torch.empty((1, n, n), dtype=torch.complex128, device=dev)
        lb.lb_expm_pade(ctx, Lb, Ld, torch.tensor([0.05], dtype=torch.float64, device=dev), m.dt, P)
        P_host = P[0].cpu().contiguous()
        for b in (1, 8, 32, 128):
            x0 = np.zeros((b, n), dtype=np.complex128)
            x0[:, 0] = 1.0
            Xd = torch.from_numpy(x0).to(dev)
            Xh = torch.from_numpy(x0.copy())
            reps = 50

            def kernel_trial():
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(reps):
                    lb.lb_propagate_batch(ctx, P, Xd, 1, "fp64")
                e.record(stream)
                e.synchronize()
                return a.elapsed_time(e) * 1e6 / reps / b

            def host_trial(fn):
                t0 = time.perf_counter_ns()
                for _ in range(reps):
                    fn()
                return (time.perf_counter_ns() - t0) / reps / b

            meas, trials = {}, {}
            for name, trial in (("kernel", kernel_trial),
                                ("resident", lambda: host_trial(lambda: lb.lb_propagate_resident(ctx, P[0], Xh))),
                                ("host", lambda: host_trial(lambda: lb.lb_propagate_host(ctx, P_host, Xh)))):
                trial()  # warm-up: one untimed trial of 50 calls
                trials[name] = [trial() for _ in range(5)]
                meas[name] = med(trials[name])
            row = {"d": m.d, "batch": b}
            for name, f in timing.MODELS:
                ideal = f(n, b, probes)
                row[name] = {"idealized_ns": ideal, "measured_ns": meas[name], "ratio": meas[name] / ideal,
                             "trials_ns": trials[name]}
            ideal = timing.cost_host(n, b, probes_measured_alloc)
            row["host"]["idealized_measured_alloc_ns"] = ideal
            row["host"]["ratio_measured_alloc"] = meas["host"] / ideal
            out["rows"].append(row)
    lb.lb_sync_status(ctx)
    ctx.close()
    return out


def control_reuse(lb, dev, time_ms):
    """Reuse of slice propagators for nearby controls (the paper's discussion
    recommends it for GRAPE line searches): P and dP/du for 100 slices at
    d = 9 once (lb_expm_frechet), then P(u + delta) ~ P + delta dP
    (lb_control_update) against a full FP64 rebuild at u + delta."""
    import numpy as np
    import torch

    from workloads import transmon_chain

    m = transmon_chain(2)
    n, S = 81, 100
    ctx = lb.Context(dev.index or 0, max_n=n, max_batch=4, max_slices=S)

    def dput(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
    Ld = torch.empty_like(Lb)
    lb.lb_assemble(ctx, dput(m.H0), dput(m.jumps), Lb)
    lb.lb_assemble(ctx, dput(m.X), None, Ld)
    u0 = 0.05 * np.sin(0.3 * np.arange(S))
    delta = 1e-3
    u, du = dput(u0), dput(np.full(S, delta))
    u1 = dput(u0 + delta)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
    dP, Pn, Pr = torch.empty_like(P), torch.empty_like(P), torch.empty_like(P)
    t_fre = time_ms(lambda: lb.lb_expm_frechet(ctx, Lb, Ld, u, m.dt, P, dP))
    t_upd = time_ms(lambda: lb.lb_control_update(P, dP, du, Pn))
    t_reb = time_ms(lambda: lb.lb_expm_pade(ctx, Lb, Ld, u1, m.dt, Pr))
    lb.lb_sync_status(ctx)
    err = float(torch.max(torch.linalg.matrix_norm(Pn - Pr) / torch.linalg.matrix_norm(Pr)))
    ctx.close()
    return {"workload": "d=9, 100 slices: P and dP/du once, then propagators for u + 1e-3 by the first-order "
                        "update vs an FP64 rebuild",
            "frechet_build_ms": t_fre, "update_ms": t_upd, "rebuild_ms": t_reb,
            "update_speedup": t_reb / t_upd, "update_rel_error": err}


def paper_model_breakdown(lb, dev):
    """Build-time split of the paper's GRAPE landscape-point model (H0 =
    diag(0..d-1), drive a + a^+, T1 = 50, T2 = 30, dt = 0.5; 3 / 5 / 6
    squarings per segment at d = 3 / 9 / 27) in the terms of its build
    breakdown table: solve, Pade products, squarings, other (norm, scaling,
    checks), per build, for the FP64 and split-BF16 forms."""
    import numpy as np
    import torch

    from workloads.transmon import paper_grape_model

    def dput(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    res = {}
    for d, S in ((3, 100), (9, 100), (27, 20)):
        m = paper_grape_model(d)
        n = d * d
        ctx = lb.Context(dev.index or 0, max_n=n, max_batch=1, max_slices=S)
        Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
        Ld = torch.empty_like(Lb)
        lb.lb_assemble(ctx, dput(m.H0), dput(m.jumps), Lb)
        lb.lb_assemble(ctx, dput(m.X), None, Ld)
        u = dput(0.1 * np.sin(0.3 * np.arange(S)))
        P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)
        s_out = torch.empty(S, dtype=torch.int32, device=dev)
        entry = {}
        for prec in ("fp64", "bf16x3"):
            lb.lb_expm_pade(ctx, Lb, Ld, u, m.dt, P, prec=prec, s_out=s_out)  # warm-up
            lb.lb_sync_status(ctx)
            reps = 3
            lb.lb_set_stage_timing(ctx, True)
            for _ in range(reps):
                lb.lb_expm_pade(ctx, Lb, Ld, u, m.dt, P, prec=prec, s_out=s_out)
            lb.lb_sync_status(ctx)
            st, _ = lb.lb_stage_times(ctx)
            lb.lb_set_stage_timing(ctx, False)
            per = {k: v / (reps * S) for k, v in st.items()}  # ms per build
            tot = sum(per.values())
            entry[prec] = {"build_ms": tot,
                           "solve_pct": 100 * per["lu_solve"] / tot,
                           "pade_products_pct": 100 * per["pade_products"] / tot,
                           "squarings_pct": 100 * per["squarings"] / tot,
                           "other_pct": 100 * (per["prepare"] + per["check"]) / tot}
        entry["s_per_segment"] = sorted(set(int(x) for x in s_out.cpu().numpy()))
        entry["builds"] = S
        res["d%d" % d] = entry
        ctx.close()
    return res

def measure_peaks(lb):
    """The arithmetic ceilings of this GPU, measured by the library's probes
    in this run (TFLOP/s; None where a probe failed)."""
    out = {}
    for key, fn in (("dfma", lb.lb_probe_dfma), ("ffma", lb.lb_probe_ffma), ("dmma", lb.lb_probe_dmma),
                    ("bf16_tc", lb.lb_probe_bf16_tc)):
        try:
            out[key] = fn()
        except lb.LBError as e:
            out[key] = None
            out[key + "_error"] = e.name
    return out


def form_errors(lb, ctx, w, dev, forms, run_form):
    """Accuracy of each form in this run: two sampled propagators against the
    oracle's Pade build and two sampled final states against the oracle's
    Taylor route through all 200 slices (no dense propagator needed)."""
    import numpy as np

    import oracle as O
    from oracle import expmv as E

    Lb = O.lindbladian(w["H0"], w["jumps"])
    Ld = O.drive_generator(w["X"])
    sl, st = (0, w["nslices"] - 1), (0, w["B"] - 1)
    P_ref = {s: O.expm_pade13(O.slice_generator(Lb, Ld, w["u"][s]) * w["dt"]) for s in sl}
    X_ref, _ = E.expmv_chain(Lb, Ld, w["u"], w["dt"], w["states"][list(st)])
    out = {}
    for f in forms:
        P, R, s_out = run_form(f)
        eP = max(float(np.linalg.norm(P[s].cpu().numpy() - P_ref[s]) / np.linalg.norm(P_ref[s])) for s in sl)
        Rg = R.cpu().numpy()
        eX = max(float(np.linalg.norm(Rg[q] - X_ref[k])) for k, q in enumerate(st))
        out[f] = {"propagator_rel_frobenius": eP, "state_abs_frobenius_after_200_steps": eX,
                  "sampled": "propagators of slices %d and %d vs the oracle's Pade build; final states %d and %d vs "
                             "the oracle's Taylor route through the 200 slices" % (sl + st),
                  "squarings": sorted(set(int(x) for x in s_out))}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2603_18052_gb300 import _build, accounting, lb
    from workloads import make_workload

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    w = make_workload(WORKLOAD, **({"nslices": 8, "B": 16} if args.profile_size else {}))
    n, S, B, dt = w["n"], w["nslices"], w["B"], w["dt"]
    ctx = lb.Context(local, max_n=n, max_batch=B, max_slices=S)
    stream = torch.cuda.current_stream()
    peaks = measure_peaks(lb) if not args.headline_only else {}
    fp64_peak = 1e12 * peaks["dfma"] if peaks.get("dfma") else FP64_PEAK
    fp32_peak = 1e12 * peaks["ffma"] if peaks.get("ffma") else FP32_PEAK
    bf16_peak = 1e12 * peaks["bf16_tc"] if peaks.get("bf16_tc") else BF16_PEAK
    peak_src = {"fp64": "lb_probe_dfma, this run" if peaks.get("dfma") else "derived from unit counts",
                "fp32": "lb_probe_ffma, this run" if peaks.get("ffma") else "derived from unit counts",
                "bf16": "lb_probe_bf16_tc, this run" if peaks.get("bf16_tc") else "MEASURED_PEAKS.json bf16_tflops"}

    def dput(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    H0, Ls, X, u = dput(w["H0"]), dput(w["jumps"]), dput(w["X"]), dput(w["u"])
    R = dput(w["states"])
    Lb = torch.empty((n, n), dtype=torch.complex128, device=dev)
    Ld = torch.empty_like(Lb)
    P = torch.empty((S, n, n), dtype=torch.complex128, device=dev)

    def step(form, ev=None, H0=H0, Ls=Ls, X=X, u=u, R=R, s_out=None):
        pb, pp, renorm = FORMS[form]
        if ev is not None:
            ev[0].record(stream)
        lb.lb_assemble(ctx, H0, Ls, Lb)
        lb.lb_assemble(ctx, X, None, Ld)
        if ev is not None:
            ev[1].record(stream)
        lb.lb_expm_pade(ctx, Lb, Ld, u, dt, P, prec=pb, s_out=s_out)
        if ev is not None:
            ev[2].record(stream)
        lb.lb_propagate_batch(ctx, P, R, steps_per_slice=1, prec=pp, renorm_trace=renorm)
        if ev is not None:
            ev[3].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        from paper_2603_18052_gb300 import ranks

        return ranks.max_over_ranks(x, dev)

    def timed(form, steps, warmup, sampler=None, ntrials=5):
        """warmup untimed steps, then `steps` timed steps in up to five
        trials of consecutive steps; ms_per_step is the median over the
        trials of the trial's time per step (max over ranks)."""
        for _ in range(warmup):
            step(form)
        lb.lb_sync_status(ctx)
        lb.lb_set_stage_timing(ctx, True)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        ntr = max(1, min(ntrials, steps))
        sizes = [steps // ntr + (1 if t < steps % ntr else 0) for t in range(ntr)]
        tev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ntr)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        if sampler:
            sampler.start()
        n0 = lb.lb_launch_count()
        e0.record(stream)
        k = 0
        for t in range(ntr):
            tev[t][0].record(stream)
            for _ in range(sizes[t]):
                step(form, evs[k])
                k += 1
            tev[t][1].record(stream)
        e1.record(stream)
        n1 = lb.lb_launch_count()
        barrier()
        clocks = sampler.stop() if sampler else None
        lb.lb_sync_status(ctx)
        trial = [tev[t][0].elapsed_time(tev[t][1]) / sizes[t] for t in range(ntr)]
        med = max_over_ranks(statistics.median(trial))
        total_ms = max_over_ranks(e0.elapsed_time(e1))
        stages, chunks = lb.lb_stage_times(ctx)
        kern_ms, kern_fl, kern_n = lb.lb_kernel_times(ctx)
        lb.lb_set_stage_timing(ctx, False)
        ph = {"assemble_ms": 0.0, "build_ms": 0.0, "propagate_ms": 0.0}
        for ev in evs:
            ph["assemble_ms"] += ev[0].elapsed_time(ev[1]) / steps
            ph["build_ms"] += ev[1].elapsed_time(ev[2]) / steps
            ph["propagate_ms"] += ev[2].elapsed_time(ev[3]) / steps
        stages = {k: v / steps for k, v in stages.items()}
        return dict(ms_per_step=med, mean_ms_per_step=total_ms / steps, trial_ms_per_step=trial, steps=steps,
                    warmup=warmup, phases=ph, build_stages_ms=stages, launches=(n1 - n0) // steps, clocks=clocks,
                    step_ms=[ev[0].elapsed_time(ev[3]) for ev in evs],
                    sliced_kernel={"ms": kern_ms / steps, "flops": kern_fl / steps, "launches": kern_n // steps})

    t_tune = time.perf_counter()
    tuned = lb.lb_autotune(ctx, n, S, B) if not args.no_autotune else 0
    t_tune = time.perf_counter() - t_tune
    sampler = ClockSampler(local)
    if args.headline_only:
        form = args.form or HEADLINE
        r = timed(form, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps({"headline_only": True, "form": form, "ms_per_step": r["ms_per_step"],
                              "steps": args.steps, "warmup": args.warmup, "slices": S, "states": B,
                              "build_stages_ms": r["build_stages_ms"], "phases_ms": r["phases"],
                              "launches_per_step": r["launches"]}), flush=True)
        ctx.close()
        return
    res = {HEADLINE: timed(HEADLINE, args.steps, args.warmup, sampler)}
    # the other forms: a bounded number of steps (the complex FP64 form takes
    # seconds per step), five trials of one step each
    for f in FORMS:
        if f != HEADLINE:
            res[f] = timed(f, min(args.steps, 5), 1 if f == "fp64" else min(args.warmup, 3))
    head = res[HEADLINE]
    mixed_form = min(MIXED_FORMS, key=lambda f: res[f]["ms_per_step"])

    # end to end through the public API with host buffers: H2D of every input
    # from pinned memory, the three calls, D2H of the final states
    host = {k: torch.from_numpy(np.ascontiguousarray(w[k])).pin_memory()
            for k in ("H0", "jumps", "X", "u", "states")}
    out_host = torch.empty_like(host["states"]).pin_memory()
    dbuf = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_host.numel() * out_host.element_size()

    def e2e_step():
        for k, v in host.items():
            dbuf[k].copy_(v, non_blocking=True)
        step(HEADLINE, None, dbuf["H0"], dbuf["jumps"], dbuf["X"], dbuf["u"], dbuf["states"])
        out_host.copy_(dbuf["states"], non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    f1.record(stream)
    barrier()
    lb.lb_sync_status(ctx)
    e2e_ms = max_over_ranks(f0.elapsed_time(f1)) / args.steps

    # accuracy of every form in this run (one step from the initial states)
    s_dev = torch.empty(S, dtype=torch.int32, device=dev)

    def run_form(f):
        Rf = dput(w["states"])
        step(f, R=Rf, s_out=s_dev)
        lb.lb_sync_status(ctx)
        return P, Rf, s_dev.cpu().numpy()

    errors = form_errors(lb, ctx, w, dev, list(FORMS), run_form) if rank == 0 else {}
    squarings = [int(x) for x in run_form(HEADLINE)[2]]

    units = B * S  # state-steps per step per rank

    def form_line(f):
        r = res[f]
        return {"value": world * units / (r["ms_per_step"] / 1e3), "unit": "state-steps/s",
                "builds_per_s": world * S / (r["ms_per_step"] / 1e3), "ms_per_step": r["ms_per_step"],
                "mean_ms_per_step": r["mean_ms_per_step"], "trial_ms_per_step": r["trial_ms_per_step"],
                "steps": r["steps"], "warmup": r["warmup"], "phases_ms": r["phases"],
                "build_stages_ms": r["build_stages_ms"], "launches_per_step": r["launches"], "dtype": DTYPES[f],
                "precision": PRECISION_DESC[f], "error": errors.get(f)}

    value = world * units / (head["ms_per_step"] / 1e3)
    builds = world * S / (head["ms_per_step"] / 1e3)

    # roofline of the dominant kernel of the headline form: the sliced FP64
    # product (ozgemm_kernel) on the BF16 tensor cores, every launch of the
    # timed steps bracketed by CUDA events on its stream (lb_kernel_times);
    # the work counted is its 45 BF16 digit products per FP64 multiply-add
    sk = head["sliced_kernel"]
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "ozgemm_d27_traffic.json")
    if os.path.exists(tfile):
        t = json.load(open(tfile))
        if t.get("per_launch_bytes") and t.get("kernel_version") == OZ_KERNEL_VERSION:
            traffic = t["per_launch_bytes"]
    ach = sk["flops"] / (sk["ms"] / 1e3) if sk["ms"] > 0 else 0.0
    roofline = {
        "bound": "tensor", "kernel": "ozgemm_kernel: the sliced FP64 products (the Pade products A^4, A^6, A^6 Z1, "
                                     "A^6 Z2 and U = A W, the LU and solve block products and the diagonal blocks' "
                                     "64-wide products, the propagation steps; the masked squaring launches excepted)",
        "achieved": ach / 1e12, "peak": bf16_peak / 1e12, "unit": "TFLOP/s", "frac": ach / bf16_peak,
        "traffic": traffic, "peak_source": peak_src["bf16"] + " (dense BF16 tcgen05, burst)",
        "launches_per_step": sk["launches"], "kernel_ms_per_step": sk["ms"],
        "algorithmic_flops_per_step": sk["flops"],
        "flops_note": "digit-product FLOPs: 45 BF16 products (the digit pairs i + j <= 10 of nine digits per "
                      "operand) x 2 M N K per FP64 product M x N x K; the padded rows and columns of the 128 x BN "
                      "tiles are not counted",
        "fp64_equivalent_tflops": ach / 45.0 / 1e12,
        "fp64_equivalent_vs_dfma_peak": (ach / 45.0) / fp64_peak,
        "share_of_step": sk["ms"] / head["ms_per_step"],
        "stage_ms": {k: head["build_stages_ms"][k] for k in ("pade_products", "lu_solve", "squarings")},
    }

    # the FP64-pipe form's roofline: the real FP64 GEMM (rgemm_kernel<double>)
    # of the LU and solve, the squarings and the propagation, from the
    # stage and phase events
    nat = res[FP64_NATIVE]
    st = nat["build_stages_ms"]
    prop_ms = nat["phases"]["propagate_ms"]
    n3 = float(n) ** 3
    fl_solve = S * accounting.build_flops_real_solve(n)
    fl_sq = sum(squarings) * 2 * n3
    fl_prop = S * B * accounting.state_step_flops_real(n)
    gemm_ms = st["lu_solve"] + st["squarings"] + prop_ms
    gemm_flops = fl_solve + fl_sq + fl_prop
    ach64 = gemm_flops / (gemm_ms / 1e3)
    roofline_native = {
        "bound": "alu", "kernel": "rgemm_kernel<double>: the LU updates and substitutions, the squarings and the "
                                  "propagation steps of the FP64-pipe real-coordinate form",
        "achieved": ach64 / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
        "peak_source": peak_src["fp64"] + " (DFMA, burst)",
        "algorithmic_flops_per_step": gemm_flops,
        "flops_note": "real FLOPs, 2 per real multiply-add, n = 729: per slice the LU 2 n^3/3 and the n-RHS solve "
                      "2 n^3, s squarings at 2 n^3; per state-step 2 n^2 (B = 256, 200 steps)",
        "share_of_step": gemm_ms / nat["ms_per_step"],
        "stage_ms": {"lu_solve": st["lu_solve"], "squarings": st["squarings"], "propagation": prop_ms},
        "lu_solve_frac": (fl_solve / (st["lu_solve"] / 1e3)) / fp64_peak,
        "squarings_frac": (fl_sq / (st["squarings"] / 1e3)) / fp64_peak if st["squarings"] > 0 else None,
        "propagation_frac": (fl_prop / (prop_ms / 1e3)) / fp64_peak}

    def prop_roof(f):
        ms = res[f]["phases"]["propagate_ms"]
        if f == "fp64_sliced":
            fl, peak, note = S * B * accounting.state_step_flops_real(n) * 45, bf16_peak, \
                "45 BF16 digit products per real multiply-add, 2 n^2 real FLOP per state-step, against the BF16 " \
                "tcgen05 probe (the states sliced every step, the propagators once per chunk)"
        elif f == "fp64_hermitian":
            fl, peak, note = S * B * accounting.state_step_flops_real(n), fp64_peak, \
                "2 n^2 real FLOP per state-step on the real coordinates against the DFMA probe"
        elif f in ("fp64",):
            fl, peak, note = S * B * accounting.state_step_flops(n), fp64_peak, \
                "8 n^2 FLOP per state-step against the DFMA probe (Gauss form: 6 executed per 8 counted)"
        elif f == "bf16x3":
            fl, peak, note = S * B * accounting.state_step_flops(n), bf16_peak / 5.0, \
                "useful 8 n^2 FLOP per state-step (Eq. 4); peak = BF16 tcgen05 probe / 5 (five BF16 products per " \
                "real product)"
        else:
            fl, peak, note = S * B * accounting.state_step_flops(n), fp32_peak, \
                "8 n^2 FLOP per state-step against the FFMA probe"
        a = fl / (ms / 1e3)
        return {"bound": "tensor" if f in ("bf16x3", "fp64_sliced") else "alu", "achieved": a / 1e12,
                "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": a / peak, "ms": ms, "note": note}

    mixed_line = {"form": mixed_form, **form_line(mixed_form),
                  "forms": {f: form_line(f) for f in MIXED_FORMS},
                  "speedup_vs_fp64_headline": head["ms_per_step"] / res[mixed_form]["ms_per_step"],
                  "roofline_propagation": prop_roof(mixed_form)}
    line = {
        "metric": METRIC, "value": value, "unit": "state-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "arithmetic": "FP64 inputs and results; the dense FP64 products run on the BF16 tensor cores as exact "
                      "digit slices (Ozaki scheme) with FP64-size rounding error; the FP64-pipe form is under "
                      "fp64_native",
        "builds_per_s": builds, "form": HEADLINE,
        "config": {"workload": WORKLOAD_DESC,
                   "precision": PRECISION_DESC[HEADLINE],
                   "timing": "median over 5 trials of consecutive steps of the time per step (CUDA events on the "
                             "launching stream); mean_ms_per_step beside it",
                   "l2": "no flush: every step streams 0.85 GB of real propagators (1.7 GB complex) plus ~8 GB "
                         "of build scratch, far larger than the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "mean_ms_per_step": head["mean_ms_per_step"], "trial_ms_per_step": head["trial_ms_per_step"],
        "phases_ms": head["phases"], "build_stages_ms": head["build_stages_ms"], "error": errors.get(HEADLINE),
        "mixed": mixed_line,
        "forms": {f: form_line(f) for f in FORMS},
        "peaks_measured_tflops": peaks,
        "roofline": roofline,
        "roofline_fp64_native": roofline_native,
        "fp64_native": {"form": FP64_NATIVE, **form_line(FP64_NATIVE),
                        "headline_speedup": nat["ms_per_step"] / head["ms_per_step"]},
        "roofline_propagation": {f: prop_roof(f) for f in FORMS},
        "e2e": {"value": world * units / (e2e_ms / 1e3), "unit": "state-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "autotune": {"shapes": tuned, "seconds": t_tune},
        "gpu_launches": head["launches"] * args.steps,
        "gpu_launches_per_step": head["launches"],
        "clocks": head["clocks"],
    }
    line["other_workloads"] = other_workloads(lb, accounting, dev, stream, fp64_peak=fp64_peak, fp32_peak=fp32_peak,
                                              bf16_peak=bf16_peak)
    line["other_workloads"]["mixed_instances"] = mixed_instances(lb, ctx, dev, stream, args.instances,
                                                                 5)
    if rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, 6)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if rank == 0 and args.trials:  # raw timings, one JSON object per line
        with open(args.trials, "a") as fh:
            for f, r in res.items():
                for k, v in enumerate(r["step_ms"]):
                    fh.write(json.dumps({"kind": "d27_chain_step", "form": f, "step": k, "ms": v}) + "\n")
                for k, v in enumerate(r["trial_ms_per_step"]):
                    fh.write(json.dumps({"kind": "d27_chain_trial", "form": f, "trial": k, "ms_per_step": v}) + "\n")
            for row in line["other_workloads"]["gpu_timing_models"]["rows"]:
                for name in ("kernel", "resident", "host"):
                    for i, v in enumerate(row[name]["trials_ns"]):
                        fh.write(json.dumps({"kind": "gpu_timing_model", "model": name, "d": row["d"],
                                             "batch": row["batch"], "trial": i, "ns_per_state_step": v}) + "\n")
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
