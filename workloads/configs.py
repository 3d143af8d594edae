"""Named synthetic workloads.

Each entry fixes the transmon model, the control schedule, the batch of
initial states and the step counts.  ``make_workload`` can shrink the batch,
slice count or step count for tests while keeping the same model and seeds.
"""

import numpy as np

from .rng import ginibre_states, stream_seed, uniform01
from .transmon import transmon_chain

SEED_BASE = 0x5EED0000

CONFIGS = {
    # one transmon, d=3: a 9x9 propagator, one state, 10^4 steps, constant u
    "d3_single": dict(nq=1, nslices=1, steps_per_slice=10000, B=1, u_const=0.05, seed=SEED_BASE + 0),
    # two coupled transmons, d=9: 81x81, 1024 states, 1000 steps, constant u
    "d9_batch": dict(nq=2, nslices=1, steps_per_slice=1000, B=1024, u_const=0.05, seed=SEED_BASE + 1),
    # three-transmon chain, d=27: 729x729, 200 slices with u ~ U(-0.1, 0.1),
    # one step per slice, 256 states
    "d27_chain": dict(nq=3, nslices=200, steps_per_slice=1, B=256, u_range=0.1, seed=SEED_BASE + 2),
}


def make_workload(name, B=None, nslices=None, steps_per_slice=None, seed=None):
    """Return a dict with the model and the seeded inputs of workload ``name``.

    Keys: d, n, dt, H0 (d,d), X (d,d), jumps (K,d,d), u (nslices,),
    states (B, n), nslices, steps_per_slice, B, seed.
    """
    cfg = dict(CONFIGS[name])
    if B is not None:
        cfg["B"] = B
    if nslices is not None:
        cfg["nslices"] = nslices
    if steps_per_slice is not None:
        cfg["steps_per_slice"] = steps_per_slice
    if seed is not None:
        cfg["seed"] = seed
    model = transmon_chain(cfg["nq"])
    S = cfg["nslices"]
    if "u_const" in cfg:
        u = np.full(S, cfg["u_const"], dtype=np.float64)
    else:
        r = cfg["u_range"]
        u = (2.0 * uniform01(stream_seed(cfg["seed"], "controls"), S) - 1.0) * r
    states = ginibre_states(stream_seed(cfg["seed"], "states"), model.d, cfg["B"])
    return dict(name=name, d=model.d, n=model.d * model.d, dt=model.dt, H0=model.H0, X=model.X,
                jumps=model.jumps, u=u, states=states, nslices=S,
                steps_per_slice=cfg["steps_per_slice"], B=cfg["B"], seed=cfg["seed"],
                model=model)


MIXED_INSTANCES = dict(count=4096, ratio=(8, 4, 1), nslices=50, Bmax=64, u_range=0.1, seed=SEED_BASE + 3)


def make_instances(count=None, seed=None):
    """The mixed-size batch: instances with d drawn from {3, 9, 27} in ratio
    8:4:1 (exact counts by rounding, shuffled by the seed), 50 control slices
    each with u ~ U(-0.1, 0.1), and B ~ U{1..64} Ginibre states.

    Returns a list of dicts (nq, d, u, states) and the shared transmon models
    per nq."""
    cfg = dict(MIXED_INSTANCES)
    if count is not None:
        cfg["count"] = count
    if seed is not None:
        cfg["seed"] = seed
    N, r = cfg["count"], cfg["ratio"]
    tot = sum(r)
    counts = [int(round(N * x / tot)) for x in r]
    counts[0] += N - sum(counts)
    nqs = np.concatenate([np.full(c, q) for q, c in zip((1, 2, 3), counts)]).astype(int)
    perm = np.argsort(uniform01(stream_seed(cfg["seed"], "order"), N), kind="stable")
    nqs = nqs[perm]
    models = {q: transmon_chain(q) for q in (1, 2, 3)}
    Bs = 1 + (uniform01(stream_seed(cfg["seed"], "batch"), N) * cfg["Bmax"]).astype(int)
    out = []
    for i in range(N):
        q = int(nqs[i])
        u = (2.0 * uniform01(stream_seed(cfg["seed"], "u%d" % i), cfg["nslices"]) - 1.0) * cfg["u_range"]
        st = ginibre_states(stream_seed(cfg["seed"], "s%d" % i), models[q].d, int(Bs[i]))
        out.append(dict(nq=q, d=models[q].d, u=u, states=st))
    return out, models
