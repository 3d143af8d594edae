"""GRAPE with a learned warm start.

The GRAPE landscape point of Sec. 2.5 (one propagator per control slice,
Eq. 5) gives the fidelity F of a piecewise-constant control and its gradient
(lb_grape_grad).  Plain GRAPE maximises F from a random start with Adam steps
(lb_adam_step_f64).  A small MLP (BF16 weights, FP32 accumulation; its
forward, backward and Adam kernels are the library's) is trained on GRAPE
solutions that the library itself generates, and proposes the starting
control for new targets.

Problems: a chain of nq = 1 or 2 transmons (d = 3 or 9), 100 slices of
0.1 ns, target R_x(theta) on transmon 0's qubit subspace (identity on the
other qubit), jump rates gamma1 and gamma_phi per instance.  The figure of
merit is the average gate fidelity on the computational subspace,
F_avg = (d_c F + 1) / (d_c + 1), with F = Re sum_b <X_target,b, X_T,b> / d_c^2
over the d_c^2 basis operators |i><j|.

Every arithmetic step runs in the library's kernels; this module only moves
tensors and loops.  `experiment_batched` runs the experiment at the
configured scale: thousands of GRAPE optimisations advance together, one
lb_grape_grad_batch call per iteration for all of them.
"""

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import lb
from workloads.rng import stream_seed, uniform01
from workloads.transmon import transmon_chain

NSLICES = 100
DT = 0.1
U_SCALE = 0.2  # network outputs are u / U_SCALE


def _rx(theta):
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def _vec(M):
    return np.ascontiguousarray(M).reshape(-1)


class GateProblem:
    """Device tensors of one gate-synthesis problem."""

    def __init__(self, ctx, nq, theta, gamma1, gamma_phi, dev):
        m = transmon_chain(nq, gamma1=gamma1, gamma_phi=gamma_phi)
        self.nq, self.d, self.n = nq, m.d, m.d * m.d
        self.theta, self.gamma1, self.gamma_phi = theta, gamma1, gamma_phi
        self.dc = 2 ** nq
        d = m.d
        # computational basis states |k> of the qubit subspace inside the chain
        comp = []
        for k in range(self.dc):
            bits = [(k >> (nq - 1 - q)) & 1 for q in range(nq)]
            idx = 0
            for bq in bits:
                idx = idx * 3 + bq
            comp.append(idx)
        Ut = _rx(theta)
        for _ in range(nq - 1):
            Ut = np.kron(Ut, np.eye(2))
        B = self.dc * self.dc
        X0 = np.zeros((B, d * d), dtype=np.complex128)
        Xt = np.zeros((B, d * d), dtype=np.complex128)
        for i in range(self.dc):
            for j in range(self.dc):
                b = i * self.dc + j
                E = np.zeros((d, d), dtype=np.complex128)
                E[comp[i], comp[j]] = 1.0
                X0[b] = _vec(E)
                T = np.zeros((d, d), dtype=np.complex128)
                Tc = Ut[:, [i]] @ Ut[:, [j]].conj().T  # U |i><j| U^+
                for a in range(self.dc):
                    for c in range(self.dc):
                        T[comp[a], comp[c]] = Tc[a, c]
                Xt[b] = _vec(T)
        put = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
        self.Lb = torch.empty((self.n, self.n), dtype=torch.complex128, device=dev)
        self.Ld = torch.empty_like(self.Lb)
        lb.lb_assemble(ctx, put(m.H0), put(m.jumps), self.Lb)
        lb.lb_assemble(ctx, put(m.X), None, self.Ld)
        self.X0, self.Xt = put(X0), put(Xt)

    def features(self):
        """Network input: (theta / pi, scaled log rates, d / 9)."""
        return np.array([self.theta / math.pi, (math.log10(self.gamma1) + 4.5) / 0.5,
                         (math.log10(self.gamma_phi) + 4.8) / 0.5, self.d / 9.0], dtype=np.float32)

    def f_avg(self, F):
        return (self.dc * F + 1.0) / (self.dc + 1.0)


def grape(ctx, prob, u0, target=0.999, max_iter=300, lr=0.01, history=None):
    """Adam ascent of F from u0 (device float64, modified in place).  Returns
    (iterations to reach F_avg >= target or max_iter, best F_avg, seconds);
    `history` (a list) receives F_avg of every iteration."""
    dev = u0.device
    u = u0
    g = torch.zeros_like(u)
    m = torch.zeros_like(u)
    v = torch.zeros_like(u)
    F = torch.zeros(1, dtype=torch.float64, device=dev)
    best = -1.0
    t0 = time.perf_counter()
    it = 0
    for it in range(1, max_iter + 1):
        lb.lb_grape_grad(ctx, prob.Lb, prob.Ld, u, DT, 1, prob.X0, prob.Xt, F, g)
        fa = prob.f_avg(float(F.item()))
        best = max(best, fa)
        if history is not None:
            history.append(fa)
        if fa >= target:
            break
        lb.lb_adam_step_f64(u, g, m, v, it, lr=lr, ascend=True)
    torch.cuda.synchronize()
    return it, best, time.perf_counter() - t0


def grape_batch(ctx, probs, U, target, max_iter=300, lr=0.01, prec="fp64"):
    """Plain GRAPE (Adam ascent of F) for K problems of one size at once:
    one lb_grape_grad_batch call and one lb_adam_step_f64 over all K x
    NSLICES controls per iteration.  U (K, NSLICES, device float64) holds the
    starting controls and receives, for every problem that reached F_avg >=
    target, the control of the iteration where it first did (the last one
    otherwise).  Returns (iterations per problem: the first iteration at the
    target, or max_iter; best F_avg per problem; seconds of the batch)."""
    K = len(probs)
    dev = U.device
    Lb = torch.stack([p.Lb for p in probs]).contiguous()
    X0 = torch.stack([p.X0 for p in probs]).contiguous()
    Xt = torch.stack([p.Xt for p in probs]).contiguous()
    dc = probs[0].dc
    g, m, v = torch.zeros_like(U), torch.zeros_like(U), torch.zeros_like(U)
    F = torch.zeros(K, dtype=torch.float64, device=dev)
    iters = np.full(K, max_iter)
    best = np.full(K, -1.0)
    done = np.zeros(K, dtype=bool)
    saved = U.clone()
    t0 = time.perf_counter()
    for it in range(1, max_iter + 1):
        lb.lb_grape_grad_batch(ctx, Lb, probs[0].Ld, U, DT, 1, X0, Xt, F, g, prec=prec)
        fa = (dc * F.cpu().numpy() + 1.0) / (dc + 1.0)
        best = np.maximum(best, fa)
        new = (fa >= target) & ~done
        if new.any():
            idx = torch.from_numpy(np.nonzero(new)[0]).to(dev)
            saved[idx] = U[idx]
            iters[new] = it
            done |= new
            if done.all():
                break
        lb.lb_adam_step_f64(U, g, m, v, it, lr=lr, ascend=True)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    if done.any():
        idx = torch.from_numpy(np.nonzero(done)[0]).to(dev)
        U[idx] = saved[idx]
    return iters, best, secs


def random_u(seed, dev):
    return torch.from_numpy((2.0 * uniform01(seed, NSLICES) - 1.0) * 0.1).to(dev)


def sample_problems(ctx, seed, count, nq, dev):
    """theta ~ U[pi/4, pi], log-uniform gamma1 in [1e-5, 1e-4] and gamma_phi
    in [5e-6, 5e-5]."""
    r = uniform01(stream_seed(seed, "params%d" % nq), 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        th = math.pi / 4 + r[k, 0] * (math.pi - math.pi / 4)
        g1 = 10 ** (-5 + r[k, 1])
        gp = 5e-6 * 10 ** r[k, 2]
        out.append(GateProblem(ctx, nq, th, g1, gp, dev))
    return out


class WarmStartNet:
    """dims[0] -> 256 -> 256 -> 256 -> NSLICES MLP; FP32 master weights, BF16
    copy for the forward pass, Adam moments."""

    def __init__(self, dev, dims=(4, 256, 256, 256, NSLICES), seed=7):
        self.dims = list(dims)
        self.dev = dev
        nW = sum(self.dims[l + 1] * self.dims[l] for l in range(len(self.dims) - 1))
        nb = sum(self.dims[1:])
        r = uniform01(seed, nW)
        parts, o = [], 0
        for l in range(len(self.dims) - 1):
            sz = self.dims[l + 1] * self.dims[l]
            lim = math.sqrt(6.0 / (self.dims[l] + self.dims[l + 1]))
            parts.append((2 * r[o: o + sz] - 1) * lim)
            o += sz
        self.W = torch.from_numpy(np.concatenate(parts).astype(np.float32)).to(dev)
        self.W16 = self.W.to(torch.bfloat16)
        self.b = torch.zeros(nb, dtype=torch.float32, device=dev)
        self.mW, self.vW = torch.zeros_like(self.W), torch.zeros_like(self.W)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.step = 0

    def _buffers(self, batch):
        acts = torch.empty(batch * sum(self.dims[1:]), dtype=torch.float32, device=self.dev)
        return acts

    def predict(self, x):
        acts = self._buffers(x.shape[0])
        lb.lb_mlp_forward(self.dims, self.W16, self.b, x, acts)
        return acts[-x.shape[0] * self.dims[-1]:].view(x.shape[0], self.dims[-1])

    def train(self, X, Y, epochs=400, batch=64, lr=1e-3, seed=11):
        """Minibatch Adam on the mean squared error."""
        N = X.shape[0]
        gW, gb = torch.empty_like(self.W), torch.empty_like(self.b)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        losses = []
        for ep in range(epochs):
            perm = np.argsort(uniform01(stream_seed(seed, "ep%d" % ep), N))
            for s0 in range(0, N, batch):
                idx = torch.from_numpy(perm[s0: s0 + batch]).to(self.dev)
                xb, yb = X[idx].contiguous(), Y[idx].contiguous()
                B = xb.shape[0]
                acts = self._buffers(B)
                lb.lb_mlp_forward(self.dims, self.W16, self.b, xb, acts)
                out = acts[-B * self.dims[-1]:].view(B, self.dims[-1])
                dy = torch.empty_like(out)
                lb.lb_mse_loss_grad(out, yb, dy, loss)
                scratch = torch.empty(2 * B * max(self.dims), dtype=torch.float32, device=self.dev)
                lb.lb_mlp_backward(self.dims, self.W16, xb, acts, dy, gW, gb, scratch)
                self.step += 1
                lb.lb_adam_step(self.W, gW, self.mW, self.vW, self.step, lr=lr, p_bf16=self.W16)
                lb.lb_adam_step(self.b, gb, self.mb, self.vb, self.step, lr=lr)
            losses.append(float(loss.item()))
        return losses


def experiment(nq=1, n_train=128, n_test=8, max_iter=300, target=0.999, seed=0x5EED0004, dev=None,
               epochs=400, log=print):
    """Generate GRAPE solutions with the library, train the network on them,
    then compare iterations and wall time to the target fidelity from the
    network's proposal and from a random start on held-out problems.  Where
    plain GRAPE does not reach the target within max_iter, the instance's
    threshold is its best plain F_avg minus 1e-4."""
    dev = dev or torch.device("cuda:0")
    d = 3 ** nq
    ctx = lb.Context(dev.index or 0, max_n=d * d, max_batch=(2 ** nq) ** 2, max_slices=NSLICES)
    t0 = time.perf_counter()
    train = sample_problems(ctx, stream_seed(seed, "train"), n_train, nq, dev)
    X, Y, train_iters, train_best = [], [], [], []
    for k, p in enumerate(train):
        u = random_u(stream_seed(seed, "u%d" % k), dev)
        it, best, _ = grape(ctx, p, u, target=target, max_iter=max_iter)
        X.append(p.features())
        Y.append((u / U_SCALE).float().cpu().numpy())
        train_iters.append(it)
        train_best.append(best)
    t_data = time.perf_counter() - t0
    log("dataset: %d GRAPE solutions in %.1f s, median iterations %d, median best F_avg %.5f"
        % (n_train, t_data, int(np.median(train_iters)), float(np.median(train_best))))
    net = WarmStartNet(dev)
    Xd = torch.from_numpy(np.array(X)).to(dev)
    Yd = torch.from_numpy(np.array(Y)).to(dev)
    t1 = time.perf_counter()
    losses = net.train(Xd, Yd, epochs=epochs)
    t_train = time.perf_counter() - t1
    log("training: %d epochs in %.1f s, loss %.4g -> %.4g" % (epochs, t_train, losses[0], losses[-1]))
    test = sample_problems(ctx, stream_seed(seed, "test"), n_test, nq, dev)
    rows = []
    for k, p in enumerate(test):
        # plain GRAPE from a random start, run to max_iter: its best F_avg sets
        # the instance's threshold min(target, F*_plain - 1e-4)
        u_rand = random_u(stream_seed(seed, "test_u%d" % k), dev)
        hist = []
        _, best_r, t_full = grape(ctx, p, u_rand, target=2.0, max_iter=max_iter, history=hist)
        thr = min(target, best_r - 1e-4)
        it_r = next(i + 1 for i, f in enumerate(hist) if f >= thr)
        t_r = t_full * it_r / len(hist)
        xin = torch.from_numpy(p.features()[None, :]).to(dev)
        u_warm = (net.predict(xin)[0].double() * U_SCALE).contiguous()
        it_w, best_w, t_w = grape(ctx, p, u_warm, target=thr, max_iter=max_iter)
        rows.append(dict(theta=p.theta, gamma1=p.gamma1, gamma_phi=p.gamma_phi, threshold=thr, warm_iters=it_w,
                         warm_best=best_w, warm_s=t_w, random_iters=it_r, random_best=best_r, random_s=t_r))
        log("test %d: threshold %.5f  warm %d it (%.2f s)  random %d it (%.2f s)"
            % (k, thr, it_w, t_w, it_r, t_r))
    ctx.close()
    med = lambda key: float(np.median([r[key] for r in rows]))
    return dict(nq=nq, d=d, nslices=NSLICES, dt=DT, target_f_avg=target, max_iter=max_iter, n_train=n_train,
                n_test=n_test, dataset_seconds=t_data, train_seconds=t_train, final_loss=losses[-1],
                median_warm_iters=med("warm_iters"), median_random_iters=med("random_iters"),
                median_warm_seconds=med("warm_s"), median_random_seconds=med("random_s"),
                warm_reached=sum(r["warm_best"] >= r["threshold"] for r in rows),
                random_reached=sum(r["random_best"] >= r["threshold"] for r in rows),
                target_reached_plain=sum(r["random_best"] >= target for r in rows), tests=rows)


def iteration_seconds(ctx, prob, reps=20):
    """Wall time of one plain-GRAPE iteration of a single problem (one
    lb_grape_grad call and one Adam step), the median of `reps`: the
    per-instance time the batched runs' iteration counts are converted
    with."""
    u = random_u(1, prob.Lb.device)
    g, m, v = torch.zeros_like(u), torch.zeros_like(u), torch.zeros_like(u)
    F = torch.zeros(1, dtype=torch.float64, device=u.device)
    ts = []
    for r in range(reps + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lb.lb_grape_grad(ctx, prob.Lb, prob.Ld, u, DT, 1, prob.X0, prob.Xt, F, g)
        F.item()
        lb.lb_adam_step_f64(u, g, m, v, r + 1, lr=0.01, ascend=True)
        torch.cuda.synchronize()
        if r >= 2:
            ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def experiment_batched(n_train=(20000, 1024), n_test=100, max_iter=300, targets=(0.999, 0.96),
                       batch=(2048, 128), precs=("fp64", "fp32"), seed=0x5EED0004, dev=None, epochs=60,
                       train_batch=256, log=print):
    """The warm-start experiment at the configured scale, with every GRAPE run
    batched (lb_grape_grad_batch): n_train[i] library-generated GRAPE
    solutions at d = 3 and d = 9 (batches of batch[i] problems, products in
    precs[i]), one network trained on both sizes (d is an input), then per
    size n_test held-out problems solved from a random start and from the
    network's proposal (FP64), both to the threshold targets[i] fixed before
    the runs.  Reports iteration counts (medians and the share of problems
    reaching the threshold) and wall times per instance (iterations x the
    measured time of one single-problem iteration)."""
    dev = dev or torch.device("cuda:0")
    X, Y = [], []
    res = dict(nslices=NSLICES, dt=DT, max_iter=max_iter, sizes={})
    for nq, ntr, K, prec, target in zip((1, 2), n_train, batch, precs, targets):
        d = 3 ** nq
        ctx = lb.Context(dev.index or 0, max_n=d * d, max_batch=(2 ** nq) ** 2 * K, max_slices=K * NSLICES)
        t0 = time.perf_counter()
        its, bests = [], []
        for b0 in range(0, ntr, K):
            k = min(K, ntr - b0)
            probs = sample_problems(ctx, stream_seed(seed, "train%d_%d" % (nq, b0)), k, nq, dev)
            U = torch.stack([random_u(stream_seed(seed, "u%d_%d" % (nq, b0 + i)), dev) for i in range(k)]).contiguous()
            it, best, _ = grape_batch(ctx, probs, U, target, max_iter=max_iter, prec=prec)
            its.extend(it.tolist())
            bests.extend(best.tolist())
            X.extend(p.features() for p in probs)
            Y.extend((U / U_SCALE).float().cpu().numpy())
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        res["sizes"]["d%d" % d] = dict(d=d, n_train=ntr, target_f_avg=target, batch=K, product_precision=prec,
                                       dataset_seconds=t_data, dataset_median_iters=float(np.median(its)),
                                       dataset_median_best=float(np.median(bests)),
                                       dataset_reached=int(np.sum(np.array(bests) >= target)))
        log("d=%d dataset: %d GRAPE solutions in %.1f s (%d reached %.3g)" % (d, ntr, t_data,
                                                                         res["sizes"]["d%d" % d]["dataset_reached"],
                                                                         target))
        ctx.close()
    net = WarmStartNet(dev)
    Xd = torch.from_numpy(np.array(X, dtype=np.float32)).to(dev)
    Yd = torch.from_numpy(np.array(Y, dtype=np.float32)).to(dev)
    t1 = time.perf_counter()
    losses = net.train(Xd, Yd, epochs=epochs, batch=train_batch)
    res["train_seconds"] = time.perf_counter() - t1
    res["train_samples"] = int(Xd.shape[0])
    res["loss_first_last"] = [losses[0], losses[-1]]
    log("training: %d samples, %d epochs in %.1f s, loss %.4g -> %.4g" % (Xd.shape[0], epochs, res["train_seconds"],
                                                                        losses[0], losses[-1]))
    for nq, target in zip((1, 2), targets):
        d = 3 ** nq
        ctx = lb.Context(dev.index or 0, max_n=d * d, max_batch=(2 ** nq) ** 2 * n_test, max_slices=n_test * NSLICES)
        probs = sample_problems(ctx, stream_seed(seed, "test%d" % nq), n_test, nq, dev)
        U_r = torch.stack([random_u(stream_seed(seed, "test_u%d_%d" % (nq, i)), dev) for i in range(n_test)])
        it_r, best_r, s_r = grape_batch(ctx, probs, U_r.contiguous(), target, max_iter=max_iter)
        feats = torch.from_numpy(np.array([p.features() for p in probs])).to(dev)
        U_w = (net.predict(feats).double() * U_SCALE).contiguous()
        it_w, best_w, s_w = grape_batch(ctx, probs, U_w, target, max_iter=max_iter)
        t_it = iteration_seconds(ctx, probs[0])
        ok_r, ok_w = best_r >= target, best_w >= target
        r = res["sizes"]["d%d" % d]
        r.update(n_test=n_test, threshold=target, seconds_per_iteration=t_it,
                 random_reached=int(ok_r.sum()), warm_reached=int(ok_w.sum()),
                 median_random_iters=float(np.median(it_r)), median_warm_iters=float(np.median(it_w)),
                 median_random_seconds=float(np.median(it_r)) * t_it,
                 median_warm_seconds=float(np.median(it_w)) * t_it,
                 batched_seconds_random=s_r, batched_seconds_warm=s_w,
                 median_random_best=float(np.median(best_r)), median_warm_best=float(np.median(best_w)),
                 plain_reached_0999=int((best_r >= 0.999).sum()))
        log("d=%d test: threshold %.4g  warm median %g it (%d/%d reached)  random median %g it (%d/%d reached)"
            % (d, target, r["median_warm_iters"], r["warm_reached"], n_test, r["median_random_iters"],
               r["random_reached"], n_test))
        ctx.close()
    return res


def main():
    ap = argparse.ArgumentParser(description="warm-start GRAPE experiment")
    ap.add_argument("--nq", type=int, default=1)
    ap.add_argument("--train", type=int, default=128)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--max-iter", type=int, default=300)
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--target", type=float, default=0.999)
    ap.add_argument("--out", default=None)
    ap.add_argument("--batched", action="store_true",
                    help="the configured scale: batched GRAPE at d = 3 and 9, one network for both")
    ap.add_argument("--train3", type=int, default=20000)
    ap.add_argument("--train9", type=int, default=1024)
    a = ap.parse_args()
    if a.batched:
        res = experiment_batched(n_train=(a.train3, a.train9), n_test=a.test, max_iter=a.max_iter,
                                 epochs=a.epochs)
        print(json.dumps(res))
        if a.out:
            os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
            json.dump(res, open(a.out, "w"), indent=1)
        return
    res = experiment(nq=a.nq, n_train=a.train, n_test=a.test, max_iter=a.max_iter, target=a.target,
                     epochs=a.epochs)
    print(json.dumps({k: v for k, v in res.items() if k != "tests"}))
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        json.dump(res, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
