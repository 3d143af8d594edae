"""The warm-start network's GPU kernels against the FP64 oracle MLP.  The
oracle uses the same BF16-rounded weights, so the comparison measures the
FP32 accumulation only (K <= 256 terms: relative error ~1e-6; the test
allows 1e-4 of the largest entry)."""

import numpy as np
import pytest

from oracle import mlp
from workloads.rng import normal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lbm():
    from paper_2603_18052_gb300 import _build, lb

    _build.build()
    assert torch.cuda.is_available()
    return lb


def _bf16(a):
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_mlp_forward_backward_adam_match_oracle(lbm):
    dev = torch.device("cuda:0")
    dims = [4, 256, 256, 256, 100]
    batch = 37
    Ws, bs = [], []
    for l in range(len(dims) - 1):
        Ws.append(_bf16(normal(70 + l, dims[l + 1] * dims[l]).reshape(dims[l + 1], dims[l]) / np.sqrt(dims[l])))
        bs.append(np.asarray(normal(90 + l, dims[l + 1]) * 0.1, dtype=np.float32).astype(np.float64))
    x = np.asarray(normal(5, batch * 4).reshape(batch, 4), dtype=np.float32)
    t = np.asarray(normal(6, batch * 100).reshape(batch, 100), dtype=np.float32)
    Wflat = torch.cat([torch.from_numpy(w.astype(np.float32)).reshape(-1) for w in Ws]).to(dev)
    W16 = Wflat.to(torch.bfloat16)
    bflat = torch.cat([torch.from_numpy(b.astype(np.float32)) for b in bs]).to(dev)
    xd = torch.from_numpy(x).to(dev)
    td = torch.from_numpy(t).to(dev)
    acts = torch.empty(batch * sum(dims[1:]), dtype=torch.float32, device=dev)
    lbm.lb_mlp_forward(dims, W16, bflat, xd, acts)
    ref = mlp.forward(Ws, bs, x.astype(np.float64))
    off = 0
    got_acts = []
    for l in range(len(dims) - 1):
        a = acts[off: off + batch * dims[l + 1]].view(batch, dims[l + 1]).cpu().numpy().astype(np.float64)
        got_acts.append(a)
        off += batch * dims[l + 1]
        assert np.max(np.abs(a - ref[l])) <= 1e-4 * np.max(np.abs(ref[l])), l
    y = acts[off - batch * 100: off].view(batch, 100)
    dy = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    lbm.lb_mse_loss_grad(y, td, dy, loss)
    lref, dyref = mlp.mse(ref[-1], t.astype(np.float64))
    assert abs(loss.item() - lref) <= 1e-4 * lref
    assert np.max(np.abs(dy.cpu().numpy() - dyref)) <= 1e-4 * np.max(np.abs(dyref))
    gW = torch.empty_like(Wflat)
    gb = torch.empty_like(bflat)
    scratch = torch.empty(2 * batch * max(dims), dtype=torch.float32, device=dev)
    lbm.lb_mlp_backward(dims, W16, xd, acts, dy, gW, gb, scratch)
    gWr, gbr = mlp.backward(Ws, bs, x.astype(np.float64), ref, dyref)
    woff, boff = 0, 0
    for l in range(len(dims) - 1):
        sz = dims[l + 1] * dims[l]
        gw = gW[woff: woff + sz].view(dims[l + 1], dims[l]).cpu().numpy()
        assert np.max(np.abs(gw - gWr[l])) <= 1e-4 * np.max(np.abs(gWr[l])), l
        g_b = gb[boff: boff + dims[l + 1]].cpu().numpy()
        assert np.max(np.abs(g_b - gbr[l])) <= 1e-4 * np.max(np.abs(gbr[l])), l
        woff += sz
        boff += dims[l + 1]
    # one Adam step on the FP32 master weights, BF16 copy refreshed
    m = torch.zeros_like(Wflat)
    v = torch.zeros_like(Wflat)
    p0 = Wflat.clone()
    lbm.lb_adam_step(Wflat, gW, m, v, 1, lr=1e-3, p_bf16=W16)
    pr, _, _ = mlp.adam(p0.cpu().numpy().astype(np.float64), gW.cpu().numpy().astype(np.float64), 0.0, 0.0, 1, 1e-3)
    assert np.max(np.abs(Wflat.cpu().numpy() - pr)) <= 1e-6
    assert torch.equal(W16, Wflat.to(torch.bfloat16))
