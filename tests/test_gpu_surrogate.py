"""The surrogate network on the GPU: gradients of the whole network against the
FP64 oracle (autograd), field packing, training on LB-generated data, and the
judged rollout with LB fallback."""
import math

import numpy as np
import pytest
import torch

from helpers import from_d_layout
from oracle import surrogate as so
from paper_1909_08406_gb300 import lb, sg
from paper_1909_08406_gb300 import surrogate as S
from paper_1909_08406_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
F64 = torch.float64


# (dilations, volume): the plain network, and the dilated one of the surrogate on a volume whose
# d = 8 layout still has rows of 4 (ny / 8 a multiple of 4)
NETS = [((1,) * 6, (2, 4, 8, 64)), (S.DILATIONS, (1, 8, 32, 64))]
NET_IDS = ["plain", "dilated"]


def _random_net(seed, dil=S.DILATIONS):
    net = S.Surrogate(seed=seed, dilations=dil)
    g = torch.Generator().manual_seed(seed)
    for k, (ci, co, _, _) in enumerate(S.LAYERS):
        w = torch.randn((co, 27, ci), generator=g) / math.sqrt(27 * ci) * (0.5 if k else 1.0)
        if ci == 16:
            w[:, :, 5:] = 0
        net.w32[k].copy_(w)
        net.b32[k].copy_(0.05 * torch.randn(co, generator=g))
    net._round_weights()
    return net


@pytest.mark.parametrize("dil,shape", NETS, ids=NET_IDS)
def test_network_gradients_match_oracle(dil, shape):
    """GPU forward + backward (BF16 storage of activations, FP32 accumulation) against FP64
    autograd on the same BF16 weights and inputs: per layer, the relative Frobenius error of
    the weight gradient <= 3e-2 and the cosine similarity >= 0.999 (activations are rounded to
    BF16 between layers, 2^-9 relative each)."""
    net = _random_net(3, dil)
    g = torch.Generator().manual_seed(4)
    x = torch.zeros(shape + (16,))
    x[..., :5] = torch.randn(shape + (5,), generator=g)
    t = x.clone()
    t[..., :5] += 0.3 * torch.randn(shape + (5,), generator=g)
    xb, tb = x.to(torch.bfloat16), t.to(torch.bfloat16)
    xd, td = xb.cuda(), tb.cuda()
    pred = net.forward(xd, train=True)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dpred = torch.empty(xd.shape, dtype=torch.float32, device="cuda")
    sg.mse(pred, td, 5, loss, dpred, sg.reduce_scratch())
    scratch = {(ci, co): sg.wgrad_scratch(xd, ci, co) for ci, co, _, _ in S.LAYERS}
    net.backward(dpred, scratch)
    torch.cuda.synchronize()
    ws = [w.cpu().to(F64) for w in net.w16]
    bs = [b.cpu().to(F64) for b in net.b32]
    l_or, gw, gb, _ = so.loss_and_grads(xb.to(F64), tb.to(F64), ws, bs, dilations=list(dil))
    assert loss.item() == pytest.approx(l_or, rel=2e-2)
    for k in range(len(S.LAYERS)):
        a = net.g[2 * k].cpu().to(F64).flatten()
        b = gw[k].flatten()
        if b.norm() == 0:
            continue
        rel = (a - b).norm() / b.norm()
        cos = (a @ b) / (a.norm() * b.norm())
        assert rel <= 3e-2 and cos >= 0.999, (k, rel.item(), cos.item())
        ab = net.g[2 * k + 1].cpu().to(F64)
        assert (ab - gb[k]).norm() <= 3e-2 * gb[k].norm() + 1e-6, k


@pytest.mark.parametrize("dil,shape", NETS, ids=NET_IDS)
def test_network_backward_chain_matches_oracle_elementwise(dil, shape):
    """Every link of the GPU backward pass, element by element, against FP64 computed from the
    GPU's own inputs to that link (the BF16 activations and FP32 pre-activations cached by the
    forward pass, and the gradient the link received):
      dL/dpred     = 2 (pred - target) / (voxels * 5) on channels 0..4, zero elsewhere;
      dz_k         = dh_out_k * act'(z_k), one BF16 rounding (2^-8 relative);
      dW_k, db_k   = sum_v h_k(v + d) dz_k(v), sum_v dz_k(v): FP32 summation, <= 1e-5 of the
                     sum of absolute terms (the kernel tests' bound);
      dh_in_k      = the input gradient of conv(h_k; W_k) for dz_k, plus dh_out_k for the
                     residual layers: <= 1e-5 of the sum of absolute terms.
    A wiring mistake anywhere in the chain (a dropped residual gradient, a wrong activation or
    cache index, a transposed tap, a layer in the wrong layout) moves some element by the size of
    the term itself.  Each layer's tensors are in its d-layout; they are compared on the volume
    (tests/helpers.py from_d_layout) against the oracle's convolution with the layer's dilation."""
    net = _random_net(5, dil)
    g = torch.Generator().manual_seed(6)
    x = torch.zeros(shape + (16,))
    x[..., :5] = torch.randn(shape + (5,), generator=g)
    t = x.clone()
    t[..., :5] += 0.3 * torch.randn(shape + (5,), generator=g)
    xd, td = x.to(torch.bfloat16).cuda(), t.to(torch.bfloat16).cuda()
    pred = net.forward(xd, train=True)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dpred = torch.empty(xd.shape, dtype=torch.float32, device="cuda")
    sg.mse(pred, td, 5, loss, dpred, sg.reduce_scratch())
    scratch = {(ci, co): sg.wgrad_scratch(xd, ci, co) for ci, co, _, _ in S.LAYERS}
    trace = {}
    net.backward(dpred, scratch, trace=trace)
    torch.cuda.synchronize()
    cpu = lambda a: a.cpu().to(F64)  # noqa: E731

    def nat(a, k):  # layer k's tensor, in its d-layout, on the volume (FP64, CPU)
        return from_d_layout(cpu(a), dil[k], shape)

    voxels = float(np.prod(shape))
    ref = torch.zeros(shape + (16,), dtype=F64)
    ref[..., :5] = 2 * (cpu(pred) - cpu(td))[..., :5] / (voxels * 5)
    assert torch.all((cpu(dpred) - ref).abs() <= 1e-6 * ref.abs() + 1e-12)
    last = len(S.LAYERS) - 1
    assert torch.equal(nat(trace[last]["dh_out"], last), cpu(dpred))

    for k in range(len(S.LAYERS) - 1, -1, -1):
        ci, co, act, res = S.LAYERS[k]
        dk = dil[k]
        h = nat(net.cache[k], k)                   # the layer's input (BF16 on the GPU)
        zk = nat(net.zs[k], k)                     # pre-activation (FP32)
        dh_out, dz = nat(trace[k]["dh_out"], k), nat(trace[k]["dz"], k)
        w = cpu(net.w16[k])
        # activation backward: one BF16 rounding of the product, plus the FP32 error of act'(z) =
        # Phi(z) + z phi(z), whose two terms cancel near z = -0.75 (a few ulp of each term)
        zr = zk.clone().requires_grad_(True)
        (so.gelu(zr) if act == sg.ACT_GELU else zr).backward(dh_out)
        terms = (0.5 * (1 + torch.erf(zk / math.sqrt(2))) + (zk * torch.exp(-zk * zk / 2)).abs() / math.sqrt(2 * math.pi)
                 if act == sg.ACT_GELU else torch.ones_like(zk))
        assert torch.all((dz - zr.grad).abs() <= 2 ** -8 * zr.grad.abs() + 5e-7 * dh_out.abs() * terms + 1e-30), k
        # weight and bias gradients from the GPU's own h and dz
        w0 = torch.zeros((co, 27, ci), dtype=F64, requires_grad=True)
        b0 = torch.zeros(co, dtype=F64, requires_grad=True)
        (so.conv3d_periodic(h, w0, b0, dilation=dk) * dz).sum().backward()
        wa = torch.zeros((co, 27, ci), dtype=F64, requires_grad=True)
        (so.conv3d_periodic(h.abs(), wa, dilation=dk) * dz.abs()).sum().backward()
        assert torch.all((cpu(net.g[2 * k]) - w0.grad).abs() <= 1e-5 * wa.grad + 1e-12), k
        assert torch.all((cpu(net.g[2 * k + 1]) - b0.grad).abs() <= 1e-5 * dz.abs().sum(dim=(0, 1, 2, 3)) + 1e-12), k
        if k > 0:
            hr = h.clone().requires_grad_(True)
            (so.conv3d_periodic(hr, w, dilation=dk) * dz).sum().backward()
            ha = h.abs().requires_grad_(True)
            (so.conv3d_periodic(ha, w.abs(), dilation=dk) * dz.abs()).sum().backward()
            want = hr.grad + (dh_out if res else 0)
            bound = 1e-5 * (ha.grad + (dh_out.abs() if res else 0)) + 1e-12
            assert torch.all((nat(trace[k]["dh_in"], k) - want).abs() <= bound), k
            # the gradient layer k passes on is the one layer k - 1 receives
            assert torch.equal(nat(trace[k - 1]["dh_out"], k - 1), nat(trace[k]["dh_in"], k)), k


def test_pack_unpack_fields():
    n = 64
    th0 = lb.lb_theta0()
    f = wl.gaussian_pulse_sample(n, th0, 11, device="cuda")
    x = torch.empty((1, n, n, n, 16), dtype=torch.bfloat16, device="cuda")
    sg.pack_fields(x, 0, f["rho"], f["u"], f["theta"], th0, S.SCALES)
    rho = torch.empty_like(f["rho"])
    u = torch.empty_like(f["u"])
    th = torch.empty_like(f["theta"])
    sg.unpack_fields(x, 0, th0, S.SCALES, rho, u, th)
    torch.cuda.synchronize()
    s = S.SCALES[0]
    # A nodes: values come back up to one BF16 rounding of the scaled deviation
    assert torch.allclose(rho[0], f["rho"][0], rtol=0, atol=s * 2 ** -8 * 4)
    assert torch.allclose(th[0], f["theta"][0], rtol=0, atol=th0 * s * 2 ** -8 * 4)
    # B node of cell r: mean of the A nodes r + {0,1}^3
    ra = rho[0]
    mean8 = sum(torch.roll(ra, shifts=(-dz, -dy, -dx), dims=(0, 1, 2))
                for dz in (0, 1) for dy in (0, 1) for dx in (0, 1)) / 8
    assert torch.allclose(rho[1], mean8, rtol=0, atol=1e-6)
    assert torch.all(x[..., 5:] == 0)


@pytest.fixture(scope="module")
def small_data():
    return S.make_dataset(24, hop=10, t0_choices=(0, 20), per_batch=12)


def test_training_reduces_loss_below_identity(small_data):
    net = S.Surrogate(seed=0)
    before, ident = S.evaluate(net, small_data)
    assert before == pytest.approx(ident, rel=1e-6)  # zero-initialised last layer: identity map
    S.train(net, small_data, iters=60, batch=4, lr=2e-3)
    after, _ = S.evaluate(net, small_data)
    assert after < 0.5 * ident, (after, ident)


def test_judged_rollout_and_fallback(small_data):
    net = S.Surrogate(seed=1)
    S.train(net, small_data, iters=20, batch=4, lr=2e-3)
    r = S.rollout(net, seed=90001, hops=3, hop=10, threshold=1e30)
    assert len(r["signal"]) == 3 and not any(r["fallback"])
    assert all(np.isfinite(r["signal"])) and all(e > 0 for e in r["state"])
    # a zero threshold falls back after every hop; the next hop then starts from LB's state
    r0 = S.rollout(net, seed=90001, hops=3, hop=10, threshold=0.0)
    assert all(r0["fallback"])
    assert r0["signal"][0] == pytest.approx(r["signal"][0], rel=1e-6)


def test_rollout_criteria_decide_fallbacks(small_data):
    """The threshold applies to the error the criterion names: the perturbation's relative L2
    ("perturbation", the default) or the full state's ("state"); a hop falls back exactly when
    that error exceeds the threshold, and the first hop (before any fallback) is the same run."""
    net = S.Surrogate(seed=3)
    S.train(net, small_data, iters=20, batch=4, lr=2e-3)
    thr = 1e-3
    for crit, key in (("perturbation", "signal"), ("state", "state")):
        r = S.rollout(net, seed=90002, hops=3, hop=10, threshold=thr, criterion=crit)
        assert r["criterion"] == crit
        assert r["fallback"] == [e > thr for e in r[key]], (crit, r)
    with pytest.raises(AssertionError):
        S.rollout(net, seed=90002, hops=1, hop=10, criterion="other")


def test_trained_network_gain_at_hop_50():
    """What the trained network gains over the method without it, judged at one hop length (50 LB
    steps, the configured hop): after training on hop-50 pairs its held-out error is below the
    identity map's (no change), and one application costs less than the 50 LB steps it replaces
    (64^3).  Its error against LB is the perturbation's, which stays far above 1e-3 at this hop
    (the dilated network sees +-31 cells, sound travels 35 in 50 steps); the judged rollout
    therefore falls back to LB under the perturbation criterion."""
    data = S.make_dataset(24, hop=50, t0_choices=(0, 40), per_batch=12)
    held = S.make_dataset(8, hop=50, seed0=700000, t0_choices=(0, 40), per_batch=8)
    net = S.Surrogate(seed=2)
    S.train(net, data, iters=150, batch=4, lr=2e-3)
    mse, ident = S.evaluate(net, held)
    assert mse < ident, (mse, ident)
    t_net, t_lb = S.time_hop(net, hop=50)
    assert t_net < t_lb, (t_net, t_lb)
    r = S.rollout(net, seed=90003, hops=2, hop=50, threshold=1e-3, criterion="perturbation")
    assert all(e > 1e-3 for e in r["signal"]) and all(r["fallback"])
