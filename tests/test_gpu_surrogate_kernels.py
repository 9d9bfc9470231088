"""Surrogate kernels against the FP64 oracle on identical BF16 inputs.

Bounds: the kernels read the same BF16 values the oracle reads in FP64 and
accumulate products exactly representable in FP32, so the FP32 results differ
from the oracle only by FP32 summation error: <= 1e-5 of the sum of absolute
terms for the convolution (K <= 864) and the weight gradient.  BF16 outputs
are compared after allowing one BF16 rounding (2^-8 relative)."""
import math

import numpy as np
import pytest
import torch

from oracle import surrogate as so
from paper_1909_08406_gb300 import sg

pytestmark = pytest.mark.gpu
F64 = torch.float64


def _rand(shape, g, scale=1.0):
    return (scale * torch.randn(shape, generator=g, dtype=torch.float32)).to(torch.bfloat16)


@pytest.fixture(params=[sg.CONV_TCGEN05, sg.CONV_MMA_SYNC], ids=["tcgen05", "mma_sync"])
def impl(request):
    prev = sg.set_conv_impl(request.param)
    yield request.param
    sg.set_conv_impl(prev)


# tcgen05 kernel: (2, 3, 4, 64) 12 tiles, one per CTA, with rows wrapping in y; (1, 4, 8, 64)
# interior and wrapping row pairs; (4, 6, 64, 64) 768 tiles over at most 152 CTAs: runs of z that
# end inside a column and continue in the next, both epilogue groups, the accumulator ring reused
@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16), (16, 16)])
@pytest.mark.parametrize("shape", [(1, 4, 8, 64), (2, 3, 4, 64), (4, 6, 64, 64)])
def test_conv_forward_matches_oracle(cin, cout, shape, impl):
    g = torch.Generator().manual_seed(cin + cout + shape[0])
    x = _rand(shape + (cin,), g)
    w = _rand((cout, 27, cin), g, 1 / math.sqrt(27 * cin))
    b = torch.randn(cout, generator=g) * 0.1
    xd, wd, bd = x.cuda(), w.cuda(), b.cuda()
    z = torch.empty(shape + (cout,), dtype=torch.float32, device="cuda")
    y = sg.conv3d_fwd(xd, wd, bd, act=sg.ACT_GELU, res_in=(cin == cout), z_out=z)
    torch.cuda.synchronize()
    zr = so.conv3d_periodic(x.to(F64), w.to(F64), b.to(F64))
    absum = so.conv3d_periodic(x.to(F64).abs(), w.to(F64).abs(), b.to(F64).abs())
    assert torch.all((z.cpu().to(F64) - zr).abs() <= 1e-5 * absum + 1e-7)
    yr = so.gelu(zr) + (x.to(F64) if cin == cout else 0)
    assert torch.allclose(y.cpu().to(F64), yr, rtol=2 ** -7, atol=1e-6 * (1 + absum.max().item()))
    sg.status()


def test_conv_forward_f32_with_add(impl):
    g = torch.Generator().manual_seed(3)
    shape = (1, 2, 4, 64)
    x = _rand(shape + (32,), g)
    w = _rand((16, 27, 32), g, 0.05)
    add = torch.randn(shape + (16,), generator=g, dtype=torch.float32)
    y = sg.conv3d_fwd_f32(x.cuda(), w.cuda(), add=add.cuda())
    sg.status()
    ref = so.conv3d_periodic(x.to(F64), w.to(F64)) + add.to(F64)
    assert torch.allclose(y.cpu().to(F64), ref, rtol=1e-5, atol=1e-5)


# tcgen05 kernel (rows in pairs): (2, 4, 8, 64) one pair per CTA (32 pairs), windows wrapping in y
# and z; (3, 5, 12, 64) 90 pairs, one per CTA, odd nz; (4, 6, 64, 64) 768 pairs over at most 152
# CTAs, five or six each (accumulation over pairs, both operand rings wrapping)
@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16), (16, 16)])
@pytest.mark.parametrize("shape", [(2, 4, 8, 64), (3, 5, 12, 64), (4, 6, 64, 64)])
def test_weight_and_bias_gradient_matches_oracle(cin, cout, shape, impl):
    g = torch.Generator().manual_seed(10 + cin + cout)
    x = _rand(shape + (cin,), g)
    dz = _rand(shape + (cout,), g)
    dw = torch.empty((cout, 27, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    xd, dzd = x.cuda(), dz.cuda()
    sg.conv3d_wgrad(xd, dzd, dw, db, sg.wgrad_scratch(xd, cin, cout))
    sg.status()
    # oracle: d/dw of sum(dz * conv(x, w)) by autograd in FP64
    w0 = torch.zeros((cout, 27, cin), dtype=F64, requires_grad=True)
    b0 = torch.zeros(cout, dtype=F64, requires_grad=True)
    (so.conv3d_periodic(x.to(F64), w0, b0) * dz.to(F64)).sum().backward()
    # element-wise bound: FP32 summation error of each element's own sum of absolute terms
    wa = torch.zeros((cout, 27, cin), dtype=F64, requires_grad=True)
    (so.conv3d_periodic(x.to(F64).abs(), wa) * dz.to(F64).abs()).sum().backward()
    assert torch.all((dw.cpu().to(F64) - w0.grad).abs() <= 1e-5 * wa.grad + 1e-12)
    assert torch.allclose(db.cpu().to(F64), b0.grad, rtol=1e-5, atol=1e-3)


@pytest.mark.parametrize("cin,cout", [(32, 32), (32, 16)])
def test_input_gradient_is_conv_with_transposed_weights(cin, cout, impl):
    g = torch.Generator().manual_seed(20 + cout)
    shape = (1, 4, 4, 64)
    x = _rand(shape + (cin,), g)
    w = _rand((cout, 27, cin), g, 1 / math.sqrt(27 * cin))
    dz = _rand(shape + (cout,), g)
    wt = sg.transpose_weights(w.cuda())
    dx = sg.conv3d_fwd_f32(dz.cuda(), wt)
    torch.cuda.synchronize()
    xr = x.to(F64).requires_grad_(True)
    (so.conv3d_periodic(xr, w.to(F64)) * dz.to(F64)).sum().backward()
    assert torch.allclose(dx.cpu().to(F64), xr.grad, rtol=1e-5, atol=1e-5)


def test_gelu_backward_matches_oracle():
    g = torch.Generator().manual_seed(5)
    z = 3 * torch.randn(10000, generator=g, dtype=torch.float32)
    dy = torch.randn(10000, generator=g, dtype=torch.float32)
    dz = sg.act_backward(dy.cuda(), z.cuda(), sg.ACT_GELU)
    torch.cuda.synchronize()
    zr = z.to(F64).requires_grad_(True)
    (so.gelu(zr) * dy.to(F64)).sum().backward()
    assert torch.allclose(dz.cpu().to(F64), zr.grad, rtol=2 ** -7, atol=1e-6)


def test_mse_and_rel_l2():
    g = torch.Generator().manual_seed(6)
    shape = (2, 2, 4, 64, 16)
    a = _rand(shape, g)
    b = _rand(shape, g)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dpred = torch.empty(shape, dtype=torch.float32, device="cuda")
    scratch = sg.reduce_scratch()
    sg.mse(a.cuda(), b.cuda(), 5, loss, dpred, scratch)
    rel = torch.empty(2, dtype=torch.float32, device="cuda")
    sg.rel_l2(a.cuda(), b.cuda(), 5, rel, scratch)
    torch.cuda.synchronize()
    d = (a.to(F64) - b.to(F64))[..., :5]
    assert loss.item() == pytest.approx((d * d).mean().item(), rel=1e-5)
    ref_dp = torch.zeros(shape, dtype=F64)
    ref_dp[..., :5] = 2 * d / d.numel()
    assert torch.allclose(dpred.cpu().to(F64), ref_dp, rtol=1e-5, atol=1e-12)
    for k in range(2):
        r = (d[k] ** 2).sum().sqrt() / (b.to(F64)[k, ..., :5] ** 2).sum().sqrt()
        assert rel[k].item() == pytest.approx(r.item(), rel=1e-5)
