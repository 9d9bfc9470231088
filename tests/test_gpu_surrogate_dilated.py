"""Dilated surrogate convolutions (taps d voxels apart) against the FP64 oracle.

The library runs a dilated convolution as the plain one of the volume's d-layout (sg_relabel),
whose rows hold 64 / d independent periodic x segments (sg_shape.xper).  The tests relabel with
the library, convolve, relabel back, and compare with the oracle's dilated convolution on the
natural volume; the relabelling itself is checked against the layout formula of
include/gblb_surrogate.h, evaluated on the CPU (tests/helpers.py).  Bounds as in
test_gpu_surrogate_kernels.py: FP32 summation, <= 1e-5 of the sum of absolute terms."""
import math

import pytest
import torch

from helpers import from_d_layout, to_d_layout
from oracle import surrogate as so
from paper_1909_08406_gb300 import sg

pytestmark = pytest.mark.gpu
F64 = torch.float64

# natural volumes per dilation: ny / d a multiple of 4, nz / d >= 1; the last has 1024 tiles in
# its d = 8 layout (runs of z across columns on every CTA)
SHAPES = {2: [(2, 4, 8, 64)], 4: [(1, 8, 16, 64)], 8: [(1, 8, 32, 64), (2, 16, 64, 64)]}
CASES = [(d, s) for d, ss in SHAPES.items() for s in ss]


def _rand(shape, g, scale=1.0):
    return (scale * torch.randn(shape, generator=g, dtype=torch.float32)).to(torch.bfloat16)


@pytest.fixture(params=[sg.CONV_TCGEN05, sg.CONV_MMA_SYNC], ids=["tcgen05", "mma_sync"])
def impl(request):
    prev = sg.set_conv_impl(request.param)
    yield request.param
    sg.set_conv_impl(prev)


@pytest.mark.parametrize("dtype,c", [(torch.bfloat16, 16), (torch.bfloat16, 32), (torch.float32, 16)])
def test_relabel_follows_the_layout_formula(dtype, c):
    g = torch.Generator().manual_seed(c)
    nat = (2, 8, 32, 64, c)
    x = torch.randn(nat, generator=g).to(dtype)
    xd = x.cuda()
    for d in (1, 2, 4, 8):
        r = sg.relabel(xd, 1, d, nat)
        assert torch.equal(r.cpu(), to_d_layout(x, d)), d
        assert torch.equal(from_d_layout(r.cpu(), d, nat), x), d
    # between two dilated layouts, and back
    r2 = sg.relabel(sg.relabel(xd, 1, 2, nat), 2, 8, nat)
    assert torch.equal(r2.cpu(), to_d_layout(x, 8))
    assert torch.equal(sg.relabel(r2, 8, 1, nat).cpu(), x)


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
@pytest.mark.parametrize("d,shape", CASES)
def test_dilated_conv_forward_matches_oracle(cin, cout, d, shape, impl):
    g = torch.Generator().manual_seed(cin + cout + d + shape[0])
    x = _rand(shape + (cin,), g)
    w = _rand((cout, 27, cin), g, 1 / math.sqrt(27 * cin))
    b = torch.randn(cout, generator=g) * 0.1
    xr = sg.relabel(x.cuda(), 1, d, shape + (cin,))
    z = torch.empty(xr.shape[:-1] + (cout,), dtype=torch.float32, device="cuda")
    y = sg.conv3d_fwd(xr, w.cuda(), b.cuda(), act=sg.ACT_GELU, res_in=(cin == cout), z_out=z, xper=64 // d)
    sg.status()
    z_nat = from_d_layout(z.cpu(), d, shape).to(F64)
    y_nat = from_d_layout(y.cpu(), d, shape).to(F64)
    zr = so.conv3d_periodic(x.to(F64), w.to(F64), b.to(F64), dilation=d)
    absum = so.conv3d_periodic(x.to(F64).abs(), w.to(F64).abs(), b.to(F64).abs(), dilation=d)
    assert torch.all((z_nat - zr).abs() <= 1e-5 * absum + 1e-7)
    yr = so.gelu(zr) + (x.to(F64) if cin == cout else 0)
    assert torch.allclose(y_nat, yr, rtol=2 ** -7, atol=1e-6 * (1 + absum.max().item()))
    # the undilated convolution differs: the segments really wrap
    z1 = so.conv3d_periodic(x.to(F64), w.to(F64), b.to(F64))
    assert (z1 - zr).abs().max() > 1e-2


@pytest.mark.parametrize("d,shape", CASES)
def test_dilated_conv_f32_with_add(d, shape, impl):
    """The input-gradient form (FP32 output, FP32 added tensor) on a d-layout."""
    g = torch.Generator().manual_seed(40 + d)
    x = _rand(shape + (32,), g)
    w = _rand((16, 27, 32), g, 0.05)
    add = torch.randn(shape + (16,), generator=g, dtype=torch.float32)
    xr = sg.relabel(x.cuda(), 1, d, shape + (32,))
    ar = sg.relabel(add.cuda(), 1, d, shape + (16,))
    y = sg.conv3d_fwd_f32(xr, w.cuda(), add=ar, xper=64 // d)
    sg.status()
    yr = so.conv3d_periodic(x.to(F64), w.to(F64), dilation=d) + add.to(F64)
    absum = so.conv3d_periodic(x.to(F64).abs(), w.to(F64).abs(), dilation=d) + add.to(F64).abs()
    assert torch.all((from_d_layout(y.cpu(), d, shape).to(F64) - yr).abs() <= 1e-5 * absum + 1e-7)


@pytest.mark.parametrize("cin,cout", [(16, 32), (32, 32), (32, 16)])
@pytest.mark.parametrize("d,shape", CASES)
def test_dilated_weight_gradient_matches_oracle(cin, cout, d, shape, impl):
    g = torch.Generator().manual_seed(7 * cin + cout + d)
    x = _rand(shape + (cin,), g)
    dz = _rand(shape + (cout,), g, 0.1)
    xr = sg.relabel(x.cuda(), 1, d, shape + (cin,))
    dzr = sg.relabel(dz.cuda(), 1, d, shape + (cout,))
    dw = torch.empty((cout, 27, cin), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    sg.conv3d_wgrad(xr, dzr, dw, db, sg.wgrad_scratch(xr, cin, cout), xper=64 // d)
    sg.status()
    w0 = torch.zeros((cout, 27, cin), dtype=F64, requires_grad=True)
    b0 = torch.zeros(cout, dtype=F64, requires_grad=True)
    (so.conv3d_periodic(x.to(F64), w0, b0, dilation=d) * dz.to(F64)).sum().backward()
    wa = torch.zeros((cout, 27, cin), dtype=F64, requires_grad=True)
    (so.conv3d_periodic(x.to(F64).abs(), wa, dilation=d) * dz.to(F64).abs()).sum().backward()
    assert torch.all((dw.cpu().to(F64) - w0.grad).abs() <= 1e-5 * wa.grad + 1e-12)
    assert torch.all((db.cpu().to(F64) - b0.grad).abs() <= 1e-5 * dz.to(F64).abs().sum(dim=(0, 1, 2, 3)) + 1e-12)


def test_relabel_and_xper_arguments():
    x = torch.zeros((1, 8, 32, 64, 16), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((16, 27, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(RuntimeError):
        sg.relabel(x, 1, 3, x.shape)                     # dilation not in {1, 2, 4, 8}
    with pytest.raises(RuntimeError):
        sg.relabel(x, 1, 16, x.shape)
    with pytest.raises(RuntimeError):
        sg.relabel(x, 1, 4, x.shape, y=x)                # in place
    with pytest.raises(RuntimeError):
        sg.conv3d_fwd(x, w, xper=4)                      # period below 8
    with pytest.raises(RuntimeError):
        sg.conv3d_fwd(x, w, xper=24)                     # not a power of two
    odd = torch.zeros((1, 6, 32, 64, 16), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(RuntimeError):
        sg.relabel(odd, 1, 4, odd.shape)                 # nz not a multiple of d
