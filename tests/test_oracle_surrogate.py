"""Pins of the surrogate oracle: the periodic convolution (plain and dilated) against explicit
loops, an impulse and the case where the dilation equals the period; GELU against its definition;
the autograd gradients against central finite differences on a tiny network, plain and dilated."""
import math

import numpy as np
import pytest
import torch

from oracle import surrogate as so

F64 = torch.float64


def test_conv3d_periodic_matches_explicit_loops():
    g = torch.Generator().manual_seed(0)
    x = torch.randn((2, 3, 4, 5, 3), generator=g, dtype=F64)
    w = torch.randn((4, 27, 3), generator=g, dtype=F64)
    b = torch.randn(4, generator=g, dtype=F64)
    assert torch.allclose(so.conv3d_periodic(x, w, b), so.conv3d_bruteforce(x, w, b), rtol=0, atol=1e-12)


def test_conv3d_tap_convention():
    """A single nonzero tap (dz, dy, dx) = (1, 0, -1) reads x[z+1][y][x-1]."""
    x = torch.zeros((1, 4, 4, 4, 1), dtype=F64)
    x[0, 2, 1, 0, 0] = 1.0
    w = torch.zeros((1, 27, 1), dtype=F64)
    w[0, (1 + 1) * 9 + (0 + 1) * 3 + (-1 + 1), 0] = 1.0
    out = so.conv3d_periodic(x, w)
    # out[z][y][x] = x[z+1][y][x-1] -> nonzero at z = 1, y = 1, x = 1
    assert out[0, 1, 1, 1, 0] == 1.0 and out.abs().sum() == 1.0


@pytest.mark.parametrize("d", [2, 3])
def test_dilated_conv3d_matches_explicit_loops(d):
    g = torch.Generator().manual_seed(d)
    x = torch.randn((1, 4, 6, 7, 2), generator=g, dtype=F64)
    w = torch.randn((3, 27, 2), generator=g, dtype=F64)
    b = torch.randn(3, generator=g, dtype=F64)
    got = so.conv3d_periodic(x, w, b, dilation=d)
    assert torch.allclose(got, so.conv3d_bruteforce(x, w, b, dilation=d), rtol=0, atol=1e-12)
    assert not torch.allclose(got, so.conv3d_periodic(x, w, b), rtol=0, atol=1e-6)


def test_dilated_conv3d_impulse_response():
    """A unit impulse at (z, y, x) = (3, 5, 2) and one tap (dz, dy, dx) = (-1, +1, +1) at dilation 4:
    out[v] = x[v + 4 (dz, dy, dx)], nonzero only at v = (3 + 4, 5 - 4, 2 - 4) mod 8."""
    x = torch.zeros((1, 8, 8, 8, 1), dtype=F64)
    x[0, 3, 5, 2, 0] = 1.0
    w = torch.zeros((1, 27, 1), dtype=F64)
    w[0, (-1 + 1) * 9 + (1 + 1) * 3 + (1 + 1), 0] = 1.0
    out = so.conv3d_periodic(x, w, dilation=4)
    assert out[0, 7, 1, 6, 0] == 1.0 and out.abs().sum() == 1.0


def test_dilation_equal_to_the_period_folds_the_taps():
    """With dilation d equal to the period along every axis, each tap reads the node itself: the
    convolution is the sum of the 27 taps applied to the voxel."""
    g = torch.Generator().manual_seed(7)
    x = torch.randn((2, 4, 4, 4, 3), generator=g, dtype=F64)
    w = torch.randn((5, 27, 3), generator=g, dtype=F64)
    out = so.conv3d_periodic(x, w, dilation=4)
    ref = torch.einsum("ci,bzyxi->bzyxc", w.sum(dim=1), x)
    assert torch.allclose(out, ref, rtol=0, atol=1e-12)


def test_gelu_definition():
    z = torch.linspace(-4, 4, 17, dtype=F64)
    ref = torch.tensor([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z.tolist()], dtype=F64)
    assert torch.allclose(so.gelu(z), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dil", [None, (1, 2, 2, 4, 2, 1)])
def test_gradients_match_finite_differences(dil):
    g = torch.Generator().manual_seed(1)
    shape = (1, 3, 4, 4)
    x = torch.zeros(shape + (16,), dtype=F64)
    x[..., :5] = 0.5 * torch.randn(shape + (5,), generator=g, dtype=F64)
    t = x.clone()
    t[..., :5] += 0.1 * torch.randn(shape + (5,), generator=g, dtype=F64)
    ws = [0.2 * torch.randn((co, 27, ci), generator=g, dtype=F64) / math.sqrt(27 * ci) for ci, co, _, _ in so.LAYERS]
    bs = [0.05 * torch.randn(co, generator=g, dtype=F64) for _, co, _, _ in so.LAYERS]
    loss, gw, gb, _ = so.loss_and_grads(x, t, ws, bs, dilations=dil)
    rng = np.random.default_rng(2)
    h = 1e-6
    for layer in (0, 2, 5):
        for _ in range(4):
            idx = tuple(int(rng.integers(0, n)) for n in ws[layer].shape)
            wp = [w.clone() for w in ws]
            wm = [w.clone() for w in ws]
            wp[layer][idx] += h
            wm[layer][idx] -= h
            lp = so.mse(so.forward(x, wp, bs, dil)[0], t, 5).item()
            lm = so.mse(so.forward(x, wm, bs, dil)[0], t, 5).item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gw[layer][idx].item()) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (layer, idx)
        k = int(rng.integers(0, bs[layer].shape[0]))
        bp = [b.clone() for b in bs]
        bm = [b.clone() for b in bs]
        bp[layer][k] += h
        bm[layer][k] -= h
        fd = (so.mse(so.forward(x, ws, bp, dil)[0], t, 5).item() -
              so.mse(so.forward(x, ws, bm, dil)[0], t, 5).item()) / (2 * h)
        assert abs(fd - gb[layer][k].item()) <= 1e-7 * max(1.0, abs(fd)) + 1e-9
