"""Pins of the surrogate oracle: the periodic convolution against explicit loops,
GELU against its definition, and the autograd gradients against central
finite differences on a tiny network."""
import math

import numpy as np
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


def test_gelu_definition():
    z = torch.linspace(-4, 4, 17, dtype=F64)
    ref = torch.tensor([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z.tolist()], dtype=F64)
    assert torch.allclose(so.gelu(z), ref, rtol=0, atol=1e-15)


def test_gradients_match_finite_differences():
    g = torch.Generator().manual_seed(1)
    shape = (1, 3, 4, 4)
    x = torch.zeros(shape + (16,), dtype=F64)
    x[..., :5] = 0.5 * torch.randn(shape + (5,), generator=g, dtype=F64)
    t = x.clone()
    t[..., :5] += 0.1 * torch.randn(shape + (5,), generator=g, dtype=F64)
    ws = [0.2 * torch.randn((co, 27, ci), generator=g, dtype=F64) / math.sqrt(27 * ci) for ci, co, _, _ in so.LAYERS]
    bs = [0.05 * torch.randn(co, generator=g, dtype=F64) for _, co, _, _ in so.LAYERS]
    loss, gw, gb, _ = so.loss_and_grads(x, t, ws, bs)
    rng = np.random.default_rng(2)
    h = 1e-6
    for layer in (0, 2, 5):
        for _ in range(4):
            idx = tuple(int(rng.integers(0, n)) for n in ws[layer].shape)
            wp = [w.clone() for w in ws]
            wm = [w.clone() for w in ws]
            wp[layer][idx] += h
            wm[layer][idx] -= h
            lp = so.mse(so.forward(x, wp, bs)[0], t, 5).item()
            lm = so.mse(so.forward(x, wm, bs)[0], t, 5).item()
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gw[layer][idx].item()) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (layer, idx)
        k = int(rng.integers(0, bs[layer].shape[0]))
        bp = [b.clone() for b in bs]
        bm = [b.clone() for b in bs]
        bp[layer][k] += h
        bm[layer][k] -= h
        fd = (so.mse(so.forward(x, ws, bp)[0], t, 5).item() - so.mse(so.forward(x, ws, bm)[0], t, 5).item()) / (2 * h)
        assert abs(fd - gb[layer][k].item()) <= 1e-7 * max(1.0, abs(fd)) + 1e-9
