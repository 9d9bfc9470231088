"""FP64 CPU oracle of the surrogate network (3D convolutional neural operator).

TEST INFRASTRUCTURE ONLY (tests and smoke check); shares no code with the
CUDA kernels.  Plain PyTorch CPU ops in float64: the periodic 3x3x3
convolution is torch's conv3d on a circularly padded input, gradients come
from autograd.  Layouts follow the C ABI (include/gblb_surrogate.h):
activations x[b][z][y][x][c] (channels last), weights w[cout][tap][cin] with
tap = (dz+1)*9 + (dy+1)*3 + (dx+1), so that
    z[v][co] = bias[co] + sum_{tap,ci} w[co][tap][ci] x[v + d(tap)][ci].

With dilation d the taps sit d voxels apart,
    z[v][co] = bias[co] + sum_{tap,ci} w[co][tap][ci] x[v + d * d(tap)][ci],
still periodic over the volume.

Network (6 layers): 16 -> 32 (GELU), four 32 -> 32 residual layers
y = x + GELU(conv(x)), and 32 -> 16 linear with the input added
(prediction = input + conv(h)), each layer with its own dilation.  GELU is
z Phi(z) with the Gaussian CDF Phi.
"""
import math

import torch
import torch.nn.functional as F

F64 = torch.float64
LAYERS = [(16, 32, "gelu", False), (32, 32, "gelu", True), (32, 32, "gelu", True), (32, 32, "gelu", True),
          (32, 32, "gelu", True), (32, 16, "none", False)]


def w_to_conv(w):
    """[cout][27][cin] -> torch conv3d weight [cout][cin][3][3][3] (kd, kh, kw) = (dz+1, dy+1, dx+1)."""
    co, taps, ci = w.shape
    assert taps == 27
    return w.permute(0, 2, 1).reshape(co, ci, 3, 3, 3)


def conv3d_periodic(x, w, bias=None, dilation=1):
    """x: [b][z][y][x][cin] float64, w: [cout][27][cin] -> [b][z][y][x][cout]; taps `dilation`
    voxels apart (the circular padding is as wide)."""
    d = dilation
    xp = x.permute(0, 4, 1, 2, 3)
    for dim in (2, 3, 4):  # periodic padding: index (i - d) mod n for i = 0 .. n + 2d - 1
        n = xp.shape[dim]
        xp = xp.index_select(dim, torch.arange(-d, n + d) % n)
    out = F.conv3d(xp, w_to_conv(w), bias=bias, dilation=d)
    return out.permute(0, 2, 3, 4, 1)


def conv3d_bruteforce(x, w, bias=None, dilation=1):
    """The same periodic convolution by explicit loops (small inputs only)."""
    b_, nz, ny, nx, ci = x.shape
    co = w.shape[0]
    out = torch.zeros((b_, nz, ny, nx, co), dtype=F64)
    for b in range(b_):
        for z in range(nz):
            for y in range(ny):
                for xx in range(nx):
                    acc = torch.zeros(co, dtype=F64) if bias is None else bias.clone().to(F64)
                    for tap in range(27):
                        dz, dy, dx = (dilation * (tap // 9 - 1), dilation * ((tap // 3) % 3 - 1),
                                      dilation * (tap % 3 - 1))
                        v = x[b, (z + dz) % nz, (y + dy) % ny, (xx + dx) % nx]
                        acc = acc + w[:, tap, :] @ v
                    out[b, z, y, xx] = acc
    return out


def gelu(z):
    return 0.5 * z * (1.0 + torch.erf(z / math.sqrt(2.0)))


def forward(x, weights, biases, dilations=None):
    """Whole network (layer k with dilation dilations[k], default 1); returns (prediction, list of
    (pre-activation, layer output))."""
    dil = dilations or [1] * len(LAYERS)
    h = x
    trace = []
    for (ci, co, act, res), w, b, d in zip(LAYERS, weights, biases, dil):
        z = conv3d_periodic(h, w, b, dilation=d)
        y = gelu(z) if act == "gelu" else z
        if res:
            y = h + y
        trace.append((z, y))
        h = y
    pred = x + h  # last layer: prediction = input + conv
    return pred, trace


def mse(pred, target, nch):
    d = pred[..., :nch] - target[..., :nch]
    return (d * d).mean()


def loss_and_grads(x, target, weights, biases, nch=5, dilations=None):
    """FP64 loss and gradients of all weights and biases by autograd."""
    ws = [w.detach().clone().to(F64).requires_grad_(True) for w in weights]
    bs = [b.detach().clone().to(F64).requires_grad_(True) for b in biases]
    pred, _ = forward(x.to(F64), ws, bs, dilations)
    loss = mse(pred, target.to(F64), nch)
    loss.backward()
    return loss.item(), [w.grad for w in ws], [b.grad for b in bs], pred.detach()
