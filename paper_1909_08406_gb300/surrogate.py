"""Learned surrogate: a 3D convolutional neural operator that advances the
macroscopic fields (rho, u, theta) of the RD3Q41 solver K lattice Boltzmann
steps per application, trained on data the solver generates, with the plain
LB method as its fallback and as the arbiter of its rollout error.

Network (6 layers, 3x3x3 periodic convolutions, BF16 weights and activations,
FP32 accumulation, all in the kernels of include/gblb_surrogate.h):
    h1 = GELU(conv(x))                       16 -> 32
    h2..h5 = h + GELU(conv(h))               32 -> 32 (residual)
    pred = x + conv(h5)                      32 -> 16 (5 used)
on the A sub-lattice fields of a 64^3 grid (channels (rho-1)/s, u/s, (theta/theta0-1)/s).
The taps of layer k sit DILATIONS[k] voxels apart (1, 2, 4, 8, 8, 8: a receptive field of
+-31 voxels, against +-6 undilated); each layer runs on its input's d-layout (sg.relabel), where
the dilated convolution is the plain one with rows of 64 / d-voxel periodic segments.
Training: mean-squared error, Adam on FP32 master weights.  Orchestration
lives here (argument marshalling, loops); every arithmetic step is a kernel
of libgblb.so.  torch supplies device memory only.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import lb, sg
from . import workloads as wl

LAYERS = [(16, 32, sg.ACT_GELU, False), (32, 32, sg.ACT_GELU, True), (32, 32, sg.ACT_GELU, True),
          (32, 32, sg.ACT_GELU, True), (32, 32, sg.ACT_GELU, True), (32, 16, sg.ACT_NONE, False)]
DILATIONS = (1, 2, 4, 8, 8, 8)
NCH = 5           # physical channels
SCALES = (5e-3, 5e-3, 5e-3)
NU = 0.01


class Surrogate:
    def __init__(self, seed=0, device="cuda", dilations=DILATIONS):
        rng = np.random.default_rng(seed)
        self.device = device
        self.dil = tuple(dilations)
        self.w32, self.b32, self.w16 = [], [], []
        for k, (ci, co, act, res) in enumerate(LAYERS):
            fan = 27 * ci
            gain = 0.0 if k == len(LAYERS) - 1 else (0.5 if res else 1.0)
            w = torch.from_numpy((gain / math.sqrt(fan)) * rng.standard_normal((co, 27, ci))).float()
            if ci == 16:
                w[:, :, NCH:] = 0  # padded input channels carry no weight
            self.w32.append(w.to(device))
            self.b32.append(torch.zeros(co, dtype=torch.float32, device=device))
            self.w16.append(torch.empty((co, 27, ci), dtype=torch.bfloat16, device=device))
        self.params = [p for pair in zip(self.w32, self.b32) for p in pair]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.g = [torch.zeros_like(p) for p in self.params]
        self.t = 0
        self._round_weights()

    def _round_weights(self):
        # BF16 copies of the FP32 master weights (an Adam call with a zero step only rounds)
        for w32, w16, m, v in zip(self.w32, self.w16, self.m[0::2], self.v[0::2]):
            zero = torch.zeros_like(w32)
            sg.adam(w32, zero, torch.zeros_like(m), torch.zeros_like(v), w16, 0.0, 1)

    def forward(self, x, train=False):
        """x: [B][nz][ny][64][16] BF16 -> prediction (BF16, same shape).  Keeps, for the backward
        pass, each layer's input (cache) and FP32 pre-activation (zs) in that layer's d-layout."""
        nat = tuple(x.shape[:-1])
        h, cur = x, 1
        self.cache, self.zs = [], []
        for k, (ci, co, act, res) in enumerate(LAYERS):
            d = self.dil[k]
            if d != cur:
                h = sg.relabel(h, cur, d, nat + (h.shape[-1],))
                cur = d
            last = k == len(LAYERS) - 1
            add = None
            if last:
                add = x if d == 1 else sg.relabel(x, 1, d, nat + (x.shape[-1],))
            z = torch.empty(h.shape[:-1] + (co,), dtype=torch.float32, device=x.device) if train else None
            self.cache.append(h)
            h = sg.conv3d_fwd(h, self.w16[k], self.b32[k], act=act, res_in=res, add=add, z_out=z, xper=64 // d)
            self.zs.append(z)
        return h if cur == 1 else sg.relabel(h, cur, 1, nat + (h.shape[-1],))

    def backward(self, dpred, scratch_w, trace=None):
        """Gradients of all weights and biases from dL/dpred (FP32, [..][16], natural layout).  If
        `trace` is a dict, it receives per layer k, in the layer's d-layout, the gradient arriving
        at the layer's output ("dh_out", FP32), the pre-activation gradient ("dz", BF16) and the
        gradient passed to its input ("dh_in", FP32; layers k > 0)."""
        nat = tuple(dpred.shape[:-1])
        dh, cur = dpred, 1
        for k in range(len(LAYERS) - 1, -1, -1):
            ci, co, act, res = LAYERS[k]
            d = self.dil[k]
            if d != cur:
                dh = sg.relabel(dh, cur, d, nat + (dh.shape[-1],))
                cur = d
            dz = sg.act_backward(dh, self.zs[k], act)
            sg.conv3d_wgrad(self.cache[k], dz, self.g[2 * k], self.g[2 * k + 1], scratch_w[(ci, co)], xper=64 // d)
            if trace is not None:
                trace[k] = {"dh_out": dh, "dz": dz}
            if k > 0:
                wt = sg.transpose_weights(self.w16[k])
                dh = sg.conv3d_fwd_f32(dz, wt, add=dh if res else None, xper=64 // d)
                if trace is not None:
                    trace[k]["dh_in"] = dh

    def adam_step(self, lr):
        self.t += 1
        for k in range(len(LAYERS)):
            sg.adam(self.w32[k], self.g[2 * k], self.m[2 * k], self.v[2 * k], self.w16[k], lr, self.t)
            sg.adam(self.b32[k], self.g[2 * k + 1], self.m[2 * k + 1], self.v[2 * k + 1], None, lr, self.t)


def _fields_buffers(n, device="cuda"):
    return (torch.empty((2, n, n, n), dtype=torch.float64, device=device),
            torch.empty((3, 2, n, n, n), dtype=torch.float64, device=device),
            torch.empty((2, n, n, n), dtype=torch.float64, device=device))


@dataclass
class Dataset:
    x: torch.Tensor
    y: torch.Tensor
    t0: list = field(default_factory=list)


def make_dataset(count, hop=50, n=64, seed0=5000, t0_choices=(0, 100, 250, 500), per_batch=32, device="cuda"):
    """Pairs (state at t0, state at t0 + hop) from `count` LB runs of Gaussian pulses with theta
    perturbations (seeds seed0..), FP32 LB on an n^3 grid, advanced in batches."""
    th0 = lb.lb_theta0()
    tau = NU / th0
    X = torch.empty((count, n, n, n, 16), dtype=torch.bfloat16, device=device)
    Y = torch.empty_like(X)
    rho, u, th = _fields_buffers(n, device)
    t0s = [t0_choices[k % len(t0_choices)] for k in range(count)]
    order = sorted(range(count), key=lambda k: t0s[k])
    for start in range(0, count, per_batch):
        ids = order[start:start + per_batch]
        groups = {}
        for k in ids:
            groups.setdefault(t0s[k], []).append(k)
        for t0, ks in groups.items():
            b = lb.lb_batch_init([(n, n, n)] * len(ks), [tau] * len(ks), "f32")
            try:
                for j, k in enumerate(ks):
                    f = wl.gaussian_pulse_sample(n, th0, seed0 + k, device=device)
                    lb.lb_set_fields(lb.lb_batch_sim(b, j), f["rho"], f["u"], f["theta"])
                lb.lb_batch_step(b, t0, lb.LB_BATCH_GRAPH)
                for j, k in enumerate(ks):
                    lb.lb_get_moments(lb.lb_batch_sim(b, j), rho, u, th)
                    sg.pack_fields(X[k:k + 1], 0, rho, u, th, th0, SCALES)
                lb.lb_batch_step(b, hop, lb.LB_BATCH_GRAPH)
                for j, k in enumerate(ks):
                    lb.lb_get_moments(lb.lb_batch_sim(b, j), rho, u, th)
                    sg.pack_fields(Y[k:k + 1], 0, rho, u, th, th0, SCALES)
                lb.lb_batch_sync(b)
            finally:
                lb.lb_batch_destroy(b)
    return Dataset(X, Y, t0s)


def train(net, data, iters, batch=4, lr=1e-3, seed=0, log_every=0):
    """Adam on minibatches drawn (seeded) from the dataset; returns the loss history (host floats)."""
    rng = np.random.default_rng(seed)
    count = data.x.shape[0]
    shape = (batch,) + tuple(data.x.shape[1:])
    xb = torch.empty(shape, dtype=torch.bfloat16, device=data.x.device)
    yb = torch.empty_like(xb)
    dpred = torch.empty(shape, dtype=torch.float32, device=data.x.device)
    loss = torch.empty(1, dtype=torch.float32, device=data.x.device)
    rs = sg.reduce_scratch()
    scratch_w = {(ci, co): sg.wgrad_scratch(xb, ci, co) for ci, co, _, _ in LAYERS}
    hist = []
    for it in range(iters):
        idx = rng.integers(0, count, size=batch)
        for j, k in enumerate(idx):
            xb[j].copy_(data.x[int(k)])  # device-to-device gather of the minibatch
            yb[j].copy_(data.y[int(k)])
        pred = net.forward(xb, train=True)
        sg.mse(pred, yb, NCH, loss, dpred, rs)
        net.backward(dpred, scratch_w)
        net.adam_step(lr * (0.5 * (1 + math.cos(math.pi * it / max(1, iters)))))
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, loss.item()))
    return hist


def evaluate(net, data, batch=4):
    """Mean MSE of the network and of the identity map (no change) on a dataset."""
    loss = torch.empty(1, dtype=torch.float32, device=data.x.device)
    dpred = torch.empty((batch,) + tuple(data.x.shape[1:]), dtype=torch.float32, device=data.x.device)
    rs = sg.reduce_scratch()
    tot, ident = 0.0, 0.0
    count = data.x.shape[0]
    nb = 0
    for s in range(0, count - batch + 1, batch):
        xb, yb = data.x[s:s + batch], data.y[s:s + batch]
        pred = net.forward(xb)
        sg.mse(pred, yb, NCH, loss, dpred, rs)
        tot += loss.item()
        sg.mse(xb, yb, NCH, loss, dpred, rs)
        ident += loss.item()
        nb += 1
    return tot / nb, ident / nb


def rollout(net, seed, hops=20, hop=50, n=64, threshold=1e-3, fallback=True, criterion="perturbation"):
    """Judged rollout from one Gaussian-pulse initial condition: the surrogate advances the
    fields hop by hop; LB runs alongside as the arbiter.  After each hop the relative L2 error
    of the predicted fields against LB is measured; above `threshold` (with fallback on) the
    state is reset to LB's (an LB fallback).  Errors: over the normalised deviation channels,
    i.e. of the perturbation (rho - 1, u, theta/theta0 - 1) relative to LB's perturbation
    ('signal'), and over the full state (rho, u, theta/theta0) ('state'): with equal channel
    scales s the state error is s ||x - ref|| / sqrt(sum over A nodes of rho^2 + u^2 +
    (theta/theta0)^2), the denominator taken at rest (2 n^3; the perturbations change it by
    less than 1%).  `criterion` picks the error the threshold applies to: "perturbation"
    (the signal error) or "state".  The state is ~1 while the perturbation is ~1e-3 of it, so a
    state error of 1e-3 allows a perturbation error of order one."""
    assert criterion in ("perturbation", "state")
    th0 = lb.lb_theta0()
    tau = NU / th0
    assert SCALES[0] == SCALES[1] == SCALES[2]
    ctx = lb.lb_init((n, n, n), tau, "f32")
    rho, u, th = _fields_buffers(n)
    x = torch.empty((1, n, n, n, 16), dtype=torch.bfloat16, device="cuda")
    ref = torch.empty_like(x)
    zero = torch.zeros_like(x)
    rs = sg.reduce_scratch()
    err = torch.empty(1, dtype=torch.float32, device="cuda")
    nrm = torch.empty(1, dtype=torch.float32, device="cuda")
    out = {"signal": [], "state": [], "fallback": [], "criterion": criterion, "threshold": threshold}
    try:
        f = wl.gaussian_pulse_sample(n, th0, seed, device="cuda")
        lb.lb_set_fields(ctx, f["rho"], f["u"], f["theta"])
        lb.lb_get_moments(ctx, rho, u, th)
        sg.pack_fields(x, 0, rho, u, th, th0, SCALES)
        for _ in range(hops):
            x = net.forward(x)
            lb.lb_step(ctx, hop)
            lb.lb_get_moments(ctx, rho, u, th)
            sg.pack_fields(ref, 0, rho, u, th, th0, SCALES)
            sg.rel_l2(x, ref, NCH, err, rs)
            sg.rel_l2(ref, zero, NCH, nrm, rs)  # ||ref|| (the kernel returns ||a|| when b = 0)
            e_sig = err.item()
            e_state = SCALES[0] * e_sig * nrm.item() / math.sqrt(2.0 * n ** 3)
            fb = fallback and (e_sig if criterion == "perturbation" else e_state) > threshold
            out["signal"].append(e_sig)
            out["state"].append(e_state)
            out["fallback"].append(bool(fb))
            if fb:
                x.copy_(ref)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    return out


def time_hop(net, hop=50, n=64, reps=5):
    """Wall time (ms, CUDA events) of one surrogate application and of `hop` LB FP32 steps on n^3."""
    th0 = lb.lb_theta0()
    x = torch.zeros((1, n, n, n, 16), dtype=torch.bfloat16, device="cuda")
    ctx = lb.lb_init((n, n, n), NU / th0, "f32")
    try:
        f = wl.gaussian_pulse_sample(n, th0, 1, device="cuda")
        lb.lb_set_fields(ctx, f["rho"], f["u"], f["theta"])
        lb.lb_tune(ctx, reps=3)
        for _ in range(2):
            net.forward(x)
            lb.lb_step(ctx, hop)
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        for _ in range(reps):
            net.forward(x)
        e[1].record()
        e[2].record()
        for _ in range(reps):
            lb.lb_step(ctx, hop)
        e[3].record()
        torch.cuda.synchronize()
        lb.lb_sync(ctx)
        return e[0].elapsed_time(e[1]) / reps, e[2].elapsed_time(e[3]) / reps
    finally:
        lb.lb_destroy(ctx)
