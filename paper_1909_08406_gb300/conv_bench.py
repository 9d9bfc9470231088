"""Timing of the surrogate's forward convolution kernels (tcgen05 and mma.sync).

    python -m paper_1909_08406_gb300.conv_bench [--impl tcgen05|mma_sync|both]
        [--layers 16x32,32x32,32x16] [--batch 1,4] [--reps 20] [--warmup 3]

Runs sg_conv3d_fwd with the fused GELU epilogue (and the residual when cin ==
cout) on random BF16 activations of batch x 64^3 x cin voxels and weights of
scale 1/sqrt(27 cin), times `reps` launches with CUDA events after `warmup`
launches, and prints one JSON object: per kernel, layer and batch the time per
launch (microseconds) and the rate (TFLOP/s, 2 * voxels * 27 * cin * cout).
Then checks the tensor-core status flag (sg_status).
"""
from __future__ import annotations

import argparse
import json
import math
import sys


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--impl", default="both", choices=["tcgen05", "mma_sync", "both"])
    p.add_argument("--layers", default="16x32,32x32,32x16")
    p.add_argument("--batch", default="1,4")
    p.add_argument("--reps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    a = p.parse_args(argv)
    import torch
    from . import sg
    impls = {"tcgen05": sg.CONV_TCGEN05, "mma_sync": sg.CONV_MMA_SYNC}
    names = list(impls) if a.impl == "both" else [a.impl]
    layers = [tuple(int(v) for v in L.split("x")) for L in a.layers.split(",")]
    batches = [int(b) for b in a.batch.split(",")]
    out = {}
    prev = None
    for name in names:
        old = sg.set_conv_impl(impls[name])
        prev = old if prev is None else prev
        for cin, cout in layers:
            for batch in batches:
                shape = (batch, 64, 64, 64)
                g = torch.Generator(device="cuda").manual_seed(cin * 100 + cout)
                x = torch.randn(shape + (cin,), device="cuda", generator=g).to(torch.bfloat16)
                w = (torch.randn((cout, 27, cin), device="cuda", generator=g) / math.sqrt(27 * cin)).to(torch.bfloat16)
                b = torch.zeros(cout, device="cuda")
                y = torch.empty(shape + (cout,), device="cuda", dtype=torch.bfloat16)
                for _ in range(a.warmup):
                    sg.conv3d_fwd(x, w, b, act=sg.ACT_GELU, res_in=(cin == cout), y=y)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(a.reps):
                    sg.conv3d_fwd(x, w, b, act=sg.ACT_GELU, res_in=(cin == cout), y=y)
                e1.record()
                e1.synchronize()
                ms = e0.elapsed_time(e1) / a.reps
                flops = 2.0 * batch * 64 ** 3 * 27 * cin * cout
                out[f"{name} {cin}->{cout} b{batch}"] = {"us": round(ms * 1e3, 2),
                                                         "tflops": round(flops / (ms * 1e-3) / 1e12, 1)}
        sg.status()
    if prev is not None:
        sg.set_conv_impl(prev)
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
