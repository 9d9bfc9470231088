"""Surrogate experiment (64^3 fields, Gaussian pulses with theta perturbations):
generate LB training pairs, train the network on the GPU, report held-out
error against the identity map, a judged 20-hop rollout with LB fallback, and
the time of one surrogate application against the LB steps it replaces.

    python -m paper_1909_08406_gb300.surrogate_experiment [--count 2000] [--iters 1500] [--hop 50]
        [--dilations 1,2,4,8,8,8]

Prints one JSON object.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--count", type=int, default=2000, help="LB runs (training pairs)")
    p.add_argument("--test", type=int, default=64, help="held-out LB runs")
    p.add_argument("--iters", type=int, default=1500)
    p.add_argument("--batch", type=int, default=4)
    p.add_argument("--lr", type=float, default=1e-3)
    p.add_argument("--hop", type=int, default=50, help="LB steps per surrogate application")
    p.add_argument("--hops", type=int, default=20)
    p.add_argument("--threshold", type=float, default=1e-3)
    p.add_argument("--rollouts", type=int, default=4)
    p.add_argument("--dilations", default="1,2,4,8,8,8", help="tap spacing of the six layers")
    a = p.parse_args(argv)
    dil = tuple(int(v) for v in a.dilations.split(","))

    from . import surrogate as S

    torch.cuda.set_device(0)
    out = {"config": vars(a), "receptive_field_cells": sum(dil), "sound_travel_cells_per_hop": None}
    import math
    from . import lb
    cs = math.sqrt(5 * lb.lb_theta0() / 3)
    out["sound_travel_cells_per_hop"] = cs * a.hop
    t0 = time.perf_counter()
    train = S.make_dataset(a.count, hop=a.hop, t0_choices=(0, 100, 250, 500))
    test = S.make_dataset(a.test, hop=a.hop, seed0=900000, t0_choices=(0, 100, 250, 500))
    torch.cuda.synchronize()
    out["data_seconds"] = time.perf_counter() - t0
    net = S.Surrogate(seed=0, dilations=dil)
    t0 = time.perf_counter()
    hist = S.train(net, train, a.iters, batch=a.batch, lr=a.lr, log_every=max(1, a.iters // 10))
    torch.cuda.synchronize()
    out["train_seconds"] = time.perf_counter() - t0
    out["loss_history"] = hist
    mse, ident = S.evaluate(net, test)
    out["heldout_mse"] = mse
    out["heldout_mse_identity"] = ident
    free = [S.rollout(net, seed=990000 + k, hops=a.hops, hop=a.hop, fallback=False) for k in range(a.rollouts)]
    out["rollout_state_rel_l2"] = [np.round(r["state"], 6).tolist() for r in free]
    out["rollout_signal_rel_l2"] = [np.round(r["signal"], 4).tolist() for r in free]
    t_net, t_lb = S.time_hop(net, hop=a.hop)
    out["ms_surrogate_per_hop"] = t_net
    out["ms_lb_per_hop"] = t_lb
    out["speedup_no_fallback"] = t_lb / t_net
    # judged rollouts under both readings of "1e-3 relative L2": the perturbation (the default) and
    # the full state.  A hop that falls back costs the surrogate application and the LB hop that
    # replaces it; the rollout's cost is set against hops x the LB hop (plain LB for the same steps)
    for crit in ("perturbation", "state"):
        rolls = [S.rollout(net, seed=990000 + k, hops=a.hops, hop=a.hop, threshold=a.threshold, criterion=crit)
                 for k in range(a.rollouts)]
        rate = float(np.mean([np.mean(r["fallback"]) for r in rolls]))
        cost = a.hops * (t_net + rate * t_lb)
        out[f"judged_{crit}"] = {"fallback_rate": rate, "ms_rollout_with_fallbacks": cost,
                                 "ms_plain_lb": a.hops * t_lb, "speedup_vs_lb": a.hops * t_lb / cost,
                                 "final_signal_rel_l2": [r["signal"][-1] for r in rolls]}
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
