"""lb_conserved_noalloc: the conservation sums for callers that cannot allocate
device memory (they run under another allocator's memory budget, or in loops
that must not pay cudaMalloc's implicit synchronisation).  Its output must match
lb_conserved on the same state, on two calls in a row (the calls share one
fixed scratch array, so the second call must not see the first's leftovers)."""
import numpy as np
import pytest
import torch

from helpers import TORCH_DTYPE
from paper_1909_08406_gb300 import lb
from paper_1909_08406_gb300 import workloads as wl


def test_rejects_more_planes_than_the_fixed_scratch():
    """2 * 2049 planes exceed the fixed scratch: LB_ERR_ARG before any device work (the dummy
    pointers are never dereferenced)."""
    L = lb._bind_noalloc()
    dummy = lb.ctypes.c_void_p(256)
    st = L.lb_conserved_noalloc(dummy, lb._Grid(8, 8, 2049), 1, dummy, None)
    assert st == -1
    assert b"4096" in L.lb_conserved_noalloc_error()


@pytest.mark.parametrize("bad", ["out_dtype", "out_size", "pop_dtype", "pop_size", "host"])
def test_wrapper_rejects_mismatched_tensors(bad):
    """The Python wrapper refuses tensors whose element type, size or device does not match the
    grid and precision, before any call into the library (CPU tensors: nothing reaches a GPU)."""
    shape = (4, 3, 2)
    n = 2 * 41 * 4 * 3 * 2
    pop = torch.zeros(n, dtype=torch.float16)
    out = torch.zeros(5, dtype=torch.float64)
    if bad == "out_dtype":
        out = torch.zeros(5, dtype=torch.float32)
    elif bad == "out_size":
        out = torch.zeros(4, dtype=torch.float64)
    elif bad == "pop_dtype":
        pop = torch.zeros(n, dtype=torch.float32)
    elif bad == "pop_size":
        pop = torch.zeros(n - 1, dtype=torch.float16)
    with pytest.raises(ValueError):
        lb.lb_conserved_noalloc(pop, shape, "f16", out)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_noalloc_matches_lb_conserved_twice(prec):
    shape = (24, 10, 6)
    th0 = lb.lb_theta0()
    fl = wl.random_fields(*shape, th0, seed=31, du=0.03, drho=0.03, dtheta=0.03)
    ctx = lb.lb_init(shape, 0.4, prec)
    try:
        lb.lb_set_fields(ctx, fl["rho"].cuda(), fl["u"].cuda(), fl["theta"].cuda())
        lb.lb_step(ctx, 5)
        ref = lb.lb_conserved(ctx)
        raw = torch.empty((2, 41, shape[2], shape[1], shape[0]), dtype=TORCH_DTYPE[prec], device="cuda")
        lb.lb_get_state(ctx, raw)
        lb.lb_sync(ctx)
    finally:
        lb.lb_destroy(ctx)
    nodes = 2 * shape[0] * shape[1] * shape[2]
    for _ in range(2):
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        lb.lb_conserved_noalloc(raw, shape, prec, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same per-node FP64 sums, summed in a different order: the tolerances of the other tests
        assert got[0] == pytest.approx(ref[0], rel=1e-13)
        assert np.max(np.abs(got[1:4] - ref[1:4])) < 1e-12 * nodes
        assert got[4] == pytest.approx(ref[4], rel=1e-13)
