"""Thin Python binding of the C ABI in ``include/gblb.h`` (argument marshalling only).

Every function has the name of its C counterpart.  Array arguments may be
torch tensors (CPU or CUDA) or numpy arrays; they must be float64 and
C-contiguous in the layouts of ``gblb.h``.  CUDA tensors are passed as device
pointers, everything else as host pointers.  The stream defaults to torch's
current stream.  All compute happens in ``libgblb.so``; if the library is
missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgblb.so")

LB_OK = 0
STATUS = {0: "LB_OK", -1: "LB_ERR_ARG", -2: "LB_ERR_OOM", -3: "LB_ERR_CUDA", -4: "LB_ERR_THETA0",
          -5: "LB_ERR_UNSTABLE", -6: "LB_ERR_TIMEOUT", -7: "LB_ERR_STATE"}
PRECISION = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}
LB_RD3Q41 = 41
LB_FLAG_PAPER_LITERAL = 1
LB_FLAG_STAGED = 2
LB_FLAG_ENTROPIC = 4
LB_FLAG_ENTROPIC_PATH = 8
LB_KERNEL_AUTO, LB_KERNEL_DIRECT1, LB_KERNEL_DIRECT2, LB_KERNEL_DIRECT2R, LB_KERNEL_STAGED, LB_KERNEL_WARPSPEC = -1, 0, 1, 2, 3, 4
LB_KERNEL_DIRECT2X, LB_KERNEL_DIRECT2XL = 5, 6
LB_HALO = 2  # halo planes at each end of a padded z slab (lb_halo_pack)
KERNEL_NAMES = {0: "k_step (direct, 1 node/thread)", 1: "k_step2 (direct, 2 rows/thread, FP32x2)",
                2: "k_step2 (direct, 2 rows/thread, FP32x2, 4 CTAs/SM)", 3: "k_step_tma (TMA-staged)",
                4: "k_step_ws (TMA-staged, warp-specialised, FP32x2)",
                5: "k_step2x (direct, 2 x-adjacent nodes/thread, FP32x2, paired 16-bit access)",
                6: "k_step2x (x pairs, 2 rows/block, next row prefetched into L2)"}


class LbError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libgblb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(or python -m paper_1909_08406_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.lb_velocity_set.argtypes = [vp, vp]
        L.lb_theta0.restype = dp
        L.lb_init.argtypes = [ctypes.POINTER(vp), _Grid, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_uint, vp]
        L.lb_set_stream.argtypes = [vp, vp]
        L.lb_set_fields.argtypes = [vp, vp, vp, vp, ctypes.c_int]
        L.lb_step.argtypes = [vp, i64]
        L.lb_get_moments.argtypes = [vp, vp, vp, vp, ctypes.c_int]
        L.lb_conserved.argtypes = [vp, vp]
        L.lb_get_populations.argtypes = [vp, vp, ctypes.c_int]
        L.lb_set_populations.argtypes = [vp, vp, ctypes.c_int]
        L.lb_state_bytes.argtypes = [vp]
        L.lb_state_bytes.restype = i64
        L.lb_get_state.argtypes = [vp, vp, ctypes.c_int]
        L.lb_set_state.argtypes = [vp, vp, ctypes.c_int]
        L.lb_step_variant.argtypes = [vp]
        L.lb_step_variant.restype = ctypes.c_int
        L.lb_set_step_kernel.argtypes = [vp, ctypes.c_int]
        L.lb_set_step_kernel.restype = ctypes.c_int
        L.lb_tune.argtypes = [vp, ctypes.c_int, vp, vp]
        L.lb_tune.restype = ctypes.c_int
        L.lb_time.argtypes = [vp]
        L.lb_time.restype = i64
        L.lb_set_walls.argtypes = [vp, ctypes.c_int, vp, vp]
        L.lb_set_walls.restype = ctypes.c_int
        L.lb_wall_density.argtypes = [vp, vp]
        L.lb_wall_density.restype = ctypes.c_int
        L.lb_set_wall_columns.argtypes = [vp, vp, vp]
        L.lb_set_wall_columns.restype = ctypes.c_int
        L.lb_get_grid.argtypes = [vp, ctypes.POINTER(_Grid)]
        L.lb_get_grid.restype = ctypes.c_int
        L.lb_conserved_planes.argtypes = [vp, i64, i64, ctypes.POINTER(ctypes.c_double)]
        L.lb_conserved_planes.restype = ctypes.c_int
        L.lb_halo_bytes.argtypes = [vp, ctypes.POINTER(i64)]
        L.lb_halo_bytes.restype = ctypes.c_int
        L.lb_halo_pack.argtypes = [vp, ctypes.c_int, vp]
        L.lb_halo_pack.restype = ctypes.c_int
        L.lb_halo_unpack.argtypes = [vp, ctypes.c_int, vp]
        L.lb_halo_unpack.restype = ctypes.c_int
        L.lb_set_stochastic_rounding.argtypes = [vp, ctypes.c_int, ctypes.c_uint64]
        L.lb_set_stochastic_rounding.restype = ctypes.c_int
        L.lb_set_nonideal.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp]
        L.lb_set_nonideal.restype = ctypes.c_int
        L.lb_nonideal_constants.argtypes = [ctypes.c_int, dp, dp, ctypes.POINTER(dp), ctypes.POINTER(dp)]
        L.lb_nonideal_constants.restype = ctypes.c_int
        L.lb_sync.argtypes = [vp]
        L.lb_destroy.argtypes = [vp]
        L.lb_last_error.argtypes = [vp]
        L.lb_last_error.restype = ctypes.c_char_p
        for name in ("lb_velocity_set", "lb_init", "lb_set_stream", "lb_set_fields", "lb_step", "lb_get_moments",
                     "lb_conserved", "lb_get_populations", "lb_set_populations", "lb_get_state", "lb_set_state",
                     "lb_sync", "lb_destroy"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status, ctx):
    if status != LB_OK:
        msg = lib().lb_last_error(ctx)
        raise LbError(status, msg.decode() if msg else "")


def _ptr(a, writable=False):
    """(pointer, on_device) of a float64 C-contiguous torch tensor / numpy array (or None)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if writable and not a.flags["WRITEABLE"]:
            raise ValueError("array is read-only")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a, writable=False):
    if a is None:
        return None, 0
    dt = a.dtype
    if str(dt) not in ("float64", "torch.float64"):
        raise TypeError("arrays crossing the interface are float64")
    return _ptr(a, writable)


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def lb_velocity_set():
    """(c2 [41,3] int32 doubled components, w [41] float64) in the library's population order."""
    c2 = np.zeros((41, 3), dtype=np.int32)
    w = np.zeros(41)
    _check(lib().lb_velocity_set(c2.ctypes.data, w.ctypes.data), None)
    return c2, w


def lb_theta0():
    return lib().lb_theta0()


def lb_init(grid, tau, precision="f32", theta0=0.0, velocity_set=LB_RD3Q41, flags=0, stream=None):
    """Create a context; grid = (nx, ny, nz).  Returns an opaque handle (int)."""
    nx, ny, nz = (int(v) for v in grid)
    h = ctypes.c_void_p()
    st = lib().lb_init(ctypes.byref(h), _Grid(nx, ny, nz), int(velocity_set), float(theta0), float(tau),
                       PRECISION[precision] if isinstance(precision, str) else int(precision), int(flags),
                       _stream(stream))
    _check(st, None)
    return h.value


def lb_set_stream(ctx, stream=None):
    _check(lib().lb_set_stream(ctx, _stream(stream)), ctx)


def lb_set_fields(ctx, rho, u, theta):
    (pr, d0), (pu, d1), (pt, d2) = _f64(rho), _f64(u), _f64(theta)
    if not (d0 == d1 == d2):
        raise ValueError("rho, u, theta must all be on the host or all on the device")
    _check(lib().lb_set_fields(ctx, pr, pu, pt, d0), ctx)


def lb_step(ctx, n=1):
    _check(lib().lb_step(ctx, int(n)), ctx)


def lb_get_moments(ctx, rho=None, u=None, theta=None):
    ps = [_f64(a, writable=True) for a in (rho, u, theta)]
    devs = {d for (p, d) in ps if p is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be on the host or all on the device")
    _check(lib().lb_get_moments(ctx, ps[0][0], ps[1][0], ps[2][0], devs.pop() if devs else 0), ctx)


def lb_conserved(ctx):
    out = np.zeros(5)
    _check(lib().lb_conserved(ctx, out.ctypes.data), ctx)
    return out


def lb_get_populations(ctx, f):
    p, d = _f64(f, writable=True)
    _check(lib().lb_get_populations(ctx, p, d), ctx)


def lb_set_populations(ctx, f):
    p, d = _f64(f)
    _check(lib().lb_set_populations(ctx, p, d), ctx)


def lb_state_bytes(ctx):
    return int(lib().lb_state_bytes(ctx))


def lb_get_state(ctx, raw):
    p, d = _ptr(raw, writable=True)
    _check(lib().lb_get_state(ctx, p, d), ctx)


def lb_set_state(ctx, raw):
    p, d = _ptr(raw)
    _check(lib().lb_set_state(ctx, p, d), ctx)


def lb_step_variant(ctx):
    return int(lib().lb_step_variant(ctx))


def lb_set_step_kernel(ctx, kernel):
    _check(lib().lb_set_step_kernel(ctx, int(kernel)), ctx)


def lb_tune(ctx, reps=3):
    """Autotune the step kernel; returns (kernel, ms_per_step)."""
    k, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib().lb_tune(ctx, int(reps), ctypes.byref(k), ctypes.byref(ms)), ctx)
    return k.value, ms.value


LB_EOS = {"vdw": 1, "peng_robinson": 2, "carnahan_starling": 3}


def lb_nonideal_constants(eos, theta_star, rho_c=1.0):
    """(a, b) of equation of state `eos` with its critical point at rho_c and
    theta_c = theta0 / theta_star."""
    a, b = ctypes.c_double(), ctypes.c_double()
    kind = LB_EOS[eos] if isinstance(eos, str) else int(eos)
    status = lib().lb_nonideal_constants(kind, float(theta_star), float(rho_c), ctypes.byref(a), ctypes.byref(b))
    if status != LB_OK:
        raise LbError(status, "lb_nonideal_constants: unknown equation of state or bad theta_star / rho_c")
    return a.value, b.value


def lb_set_nonideal(ctx, a=None, b=None, kappa=0.0, eta=0.5, eos="vdw"):
    """Isothermal nonideal fluid with the paper's momentum-conserving force, for the equation
    of state `eos` ("vdw", "peng_robinson" or "carnahan_starling", or its LB_EOS_* number) with
    constants a, b; a = None restores the energy-conserving update."""
    if a is None:
        _check(lib().lb_set_nonideal(ctx, 0, 0.0, 0.0, 0.0, 0.0), ctx)
        return
    kind = LB_EOS[eos] if isinstance(eos, str) else int(eos)
    _check(lib().lb_set_nonideal(ctx, kind, float(a), float(b), float(kappa), float(eta)), ctx)


def lb_conserved_planes(ctx, z0, z1):
    """lb_conserved over the planes z0 <= z < z1 of both sub-lattices (a slab's interior)."""
    out = (ctypes.c_double * 5)()
    _check(lib().lb_conserved_planes(ctx, int(z0), int(z1), out), ctx)
    return [out[k] for k in range(5)]


def lb_halo_bytes(ctx):
    """Bytes of one halo message of a padded z slab (see gblb.h)."""
    n = ctypes.c_int64()
    _check(lib().lb_halo_bytes(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def lb_halo_pack(ctx, side, buf):
    """Interior planes for a neighbour's halo into the device tensor buf (side 1: the top ones,
    for rank + 1; side 0: the bottom ones, for rank - 1)."""
    p, dev = _ptr(buf, writable=True)
    if not dev or buf.numel() * buf.element_size() < lb_halo_bytes(ctx):
        raise ValueError("lb_halo_pack: buf must be a device tensor of lb_halo_bytes bytes")
    _check(lib().lb_halo_pack(ctx, int(side), p), ctx)


def lb_halo_unpack(ctx, side, buf):
    """This slab's halo from the device tensor buf (side 0: lower, from rank - 1; side 1: upper,
    from rank + 1)."""
    p, dev = _ptr(buf)
    if not dev or buf.numel() * buf.element_size() < lb_halo_bytes(ctx):
        raise ValueError("lb_halo_unpack: buf must be a device tensor of lb_halo_bytes bytes")
    _check(lib().lb_halo_unpack(ctx, int(side), p), ctx)


def lb_set_stochastic_rounding(ctx, seed=None):
    """Stochastic rounding of the BF16 store with the given 64-bit seed (the step counter starts
    again at 0); seed = None restores round to nearest."""
    if seed is None:
        _check(lib().lb_set_stochastic_rounding(ctx, 0, 0), ctx)
    else:
        _check(lib().lb_set_stochastic_rounding(ctx, 1, int(seed) & 0xFFFFFFFFFFFFFFFF), ctx)


def lb_grid_of(ctx):
    """(nx, ny, nz) of a context."""
    g = _Grid()
    _check(lib().lb_get_grid(ctx, ctypes.byref(g)), ctx)
    return g.nx, g.ny, g.nz


def lb_set_walls(ctx, bottom=None, top=None):
    """Kinetic walls normal to z: bottom, top = (u_x, u_y, theta) of each wall, each entry a
    number (the same for every cell column) or an array [ny][nx] (per column); None for both
    restores the periodic grid."""
    if bottom is None and top is None:
        _check(lib().lb_set_walls(ctx, 0, None, None), ctx)
        return
    if all(np.ndim(v) == 0 for v in tuple(bottom) + tuple(top)):
        b = (ctypes.c_double * 4)(float(bottom[0]), float(bottom[1]), 0.0, float(bottom[2]))
        t = (ctypes.c_double * 4)(float(top[0]), float(top[1]), 0.0, float(top[2]))
        _check(lib().lb_set_walls(ctx, 1, ctypes.cast(b, ctypes.c_void_p), ctypes.cast(t, ctypes.c_void_p)), ctx)
        return
    nx, ny, _ = lb_grid_of(ctx)
    arrs = [np.ascontiguousarray(np.stack([np.broadcast_to(np.asarray(v, dtype=np.float64), (ny, nx))
                                           for v in w])) for w in (bottom, top)]
    _check(lib().lb_set_wall_columns(ctx, arrs[0].ctypes.data, arrs[1].ctypes.data), ctx)


def lb_wall_density(ctx):
    """rho_w of every cell column of the bottom and the top wall in the last step, [2][ny][nx]."""
    nx, ny, _ = lb_grid_of(ctx)
    out = np.empty((2, ny, nx))
    _check(lib().lb_wall_density(ctx, out.ctypes.data), ctx)
    return out


def lb_time(ctx):
    return int(lib().lb_time(ctx))


def lb_sync(ctx):
    _check(lib().lb_sync(ctx), ctx)


def lb_destroy(ctx):
    _check(lib().lb_destroy(ctx), ctx)


def lb_last_error(ctx=None):
    m = lib().lb_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# Batched sweep of independent simulations
# ---------------------------------------------------------------------------
LB_BATCH_GRAPH = 0
LB_BATCH_PERSISTENT = 1
LB_BATCH_SEQUENTIAL = 2
_batch_bound = False


def _bind_batch():
    global _batch_bound
    if _batch_bound:
        return lib()
    L = lib()
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.lb_batch_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_uint, vp]
    L.lb_batch_size.argtypes = [vp]
    L.lb_batch_size.restype = ctypes.c_int
    L.lb_batch_sim.argtypes = [vp, ctypes.c_int]
    L.lb_batch_sim.restype = vp
    L.lb_batch_tune.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.lb_batch_get_tile.argtypes = [vp, vp, vp]
    L.lb_batch_set_tile.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.lb_batch_set_rows.argtypes = [vp, ctypes.c_int]
    L.lb_batch_get_rows.argtypes = [vp]
    L.lb_batch_get_rows.restype = ctypes.c_int
    L.lb_batch_get_plan.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    L.lb_batch_step.argtypes = [vp, i64, ctypes.c_int]
    L.lb_batch_set_wait.argtypes = [vp, ctypes.c_longlong, ctypes.c_uint]
    L.lb_batch_sync.argtypes = [vp]
    L.lb_batch_destroy.argtypes = [vp]
    L.lb_batch_last_error.argtypes = [vp]
    L.lb_batch_last_error.restype = ctypes.c_char_p
    for name in ("lb_batch_init", "lb_batch_tune", "lb_batch_get_tile", "lb_batch_set_tile", "lb_batch_set_rows",
                 "lb_batch_get_plan", "lb_batch_step", "lb_batch_set_wait", "lb_batch_sync", "lb_batch_destroy"):
        getattr(L, name).restype = ctypes.c_int
    _batch_bound = True
    return L


def _bcheck(status, b):
    if status != LB_OK:
        msg = _bind_batch().lb_batch_last_error(b)
        raise LbError(status, msg.decode() if msg else "")


def lb_batch_init(grids, taus, precision="f32", flags=0, stream=None):
    """grids: list of (nx, ny, nz); taus: list of tau.  Returns an opaque batch handle."""
    L = _bind_batch()
    n = len(grids)
    garr = (_Grid * n)(*[_Grid(*(int(v) for v in g)) for g in grids])
    tarr = (ctypes.c_double * n)(*[float(t) for t in taus])
    h = ctypes.c_void_p()
    st = L.lb_batch_init(ctypes.byref(h), n, ctypes.cast(garr, ctypes.c_void_p), ctypes.cast(tarr, ctypes.c_void_p),
                         PRECISION[precision] if isinstance(precision, str) else int(precision), int(flags),
                         _stream(stream))
    _bcheck(st, None)
    return h.value


def lb_batch_size(b):
    return int(_bind_batch().lb_batch_size(b))


def lb_batch_sim(b, sim):
    """Context handle of simulation `sim` (owned by the batch: use with lb_set_fields etc., never lb_destroy)."""
    h = _bind_batch().lb_batch_sim(b, int(sim))
    if not h:
        raise IndexError(sim)
    return h


def lb_batch_tune(b, reps=3):
    """Autotune the tile shape and rows per thread of both batched modes; returns the graph
    mode's (tx, ry, ms_per_step)."""
    tx, ry, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _bcheck(_bind_batch().lb_batch_tune(b, int(reps), ctypes.byref(tx), ctypes.byref(ry), ctypes.byref(ms)), b)
    return tx.value, ry.value, ms.value


def lb_batch_get_tile(b):
    tx, ry = ctypes.c_int(), ctypes.c_int()
    _bcheck(_bind_batch().lb_batch_get_tile(b, ctypes.byref(tx), ctypes.byref(ry)), b)
    return tx.value, ry.value


def lb_batch_set_tile(b, tx, ry):
    _bcheck(_bind_batch().lb_batch_set_tile(b, int(tx), int(ry)), b)


def lb_batch_set_rows(b, rows_per_thread):
    """1 or 2 rows per thread (2: packed FP32x2 on (y, y + 1); FP32 arithmetic, every ny even)."""
    _bcheck(_bind_batch().lb_batch_set_rows(b, int(rows_per_thread)), b)


def lb_batch_get_rows(b):
    return int(_bind_batch().lb_batch_get_rows(b))


def lb_batch_get_plan(b, mode):
    """(tx, ry, rows_per_thread) of LB_BATCH_GRAPH or LB_BATCH_PERSISTENT."""
    tx, ry, rows = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(_bind_batch().lb_batch_get_plan(b, int(mode), ctypes.byref(tx), ctypes.byref(ry), ctypes.byref(rows)), b)
    return tx.value, ry.value, rows.value


def lb_batch_step(b, n, mode=LB_BATCH_GRAPH):
    _bcheck(_bind_batch().lb_batch_step(b, int(n), int(mode)), b)


def lb_batch_set_wait(b, limit_cycles, extra_arrivals=0):
    _bcheck(_bind_batch().lb_batch_set_wait(b, int(limit_cycles), int(extra_arrivals)), b)


def lb_batch_sync(b):
    _bcheck(_bind_batch().lb_batch_sync(b), b)


def lb_batch_destroy(b):
    _bcheck(_bind_batch().lb_batch_destroy(b), b)


def _bind_noalloc():
    L = lib()
    if not getattr(L, "_noalloc_bound", False):
        L.lb_conserved_noalloc.argtypes = [ctypes.c_void_p, _Grid, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.lb_conserved_noalloc.restype = ctypes.c_int
        L.lb_conserved_noalloc_error.restype = ctypes.c_char_p
        L._noalloc_bound = True
    return L


def lb_conserved_noalloc(populations, grid, precision, out, stream=None):
    """Conservation sums of stored populations (device tensor in the raw layout of lb_get_state)
    into `out` (device float64 tensor of 5), with no device allocation.  The tensors' element
    types, sizes and device are checked here, before the call: a mismatch would otherwise become
    an out-of-bounds access on the GPU."""
    import torch
    L = _bind_noalloc()
    if isinstance(precision, str):
        if precision not in PRECISION:
            raise ValueError(f"unknown precision {precision!r}")
        prec = PRECISION[precision]
    else:
        prec = int(precision)
    es = {PRECISION[k]: v for k, v in STORAGE_BYTES.items()}.get(prec)
    if es is None:
        raise ValueError(f"unknown precision {precision!r}")
    if not (isinstance(populations, torch.Tensor) and isinstance(out, torch.Tensor)):
        raise TypeError("populations and out must be torch tensors on the device")
    if out.dtype != torch.float64 or out.numel() < 5:
        raise ValueError("out must be a float64 tensor of at least 5 elements")
    nx, ny, nz = (int(v) for v in grid)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid extents must be >= 1")
    if populations.element_size() != es:
        raise ValueError(f"populations hold {populations.element_size()}-byte elements; precision {precision!r} "
                         f"stores {es}-byte elements")
    if populations.numel() != 2 * 41 * nx * ny * nz:
        raise ValueError(f"populations hold {populations.numel()} elements, the grid needs 2*41*nx*ny*nz = "
                         f"{2 * 41 * nx * ny * nz}")
    if not (populations.is_cuda and out.is_cuda):
        raise ValueError("populations and out must be device tensors")
    here = torch.cuda.current_device()
    if populations.device.index != here or out.device.index != here:
        raise ValueError(f"populations and out must be on the current device (cuda:{here})")
    pp, _ = _ptr(populations)
    po, _ = _ptr(out, writable=True)
    st = L.lb_conserved_noalloc(pp, _Grid(nx, ny, nz), prec, po, _stream(stream))
    if st != LB_OK:
        raise LbError(st, L.lb_conserved_noalloc_error().decode())
