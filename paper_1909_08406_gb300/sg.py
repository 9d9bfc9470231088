"""Thin binding of the surrogate kernels' C ABI (include/gblb_surrogate.h).

Argument marshalling only: tensors are torch CUDA tensors (BF16 activations
and weights, FP32 accumulators / gradients); every computation runs in
libgblb.so.  Shapes: activations [batch][nz][ny][nx][channels] (nx = 64); a dilated convolution
runs on the volume's d-layout (relabel) with xper = 64 / d.
"""
from __future__ import annotations

import ctypes

import torch

from .lb import lib

_bound = False


class SgShape(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("nz", ctypes.c_int), ("ny", ctypes.c_int), ("nx", ctypes.c_int),
                ("xper", ctypes.c_int)]


ACT_NONE, ACT_GELU = 0, 1
CONV_MMA_SYNC, CONV_TCGEN05 = 0, 1


def _L():
    global _bound
    L = lib()
    if not _bound:
        vp, i64, f32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        sig = {
            "sg_conv3d_fwd": [SgShape, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp],
            "sg_conv3d_fwd_f32": [SgShape, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp],
            "sg_act_backward": [i64, ctypes.c_int, vp, vp, vp, vp],
            "sg_transpose_weights": [ctypes.c_int, ctypes.c_int, vp, vp, vp],
            "sg_wgrad_scratch_bytes": [SgShape, ctypes.c_int, ctypes.c_int],
            "sg_conv3d_wgrad": [SgShape, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp],
            "sg_reduce_scratch_bytes": [i64],
            "sg_mse": [i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp],
            "sg_rel_l2": [SgShape, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp],
            "sg_adam": [i64, vp, vp, vp, vp, vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                        ctypes.c_int, vp],
            "sg_pack_fields": [SgShape, ctypes.c_int, vp, vp, vp, ctypes.c_double, vp, vp, vp],
            "sg_unpack_fields": [SgShape, ctypes.c_int, vp, ctypes.c_double, vp, vp, vp, vp, vp],
            "sg_relabel": [SgShape, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp],
            "sg_set_conv_impl": [ctypes.c_int],
            "sg_status": [vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int64 if name.endswith("_bytes") else ctypes.c_int
        _bound = True
    return L


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")


def set_conv_impl(impl):
    """Select the forward-convolution kernel (CONV_TCGEN05, the default, or CONV_MMA_SYNC);
    returns the previous one."""
    prev = _L().sg_set_conv_impl(int(impl))
    if prev < 0:
        raise ValueError(f"unknown convolution kernel {impl}")
    return prev


def status():
    """Synchronise the current stream; raise if a tensor-core wait of a convolution ran out of time."""
    _ok(_L().sg_status(_stream()), "sg_status")


def shape_of(t, xper=0):
    b, nz, ny, nx, _ = t.shape
    return SgShape(b, nz, ny, nx, xper)


def relabelled_shape(shape, d):
    """Shape of the d-layout of a volume [batch][nz][ny][64][c] (sg_relabel)."""
    b, nz, ny, nx, c = shape
    return (b * d * d, nz // d, ny // d, nx, c)


def relabel(x, df, dt, natural, y=None):
    """x in the df-layout of a volume of shape `natural` -> its dt-layout (a new tensor unless y)."""
    if y is None:
        y = torch.empty(relabelled_shape(natural, dt), dtype=x.dtype, device=x.device)
    b, nz, ny, nx, c = natural
    _ok(_L().sg_relabel(SgShape(b, nz, ny, nx, 0), c * x.element_size(), df, dt, _p(x), _p(y), _stream()),
        "sg_relabel")
    return y


def conv3d_fwd(x, w, bias=None, act=ACT_NONE, res_in=False, add=None, z_out=None, y=None, xper=0):
    """x in a d-layout with xper = 64 / d gives the convolution with taps d voxels apart."""
    cout, _, cin = w.shape
    s = shape_of(x, xper)
    if y is None:
        y = torch.empty(x.shape[:-1] + (cout,), dtype=torch.bfloat16, device=x.device)
    _ok(_L().sg_conv3d_fwd(s, cin, cout, _p(x), _p(w), _p(bias), act, int(res_in), _p(add), _p(z_out), _p(y),
                           _stream()), "sg_conv3d_fwd")
    return y


def conv3d_fwd_f32(x, w, add=None, y=None, xper=0):
    cout, _, cin = w.shape
    if y is None:
        y = torch.empty(x.shape[:-1] + (cout,), dtype=torch.float32, device=x.device)
    _ok(_L().sg_conv3d_fwd_f32(shape_of(x, xper), cin, cout, _p(x), _p(w), _p(add), _p(y), _stream()),
        "sg_conv3d_fwd_f32")
    return y


def act_backward(dy, z, act, dz=None):
    if dz is None:
        dz = torch.empty(dy.shape, dtype=torch.bfloat16, device=dy.device)
    _ok(_L().sg_act_backward(dy.numel(), act, _p(dy), _p(z), _p(dz), _stream()), "sg_act_backward")
    return dz


def transpose_weights(w, wt=None):
    cout, _, cin = w.shape
    if wt is None:
        wt = torch.empty((cin, 27, cout), dtype=w.dtype, device=w.device)
    _ok(_L().sg_transpose_weights(cin, cout, _p(w), _p(wt), _stream()), "sg_transpose_weights")
    return wt


def wgrad_scratch(x, cin, cout):
    n = _L().sg_wgrad_scratch_bytes(shape_of(x), cin, cout)
    return torch.empty(n, dtype=torch.uint8, device=x.device)


def conv3d_wgrad(x, dz, dw, db, scratch, xper=0):
    cin, cout = x.shape[-1], dz.shape[-1]
    _ok(_L().sg_conv3d_wgrad(shape_of(x, xper), cin, cout, _p(x), _p(dz), _p(dw), _p(db), _p(scratch), _stream()),
        "sg_conv3d_wgrad")


def reduce_scratch(device="cuda"):
    return torch.empty(_L().sg_reduce_scratch_bytes(0), dtype=torch.uint8, device=device)


def mse(pred, target, nch, loss, dpred, scratch):
    voxels = pred.numel() // pred.shape[-1]
    _ok(_L().sg_mse(voxels, pred.shape[-1], nch, _p(pred), _p(target), _p(loss), _p(dpred), _p(scratch), _stream()),
        "sg_mse")


def rel_l2(a, b, nch, out, scratch):
    _ok(_L().sg_rel_l2(shape_of(a), a.shape[-1], nch, _p(a), _p(b), _p(out), _p(scratch), _stream()), "sg_rel_l2")


def adam(p, g, m, v, p16, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    _ok(_L().sg_adam(p.numel(), _p(p), _p(g), _p(m), _p(v), _p(p16), lr, beta1, beta2, eps, t, _stream()), "sg_adam")


def pack_fields(x, item, rho, u, theta, theta0, scales):
    sc = (ctypes.c_float * 3)(*scales)
    _ok(_L().sg_pack_fields(shape_of(x), item, _p(rho), _p(u), _p(theta), theta0, ctypes.cast(sc, ctypes.c_void_p),
                            _p(x), _stream()), "sg_pack_fields")


def unpack_fields(x, item, theta0, scales, rho, u, theta):
    sc = (ctypes.c_float * 3)(*scales)
    _ok(_L().sg_unpack_fields(shape_of(x), item, _p(x), theta0, ctypes.cast(sc, ctypes.c_void_p), _p(rho), _p(u),
                              _p(theta), _stream()), "sg_unpack_fields")
