"""Test helpers shared by the GPU parity tests: velocity-order mapping between
the library and the oracle, and storage decoding (the storage format is part
of the C ABI: f64 stores f_i, the 32/16-bit modes store h_i = f_i / w_i - 1)."""
import numpy as np
import torch

import oracle

TORCH_DTYPE = {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
# unit roundoff of each storage type (half the spacing at 1)
STORE_EPS = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "f16": 2.0 ** -11, "bf16": 2.0 ** -8}
# scale of the stored value: f16 stores 2^8 h (documented in gblb.h)
STORE_SCALE = {"f64": 1.0, "f32": 1.0, "f16": 256.0, "bf16": 1.0}
# largest rounding error near zero, in units of h: half the smallest subnormal spacing
STORE_TINY = {"f64": 0.0, "f32": 2.0 ** -150, "f16": 2.0 ** -25 / 256.0, "bf16": 2.0 ** -134}


def lib_to_oracle_perm():
    """perm[i] = oracle index of the library's velocity i (matched by velocity vector)."""
    from paper_1909_08406_gb300 import lb
    c2_lib, w_lib = lb.lb_velocity_set()
    c2_or = oracle.velocities_doubled()
    perm = np.array([int(np.where((c2_or == v).all(1))[0][0]) for v in c2_lib])
    assert sorted(perm.tolist()) == list(range(41))
    return perm


def to_oracle_order(f_lib, perm):
    """[2][41][...] library order -> oracle order."""
    out = np.empty_like(f_lib)
    out[:, perm] = f_lib
    return out


def to_lib_order(f_or, perm):
    return np.ascontiguousarray(f_or[:, perm])


def decode(raw, prec, w_lib):
    """Stored elements [2][41][...] (torch, any device) -> float64 f_i (numpy)."""
    v = raw.detach().to("cpu", torch.float64).numpy()
    if prec == "f64":
        return v
    w = np.asarray(w_lib)[None, :, None, None, None]
    return w * (1.0 + v / STORE_SCALE[prec])


def _d_layout_index(natural, d):
    """Index arrays (b', z', y', x') of every voxel (b, z, y, x) of a volume [b][nz][ny][nx][c] in
    its d-layout (include/gblb_surrogate.h): b' = (b d + z mod d) d + y mod d, z' = z / d,
    y' = y / d, x' = (x mod d)(nx / d) + x / d."""
    b, nz, ny, nx = natural[:4]
    B, Z, Y, X = np.meshgrid(np.arange(b), np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    idx = ((B * d + Z % d) * d + Y % d, Z // d, Y // d, (X % d) * (nx // d) + X // d)
    return tuple(torch.from_numpy(np.ascontiguousarray(i)) for i in idx)


def from_d_layout(t, d, natural):
    """A CPU tensor in the d-layout of a volume of shape `natural` back to the volume's layout."""
    return t[_d_layout_index(natural, d)]


def to_d_layout(t, d):
    """A CPU volume [b][nz][ny][nx][c] in its d-layout [b d^2][nz / d][ny / d][nx][c]."""
    b, nz, ny, nx, c = t.shape
    out = torch.empty((b * d * d, nz // d, ny // d, nx, c), dtype=t.dtype)
    out[_d_layout_index(t.shape, d)] = t
    return out
