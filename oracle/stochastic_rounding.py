"""Stochastic rounding of FP32 values to BF16 with a counter-based generator.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by ``tests/`` to
check the library's stochastic BF16 store (``lb_set_stochastic_rounding``),
never by the library.  It shares no code with the CUDA path.

The paper fixes no storage rounding (16-bit storage is an addition to it); the
definition checked here is the one the library documents:

* Rounding.  A BF16 number is the upper 16 bits of an FP32 bit pattern.  With
  r uniform in [0, 2^16), the upper half of bits(v) + r equals the magnitude
  truncation of v, or the next BF16 number away from zero with probability
  (lower 16 bits of v) / 2^16: the expected result is v itself.
* Random bits, per step t, node q (q = s nx ny nz + (z ny + y) nx + x, mod
  2^32) and population i (library order):
    k_t = H(H(lo32(seed) ^ H(hi32(seed))) + t),   s_0 = H(k_t ^ (q >> 1)),
    s_(n+1) = 1664525 s_n + 1013904223,           w_i = s_(i+1) ^ (s_(i+1) >> 16),
    r = low 16 bits of w_i (q even) or high 16 bits (q odd),
  all mod 2^32.  H is the PCG hash of Jarzynski and Olano, "Hash Functions
  for GPU Rendering" (JCGT 9(3), 2020); the recurrence is the linear
  congruential generator of Numerical Recipes (Press et al., 2nd ed., Sec. 7.1).

Parity unpinned for the generator's constants: they define one stream among
many equally good ones, so no external value fixes them.  The tests pin what
matters for the method instead: the rounding rule exactly (two neighbours,
exact mean over all 2^16 values of r) and the stream's uniformity and
independence statistically.
"""
from __future__ import annotations

import numpy as np

U32 = np.uint32


def pcg_hash(x):
    """The 32-bit PCG hash (Jarzynski and Olano 2020): an LCG step of the input, then PCG's
    random-shift output permutation and a final xorshift."""
    x = np.asarray(x, dtype=U32)
    with np.errstate(over="ignore"):
        state = x * U32(747796405) + U32(2891336453)
        word = ((state >> ((state >> U32(28)) + U32(4))) ^ state) * U32(277803737)
    return (word >> U32(22)) ^ word


def step_key(seed, t):
    """k_t for a 64-bit seed and the step number t (steps since the rounding was enabled)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    lo, hi = U32(seed & 0xFFFFFFFF), U32(seed >> 32)
    ks = pcg_hash(lo ^ pcg_hash(hi))
    with np.errstate(over="ignore"):
        return pcg_hash(ks + U32(int(t) & 0xFFFFFFFF))


def random_bits(key_t, q, i):
    """The 16 random bits r of population i (0..40) of node q for the step key key_t; q and i
    broadcast."""
    q = np.asarray(q, dtype=np.uint64).astype(U32)  # q mod 2^32
    i = np.asarray(i, dtype=np.int64)
    q, i = np.broadcast_arrays(q, i)
    s = pcg_hash(U32(key_t) ^ (q >> U32(1)))
    out = np.empty(s.shape, dtype=U32)
    with np.errstate(over="ignore"):
        for n in range(int(i.max()) + 1 if i.size else 0):
            s = s * U32(1664525) + U32(1013904223)  # s_(n+1)
            sel = i == n
            w = s[sel] ^ (s[sel] >> U32(16))
            odd = (q[sel] & U32(1)) != 0
            out[sel] = np.where(odd, w >> U32(16), w & U32(0xFFFF))
    return out


def round_bf16(v, r):
    """BF16 of the FP32 values v (returned as float64) rounded with the random bits r."""
    b = np.asarray(v, dtype=np.float32).view(U32)
    with np.errstate(over="ignore"):
        up = (b + np.asarray(r, dtype=U32)) & U32(0xFFFF0000)
    return up.view(np.float32).astype(np.float64)


def round_bf16_nearest(v):
    """BF16 of float64 values by round to nearest, ties to even (through FP32: the values these
    tests use carry no more than 24 significant bits)."""
    b = np.asarray(v, dtype=np.float32).view(U32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(U32)
    return r.view(np.float32).astype(np.float64)
