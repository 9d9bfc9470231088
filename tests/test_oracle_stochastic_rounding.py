"""Pins of the oracle's stochastic BF16 rounding (oracle/stochastic_rounding.py) against what the
rounding rule fixes exactly and what a uniform, independent generator must show statistically.

* Exactly representable values are returned unchanged for every r.
* Any other value goes to one of its two BF16 neighbours: the magnitude truncation, or the next
  BF16 number away from zero.
* Averaged over all 2^16 values of r the result equals the input exactly (the rounding is
  unbiased; round to nearest or a shifted threshold fails this).
* The 16-bit words are uniform (chi-square over 256 bins), their halves and neighbouring
  populations and nodes uncorrelated, and the step key changes the stream."""
import numpy as np
import pytest

from oracle import stochastic_rounding as sr


def _bf16_neighbours(v):
    """(truncation toward zero, next BF16 away from zero) of FP32 values, as float64."""
    b = np.asarray(v, dtype=np.float32).view(np.uint32)
    lo = (b & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    hi = ((b & np.uint32(0xFFFF0000)) + np.uint32(0x10000)).view(np.float32).astype(np.float64)
    return lo, hi


def test_representable_values_are_unchanged():
    rng = np.random.default_rng(1)
    v = sr.round_bf16_nearest(rng.normal(0, 1e-2, 4096))
    r = rng.integers(0, 1 << 16, v.size)
    assert np.array_equal(sr.round_bf16(v, r), v)


def test_result_is_one_of_the_two_neighbours():
    rng = np.random.default_rng(2)
    v = (rng.normal(0, 1, 20000) * 10.0 ** rng.integers(-6, 2, 20000)).astype(np.float32)
    r = rng.integers(0, 1 << 16, v.size)
    out = sr.round_bf16(v, r)
    lo, hi = _bf16_neighbours(v)
    assert np.all((out == lo) | (out == hi))
    # magnitude never shrinks below the truncation nor passes the next value
    assert np.all(np.abs(out) >= np.abs(lo)) and np.all(np.abs(out) <= np.abs(hi))


@pytest.mark.parametrize("v", [1.2345678e-3, -7.654321e-2, 3.3e-5, -0.9])
def test_mean_over_all_r_is_exact(v):
    v32 = np.float32(v)
    out = sr.round_bf16(np.full(1 << 16, v32), np.arange(1 << 16))
    # every term is a multiple of the BF16 spacing, so the float64 sum is exact
    assert out.sum() / (1 << 16) == float(v32)
    # round to nearest is biased for the same value
    assert sr.round_bf16_nearest(np.float64(v32)) != float(v32)


def test_random_bits_are_uniform_and_independent():
    key = sr.step_key(12345, 0)
    q = np.arange(1 << 14, dtype=np.uint64)
    i = np.arange(41)
    r = sr.random_bits(key, q[:, None], i[None, :]).astype(np.int64)  # [q][i]
    assert r.min() >= 0 and r.max() < (1 << 16)
    counts = np.bincount((r >> 8).ravel(), minlength=256)
    expected = r.size / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 255 + 5 * np.sqrt(2 * 255), chi2  # 5 sigma of the chi-square with 255 dof
    x = (r - r.mean()) / r.std()
    for a, b in ((x[0::2], x[1::2]),        # the two nodes of a pair (halves of one word)
                 (x[:, :-1], x[:, 1:]),     # neighbouring populations
                 (x[:-2], x[2:])):          # neighbouring pairs
        assert abs(float((a * b).mean())) < 5 / np.sqrt(a.size)
    # a different step or seed gives a different stream
    r1 = sr.random_bits(sr.step_key(12345, 1), q[:64, None], i[None, :])
    r2 = sr.random_bits(sr.step_key(54321, 0), q[:64, None], i[None, :])
    assert (r1 != r[:64]).mean() > 0.99 and (r2 != r[:64]).mean() > 0.99


def test_random_bits_follow_the_recurrence():
    """The words of populations i and i + 1 are successive states of the recurrence; the pair
    q, q + 1 (q even) shares one word."""
    key = sr.step_key(7, 3)
    q = np.uint64(2 * 1000)
    s0 = sr.pcg_hash(np.uint32(key) ^ np.uint32(1000))
    s = s0
    for i in range(41):
        with np.errstate(over="ignore"):
            s = s * np.uint32(1664525) + np.uint32(1013904223)
        w = int(s ^ (s >> np.uint32(16)))
        assert int(sr.random_bits(key, q, i)) == w & 0xFFFF
        assert int(sr.random_bits(key, q + np.uint64(1), i)) == w >> 16


def test_rounding_is_unbiased_over_the_generator():
    """A fixed value rounded with the generator's bits over many nodes averages to itself
    within the sampling error."""
    v = np.float32(3.21e-3)
    lo, hi = _bf16_neighbours(v)
    p = (float(v) - lo) / (hi - lo)
    n = 1 << 16
    r = sr.random_bits(sr.step_key(99, 0), np.arange(n, dtype=np.uint64), 17)
    out = sr.round_bf16(np.full(n, v), r)
    frac_up = float((out == hi).mean())
    assert abs(frac_up - p) < 5 * np.sqrt(p * (1 - p) / n), (frac_up, p)
