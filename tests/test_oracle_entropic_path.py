"""Pins of the oracle's entropic path length (oracle.path_length, collision kind "entropic_path").

alpha is the nontrivial root of Delta H(alpha) = H(f + alpha (f^eq - f)) - H(f), H = sum f ln(f/w)
(Sec. "Droplet Collision": the update with alpha beta, alpha from the H theorem).  What fixes it
independently of the oracle's own evaluation:
* the definition, evaluated here directly as a difference of H (the oracle uses the expansion in
  x_i = f^eq_i / f_i - 1);
* the small-deviation limit: for an f^eq with the moments of f whose logarithm is a sum of
  collision invariants (the exact entropic equilibrium), expanding Delta H to third order in x
  gives alpha = 2 + sum f x^3 / (3 sum f x^2) + O(x^2);
* the sign structure: Delta H < 0 on (0, alpha), > 0 beyond (convexity);
* a brute-force root on a dense grid;
* the collision keeps mass, momentum and energy and does not raise H.
A planted mistake (H without the weights) fails the limit."""
import numpy as np
import pytest

import oracle

C, W, _ = oracle.velocities()


def _state(eps, seed, skew=False):
    """A node's populations eps away from an entropic equilibrium, and the exact entropic
    equilibrium of their own moments."""
    rng = np.random.default_rng(seed)
    base = oracle.entropic_equilibrium(1.03, np.array([0.03, -0.02, 0.01]), oracle.theta0() * 1.02)
    d = rng.exponential(1.0, 41) - 1.0 if skew else rng.standard_normal(41)
    f = base * (1.0 + eps * d)
    rho, u, th = oracle.moments(f)
    return f, oracle.entropic_equilibrium(rho, u, th)


def _H(f):
    return float(np.sum(f * np.log(f / W)))


def _dH(f, feq, a):
    return _H(f + a * (feq - f)) - _H(f)


@pytest.mark.parametrize("eps,seed", [(0.1, 1), (0.03, 2), (0.1, 3)])
def test_root_of_the_direct_entropy_difference(eps, seed):
    f, feq = _state(eps, seed)
    a = oracle.path_length(f, feq)
    scale = abs(_H(feq) - _H(f))
    assert abs(_dH(f, feq, a)) <= 1e-9 * scale, (_dH(f, feq, a), scale)
    # a root of the definition, not a point where it merely looks flat
    assert _dH(f, feq, 0.99 * a) < 0 < _dH(f, feq, 1.01 * a)


@pytest.mark.parametrize("eps", [1e-2, 3e-3, 1e-3])
def test_small_deviation_limit(eps):
    f, feq = _state(eps, 5, skew=True)
    x = feq / f - 1
    lin = np.sum(f * x ** 3) / (3 * np.sum(f * x ** 2))
    a = oracle.path_length(f, feq)
    xm = np.abs(x).max()
    assert abs(a - 2 - lin) <= 0.5 * xm ** 2, (a, lin, xm)  # measured 0.155 xm^2
    assert abs(lin) > xm ** 2  # so alpha = 2 without the first-order term would fail the bound


def test_sign_structure_and_brute_force_root():
    f, feq = _state(0.1, 7)
    a = oracle.path_length(f, feq)
    x = feq / f - 1
    amax = np.inf if x.min() >= 0 else -1 / x.min()
    grid = np.linspace(1e-3, min(2 * a, 0.999 * amax), 4001)
    vals = np.array([_dH(f, feq, g) for g in grid])
    assert np.all(vals[grid < 0.995 * a] < 0) and np.all(vals[grid > 1.005 * a] > 0)
    k = np.nonzero(vals > 0)[0][0]
    assert grid[k - 1] <= a <= grid[k]


def test_equilibrium_gives_two_and_collision_is_bgk():
    feq = oracle.entropic_equilibrium(1.0, np.array([0.02, 0.0, -0.01]), oracle.theta0())
    assert oracle.path_length(feq, feq) == 2.0
    out = oracle.collide(feq.copy(), 0.7, project="entropic_path")
    assert np.allclose(out, feq, rtol=0, atol=1e-14)


@pytest.mark.parametrize("tau", [0.05, 0.5, 2.0])
def test_collision_keeps_moments_and_does_not_raise_h(tau):
    f, feq = _state(0.05, 11)
    out = oracle.collide(f.copy(), tau, project="entropic_path")
    r0, u0, t0 = oracle.moments(f)
    r1, u1, t1 = oracle.moments(out)
    assert abs(r1 - r0) <= 1e-14 and np.allclose(u1, u0, rtol=0, atol=1e-14) and abs(t1 - t0) <= 1e-14
    assert _H(out) <= _H(f) + 1e-15
    # f' = f + alpha beta (f^eq - f) with the oracle's alpha
    beta = 1 / (2 * tau + 1)
    a = oracle.path_length(f, feq)
    assert np.allclose(out, f + a * beta * (feq - f), rtol=1e-13, atol=0)


def test_planted_mistake_fails_the_limit():
    """The same root search with H = sum f ln f (weights left out) lands far from 2 + O(x)."""
    f, feq = _state(3e-3, 5, skew=True)

    def dh_wrong(a):
        g = f + a * (feq - f)
        return float(np.sum(g * np.log(g)) - np.sum(f * np.log(f)))

    lo, hi = 1e-3, 20.0
    if dh_wrong(hi) * dh_wrong(lo) < 0:
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if dh_wrong(mid) < 0 else (lo, mid)
        wrong = 0.5 * (lo + hi)
    else:
        wrong = np.nan  # no root at all: the mistake is just as visible
    x = feq / f - 1
    lin = np.sum(f * x ** 3) / (3 * np.sum(f * x ** 2))
    assert not abs(wrong - 2 - lin) <= 0.5 * np.abs(x).max() ** 2
