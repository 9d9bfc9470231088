"""Pins of the oracle's velocity set, weights and reference temperature.

Everything here is fixed by the paper independently of the oracle's code:
the shells of Table I (Sec. IV), the printed weights, the seven weight
constraints of Eq. (allWeights) (Sec. III) and the symmetry conditions of
Eq. (dvmcond).
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_weights.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, a, b, c, w = line.split()
            rows.append((name, (int(a), int(b), int(c)), float(w)))
    return rows


def test_velocity_set_shells():
    c, w, shell = oracle.velocities()
    assert c.shape == (41, 3)
    assert np.bincount(shell).tolist() == [1, 6, 6, 12, 8, 8]
    c2 = (c ** 2).sum(1)
    for sh, expected in zip(range(6), [0.0, 1.0, 4.0, 2.0, 3.0, 0.75]):
        assert np.all(c2[shell == sh] == expected)
    # distinct velocities
    assert len({tuple(v) for v in c}) == 41


def test_velocity_set_closure():
    """Closure under inversion and under reflections/permutations (Sec. III)."""
    c, _, _ = oracle.velocities()
    s = {tuple(v) for v in c}
    for v in c:
        assert tuple(-v) in s
        for perm in itertools.permutations(range(3)):
            for signs in itertools.product([1, -1], repeat=3):
                assert tuple(np.array(signs) * v[list(perm)]) in s


def test_weights_match_table1():
    c, w, shell = oracle.velocities()
    table = _table1()
    for k, (name, gen, wt) in enumerate(table, start=1):
        sel = shell == k
        assert np.all(w[sel] == wt), name
        # the shell generator (doubled) is in the shell
        g = np.array(sorted(np.abs(gen))) / 2.0
        assert any(np.array_equal(np.sort(np.abs(v)), g) for v in c[sel]), name
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.all(w > 0)
    # rest weight derived from sum w = 1 (Eq. allWeights)
    counts = [6, 6, 12, 8, 8]
    expected_w0 = 1.0 - sum(n * t[2] for n, t in zip(counts, table))
    assert w[shell == 0][0] == pytest.approx(expected_w0, abs=1e-15)
    assert w[shell == 0][0] == pytest.approx(0.19756978203204612, abs=1e-15)


def test_weight_constraints_allweights():
    """Eq. (allWeights): seven constraints on the weights, to round-off."""
    th = oracle.theta0()
    r = oracle.weight_constraints()
    scale = np.array([1, th, th ** 2, th ** 2, th ** 3, th ** 3, th ** 4]) * np.array([1, 1, 3, 1, 21, 35, 945])
    assert np.all(np.abs(r) / scale < 2e-14), r / scale


def test_theta0_is_fixed_by_the_weights():
    """theta_0 is not printed; only one value satisfies Eq. (allWeights) with the Table I weights."""
    th = oracle.theta0()
    assert th == pytest.approx(0.2948964908710634, rel=1e-15)
    bad = oracle.weight_constraints(th * (1 + 1e-6))
    assert np.max(np.abs(bad[1:])) > 1e-8


def test_lattice_isotropy_dvmcond():
    """Eq. (dvmcond): for any psi(c^2), even moments are axis-independent and odd ones vanish."""
    c, w, _ = oracle.velocities()
    c2 = (c ** 2).sum(1)
    rng = np.random.default_rng(0)
    for _ in range(5):
        psi = w * (1 + rng.uniform(-1, 1) * c2 + rng.uniform(-1, 1) * c2 ** 2)
        for n in (1, 2, 3):
            mx, my, mz = [(psi * c[:, k] ** (2 * n)).sum() for k in range(3)]
            assert mx == pytest.approx(my, rel=1e-14) and mx == pytest.approx(mz, rel=1e-14)
            for m in (1, 2):
                a = (psi * c[:, 0] ** (2 * n) * c[:, 1] ** (2 * m)).sum()
                b = (psi * c[:, 1] ** (2 * n) * c[:, 2] ** (2 * m)).sum()
                assert a == pytest.approx(b, rel=1e-14)
            for k in range(3):
                assert abs((psi * c[:, k] ** (2 * n - 1)).sum()) < 1e-15
