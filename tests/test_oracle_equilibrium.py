"""Pins of the oracle's equilibria and collision.

Independent facts used: exact rest-state moments implied by Eq. (allWeights);
the M_2, M_2', M_3, M_3' coefficients printed in Sec. V (golden file); the
cubic Hermite equilibrium of Sec. II at theta = theta_0; the exact entropic
minimiser of Eqs. (discreteentropiceq)/(fivelagrangemultipliersystem) solved
by Newton; exact conservation of the collision invariants.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def lat():
    c, w, shell = oracle.velocities()
    return c, w, shell, (c ** 2).sum(1)


def _moments(f, c, c2):
    return f.sum(), f @ c, f @ c2


def test_rest_equilibrium_exact_moments(lat, theta0):
    c, w, _, c2 = lat
    rng = np.random.default_rng(1)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        theta = theta0 * (1 + rng.uniform(-0.1, 0.1))
        ft = oracle.rest_equilibrium(rho, theta)
        assert ft.sum() == pytest.approx(rho, rel=1e-14)
        assert np.max(np.abs(ft @ c)) < 1e-15 * rho
        P = (ft[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
        assert np.allclose(P, rho * theta * np.eye(3), rtol=0, atol=1e-14 * rho * theta)
        assert ft @ c2 == pytest.approx(3 * rho * theta, rel=1e-14)


def test_rest_equilibrium_heat_flux_moment(lat, theta0):
    """R_ab(u=0) = <f~, c^2 c_a c_b> = 5 rho theta^2 (1 + M_2) with M_2 = O(eta^3) (Sec. III, V)."""
    c, _, _, c2 = lat
    for eta in (1e-2, 2e-2, 4e-2):
        theta = theta0 * (1 + eta)
        ft = oracle.rest_equilibrium(1.0, theta)
        R = (ft * c2 * c[:, 0] ** 2).sum() / (5 * theta ** 2) - 1
        Rh = (oracle.rest_equilibrium(1.0, theta0 * (1 + eta / 2)) * c2 * c[:, 0] ** 2).sum() / (
            5 * (theta0 * (1 + eta / 2)) ** 2) - 1
        assert R / Rh == pytest.approx(8.0, rel=0.05)  # cubic in eta


def _golden_m():
    out = {}
    with open(os.path.join(GOLDEN, "m_coefficients.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, p, pre, c1, c2, c3, _ = line.split()
            out[name] = (int(p), float(pre) * np.array([float(c1), float(c2), float(c3)]))
    return out


def test_m_coefficients_match_printed(theta0):
    """The departures M_2, M_2', M_3, M_3' computed from Table I reproduce the printed polynomials."""
    golden = _golden_m()
    etas = np.linspace(-0.05, 0.05, 41)
    for k, name in enumerate(["M2", "M2p", "M3", "M3p"]):
        p, printed = golden[name]
        vals = np.array([oracle.m_terms(1.0, theta0 * (1 + e))[k] * (1 + e) ** p for e in etas])
        coef = np.polynomial.polynomial.polyfit(etas, vals, 3)
        assert abs(coef[0]) < 1e-13, name
        for j in range(3):
            if printed[j] == 0:
                assert abs(coef[j + 1]) < 1e-11, (name, j, coef)
            else:
                assert coef[j + 1] == pytest.approx(printed[j], rel=5e-6), (name, j, coef)


def _hermite3(rho, u, th, c, w):
    """Cubic Hermite equilibrium of Sec. II (isothermal, reference temperature th)."""
    uc = c @ u
    usq = u @ u
    return w * rho * (1 + uc / th + (uc ** 2 - th * usq) / (2 * th ** 2) + (uc ** 3 - 3 * th * usq * uc) / (6 * th ** 3))


@pytest.mark.parametrize("project", [True, False])
def test_equilibrium_reduces_to_cubic_hermite(lat, theta0, project):
    c, w, _, _ = lat
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = oracle.equilibrium(rho, u, theta0, project)
        ref = _hermite3(rho, u, theta0, c, w)
        assert np.max(np.abs(feq - ref) / ref) < 1e-14


def test_equilibrium_converges_to_entropic_minimiser(theta0):
    """The series equilibrium approximates the exact entropic one; the gap is O(eps^4)."""
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.uniform(-1, 1, 3)
        g = rng.uniform(-1, 1)
        errs = []
        for eps in (4e-3, 2e-3, 1e-3):
            u = eps * d
            theta = theta0 * (1 + eps * g)
            a = oracle.equilibrium(1.0, u, theta, True)
            b = oracle.entropic_equilibrium(1.0, u, theta)
            errs.append(np.max(np.abs(a - b) / b))
        assert errs[-1] < 1e-10
        assert 12 < errs[0] / errs[1] < 20 and 12 < errs[1] / errs[2] < 20, errs


def test_entropic_solver_hits_constraints(lat, theta0):
    c, _, _, c2 = lat
    u = np.array([0.05, -0.02, 0.01])
    theta = theta0 * 1.03
    f = oracle.entropic_equilibrium(1.1, u, theta)
    r, j, k = _moments(f, c, c2)
    assert r == pytest.approx(1.1, rel=1e-14)
    assert np.allclose(j, 1.1 * u, rtol=0, atol=1e-15)
    assert k == pytest.approx(1.1 * (u @ u) + 3 * 1.1 * theta, rel=1e-14)


def _near_equilibrium(rng, theta0, du=0.1, deta=0.05, noise=0.05):
    rho = rng.uniform(0.8, 1.2)
    u = rng.uniform(-du, du, 3)
    theta = theta0 * (1 + rng.uniform(-deta, deta))
    feq = oracle.equilibrium(rho, u, theta, True)
    return feq * (1 + noise * rng.uniform(-1, 1, 41))


def test_collision_conserves_invariants(lat, theta0):
    c, _, _, c2 = lat
    rng = np.random.default_rng(4)
    for tau in (0.0339, 0.51, 1.0, 5.0):
        for _ in range(20):
            f = _near_equilibrium(rng, theta0)
            g = oracle.collide(f, tau, True)
            r0, j0, k0 = _moments(f, c, c2)
            r1, j1, k1 = _moments(g, c, c2)
            # round-off of 41-term sums: a few units of 1e-16
            assert abs(r1 - r0) < 4e-15 * r0
            assert np.max(np.abs(j1 - j0)) < 4e-15 * r0
            assert abs(k1 - k0) < 1e-14 * k0


def test_equilibrium_is_fixed_point(theta0):
    rng = np.random.default_rng(5)
    for _ in range(10):
        feq = oracle.equilibrium(rng.uniform(0.9, 1.1), rng.uniform(-0.05, 0.05, 3), theta0 * rng.uniform(0.97, 1.03))
        assert np.max(np.abs(oracle.collide(feq, 0.3, True) - feq) / feq) < 1e-14


def test_unprojected_momentum_defect_scaling(lat, theta0):
    """The printed series violates momentum conservation at O(u^3 eta^2) (cubic-lattice
    anisotropy of f~); the projected equilibrium removes it."""
    c, _, _, _ = lat
    d = np.array([0.8, -0.5, 0.3])

    def defect(us, eta, project):
        u = us * d
        f = oracle.equilibrium(1.0, u, theta0 * (1 + eta), project)
        return np.max(np.abs(f @ c - u))

    base = defect(0.1, 0.05, False)
    assert base > 1e-9
    assert defect(0.2, 0.05, False) / base == pytest.approx(8.0, rel=1e-6)  # cubic in u
    # quadratic in eta at leading order (an eta^3 term of opposite sign follows)
    assert defect(0.1, 0.002, False) / defect(0.1, 0.001, False) == pytest.approx(4.0, rel=0.03)
    assert defect(0.1, 0.05, True) < 1e-16


def test_second_moment_at_reference_temperature(lat, theta0):
    """At theta = theta_0 the equilibrium stress is rho u u + rho theta_0 I (Sec. II)."""
    c, _, _, _ = lat
    u = np.array([0.03, -0.07, 0.05])
    f = oracle.equilibrium(1.2, u, theta0, True)
    P = (f[:, None, None] * c[:, :, None] * c[:, None, :]).sum(0)
    assert np.allclose(P, 1.2 * np.outer(u, u) + 1.2 * theta0 * np.eye(3), rtol=0, atol=1e-15)


def test_entropic_collision_conserves_and_fixes_equilibrium():
    """With the exact entropic equilibrium the collision keeps rho, rho u and the energy to
    round-off for states far from rest, and leaves an entropic equilibrium unchanged."""
    rng = np.random.default_rng(41)
    c, w, _ = oracle.velocities()
    for _ in range(5):
        f = w * (1.0 + 0.3 * rng.uniform(-1, 1, size=41))
        out = oracle.collide(f, 0.4, project="entropic")
        m0, m1 = oracle.moments(f), oracle.moments(out)
        for a, b in zip(m0, m1):
            assert np.allclose(a, b, rtol=0, atol=1e-14)
    feq = oracle.entropic_equilibrium(1.05, np.array([0.1, -0.05, 0.02]), 1.1 * oracle.theta0())
    assert np.allclose(oracle.collide(feq, 0.4, project="entropic"), feq, rtol=1e-13, atol=0)
