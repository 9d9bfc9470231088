"""Whole-step pins of the oracle against continuum theory and symmetry.

Facts from the paper: isentropic sound speed c_s = sqrt(gamma theta_0),
gamma = 5/3 (Sec. I, Sec. VI); Prandtl number 1 and no bulk viscosity
(Sec. I, Sec. XI); nu = tau theta_0 (Sec. X, "tau = nu / c_s^2" with the
isothermal c_s^2 = theta_0, and the BGK beta = 1/(2 tau + 1), Sec. II).
From the linearised Navier-Stokes-Fourier equations (Sec. I) with these
values: a density wave at constant temperature splits into an acoustic part
(3/5 = 1/gamma of the amplitude) damped at (k^2/2)(4/3 nu + (gamma-1) chi) =
nu k^2, and an entropy part (2/5) decaying at chi k^2 = nu k^2; a shear wave
decays at nu k^2.  Lattice effects are O(k^2), so errors must shrink ~4x when
the wavelength doubles.

The grids are quasi-one-dimensional (nx x 1 x 1): a field that depends on x
only evolves identically on any periodic ny, nz.
"""
import math

import numpy as np
import pytest
from scipy.optimize import curve_fit

import oracle
from paper_1909_08406_gb300 import workloads as wl

NU = 0.01


def _run_mode(fields, N, tau, steps, project_fn):
    f = oracle.init_fields(fields["rho"].numpy(), fields["u"].numpy(), fields["theta"].numpy())
    out = []
    for _ in range(steps):
        rho, u, th = oracle.get_moments(f)
        out.append(project_fn(rho, u, th))
        f = oracle.step(f, tau, 1)
    return np.arange(steps, dtype=np.float64), np.array(out)


def _standing_wave_fit(N, theta0, steps=4000):
    tau = NU / theta0
    k = 2 * math.pi / N
    X, _, _ = wl.node_positions(N, 1, 1)
    S = np.sin(k * X.numpy())
    A = 1e-3
    t, a = _run_mode(wl.standing_wave(N, 1, 1, theta0, amplitude=A), N, tau, steps,
                     lambda rho, u, th: np.sum((rho - 1) * S) / np.sum(S * S) / A)
    cs = math.sqrt(5 * theta0 / 3)

    def model(t, As, w, phi, G, Ae, X):
        return As * np.cos(w * t + phi) * np.exp(-G * t) + Ae * np.exp(-X * t)

    p, _ = curve_fit(model, t, a, p0=[0.6, cs * k, 0.0, NU * k * k, 0.4, NU * k * k])
    return {"As": p[0], "Ae": p[4], "cs": p[1] / (cs * k), "G": p[3] / (NU * k * k), "chi": p[5] / (NU * k * k)}


@pytest.fixture(scope="module")
def wave32(theta0):
    return _standing_wave_fit(32, theta0)


@pytest.fixture(scope="module")
def wave64(theta0):
    return _standing_wave_fit(64, theta0)


def test_standing_wave_mode_split(wave32):
    """1/gamma of a constant-temperature density wave is acoustic, the rest entropic (gamma = 5/3)."""
    assert wave32["As"] == pytest.approx(0.6, abs=1e-3)
    assert wave32["Ae"] == pytest.approx(0.4, abs=1e-3)


def test_isentropic_sound_speed(wave32, wave64):
    assert wave32["cs"] == pytest.approx(1.0, abs=1e-3)
    assert wave64["cs"] == pytest.approx(1.0, abs=2.5e-4)
    # second-order convergence in the wavenumber
    assert abs(1 - wave64["cs"]) < abs(1 - wave32["cs"]) / 3


def test_acoustic_and_entropy_decay_rates(wave32, wave64):
    assert wave32["G"] == pytest.approx(1.0, abs=1e-2)
    assert wave32["chi"] == pytest.approx(1.0, abs=1e-2)
    assert wave64["G"] == pytest.approx(1.0, abs=5e-3)
    assert wave64["chi"] == pytest.approx(1.0, abs=3e-3)
    assert abs(1 - wave64["chi"]) < abs(1 - wave32["chi"]) / 3


def _decay_rate(gen, comp, N, theta0, steps=1500):
    tau = NU / theta0
    k = 2 * math.pi / N
    X, _, _ = wl.node_positions(N, 1, 1)
    X = X.numpy()
    B = np.sin(k * X) if comp == "uy" else np.cos(k * X)

    def proj(rho, u, th):
        q = u[1] if comp == "uy" else th / theta0 - 1
        return np.sum(q * B) / np.sum(B * B)

    t, a = _run_mode(gen(N, 1, 1, theta0, amplitude=1e-3), N, tau, steps, proj)
    slope = np.polyfit(t, np.log(np.abs(a)), 1)[0]
    return -slope / (NU * k * k)


def test_shear_viscosity_is_tau_theta0(theta0):
    r32 = _decay_rate(wl.shear_wave, "uy", 32, theta0)
    r64 = _decay_rate(wl.shear_wave, "uy", 64, theta0)
    assert r32 == pytest.approx(1.0, abs=5e-3)
    assert r64 == pytest.approx(1.0, abs=1.5e-3)
    assert abs(1 - r64) < abs(1 - r32) / 3


def test_isobaric_temperature_wave_prandtl_one(theta0):
    """An isobaric temperature wave is a pure entropy mode decaying at chi k^2, chi = nu (Pr = 1)."""
    r32 = _decay_rate(wl.isobaric_thermal_wave, "theta", 32, theta0)
    r64 = _decay_rate(wl.isobaric_thermal_wave, "theta", 64, theta0)
    assert r32 == pytest.approx(1.0, abs=1e-2)
    assert r64 == pytest.approx(1.0, abs=3e-3)
    assert abs(1 - r64) < abs(1 - r32) / 3


def test_global_conservation_over_many_steps(theta0):
    fields = wl.random_fields(6, 5, 4, theta0, seed=21, du=0.03, drho=0.03, dtheta=0.03)
    f0 = oracle.init_fields(fields["rho"].numpy(), fields["u"].numpy(), fields["theta"].numpy())
    c0 = oracle.conserved(f0)
    f = oracle.step(f0, 0.2, 300)
    c1 = oracle.conserved(f)
    assert abs(c1[0] - c0[0]) < 1e-12 * c0[0]
    assert np.max(np.abs(c1[1:4] - c0[1:4])) < 1e-12 * c0[0]
    assert abs(c1[4] - c0[4]) < 1e-12 * c0[4]


def _swap_xy(fields):
    rho = fields["rho"].numpy().transpose(0, 1, 3, 2)
    th = fields["theta"].numpy().transpose(0, 1, 3, 2)
    u = fields["u"].numpy().transpose(0, 1, 2, 4, 3)[[1, 0, 2]]
    return rho.copy(), u.copy(), th.copy()


def _reflect_x(rho, u, th):
    n = rho.shape[-1]
    ia = (-np.arange(n)) % n
    ib = (-np.arange(n) - 1) % n
    r = np.stack([rho[0][..., ia], rho[1][..., ib]])
    t = np.stack([th[0][..., ia], th[1][..., ib]])
    v = np.stack([np.stack([u[d][0][..., ia], u[d][1][..., ib]]) for d in range(3)])
    v[0] *= -1
    return r, v, t


def test_cubic_symmetry(theta0):
    """Swapping two axes, or reflecting one, commutes with the update (the velocity set is
    closed under the cube's symmetries, Sec. III)."""
    fields = wl.random_fields(5, 5, 3, theta0, seed=22)
    rho, u, th = fields["rho"].numpy(), fields["u"].numpy(), fields["theta"].numpy()
    steps = 15
    base = oracle.get_moments(oracle.step(oracle.init_fields(rho, u, th), 0.3, steps))

    r2, u2, t2 = _swap_xy(fields)
    out = oracle.get_moments(oracle.step(oracle.init_fields(r2, u2, t2), 0.3, steps))
    assert np.allclose(out[0], base[0].transpose(0, 1, 3, 2), rtol=0, atol=1e-13)
    assert np.allclose(out[1], base[1].transpose(0, 1, 2, 4, 3)[[1, 0, 2]], rtol=0, atol=1e-13)
    assert np.allclose(out[2], base[2].transpose(0, 1, 3, 2), rtol=0, atol=1e-13)

    r3, u3, t3 = _reflect_x(rho, u, th)
    out = oracle.get_moments(oracle.step(oracle.init_fields(r3, u3, t3), 0.3, steps))
    br, bu, bt = _reflect_x(*base)
    assert np.allclose(out[0], br, rtol=0, atol=1e-13)
    assert np.allclose(out[1], bu, rtol=0, atol=1e-13)
    assert np.allclose(out[2], bt, rtol=0, atol=1e-13)
