"""The isothermal nonideal fluid of Sec. "Nonideal Fluids and two-phase flow"
in the oracle (``oracle/nonideal.py``): the derivative stencil of Appendix A,
the momentum-conserving force of Eq. (gradientFinal), the three equations of
state (van der Waals, the Peng-Robinson type of Eq. (cspreos) and
Carnahan-Starling), and flat interfaces against Maxwell's equal-area
construction.

Pins, each independent of the oracle's formula:
  - each equation of state's free energy is consistent with its pressure
    (p = rho mu - F with mu = dF/drho, by finite differences), tends to the
    ideal gas at low density, and has its critical point where its constants
    put it: dp/drho = d2p/drho2 = 0 at (rho_c, theta_c), with the textbook
    critical compressibilities 3/8 (van der Waals) and 0.3590 at packing
    fraction 0.13044 (Carnahan-Starling); for the Peng-Robinson type this pins
    the printed formula against the printed ten-digit constants;
  - Maxwell's construction is solved to round-off (equal chemical potential
    and pressure, and equal areas) and reproduces the known van der Waals
    coexistence densities;
  - the stencil's gradient and Laplacian are second order and the corrected
    gradient of Eq. (gradient4) fourth order (error ratios 4 and 16 when the
    wavenumber halves);
  - the force conserves global momentum to round-off for any density field,
    the property the paper builds it for;
  - a flat interface at theta/theta_c = 0.9 settles on the coexisting
    densities of Maxwell's construction, for each equation of state;
  - a small density wave in either phase travels at the isothermal sound
    speed of the equation of state, sqrt(dp/drho), with an error that is
    second order in the wavenumber: the van der Waals fluid, and the
    experiment of Sec. "Sound propagation in a nonideal gas" itself, the
    Peng-Robinson type fluid at its coexisting phase densities."""
import functools
import os

import numpy as np
import pytest

import oracle
from oracle import nonideal as ni

TH0 = oracle.theta0()


EOS = {"vdw": ni.VdW, "peng_robinson": ni.PengRobinson, "carnahan_starling": ni.CarnahanStarling}


@pytest.mark.parametrize("name", list(EOS))
def test_equation_of_state_thermodynamics(name):
    e = EOS[name](0.9)
    r = np.linspace(0.05, 0.8 * min(e.rho_max(), 4.0), 400)
    # p = rho mu - F with the ideal parts theta0 rho (ln rho - 1) and theta0 ln rho added back
    F = TH0 * r * (np.log(r) - 1) + e.F_nid(r)
    assert np.abs(e.p(r) - (r * e.mu(r) - F)).max() <= 1e-14 * (1 + np.abs(e.p(r)).max())
    # mu_nid = dF_nid/drho by central differences (truncation h^2/6 times the third derivative)
    h = 1e-5
    dF = (e.F_nid(r + h) - e.F_nid(r - h)) / (2 * h)
    assert np.abs(e.mu_nid(r) - dF).max() <= 1e-8
    # the ideal gas at low density: F_nid and mu_nid vanish, p -> rho theta0
    lo = np.array([1e-9, 1e-7])
    assert np.abs(e.mu_nid(lo)).max() <= 1e-6 and np.abs(e.F_nid(lo)).max() <= 1e-13
    assert e.p(1e-7) / (1e-7 * TH0) == pytest.approx(1.0, abs=1e-6)


@pytest.mark.parametrize("name,Zc", [("vdw", 3 / 8), ("peng_robinson", None), ("carnahan_starling", 0.35896)])
def test_critical_point(name, Zc):
    e = EOS[name](1.0)  # theta0 = theta_c
    h = 1e-4
    p = e.p(np.array([1 - h, 1.0, 1 + h]))
    dp = (p[2] - p[0]) / (2 * h)
    d2p = (p[2] - 2 * p[1] + p[0]) / h ** 2
    assert abs(dp) <= 1e-8 * TH0 and abs(d2p) <= 1e-6 * TH0, (dp, d2p)
    if Zc is not None:
        assert p[1] / TH0 == pytest.approx(Zc, abs=2e-5)
    if name == "carnahan_starling":
        assert e.b / 4 == pytest.approx(0.13044, abs=1e-5)  # the critical packing fraction
    # a loop below theta_c, none above it
    r = np.linspace(0.05, 0.9 * min(e.rho_max(), 4.0), 20000)
    assert (np.gradient(EOS[name](0.9).p(r), r) < 0).any()
    assert (np.gradient(EOS[name](1.05).p(r), r)[: int(0.75 * len(r))] > 0).all()


def test_maxwell_construction():
    e = ni.VdW(0.9)
    g, l = e.maxwell()
    # van der Waals coexistence at T / T_c = 0.9, in units of the critical density
    assert g == pytest.approx(0.42574, abs=2e-5) and l == pytest.approx(1.65727, abs=2e-5)


@pytest.mark.parametrize("name,theta_star", [("vdw", 0.9), ("vdw", 0.7), ("peng_robinson", 0.9),
                                             ("peng_robinson", 0.8), ("carnahan_starling", 0.9),
                                             ("carnahan_starling", 0.7)])
def test_maxwell_equal_areas(name, theta_star):
    e = EOS[name](theta_star)
    g, l = e.maxwell()
    assert g < e.rho_scale() < l
    assert abs(e.mu(g) - e.mu(l)) <= 1e-14 and abs(e.p(g) - e.p(l)) <= 1e-14
    # the equal-area rule: the integral of p - p_sat over 1/rho between the phases vanishes
    v = np.linspace(1 / l, 1 / g, 200001)
    integrand = e.p(1 / v) - e.p(g)
    assert abs(np.trapezoid(integrand, v)) <= 1e-7 * e.p(g) * (1 / g - 1 / l)


def test_peng_robinson_has_no_coexistence_far_below_critical():
    """With the printed constants (no temperature factor in a) the Peng-Robinson type loop at
    theta/theta_c = 0.7 never rises back to a positive pressure before the attraction's pole:
    no liquid can coexist with a vapour there."""
    with pytest.raises(ValueError):
        ni.PengRobinson(0.7).maxwell()


def test_stencil_orders():
    nx = 64
    x = np.array([[[[ix + 0.5 * s for ix in range(nx)]]] for s in (0, 1)])
    errs = []
    for k in (4 * np.pi / nx, 2 * np.pi / nx):
        psi = np.sin(k * x)
        exact = k * np.cos(k * x)
        errs.append((np.abs(ni.grad2(psi)[0] - exact).max() / k, np.abs(ni.lap(psi) + k * k * psi).max() / (k * k),
                     np.abs(ni.grad4(psi)[0] - exact).max() / k))
    (g2a, la, g4a), (g2b, lb, g4b) = errs
    assert g2a / g2b == pytest.approx(4.0, rel=0.02) and la / lb == pytest.approx(4.0, rel=0.02)
    assert g4a / g4b == pytest.approx(16.0, rel=0.05)


def test_force_conserves_global_momentum():
    rng = np.random.default_rng(3)
    rho = 1.0 + 0.3 * np.clip(rng.standard_normal((2, 4, 3, 5)), -2, 2)
    g = ni.force(rho, ni.VdW(0.9), kappa=0.05)
    total = (rho[None] * g).sum(axis=(1, 2, 3, 4))
    assert np.abs(total).max() <= 1e-14 * rho.size
    assert np.abs(rho[None] * g).max() > 1e-2  # and it is not trivially zero
    # the chemical-potential formulation, rho g = -rho d2 mu, breaks it on the same field: the sum
    # of rho(n) [mu(n + 1) - mu(n - 1)] does not telescope (Eq. chempotbad)
    e = ni.VdW(0.9)
    total_mu = (-rho[None] * ni.grad2(e.mu_nid(rho))).sum(axis=(1, 2, 3, 4))
    assert np.abs(total_mu).max() > 1e-3


@functools.lru_cache(maxsize=None)
def interface(theta_star=0.9, kappa=0.05, tau=0.5, nx=64, steps=1500, width=3.0, eos=ni.VdW, eta=0.5):
    """A liquid slab in vapour (flat interfaces normal to x), started at the Maxwell densities
    with tanh profiles; returns the bulk densities after `steps` and Maxwell's."""
    e = eos(theta_star)
    g, l = e.maxwell()
    x = np.array([[[[ix + 0.5 * s for ix in range(nx)]]] for s in (0, 1)])
    rho = g + (l - g) * 0.5 * (np.tanh((x - nx / 4) / width) - np.tanh((x - 3 * nx / 4) / width))
    f = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    f = ni.step(f, tau, e, kappa, nsteps=steps, eta=eta)
    r = f.sum(axis=1)
    return r[0, 0, 0, 0], r[0, 0, 0, nx // 2], g, l


# (equation of state, kappa, vapour bound, liquid bound); measured: van der Waals +1.5% / +0.13%,
# Peng-Robinson type +1.9% / +0.23% (density ratio 9.1), Carnahan-Starling +3.1% / +0.21% (5.5).
# The two with the Carnahan-Starling repulsion take kappa = 0.02: at 0.05 the Peng-Robinson
# slab diverges.
INTERFACES = [("vdw", 0.05, 0.02, 0.003), ("peng_robinson", 0.02, 0.025, 0.004),
              ("carnahan_starling", 0.02, 0.04, 0.004)]


@pytest.mark.parametrize("name,kappa,gas_tol,liquid_tol", INTERFACES)
def test_flat_interface_reaches_maxwell_densities(name, kappa, gas_tol, liquid_tol):
    gas, liquid, g, l = interface(kappa=kappa, eos=EOS[name])
    assert abs(gas / g - 1) <= gas_tol and abs(liquid / l - 1) <= liquid_tol, (gas, liquid, g, l)


def _sound_speed(rho0, nx, eos, eps=1e-4, tau=0.5, kappa=0.05):
    """Speed of a standing density wave of one wavelength over nx cells in a uniform phase, from
    the zero crossings of its amplitude over about 1.6 periods."""
    x = np.array([[[[ix + 0.5 * s for ix in range(nx)]]] for s in (0, 1)])
    k = 2 * np.pi / nx
    cs2 = (eos.p(rho0 + 1e-7) - eos.p(rho0 - 1e-7)) / 2e-7
    rho = rho0 * (1 + eps * np.cos(k * x))
    f = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    cosx = np.cos(k * x)
    amp = []
    for _ in range(int(1.6 * 2 * np.pi / (k * np.sqrt(cs2)))):
        amp.append(((f.sum(axis=1) - rho0) * cosx).sum() / (cosx * cosx).sum())
        f = ni.step(f, tau, eos, kappa)
    a = np.array(amp)
    zc = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    return np.pi / (k * np.diff(zc).mean()), np.sqrt(cs2)


@pytest.mark.parametrize("rho0", [0.3, 1.7])  # vapour and liquid side of theta/theta_c = 0.9
def test_sound_speed_in_a_nonideal_phase(rho0):
    e = ni.VdW(0.9)
    c64, exact = _sound_speed(rho0, 64, e)
    c128, _ = _sound_speed(rho0, 128, e)
    e64, e128 = abs(c64 / exact - 1), abs(c128 / exact - 1)
    assert e64 <= 3e-3, (c64, exact)  # measured 1.2e-3 (vapour), 1.8e-3 (liquid)
    assert e64 / e128 >= 3.5, (e64, e128)  # second order: 4.0 measured


@pytest.mark.parametrize("phase", [0, 1])
def test_sound_speed_in_peng_robinson_phases(phase):
    """Sec. "Sound propagation in a nonideal gas": a small wave in each coexisting phase of the
    Peng-Robinson type fluid of Eq. (cspreos) at theta/theta_c = 0.9 (vapour 0.272, liquid 2.470)
    travels at sqrt(dp/drho); kappa = 0.02, with which its interface is stable."""
    e = ni.PengRobinson(0.9)
    rho0 = e.maxwell()[phase]
    c64, exact = _sound_speed(rho0, 64, e, kappa=0.02)
    c128, _ = _sound_speed(rho0, 128, e, kappa=0.02)
    e64, e128 = abs(c64 / exact - 1), abs(c128 / exact - 1)
    assert e64 <= 4e-3, (c64, exact)  # measured 1.6e-3 (vapour), 2.7e-3 (liquid)
    assert e64 / e128 >= 3.5, (e64, e128)  # second order: 4.0 measured


def quench(name, kappa, shape=(32, 32, 1), steps=1000, noise=0.01, seed=11, theta_star=0.9):
    """Sec. "Quenching of a liquid-gas system": a fluid at the critical density with 1% noise,
    below the critical temperature, separates into its two phases. Returns the equation of
    state, the initial and the final density fields."""
    e = EOS[name](theta_star)
    nx, ny, nz = shape
    rho = e.rho_scale() * (1 + noise * np.random.default_rng(seed).standard_normal((2, nz, ny, nx)))
    f = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    f = ni.step(f, 0.5, e, kappa, nsteps=steps)
    return e, rho, f.sum(axis=1)


# (equation of state, kappa, vapour bound, liquid bound) on the 5% and 95% density quantiles;
# measured after 1000 steps (converged from about 1000): van der Waals +1.56% / +0.10%,
# Peng-Robinson type +1.89% / -0.43% (its liquid, a third of the box, forms a curved region),
# Carnahan-Starling +3.07% / +0.19%
QUENCHES = [("vdw", 0.05, 0.02, 0.003), ("peng_robinson", 0.02, 0.025, 0.006),
            ("carnahan_starling", 0.02, 0.04, 0.004)]


@pytest.mark.parametrize("name,kappa,gas_tol,liquid_tol", QUENCHES)
def test_quench_separates_into_maxwell_phases(name, kappa, gas_tol, liquid_tol):
    e, rho0, rho = quench(name, kappa)
    g, l = e.maxwell()
    assert abs(rho.sum() - rho0.sum()) <= 1e-12 * rho.size
    gas, liquid = np.quantile(rho, 0.05), np.quantile(rho, 0.95)
    assert abs(gas / g - 1) <= gas_tol and abs(liquid / l - 1) <= liquid_tol, (gas, liquid, g, l)


def _golden_spurious():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "spurious_currents.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, pr, cs = line.split()
                rows[name] = {"peng_robinson": float(pr), "carnahan_starling": float(cs)}
    return rows


def droplet(name, eta, kappa=0.02, n=48, steps=1000, theta_star=0.9):
    """A static cylindrical liquid drop (radius n/4, tanh profile of width 2) in its vapour on an
    n x n x 1 grid. Returns the largest fluid speed |sum f c / rho + g / 2| after `steps` (the
    spurious current; the exact answer is 0) and the vapour density relative to Maxwell's."""
    e = EOS[name](theta_star)
    g, l = e.maxwell()
    s = np.arange(2)[:, None, None, None] * 0.5
    x = np.arange(n)[None, None, None, :] + s
    y = np.arange(n)[None, None, :, None] + s
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2) + np.zeros((2, 1, n, n))
    rho = g + (l - g) * 0.5 * (1 - np.tanh((r - n / 4) / 2.0))
    f = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    f = ni.step(f, 0.5, e, kappa, nsteps=steps, eta=eta)
    fpre = oracle.stream(f)
    rr = fpre.sum(axis=1)
    u = np.einsum("sqzyx,qa->aszyx", fpre, oracle.velocities()[0]) / rr + 0.5 * ni.force(rr, e, kappa, eta)
    return np.sqrt((u ** 2).sum(0)).max(), rr.min() / g - 1


@pytest.mark.parametrize("name", ["peng_robinson", "carnahan_starling"])
def test_eta_half_reduces_spurious_currents(name):
    """The printed table: Eq. (gradientFinal) with eta = 1/2 has smaller spurious currents than
    with eta = 1 (ratios 0.59 and 0.67 there). Measured on a 48 x 48 drop: 0.79 (Peng-Robinson
    type) and 0.69 (Carnahan-Starling); the vapour density is also closer to Maxwell's (+6.3%
    against +25%, and +6.4% against +16%, the drop's Laplace pressure included)."""
    paper = _golden_spurious()
    assert paper["current_eta_half"][name] < paper["current_eta_1"][name]
    u_half, gas_half = droplet(name, 0.5)
    u_one, gas_one = droplet(name, 1.0)
    assert u_half <= 0.85 * u_one, (u_half, u_one)
    assert abs(gas_half) < 0.5 * abs(gas_one), (gas_half, gas_one)


@pytest.mark.parametrize("theta_star,phase,tol", [(0.8, 0, 2e-3), (0.8, 1, 3e-3), (0.85, 0, 2e-3),
                                                  (0.85, 1, 3e-3), (0.95, 0, 6e-3), (0.95, 1, 8e-3)])
def test_sound_speed_across_temperatures(theta_star, phase, tol):
    """The sound-speed figure of Sec. "Sound propagation in a nonideal gas" spans temperatures: at
    64 cells per wavelength the wave speed follows sqrt(dp/drho) of the Peng-Robinson type fluid
    from 0.23 to 0.67 over theta/theta_c = 0.8 to 0.95 in both phases. Measured errors 5e-4 to
    5.7e-3, largest near the critical point, where the phases approach each other."""
    e = ni.PengRobinson(theta_star)
    c, exact = _sound_speed(e.maxwell()[phase], 64, e, kappa=0.02)
    assert abs(c / exact - 1) <= tol, (c, exact)


@pytest.mark.parametrize("tau", [0.5, 0.05])
def test_forced_collision_changes_momentum_by_rho_g(tau):
    """Eq. (momentumchange): the forced collision of Eq. (multiphaseEvolution) with
    u = j / rho + g / 2 keeps the mass and adds exactly rho g to the momentum of every node,
    for any tau (the forcing term carries no mass, its momentum is rho g, and the relaxation
    removes the half added to u)."""
    import ctypes
    rng = np.random.default_rng(21)
    nx, ny, nz = 4, 3, 2
    shape = (2, nz, ny, nx)
    rho = 1.0 + 0.3 * rng.random(shape)
    u = 0.05 * rng.standard_normal((3,) + shape)
    fpre = oracle.init_fields(rho, u, np.full(shape, TH0))
    fpre = fpre * (1 + 0.01 * rng.standard_normal(fpre.shape))  # off equilibrium
    g = np.ascontiguousarray(0.02 * rng.standard_normal((3,) + shape))
    out = np.empty_like(fpre)
    oracle.lib().or_collide_forced(ctypes.c_int64(nx), ctypes.c_int64(ny), ctypes.c_int64(nz), ctypes.c_double(tau),
                                   ctypes.c_int(1), oracle._p(fpre), oracle._p(g), oracle._p(out), oracle._threads(1))
    c = oracle.velocities()[0]
    r0, r1 = fpre.sum(axis=1), out.sum(axis=1)
    j0 = np.einsum("sqzyx,qa->aszyx", fpre, c)
    j1 = np.einsum("sqzyx,qa->aszyx", out, c)
    assert np.abs(r1 - r0).max() <= 1e-14
    assert np.abs(j1 - (j0 + r0[None] * g)).max() <= 1e-14


def test_carnahan_starling_slab_at_the_droplet_collision_parameters():
    """Sec. "Droplet Collision" runs the Carnahan-Starling fluid at theta/theta_c = 0.8 (density
    ratio 14) with nu_liq = 0.0303, so tau = nu / theta0 = 0.103, and kappa = 0.001 a. A flat
    slab at those parameters stays stable and settles at +14% (vapour) and +0.27% (liquid) of
    Maxwell's densities after 3000 steps (the thin interface of the small kappa costs vapour
    accuracy); at tau = 0.5 the same slab diverges."""
    e = ni.CarnahanStarling(0.8)
    gas, liquid, g, l = interface(theta_star=0.8, kappa=0.001 * e.a, tau=0.103, steps=3000, eos=ni.CarnahanStarling)
    assert np.isfinite(gas) and np.isfinite(liquid)
    assert abs(gas / g - 1) <= 0.16 and abs(liquid / l - 1) <= 0.005, (gas, liquid, g, l)


def _drop_pressure_jump(radius, n=48, steps=1000, kappa=0.05):
    """(equimolar radius, p_inside - p_outside) of a settled cylindrical van der Waals drop at
    theta/theta_c = 0.9 on an n x n x 1 grid, the pressures from the equation of state at the
    drop's centre and far corner."""
    e = ni.VdW(0.9)
    g, l = e.maxwell()
    s = np.arange(2)[:, None, None, None] * 0.5
    x = np.arange(n)[None, None, None, :] + s
    y = np.arange(n)[None, None, :, None] + s
    r = np.sqrt((x - n / 2) ** 2 + (y - n / 2) ** 2) + np.zeros((2, 1, n, n))
    rho = g + (l - g) * 0.5 * (1 - np.tanh((r - radius) / 3.0))
    f = oracle.init_fields(rho, np.zeros((3,) + rho.shape), np.full(rho.shape, TH0))
    rho = ni.step(f, 0.5, e, kappa, nsteps=steps).sum(axis=1)
    inside, outside = rho[0, 0, n // 2, n // 2], rho[0, 0, 0, 0]
    # each node stands for half a cell of the z = const plane
    r_eq = np.sqrt(0.5 * (rho - outside).sum() / (np.pi * (inside - outside)))
    return r_eq, e.p(inside) - e.p(outside)


def test_laplace_law_for_drops():
    """Young-Laplace for a cylinder: the pressure jump across a drop's interface is
    sigma / R, the same surface tension for every radius. Measured dp R = 0.02857 (R 7.4) and
    0.02986 (R 11.8) here, and 0.0297-0.0299 for R 9 to 18 on a 64-cell box: within 4.5%, the
    smallest drop's interface being a third of its radius. (The surface tension is about twice
    kappa times the integral of (drho/dx)^2 of the flat profile: the discrete force adds an
    interfacial stiffness of its own, about 0.07 at theta/theta_c = 0.9.)"""
    r1, dp1 = _drop_pressure_jump(8)
    r2, dp2 = _drop_pressure_jump(12)
    assert r1 < r2 and dp1 > dp2 > 0
    assert abs((dp1 * r1) / (dp2 * r2) - 1) <= 0.07, (dp1 * r1, dp2 * r2)


def _plane_wave_errors(m, n=48):
    """Relative errors of grad2 and lap on sin(k.x), k = 2 pi m / n, over the whole bcc grid (the
    projection of the discrete result on the exact one, minus 1), and |k|^2."""
    s = np.arange(2)[:, None, None, None] * 0.5
    z = np.arange(n)[None, :, None, None] + s
    y = np.arange(n)[None, None, :, None] + s
    x = np.arange(n)[None, None, None, :] + s
    k = 2 * np.pi * np.asarray(m, float) / n
    phase = k[0] * x + k[1] * y + k[2] * z
    psi = np.sin(phase)
    exact = np.array([k[a] * np.cos(phase) for a in range(3)])
    g = ni.grad2(psi)
    kk = float(k @ k)
    return kk, (g * exact).sum() / (exact * exact).sum() - 1, (ni.lap(psi) * psi).sum() / (-kk * (psi * psi).sum()) - 1


def test_stencil_is_isotropic():
    """Appendix A: the 15-velocity stencil's derivatives err isotropically at leading order, with
    theta_hat = 1/6: on a plane wave grad2 is short by theta_hat k^2 / 2 and the Laplacian by
    theta_hat k^2 / 4 whatever the wave's direction. Along x the stencil sums in closed form to
    (sin k + 4 sin(k/2)) / (3k) = 1 - k^2/12 + k^4/320 - ... and
    12 (1/2 - cos(k)/18 - 4 cos(k/2)/9) / k^2 = 1 - k^2/24 + ...; the direction enters only at
    k^4 (the stencil's sixth moments are not isotropic): measured differences 1.6e-5 and 5e-6
    against errors of 1.3e-2 and 6.4e-3 for |k| = 2 pi 3 / 48 along (1,0,0) and (2,2,1)/3."""
    th = 1.0 / 6.0
    kk, g_axis, l_axis = _plane_wave_errors((3, 0, 0))
    kk2, g_diag, l_diag = _plane_wave_errors((2, 2, 1))
    assert kk == pytest.approx(kk2, rel=1e-14)
    for g_err, l_err in ((g_axis, l_axis), (g_diag, l_diag)):
        assert g_err / (-th * kk / 2) == pytest.approx(1.0, abs=0.02)
        assert l_err / (-th * kk / 4) == pytest.approx(1.0, abs=0.02)
    k = np.sqrt(kk)
    assert g_axis == pytest.approx((np.sin(k) + 4 * np.sin(k / 2)) / (3 * k) - 1, abs=1e-12)
    assert l_axis == pytest.approx(12 * (0.5 - np.cos(k) / 18 - 4 * np.cos(k / 2) / 9) / kk - 1, abs=1e-12)
    assert abs(g_axis - g_diag) <= 1e-4 and abs(l_axis - l_diag) <= 5e-5


@pytest.mark.parametrize("name,kappa", [("vdw", 0.05), ("peng_robinson", 0.02)])
def test_eta_half_brings_the_vapour_to_maxwell(name, kappa):
    """The densities figure of the discretisation section: Eq. (gradientFinal) with eta = 1/2
    (half of the free-energy gradient at fourth order) puts the coexisting densities of a flat
    interface closer to Maxwell's than eta = 1 (all at second order). Measured vapour errors:
    +1.5% against +5.9% (van der Waals), +1.9% against +21.8% (Peng-Robinson type)."""
    gas_h, liq_h, g, l = interface(kappa=kappa, eos=EOS[name])  # shared with the flat-interface test
    gas_1, liq_1, _, _ = interface(kappa=kappa, eos=EOS[name], eta=1.0)
    assert abs(gas_h / g - 1) <= 0.4 * abs(gas_1 / g - 1), (gas_h, gas_1, g)
    assert abs(liq_h / l - 1) <= 0.5 * abs(liq_1 / l - 1), (liq_h, liq_1, l)
