"""Kinetic (diffuse) walls normal to z in the oracle (Sec. "Viscous heat
dissipation": kinetic boundary conditions at the walls, periodic in the other
two directions).

Pins, none of which restates the oracle's formula:
  - a gas at rest at the walls' temperature stays exactly at rest, with the
    walls' density 1 (every absorbed population comes back as the same
    equilibrium value);
  - the walls conserve mass to round-off while they exchange momentum and
    energy with the gas;
  - mirroring the channel (z -> -z with the half-cell shift that keeps the bcc
    grid on itself, walls swapped) mirrors the solution, which catches a
    misplaced top wall;
  - Couette flow with viscous heating reaches the steady temperature profile of
    Eq. (eckert), (T - T0)/dT = y/H + Ec/2 (y/H)(1 - y/H), and the linear
    velocity profile, at first order in 1/H (the kinetic boundary layer: the
    temperature jump and velocity slip at a diffuse wall are of the order of a
    mean free path);
  - a wall whose temperature varies along it (theta0 (1 + a cos kx) below,
    theta0 above) leads to the steady conduction field of Laplace's equation,
    a cos(kx) sinh(k (H - y)) / sinh(kH), again at first order in 1/H: the
    wall condition acts column by column;
  - the paper's cavity heated at the top (Sec. "2D cavity heated at the top"):
    its steady temperature is the sine series printed there.  The side walls
    at T0 are represented by images: over a period of two cavity widths the
    top wall is at T0 + dT on one width and T0 - dT on the next, whose
    solution is odd about both side-wall planes and so equals T0 on them.  At
    the paper's sections (x/L = 0.1, 0.2, 0.5 and y/H = 0.25, 0.5, 0.75) the
    lattice Boltzmann field matches the series within 0.045 dT at L = H = 16."""
import math

import numpy as np
import pytest

import oracle
from oracle.conduction import cavity_series
from paper_1909_08406_gb300 import workloads as wl

TH0 = oracle.theta0()


def _rest(nx, ny, nz):
    rho = np.ones((2, nz, ny, nx))
    u = np.zeros((3, 2, nz, ny, nx))
    th = np.full((2, nz, ny, nx), TH0)
    return oracle.init_fields(rho, u, th)


def test_rest_state_is_a_fixed_point():
    f0 = _rest(3, 2, 6)
    f1, rho_w = oracle.step_walls(f0, 0.3, 20, (0.0, 0.0, TH0), (0.0, 0.0, TH0), wall_rho=True)
    assert np.abs(f1 - f0).max() <= 1e-13 * f0.max()
    assert np.abs(rho_w - 1.0).max() <= 1e-13


def _random(nx, ny, nz, seed):
    fl = wl.random_fields(nx, ny, nz, TH0, seed=seed, du=0.03, drho=0.03, dtheta=0.03)
    return oracle.init_fields(fl["rho"].numpy(), fl["u"].numpy(), fl["theta"].numpy())


BOTTOM = (0.02, -0.01, TH0 * 1.01)
TOP = (-0.03, 0.0, TH0 * 0.98)


def test_walls_conserve_mass_and_exchange_momentum_and_energy():
    f0 = _random(3, 2, 6, 3)
    c0 = oracle.conserved(f0)
    f1 = oracle.step_walls(f0, 0.3, 50, BOTTOM, TOP)
    c1 = oracle.conserved(f1)
    assert abs(c1[0] - c0[0]) <= 1e-13 * c0[0]
    assert np.abs(c1[1:] - c0[1:]).max() > 1e-3  # the walls push and heat or cool the gas
    # the same state stepped periodically keeps every invariant
    c2 = oracle.conserved(oracle.step(f0, 0.3, 50))
    assert np.abs(c2 - c0).max() <= 1e-12 * c0[0]


def _mirror(f):
    """The channel reflected about its mid-plane: in doubled coordinates
    (x2, y2, z2) -> (x2 + 1, y2 + 1, 2 nz - 1 - z2), velocities c_z -> -c_z.  A reflection
    in z alone would send a node of one sub-lattice to no node at all; with the half-cell
    shift in x and y (a symmetry of the periodic bcc grid) A (x, y, z) goes to
    B (x, y, nz - 1 - z) and B (x, y, z) to A (x + 1, y + 1, nz - 1 - z)."""
    c2 = oracle.velocities_doubled()
    refl = np.array([int(np.where((c2 == v * np.array([1, 1, -1])).all(1))[0][0]) for v in c2])
    g = np.empty_like(f)
    g[1] = f[0][refl][:, ::-1]
    g[0] = np.roll(f[1][refl][:, ::-1], (1, 1), axis=(2, 3))
    return g


def test_mirrored_channel_gives_the_mirrored_solution():
    f0 = _random(4, 3, 5, 7)
    a = oracle.step_walls(f0, 0.4, 12, BOTTOM, TOP)
    b = oracle.step_walls(_mirror(f0), 0.4, 12, TOP, BOTTOM)
    assert np.abs(_mirror(a) - b).max() <= 1e-14 * f0.max()


def _couette(H, ec, nu=0.05, u0=0.02):
    """Steady Couette flow between a still wall at T0 (bottom) and a wall moving at u0 at
    T1 = T0 + dT (top), dT = u0^2 / (c_p Ec), c_p = 5/2, the walls at theta0 -+ dT/2 as in
    the paper's runs; returns y/H, (T - T0)/dT and u/u0 at every node plane, and the exact
    temperature profile."""
    dT = u0 * u0 / (2.5 * ec)
    f = _rest(1, 1, H)
    f = oracle.step_walls(f, nu / TH0, int(3 * H * H / nu), (0.0, 0.0, TH0 - dT / 2), (u0, 0.0, TH0 + dT / 2))
    _, u, th = oracle.get_moments(f)
    z2 = np.array([[2 * z + s for z in range(H)] for s in range(2)]).ravel()
    y = (z2 / 2.0 + 0.25) / H  # walls a quarter cell beyond the outermost node planes
    o = np.argsort(y)
    y = y[o]
    tn = ((th.reshape(2, H) - (TH0 - dT / 2)) / dT).ravel()[o]
    un = (u[0].reshape(2, H) / u0).ravel()[o]
    return y, tn, un, y + ec / 2 * y * (1 - y)


def test_couette_viscous_heating_converges_to_eq_eckert():
    errs = []
    for H in (8, 16):
        y, tn, un, ex = _couette(H, 2.0)
        errs.append((np.abs(tn - ex).max(), np.abs(un - y).max()))
    (t8, u8), (t16, u16) = errs
    assert t16 <= 0.04 and u16 <= 0.01, errs  # measured 0.037, 0.0079
    assert t8 / t16 >= 1.8 and u8 / u16 >= 1.8, errs  # first order (measured 1.93, 1.97)


@pytest.mark.parametrize("ec,bound", [(0.5, 0.03), (5.0, 0.07)])
def test_couette_eckert_numbers_of_the_paper(ec, bound):
    y, tn, un, ex = _couette(16, ec)
    assert np.abs(tn - ex).max() <= bound, np.abs(tn - ex).max()
    # at Ec = 5 the viscous heating lifts the gas above the hot wall's temperature
    assert (tn.max() > 1.1) == (ex.max() > 1.1)


def _laplace(nx, H, nu=0.1, a=0.01):
    k = 2 * math.pi / nx
    # bottom wall column x covers the doubled lateral positions 2x, 2x + 1: centre x + 1/4
    tb = (TH0 * (1 + a * np.cos(k * (np.arange(nx) + 0.25))))[None, :]
    f = oracle.init_fields(np.ones((2, H, 1, nx)), np.zeros((3, 2, H, 1, nx)), np.full((2, H, 1, nx), TH0))
    f = oracle.step_walls(f, nu / TH0, int(4 * H * H / (5.0 / 3.0 * nu)), (0.0, 0.0, tb), (0.0, 0.0, TH0))
    _, _, th = oracle.get_moments(f)
    err = 0.0
    for s in (0, 1):
        X = np.arange(nx) + 0.5 * s
        for z in range(H):
            Y = z + 0.5 * s + 0.25  # distance from the bottom wall
            exact = a * np.cos(k * X) * np.sinh(k * (H - Y)) / np.sinh(k * H)
            err = max(err, np.abs(th[s, z, 0] / TH0 - 1 - exact).max())
    return err / a


def test_wall_with_varying_temperature_gives_laplace_field():
    e8, e16 = _laplace(16, 8), _laplace(32, 16)
    assert e16 <= 0.10, (e8, e16)  # measured 0.166 and 0.089 of the amplitude
    assert e8 / e16 >= 1.7, (e8, e16)


def test_cavity_series_is_the_conduction_solution():
    """The printed series solves Laplace's equation (five-point check) with T = T0 on the side
    and bottom walls and T = T1 on the top wall away from the corners."""
    L, H = 1.0, 1.0
    h = 1e-3
    X, Y = np.meshgrid(np.linspace(0.1, 0.9, 9), np.linspace(0.1, 0.9, 9))
    lap = (cavity_series(X + h, Y, L, H) + cavity_series(X - h, Y, L, H) + cavity_series(X, Y + h, L, H)
           + cavity_series(X, Y - h, L, H) - 4 * cavity_series(X, Y, L, H)) / h ** 2
    assert np.abs(lap).max() <= 1e-3
    xs = np.linspace(0.05, 0.95, 19)
    assert np.abs(cavity_series(xs, 0.0, L, H)).max() <= 1e-12
    assert np.abs(cavity_series(0.0, xs, L, H)).max() <= 1e-12
    # the partial sum of a square wave: its ripple at distance d from a corner is about 1 / (pi N d)
    assert np.abs(cavity_series(xs[(xs > 0.09) & (xs < 0.91)], 1.0, L, H) - 1.0).max() <= 0.01


def test_cavity_heated_at_the_top_matches_the_series():
    L = H = 16
    nx, dT, nu = 2 * L, 0.01, 0.1
    # the top wall's column x covers the doubled positions 2x - 1, 2x: centre x - 1/4, so its
    # steps sit at x = 1/4 + k L; the series is evaluated at X - 1/4
    xc = np.arange(nx) - 0.25
    top = TH0 * (1 + dT * np.sign(np.sin(math.pi * xc / L)))[None, :]
    f = _rest(nx, 1, H)
    f = oracle.step_walls(f, nu / TH0, int(4 * H * H / (5.0 / 3.0 * nu)), (0.0, 0.0, TH0), (0.0, 0.0, top))
    _, _, th = oracle.get_moments(f)
    T = th[:, :, 0, :] / TH0 - 1
    X = np.array([[np.arange(nx) + 0.5 * s - 0.25 for _ in range(H)] for s in (0, 1)])
    Y = np.array([[np.full(nx, z + 0.5 * s + 0.25) for z in range(H)] for s in (0, 1)])
    err = np.abs(T - dT * cavity_series(X, Y, L, H)) / dT
    xl, yh = X / L, Y / H
    worst = 0.0
    for x0 in (0.1, 0.2, 0.5):
        worst = max(worst, err[(np.abs(xl - x0) <= 0.5 / L + 1e-9) & (yh <= 0.8)].max())
    for y0 in (0.25, 0.5, 0.75):
        worst = max(worst, err[(np.abs(yh - y0) <= 0.5 / H + 1e-9) & (xl > 0.05) & (xl < 0.95)].max())
    assert worst <= 0.045, worst  # measured 0.043
