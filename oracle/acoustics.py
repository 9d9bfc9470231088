"""Exact linear-acoustics solution of the 3D spherical pulse (Sec. VII, "3D
acoustic spherical pulse source").  TEST INFRASTRUCTURE ONLY, like the rest of
``oracle/``: used by ``tests/`` to check whole-step runs of the solver and of
the oracle against physics, never by the library.

An initial density pulse rho' = eps exp(-alpha r^2) with zero velocity, in a
loss-free gas in which it is entirely acoustic (isentropic), spreads as the
spherically symmetric solution of the wave equation with the isentropic sound
speed c.  Two independent forms are given:

* ``pulse_integral``: the Fourier-Bessel form of the section's exact solution,
  eps / (2 alpha sqrt(pi alpha)) * int_0^inf exp(-xi^2 / (4 alpha))
  cos(c xi t) sin(xi r) / (xi r) xi^2 dxi, evaluated by quadrature.  The
  printed formula has no time dependence; the factor cos(c xi t) of the
  source it cites is restored here (at t = 0 both agree).
* ``pulse_dalembert``: the same solution in closed form, from d'Alembert's
  solution for r rho': r rho'(r, t) = [(r - ct) g(r - ct) + (r + ct) g(r + ct)] / 2
  with g(s) = eps exp(-alpha s^2).

The tests pin one against the other and both against the initial condition.
"""
from __future__ import annotations

import math

import numpy as np


def pulse_integral(r, t, eps, alpha, c, n_xi=40001):
    """rho'(r, t) by trapezoidal quadrature of the Fourier-Bessel integral over
    xi in [0, sqrt(4 alpha * 50)] (the Gaussian factor is below e^-50 beyond)."""
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    xi = np.linspace(0.0, math.sqrt(4.0 * alpha * 50.0), n_xi)
    gauss = np.exp(-xi * xi / (4.0 * alpha)) * np.cos(c * xi * t) * xi * xi
    # sin(xi r) / (xi r) with its limit 1 at xi r = 0 (np.sinc(x) = sin(pi x) / (pi x))
    kern = np.sinc(np.outer(r, xi) / math.pi)
    integral = np.trapezoid(kern * gauss[None, :], xi, axis=1)
    return eps / (2.0 * alpha * math.sqrt(math.pi * alpha)) * integral


def pulse_dalembert(r, t, eps, alpha, c):
    """rho'(r, t) in closed form; at r = 0 the limit d/ds [s g(s)] at s = ct."""
    r = np.asarray(r, dtype=np.float64)
    ct = c * t

    def sg(s):
        return s * eps * np.exp(-alpha * s * s)

    with np.errstate(invalid="ignore", divide="ignore"):
        out = (sg(r - ct) + sg(r + ct)) / (2.0 * r)
    s = ct
    at0 = eps * np.exp(-alpha * s * s) * (1.0 - 2.0 * alpha * s * s)
    return np.where(r > 1e-12, out, at0)
