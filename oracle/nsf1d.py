"""Reference solution for the thermoacoustic column (Sec. "Thermal flows", the
1D case between two walls, one of them heated suddenly).

TEST INFRASTRUCTURE ONLY: loaded by the tests, never by the library.

The paper compares its lattice Boltzmann run with a Navier-Stokes-Fourier
(NSF) solution in the manner of Larkin (1967), which it does not reproduce.
This is that comparison solution, written from the equations: the NSF
equations of a monatomic ideal gas, linearised about rest (rho0 = 1,
theta0, u = 0), in one dimension z in [0, L]:

    d rho'/dt = -du/dz
    du/dt     = -dp'/dz + (4/3) nu d2u/dz2          (bulk viscosity zero, Sec. I)
    dT'/dt    = -(theta0 / c_v) du/dz + (c_p / c_v) nu d2T'/dz2   (Pr = 1)
    p'        = theta0 rho' + T'

with c_v = 3/2 and c_p = 5/2 (theta units), u = 0 at both walls, T' = 0 at
z = 0 and T' = dT at z = L for t > 0, and a gas at rest at theta0 at t = 0.
Staggered grid (rho', T' at cell centres, u at faces), explicit time steps,
central differences; the wall temperature enters through ghost cells.  The
scheme is second order in space; its step is a fraction of both the
diffusive and the acoustic limit."""
import numpy as np

CV = 1.5
CP = 2.5


def column(L, nu, dT, theta0, times, n=1024):
    """rho', T', u of the column at the given times (ascending, > 0); returns a dict
    t -> (z of the cell centres, rho', T', u at the cell centres)."""
    dx = L / n
    a_u = 4.0 / 3.0 * nu
    a_t = CP / CV * nu
    dt = min(0.2 * dx * dx / max(a_u, a_t), 0.3 * dx / np.sqrt(CP / CV * theta0))
    rho = np.zeros(n)
    T = np.zeros(n)
    u = np.zeros(n + 1)  # faces 0 .. n; u[0] = u[n] = 0
    out = {}
    t = 0.0
    for t_out in sorted(times):
        while t < t_out - 1e-12:
            h = min(dt, t_out - t)
            p = theta0 * rho + T
            dpdz = np.zeros(n + 1)
            dpdz[1:-1] = (p[1:] - p[:-1]) / dx
            uzz = np.zeros(n + 1)
            uzz[1:-1] = (u[2:] - 2 * u[1:-1] + u[:-2]) / dx ** 2
            divu = (u[1:] - u[:-1]) / dx
            Tg = np.concatenate(([-T[0]], T, [2 * dT - T[-1]]))  # T' = 0 at z = 0, dT at z = L
            Tzz = (Tg[2:] - 2 * Tg[1:-1] + Tg[:-2]) / dx ** 2
            rho = rho - h * divu
            T = T + h * (-(theta0 / CV) * divu + a_t * Tzz)
            u = u + h * (-dpdz + a_u * uzz)
            u[0] = u[-1] = 0.0
            t += h
        out[t_out] = ((np.arange(n) + 0.5) * dx, rho.copy(), T.copy(), 0.5 * (u[1:] + u[:-1]))
    return out
