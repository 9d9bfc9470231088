"""Isothermal nonideal (van der Waals) fluid on the RD3Q41 grid (Sec. "Nonideal
Fluids and two-phase flow" and Appendix A).

TEST INFRASTRUCTURE ONLY: loaded by the tests, never by the library.

Written from the paper, step by step:
  - discrete derivatives on the 15-velocity bcc stencil of Appendix A
    (c = 0, (+-1, 0, 0) and permutations, (+-1/2, +-1/2, +-1/2); weights
    14/36, 1/36, 2/36; theta_hat = 1/6):
        grad2_a psi = (1 / theta_hat) sum_i w_i c_ia psi(x + c_i)          Eq. (gradient2)
        lap psi     = (2 / theta_hat) [sum_i w_i psi(x + c_i) - psi(x)]
        grad4_a psi = grad2_a psi - (theta_hat / 2) grad2_a (lap psi)      Eq. (gradient4)
  - the van der Waals free energy, split into the ideal part theta0 rho
    (ln rho - 1) and the rest: F_nid = -theta0 rho ln(1 - b rho) - a rho^2,
    mu_nid = dF_nid/drho, p = rho theta0 / (1 - b rho) - a rho^2;
  - the force of the momentum-conserving formulation, Eq. (gradientFinal):
        rho g_a = -[rho grad2_a mu_nid + mu_nid grad2_a rho
                    - eta grad2_a F_nid - (1 - eta) grad4_a F_nid
                    + kappa grad2_b I_ab],
        I_ab = [-(1/2) |grad rho|^2 - rho lap rho] delta_ab + grad_a rho grad_b rho,
    with the derivatives of rho inside I taken with grad2 and lap;
  - one time step: stream, the density of the streamed populations, the force
    from it, then the forced BGK collision of Eq. (multiphaseEvolution)
    (or_collide_forced in the C oracle);
  - Maxwell's equal-area construction of the coexisting densities, by
    solving mu(rho_g) = mu(rho_l) and p(rho_g) = p(rho_l)."""
import numpy as np

import oracle

THETA_HAT = 1.0 / 6.0
# doubled stencil velocities and weights (Appendix A)
_STENCIL = [((0, 0, 0), 14.0 / 36.0)]
for d in range(3):
    for sgn in (1, -1):
        v = [0, 0, 0]
        v[d] = 2 * sgn
        _STENCIL.append((tuple(v), 1.0 / 36.0))
for sx in (1, -1):
    for sy in (1, -1):
        for sz in (1, -1):
            _STENCIL.append(((sx, sy, sz), 2.0 / 36.0))


def shifted(field, c2):
    """field at x + c for every node; field[s][z][y][x] on the bcc grid, c2 = 2c (doubled)."""
    out = np.empty_like(field)
    for s in (0, 1):
        t = (s + c2[0]) & 1  # sub-lattice of the target (all components share the parity)
        dx, dy, dz = ((s + c2[0]) - t) // 2, ((s + c2[1]) - t) // 2, ((s + c2[2]) - t) // 2
        out[s] = np.roll(field[t], shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return out


def grad2(psi):
    g = np.zeros((3,) + psi.shape)
    for c2, w in _STENCIL:
        if c2 == (0, 0, 0):
            continue
        sh = shifted(psi, c2)
        for a in range(3):
            if c2[a]:
                g[a] += w * (0.5 * c2[a]) * sh
    return g / THETA_HAT


def lap(psi):
    acc = np.zeros_like(psi)
    for c2, w in _STENCIL:
        acc += w * (psi if c2 == (0, 0, 0) else shifted(psi, c2))
    return 2.0 / THETA_HAT * (acc - psi)


def grad4(psi):
    return grad2(psi) - 0.5 * THETA_HAT * grad2(lap(psi))


class VdW:
    """van der Waals fluid at the lattice temperature theta0: theta0 / theta_c = theta_star,
    critical density rho_c (b = 1 / (3 rho_c), a = 27 b theta_c / 8)."""

    def __init__(self, theta_star, rho_c=1.0, theta0=None):
        self.theta0 = oracle.theta0() if theta0 is None else theta0
        self.theta_c = self.theta0 / theta_star
        self.b = 1.0 / (3.0 * rho_c)
        self.a = 27.0 * self.b * self.theta_c / 8.0

    def F_nid(self, rho):
        return -rho * self.theta0 * np.log(1.0 - self.b * rho) - self.a * rho * rho

    def mu_nid(self, rho):
        br = self.b * rho
        return -self.theta0 * np.log(1.0 - br) + self.theta0 * br / (1.0 - br) - 2.0 * self.a * rho

    def mu(self, rho):
        return self.theta0 * np.log(rho) + self.mu_nid(rho)

    def p(self, rho):
        return rho * self.theta0 / (1.0 - self.b * rho) - self.a * rho * rho

    def maxwell(self):
        """(rho_gas, rho_liquid) with equal chemical potential and pressure."""
        from scipy.optimize import brentq, fsolve
        # spinodal densities bracket the two phases
        rs = np.linspace(0.05, 2.9, 20000) / (3 * self.b)
        dp = np.gradient(self.p(rs), rs)
        neg = np.where(dp < 0)[0]
        r1, r2 = rs[neg[0]], rs[neg[-1]]

        def eqs(v):
            g, l = v
            return [self.mu(g) - self.mu(l), self.p(g) - self.p(l)]

        # a starting pressure between the spinodal extremes (and above zero, where a gas root exists)
        p_mid = 0.5 * (self.p(r1) + max(self.p(r2), 0.0))
        g0 = brentq(lambda r: self.p(r) - p_mid, 1e-12, r1)
        l0 = brentq(lambda r: self.p(r) - p_mid, r2, 0.999 / self.b)
        g, l = fsolve(eqs, [g0, l0], xtol=1e-12)
        return float(g), float(l)


def force(rho, eos, kappa, eta=0.5):
    """g^nid of Eq. (gradientFinal) for a density field rho[2][nz][ny][nx]."""
    mu = eos.mu_nid(rho)
    F = eos.F_nid(rho)
    grho = grad2(rho)
    lrho = lap(rho)
    rho_g = -(rho * grad2(mu) + mu * grho - eta * grad2(F) - (1.0 - eta) * grad4(F))
    gsq = (grho ** 2).sum(0)
    for a in range(3):
        div = np.zeros_like(rho)
        for b in range(3):
            I_ab = grho[a] * grho[b] + (-(0.5 * gsq) - rho * lrho if a == b else 0.0)
            div += grad2(I_ab)[b]
        rho_g[a] -= kappa * div
    return rho_g / rho


def step(f, tau, eos, kappa, nsteps=1, eta=0.5, nthreads=None):
    """nsteps of the nonideal update of post-collision populations f[2][41][nz][ny][nx]."""
    import ctypes
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    _, _, nz, ny, nx = f.shape
    L = oracle.lib()
    out = np.empty_like(f)
    for _ in range(nsteps):
        fpre = oracle.stream(f, nthreads)
        rho = fpre.sum(axis=1)
        g = np.ascontiguousarray(force(rho, eos, kappa, eta))
        L.or_collide_forced(ctypes.c_int64(nx), ctypes.c_int64(ny), ctypes.c_int64(nz), ctypes.c_double(tau),
                            ctypes.c_int(1), oracle._p(fpre), oracle._p(g), oracle._p(out),
                            oracle._threads(nthreads))
        f, out = out, f
    return f
