"""Isothermal nonideal fluid on the RD3Q41 grid (Sec. "Nonideal Fluids and
two-phase flow" and Appendix A): van der Waals, the Peng-Robinson type of
Eq. (cspreos) and Carnahan-Starling equations of state.

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
    mu_nid = dF_nid/drho, p = rho theta0 / (1 - b rho) - a rho^2; the other two
    split the same way (classes PengRobinson and CarnahanStarling);
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
    solving mu(rho_g) = mu(rho_l) and p(rho_g) = p(rho_l).

Pinned by tests/test_oracle_nonideal.py (critical points, thermodynamic
consistency, Maxwell, stencil orders, momentum conservation, the forced
collision's momentum change, interfaces, quench, Laplace, sound speed)."""
import functools

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


def _shifted_by_roll(field, c2):
    """field at x + c for every node; field[s][z][y][x] on the bcc grid, c2 = 2c (doubled)."""
    out = np.empty_like(field)
    for s in (0, 1):
        t = (s + c2[0]) & 1  # sub-lattice of the target (all components share the parity)
        dx, dy, dz = ((s + c2[0]) - t) // 2, ((s + c2[1]) - t) // 2, ((s + c2[2]) - t) // 2
        out[s] = np.roll(field[t], shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return out


@functools.lru_cache(maxsize=None)
def _shift_index(shape, c2):
    """The same map as flat indices: _shifted_by_roll applied to the node numbers."""
    return _shifted_by_roll(np.arange(int(np.prod(shape))).reshape(shape), c2).ravel()


def shifted(field, c2):
    """field at x + c for every node (_shifted_by_roll, as one gather)."""
    return field.ravel()[_shift_index(field.shape, c2)].reshape(field.shape)


def grad2(psi, axis=None):
    """All three components of the gradient, or only component `axis` (the same sums)."""
    axes = range(3) if axis is None else (axis,)
    g = np.zeros((3,) + psi.shape)
    for c2, w in _STENCIL:
        if not any(c2[a] for a in axes):
            continue
        sh = shifted(psi, c2)
        for a in axes:
            if c2[a]:
                g[a] += w * (0.5 * c2[a]) * sh
    return g / THETA_HAT if axis is None else g[axis] / THETA_HAT


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

    def rho_scale(self):
        """The critical density."""
        return 1.0 / (3.0 * self.b)

    def rho_max(self):
        """The density where the equation of state becomes singular."""
        return 1.0 / self.b

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
        # spinodal densities bracket the two phases: the first run of negative slope dp/drho
        # (the loop below the critical temperature; an equation of state may turn down again
        # near its own singular density, which is not part of the loop)
        rmax = 0.95 * self.rho_max()
        rs = np.linspace(0.02 * self.rho_scale(), rmax, 200000)
        dp = np.gradient(self.p(rs), rs)
        neg = np.where(dp < 0)[0]
        end = neg[0]
        while end + 1 < len(rs) and dp[end + 1] < 0:
            end += 1
        r1, r2 = rs[neg[0]], rs[end]
        top = end + 1  # the liquid branch: rising pressure after the loop
        while top + 1 < len(rs) and dp[top + 1] >= 0:
            top += 1

        def eqs(v):
            g, l = v
            return [self.mu(g) - self.mu(l), self.p(g) - self.p(l)]

        # a starting pressure between the spinodal extremes (and above zero, where a gas root
        # exists), below the top of the liquid branch
        lo, hi = max(self.p(r2), 0.0), min(self.p(r1), self.p(rs[top]))
        if not lo < hi:
            raise ValueError("no liquid-vapour coexistence at this temperature")
        p_mid = 0.5 * (lo + hi)
        g0 = brentq(lambda r: self.p(r) - p_mid, 1e-12, r1)
        l0 = brentq(lambda r: self.p(r) - p_mid, r2, rs[top])
        g, l = fsolve(eqs, [g0, l0], xtol=1e-12)
        return float(g), float(l)


def _cs_repulsion(eta):
    """Carnahan-Starling hard-sphere terms at packing eta = b rho / 4: the compressibility
    Z = (1 + eta + eta^2 - eta^3) / (1 - eta)^3, the excess free energy per particle and
    theta0, (4 eta - 3 eta^2) / (1 - eta)^2 = int_0^rho (Z - 1) / rho' drho', and its
    derivative times rho, eta (4 - 2 eta) / (1 - eta)^3."""
    Z = (1 + eta + eta * eta - eta ** 3) / (1 - eta) ** 3
    f = (4 * eta - 3 * eta * eta) / (1 - eta) ** 2
    return Z, f, eta * (4 - 2 * eta) / (1 - eta) ** 3


class PengRobinson(VdW):
    """The Peng-Robinson type equation of state of Eq. (cspreos) (Sec. "Sound propagation in a
    nonideal gas"): Carnahan-Starling repulsion with a Peng-Robinson attraction,
        p = rho theta0 Z(b rho / 4) - a rho^2 / (1 + 2 b rho - b^2 rho^2),
    a = 1.851427622 theta_c / rho_c, b = 0.353748714 / rho_c as printed there.
    The attraction's free energy is rho int_0^rho p_att / rho'^2 drho'; with
    1 + 2x - x^2 = (sqrt2 - 1 + x)(sqrt2 + 1 - x) it is
        F_att = -(a rho / (2 sqrt2 b)) ln[(1 + b rho / (sqrt2 - 1)) / (1 - b rho / (sqrt2 + 1))]."""

    def __init__(self, theta_star, rho_c=1.0, theta0=None):
        self.theta0 = oracle.theta0() if theta0 is None else theta0
        self.theta_c = self.theta0 / theta_star
        self.rho_c = rho_c
        self.a = 1.851427622 * self.theta_c / rho_c
        self.b = 0.353748714 / rho_c

    def rho_scale(self):
        return self.rho_c

    def rho_max(self):
        return (1.0 + np.sqrt(2.0)) / self.b  # the attraction's pole (before eta = 1)

    def _att_log(self, rho):
        r2 = np.sqrt(2.0)
        x = self.b * rho
        return np.log((r2 - 1 + x) / (r2 + 1 - x)) - np.log((r2 - 1) / (r2 + 1))

    def F_nid(self, rho):
        _, f, _ = _cs_repulsion(self.b * rho / 4.0)
        return rho * self.theta0 * f - (self.a * rho / (2 * np.sqrt(2.0) * self.b)) * self._att_log(rho)

    def mu_nid(self, rho):
        _, f, rdf = _cs_repulsion(self.b * rho / 4.0)
        x = self.b * rho
        return (self.theta0 * (f + rdf) - (self.a / (2 * np.sqrt(2.0) * self.b)) * self._att_log(rho)
                - self.a * rho / (1 + 2 * x - x * x))

    def p(self, rho):
        Z, _, _ = _cs_repulsion(self.b * rho / 4.0)
        x = self.b * rho
        return rho * self.theta0 * Z - self.a * rho * rho / (1 + 2 * x - x * x)


class CarnahanStarling(VdW):
    """The Carnahan-Starling equation of state (Sec. "Quenching of a liquid-gas system" and
    "Droplet Collision"): Carnahan-Starling repulsion with the van der Waals attraction,
        p = rho theta0 Z(b rho / 4) - a rho^2,   F_nid = rho theta0 f(b rho / 4) - a rho^2.
    The paper prints no constants for it; a and b put the critical point at (rho_c, theta_c):
    with g(eta) = eta Z(eta), dp/drho = d2p/drho2 = 0 there gives g'(eta_c) = eta_c g''(eta_c),
    b = 4 eta_c / rho_c and a = theta_c g'(eta_c) / (2 rho_c), where
        g'(eta) = (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4) / (1 - eta)^4,
        g''(eta) = (8 + 20 eta - 4 eta^2) / (1 - eta)^5."""

    @staticmethod
    def critical_constants():
        """(b rho_c, a rho_c / theta_c)."""
        from scipy.optimize import brentq

        def g1(e):
            return (1 + 4 * e + 4 * e * e - 4 * e ** 3 + e ** 4) / (1 - e) ** 4

        def g2(e):
            return (8 + 20 * e - 4 * e * e) / (1 - e) ** 5

        ec = brentq(lambda e: g1(e) - e * g2(e), 0.01, 0.5, xtol=1e-16)
        return 4.0 * ec, 0.5 * g1(ec)

    def __init__(self, theta_star, rho_c=1.0, theta0=None):
        self.theta0 = oracle.theta0() if theta0 is None else theta0
        self.theta_c = self.theta0 / theta_star
        self.rho_c = rho_c
        bc, ac = self.critical_constants()
        self.a = ac * self.theta_c / rho_c
        self.b = bc / rho_c

    def rho_scale(self):
        return self.rho_c

    def rho_max(self):
        return 4.0 / self.b  # eta = 1

    def F_nid(self, rho):
        _, f, _ = _cs_repulsion(self.b * rho / 4.0)
        return rho * self.theta0 * f - self.a * rho * rho

    def mu_nid(self, rho):
        _, f, rdf = _cs_repulsion(self.b * rho / 4.0)
        return self.theta0 * (f + rdf) - 2.0 * self.a * rho

    def p(self, rho):
        Z, _, _ = _cs_repulsion(self.b * rho / 4.0)
        return rho * self.theta0 * Z - self.a * rho * rho


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
            div += grad2(I_ab, axis=b)
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
