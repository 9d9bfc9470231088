/*
 * Plain FP64 CPU oracle for the energy-conserving crystallographic lattice
 * Boltzmann model RD3Q41 (Kolluru, Atif, Namburi, Ansumali, "Lattice Boltzmann
 * model for weakly compressible flows", arXiv:1909.08406).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * table or constant with the CUDA library: the velocity set is enumerated here
 * from the shell definitions of Table I, the weights are typed from Table I,
 * and every formula is written out per population, in the order the paper
 * states it, with no pair factorisation, no closed-form shortcuts and no
 * blocking.
 *
 * Section / equation map (paper numbering):
 *   - velocity shells and weights ............ Sec. IV, Table I
 *   - w_0 and theta_0 from the constraints .... Sec. III, Eq. (allWeights)
 *   - hydrodynamic moments .................... Sec. II (rho, j, E definitions)
 *   - rest-state equilibrium f~ to O(eta^3) ... Sec. V (unnumbered display
 *                                               before Eq. feqGenU3)
 *   - velocity-dependent equilibrium ......... Sec. V, Eq. (feqGenU3) with
 *                                               M_2, M_2', A_1, A_2
 *   - exact entropic equilibrium (Newton) ..... Sec. V, Eqs. (discreteentropiceq)
 *                                               and (fivelagrangemultipliersystem)
 *   - entropic path length alpha ............. Sec. "Droplet Collision" (the
 *                                               update with alpha beta, x_i)
 *   - BGK collision and streaming ............. Sec. II, discrete BGK update
 *   - bcc grid: two sc lattices offset by
 *     half a cell in every direction .......... Sec. IV
 *   - forced collision of the nonideal fluid .. Sec. "Nonideal Fluids and
 *                                               two-phase flow", Eq.
 *                                               (multiphaseEvolution); pinned by
 *                                               its momentum change, Eq.
 *                                               (momentumchange)
 *
 * Readings where the paper is silent or garbled:
 *   - theta_0 is not printed: theta_0 = sum_i w_i c_ix^2 (Eq. allWeights).
 *   - w_0 is not printed: w_0 = 1 - sum of the 40 tabulated weights.
 *   - "Delta theta" in M_2, M_2' means eta = theta/theta_0 - 1, and
 *     "Delta^n theta" means eta^n.
 *   - M_2  = <f~, c^2 c_x^2> / (5 rho theta^2) - 1 and
 *     M_2' = <f~, c_x^2 c_y^2> / (rho theta^2) - 1, the departures of the
 *     zero-velocity moments from their Maxwell-Boltzmann values; they are
 *     evaluated here by direct summation over the lattice.
 *   - The truncated series does not conserve momentum exactly (error
 *     O(u^3 eta^2)).  With project != 0 the equilibrium is corrected by
 *     f~_i c_i . dj / (rho theta), dj = rho u - sum_i f^eq_i c_i, which restores
 *     the momentum constraint of Eq. (fivelagrangemultipliersystem) and leaves
 *     mass, energy and the second moment unchanged.  project == 0 is the
 *     formula as printed.
 *   - beta = 1 / (2 tau + 1) (Delta t = 1); tau = +inf gives beta = 0.
 *   - The grid "N^3" has N^3 simple-cubic cells and 2 N^3 nodes: sub-lattice
 *     A at integer positions r, sub-lattice B at r + (1/2, 1/2, 1/2).
 *   - The kinetic wall condition the paper cites (Ansumali and Karlin 2002) is
 *     not restated there; or_step_walls writes it for this lattice as diffuse
 *     reflection with the walls a quarter cell beyond the outermost node planes
 *     and one wall density per cell column of the wall and step (see that
 *     function).
 *
 * Array layout used by every grid routine here (the oracle's own velocity
 * order, given by or_velocities):
 *   populations f[s][i][z][y][x], s in {0 (A), 1 (B)}, i in 0..40;
 *   scalar fields  a[s][z][y][x];  vector fields u[d][s][z][y][x].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 41

/* Table I weights, per shell, as printed. */
static const double TABLE_I_WEIGHTS[5] = {
    0.04743040745116578, /* sc-1   (+-1, 0, 0) and permutations      */
    0.00165687664501576, /* sc-2   (+-2, 0, 0) and permutations      */
    0.00651175327832464, /* fcc-1  (+-1, +-1, 0) and permutations    */
    0.00454087801154440, /* bcc-1  (+-1, +-1, +-1)                   */
    0.04917980624482672  /* bcc-1/2 (+-1/2, +-1/2, +-1/2)            */
};

static int C2[NV][3];  /* doubled velocity components, 2 c_i */
static double CV[NV][3];
static double W[NV];
static int SHELL[NV];
static double THETA0;
static int lattice_ready = 0;

/* Shell of a doubled velocity vector (Table I), or -1 if it is not in the set. */
static int shell_of(int dx, int dy, int dz) {
    int a[3] = {abs(dx), abs(dy), abs(dz)};
    int nz = (a[0] != 0) + (a[1] != 0) + (a[2] != 0);
    if (nz == 0) return 0;
    if (nz == 1) {
        int m = a[0] + a[1] + a[2];
        if (m == 2) return 1; /* sc-1 */
        if (m == 4) return 2; /* sc-2 */
        return -1;
    }
    if (nz == 2) {
        for (int k = 0; k < 3; ++k)
            if (a[k] != 0 && a[k] != 2) return -1;
        return 3; /* fcc-1 */
    }
    if (a[0] == 2 && a[1] == 2 && a[2] == 2) return 4; /* bcc-1 */
    if (a[0] == 1 && a[1] == 1 && a[2] == 1) return 5; /* bcc-1/2 */
    return -1;
}

static void init_lattice(void) {
    if (lattice_ready) return;
    int n = 0;
    for (int sh = 0; sh <= 5; ++sh)
        for (int dx = -4; dx <= 4; ++dx)
            for (int dy = -4; dy <= 4; ++dy)
                for (int dz = -4; dz <= 4; ++dz)
                    if (shell_of(dx, dy, dz) == sh) {
                        C2[n][0] = dx;
                        C2[n][1] = dy;
                        C2[n][2] = dz;
                        SHELL[n] = sh;
                        ++n;
                    }
    /* n == 41 by construction: 1 + 6 + 6 + 12 + 8 + 8 */
    double sum = 0.0;
    for (int i = 0; i < NV; ++i) {
        for (int d = 0; d < 3; ++d) CV[i][d] = 0.5 * C2[i][d];
        W[i] = SHELL[i] == 0 ? 0.0 : TABLE_I_WEIGHTS[SHELL[i] - 1];
        sum += W[i];
    }
    W[0] = 1.0 - sum; /* Eq. (allWeights): sum_i w_i = 1 */
    double th = 0.0;
    for (int i = 0; i < NV; ++i) th += W[i] * CV[i][0] * CV[i][0];
    THETA0 = th; /* Eq. (allWeights): sum_i w_i c_ix^2 = theta_0 */
    lattice_ready = 1;
}

static double csq(int i) {
    return CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2];
}

/* ------------------------------------------------------------------ */
/* Lattice                                                             */
/* ------------------------------------------------------------------ */

int or_nvel(void) { return NV; }

/* Velocity set in the oracle's order: c2 = doubled components [41][3],
 * w = weights [41], shell = shell index (0 rest, 1 sc-1, 2 sc-2, 3 fcc-1,
 * 4 bcc-1, 5 bcc-1/2). */
void or_velocities(int *c2, double *w, int *shell) {
    init_lattice();
    for (int i = 0; i < NV; ++i) {
        for (int d = 0; d < 3; ++d) c2[3 * i + d] = C2[i][d];
        if (w) w[i] = W[i];
        if (shell) shell[i] = SHELL[i];
    }
}

double or_theta0(void) {
    init_lattice();
    return THETA0;
}

/* Residuals of the seven weight constraints, Sec. III Eq. (allWeights):
 * sum w - 1, sum w cx^2 - th, sum w cx^4 - 3 th^2, sum w cx^2 cy^2 - th^2,
 * sum w cx^4 c^2 - 21 th^3, sum w cx^2 c^4 - 35 th^3, sum w c^8 - 945 th^4.
 * theta0 <= 0 uses the derived theta_0. */
void or_weight_constraints(double theta0, double res[7]) {
    init_lattice();
    double th = theta0 > 0 ? theta0 : THETA0;
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < NV; ++i) {
        double cx = CV[i][0], cy = CV[i][1], c2 = csq(i);
        s[0] += W[i];
        s[1] += W[i] * cx * cx;
        s[2] += W[i] * cx * cx * cx * cx;
        s[3] += W[i] * cx * cx * cy * cy;
        s[4] += W[i] * cx * cx * cx * cx * c2;
        s[5] += W[i] * cx * cx * c2 * c2;
        s[6] += W[i] * c2 * c2 * c2 * c2;
    }
    res[0] = s[0] - 1.0;
    res[1] = s[1] - th;
    res[2] = s[2] - 3.0 * th * th;
    res[3] = s[3] - th * th;
    res[4] = s[4] - 21.0 * th * th * th;
    res[5] = s[5] - 35.0 * th * th * th;
    res[6] = s[6] - 945.0 * th * th * th * th;
}

/* ------------------------------------------------------------------ */
/* Equilibria (Sec. V)                                                 */
/* ------------------------------------------------------------------ */

/* Rest-state equilibrium f~_i(rho, theta) to O(eta^3), eta = theta/theta_0 - 1. */
void or_rest_equilibrium(double rho, double theta, double *ft) {
    init_lattice();
    double eta = theta / THETA0 - 1.0;
    for (int i = 0; i < NV; ++i) {
        double s = csq(i) / THETA0; /* c_i^2 / theta_0 */
        double b1 = 0.5 * eta * (s - 3.0);
        double b2 = eta * eta / 8.0 * (s * s - 10.0 * s + 15.0);
        double b3 = eta * eta * eta / 48.0 * (s * s * s - 21.0 * s * s + 105.0 * s - 105.0);
        ft[i] = W[i] * rho * (1.0 + b1 + b2 + b3);
    }
}

/* Departures of the zero-velocity moments of f~ from their Maxwell-Boltzmann
 * values, by direct summation:
 *   out[0] = M_2   = <f~, c^2 cx^2>      / (5 rho theta^2) - 1
 *   out[1] = M_2'  = <f~, cx^2 cy^2>     / (rho theta^2)   - 1
 *   out[2] = M_3   = <f~, c^4 cx^2>      / (35 rho theta^3) - 1
 *   out[3] = M_3'  = <f~, cx^2 cy^2 c^2> / (7 rho theta^3)  - 1        */
void or_m_terms(double rho, double theta, double out[4]) {
    init_lattice();
    double ft[NV];
    or_rest_equilibrium(rho, theta, ft);
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (int i = 0; i < NV; ++i) {
        double cx = CV[i][0], cy = CV[i][1], c2 = csq(i);
        s0 += ft[i] * c2 * cx * cx;
        s1 += ft[i] * cx * cx * cy * cy;
        s2 += ft[i] * c2 * c2 * cx * cx;
        s3 += ft[i] * cx * cx * cy * cy * c2;
    }
    out[0] = s0 / (5.0 * rho * theta * theta) - 1.0;
    out[1] = s1 / (rho * theta * theta) - 1.0;
    out[2] = s2 / (35.0 * rho * theta * theta * theta) - 1.0;
    out[3] = s3 / (7.0 * rho * theta * theta * theta) - 1.0;
}

/* Energy-conserving equilibrium, Eq. (feqGenU3), term by term. */
void or_equilibrium(double rho, const double *u, double theta, int project, double *feq) {
    init_lattice();
    double ft[NV], m[4];
    or_rest_equilibrium(rho, theta, ft);
    or_m_terms(rho, theta, m);
    double M2 = m[0], M2p = m[1];
    double A1 = 2.5 * M2 / (1.0 + 2.5 * M2);
    double A2 = 5.0 * A1 * (1.0 - M2) - (3.0 + M2p - 5.0 * M2);
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NV; ++i) {
        double c2 = csq(i);
        double uc = u[0] * CV[i][0] + u[1] * CV[i][1] + u[2] * CV[i][2];
        double a = uc / theta;
        double brace = 1.0 + a - usq / (2.0 * theta) * (1.0 - A1) + 0.5 * a * a + a * a * a / 6.0 -
                       usq * c2 / (6.0 * theta * theta) * A1 + usq * uc / (6.0 * theta * theta) * A2 -
                       usq * c2 * uc / (6.0 * theta * theta * theta) * A1;
        feq[i] = ft[i] * brace;
    }
    if (project) {
        double dj[3] = {rho * u[0], rho * u[1], rho * u[2]};
        for (int i = 0; i < NV; ++i)
            for (int d = 0; d < 3; ++d) dj[d] -= feq[i] * CV[i][d];
        for (int i = 0; i < NV; ++i) {
            double cdj = CV[i][0] * dj[0] + CV[i][1] * dj[1] + CV[i][2] * dj[2];
            feq[i] += ft[i] * cdj / (rho * theta);
        }
    }
}

/* Solve the 5x5 system A x = b by Gaussian elimination with partial pivoting. */
static int solve5(double A[5][5], double b[5], double x[5]) {
    for (int k = 0; k < 5; ++k) {
        int p = k;
        for (int r = k + 1; r < 5; ++r)
            if (fabs(A[r][k]) > fabs(A[p][k])) p = r;
        if (A[p][k] == 0.0) return -1;
        if (p != k) {
            for (int c = 0; c < 5; ++c) {
                double t = A[k][c];
                A[k][c] = A[p][c];
                A[p][c] = t;
            }
            double t = b[k];
            b[k] = b[p];
            b[p] = t;
        }
        for (int r = k + 1; r < 5; ++r) {
            double f = A[r][k] / A[k][k];
            for (int c = k; c < 5; ++c) A[r][c] -= f * A[k][c];
            b[r] -= f * b[k];
        }
    }
    for (int k = 4; k >= 0; --k) {
        double s = b[k];
        for (int c = k + 1; c < 5; ++c) s -= A[k][c] * x[c];
        x[k] = s / A[k][k];
    }
    return 0;
}

/* Exact entropic equilibrium f_i = w_i rho exp(-alpha - beta.c_i - gamma c_i^2),
 * Eq. (discreteentropiceq), with the five Lagrange multipliers found by
 * Newton's method from the moment constraints of
 * Eq. (fivelagrangemultipliersystem): <f,1> = rho, <f,c> = rho u,
 * <f,c^2> = rho u^2 + 3 rho theta.  Returns the iteration count, or -1 if
 * Newton did not converge. */
int or_entropic_equilibrium(double rho, const double *u, double theta, double *feq) {
    init_lattice();
    double x[5] = {0, 0, 0, 0, 0}; /* alpha, beta_x, beta_y, beta_z, gamma */
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double target[5] = {rho, rho * u[0], rho * u[1], rho * u[2], rho * usq + 3.0 * rho * theta};
    for (int it = 0; it < 100; ++it) {
        double phi[NV][5];
        double F[5] = {0, 0, 0, 0, 0};
        double J[5][5];
        memset(J, 0, sizeof J);
        for (int i = 0; i < NV; ++i) {
            phi[i][0] = 1.0;
            phi[i][1] = CV[i][0];
            phi[i][2] = CV[i][1];
            phi[i][3] = CV[i][2];
            phi[i][4] = csq(i);
            double arg = 0.0;
            for (int k = 0; k < 5; ++k) arg += x[k] * phi[i][k];
            feq[i] = W[i] * rho * exp(-arg);
            for (int r = 0; r < 5; ++r) {
                F[r] += feq[i] * phi[i][r];
                for (int c = 0; c < 5; ++c) J[r][c] -= feq[i] * phi[i][r] * phi[i][c];
            }
        }
        double err = 0.0;
        for (int r = 0; r < 5; ++r) {
            F[r] -= target[r];
            err = fmax(err, fabs(F[r]));
        }
        if (err <= 1e-15 * rho) return it;
        double dx[5], rhs[5];
        for (int r = 0; r < 5; ++r) rhs[r] = -F[r];
        if (solve5(J, rhs, dx) != 0) return -1;
        for (int k = 0; k < 5; ++k) x[k] += dx[k];
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Moments and collision (Sec. II)                                     */
/* ------------------------------------------------------------------ */

/* rho = <f,1>, rho u = <f,c>, E = <f,c^2/2> = (rho u^2 + 3 rho theta)/2. */
void or_moments(const double *f, double *rho, double *u, double *theta) {
    init_lattice();
    double r = 0, j[3] = {0, 0, 0}, e2 = 0;
    for (int i = 0; i < NV; ++i) {
        r += f[i];
        for (int d = 0; d < 3; ++d) j[d] += f[i] * CV[i][d];
        e2 += f[i] * csq(i);
    }
    for (int d = 0; d < 3; ++d) u[d] = j[d] / r;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    *rho = r;
    *theta = (e2 / r - usq) / 3.0;
}

static double beta_of_tau(double tau) { return isinf(tau) ? 0.0 : 1.0 / (2.0 * tau + 1.0); }

/* Entropic path length (Sec. "Droplet Collision": the update written with a
 * factor alpha beta, alpha chosen so that the dynamics obeys the H theorem,
 * from x_i = f^eq_i / f_i - 1).  alpha is the nontrivial root of
 *   Delta H(alpha) = H(f + alpha (f^eq - f)) - H(f) = 0,  H(f) = sum_i f_i ln(f_i / w_i),
 * which with f_i + alpha (f^eq_i - f_i) = f_i (1 + alpha x_i) reads
 *   Delta H(alpha) = sum_i f_i [(1 + alpha x_i) ln(1 + alpha x_i) + alpha x_i ln(f_i / w_i)].
 * Delta H(0) = 0 and Delta H is convex in alpha; when H falls towards f^eq
 * (Delta H < 0 just above 0) it returns to zero once more below
 * alpha_max = min over x_i < 0 of -1/x_i (where a population reaches zero).
 * The root is bracketed (a point where Delta H < 0, one where it is > 0) and
 * bisected to the last bit.  Readings: alpha = 2 (plain BGK) when every
 * |x_i| <= 1e-7 (there the FP64 round-off of f^eq - f, and the residual of an
 * iterated f^eq's moments, dominate Delta H ~ sum f x^2; the root is 2 + O(x),
 * so f' moves by less than beta |x|^2), and when no root lies below alpha_max. */
static double path_dh(const double *f, const double *x, double a) {
    double s = 0.0;
    for (int i = 0; i < NV; ++i) {
        const double y = a * x[i];
        s += f[i] * ((1.0 + y) * log1p(y) + y * log(f[i] / W[i]));
    }
    return s;
}

double or_path_length(const double *f, const double *feq) {
    init_lattice();
    double x[NV], amax = INFINITY;
    int resolved = 0;
    for (int i = 0; i < NV; ++i) {
        x[i] = feq[i] / f[i] - 1.0;
        if (fabs(x[i]) > 1e-7) resolved = 1;
        if (x[i] < 0.0 && -1.0 / x[i] < amax) amax = -1.0 / x[i];
    }
    if (!resolved) return 2.0;
    /* hi: Delta H > 0, from 2 outwards (halfway to alpha_max at each try) */
    double hi = amax > 2.0 ? 2.0 : 0.5 * amax;
    for (int k = 0; k < 200 && path_dh(f, x, hi) <= 0.0; ++k) {
        if (isinf(amax))
            hi *= 2.0;
        else
            hi = 0.5 * (hi + amax);
    }
    if (!(path_dh(f, x, hi) > 0.0)) return 2.0;
    /* lo: Delta H < 0, from hi towards 0 */
    double lo = 0.5 * hi;
    for (int k = 0; k < 200 && path_dh(f, x, lo) >= 0.0; ++k) lo *= 0.5;
    if (!(path_dh(f, x, lo) < 0.0)) return 2.0;
    for (int k = 0; k < 200; ++k) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (path_dh(f, x, mid) < 0.0)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* The equilibrium used by the update.  kind 0: Eq. (feqGenU3) as printed;
 * 1: Eq. (feqGenU3) with the momentum projection; 2: the exact entropic
 * equilibrium, Eq. (discreteentropiceq) (NaN if Newton fails). */
static void equilibrium_of_kind(double rho, const double *u, double theta, int kind, double *feq) {
    if (kind == 2 || kind == 3) {
        if (or_entropic_equilibrium(rho, u, theta, feq) < 0)
            for (int i = 0; i < NV; ++i) feq[i] = NAN;
    } else {
        or_equilibrium(rho, u, theta, kind, feq);
    }
}

/* Discrete BGK collision f* = f + 2 beta (f^eq(rho(f), u(f), theta(f)) - f),
 * with the equilibrium of the given kind (see equilibrium_of_kind); kind 3 is
 * the exact entropic equilibrium with the entropic path length,
 * f* = f + alpha beta (f^eq - f), alpha = or_path_length(f, f^eq). */
void or_collide(const double *f, double tau, int project, double *out) {
    init_lattice();
    double rho, u[3], theta, feq[NV];
    or_moments(f, &rho, u, &theta);
    equilibrium_of_kind(rho, u, theta, project, feq);
    double b2 = 2.0 * beta_of_tau(tau);
    if (project == 3) b2 = or_path_length(f, feq) * beta_of_tau(tau);
    for (int i = 0; i < NV; ++i) out[i] = f[i] + b2 * (feq[i] - f[i]);
}

/* ------------------------------------------------------------------ */
/* Grid routines                                                       */
/* ------------------------------------------------------------------ */

static int64_t pidx(int64_t nx, int64_t ny, int64_t nz, int s, int i, int64_t z, int64_t y, int64_t x) {
    return ((((int64_t)s * NV + i) * nz + z) * ny + y) * nx + x;
}

static int64_t mod(int64_t a, int64_t n) {
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

/* Position of the node that streams into node (s, z, y, x) along velocity i:
 * in doubled coordinates the node sits at P = (2x+s, 2y+s, 2z+s) and its
 * upwind neighbour at P - 2 c_i, wrapped periodically on the 2n torus. */
static int64_t upwind(int64_t nx, int64_t ny, int64_t nz, int s, int i, int64_t z, int64_t y, int64_t x) {
    int64_t qx = mod(2 * x + s - C2[i][0], 2 * nx);
    int64_t qy = mod(2 * y + s - C2[i][1], 2 * ny);
    int64_t qz = mod(2 * z + s - C2[i][2], 2 * nz);
    int sp = (int)(qx & 1);
    return pidx(nx, ny, nz, sp, i, qz >> 1, qy >> 1, qx >> 1);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Streaming: fpre_i(x) = fpost_i(x - c_i), periodic. */
void or_stream(int64_t nx, int64_t ny, int64_t nz, const double *fpost, double *fpre, int nthreads) {
    init_lattice();
    set_threads(nthreads);
#pragma omp parallel for collapse(3) schedule(static)
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < NV; ++i)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x)
                        fpre[pidx(nx, ny, nz, s, i, z, y, x)] = fpost[upwind(nx, ny, nz, s, i, z, y, x)];
}

/* n time steps of the discrete BGK update, Sec. II.  f holds the
 * post-collision state and is advanced in place; work is a scratch array of
 * the same size. */
void or_step(int64_t nx, int64_t ny, int64_t nz, double tau, int project, int64_t nsteps, double *f, double *work,
             int nthreads) {
    init_lattice();
    set_threads(nthreads);
    for (int64_t t = 0; t < nsteps; ++t) {
        or_stream(nx, ny, nz, f, work, nthreads);
#pragma omp parallel for collapse(3) schedule(static)
        for (int s = 0; s < 2; ++s)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        double fin[NV], fout[NV];
                        for (int i = 0; i < NV; ++i) fin[i] = work[pidx(nx, ny, nz, s, i, z, y, x)];
                        or_collide(fin, tau, project, fout);
                        for (int i = 0; i < NV; ++i) f[pidx(nx, ny, nz, s, i, z, y, x)] = fout[i];
                    }
    }
}

/* One update for a list of nodes only: out[k][i] = collide(stream(fpost))
 * at node nodes[k], where nodes[k] = ((s*nz + z)*ny + y)*nx + x. */
void or_step_nodes(int64_t nx, int64_t ny, int64_t nz, double tau, int project, const double *fpost,
                   const int64_t *nodes, int64_t n, double *out, int nthreads) {
    init_lattice();
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        int64_t q = nodes[k];
        int64_t x = q % nx;
        q /= nx;
        int64_t y = q % ny;
        q /= ny;
        int64_t z = q % nz;
        int s = (int)(q / nz);
        double fin[NV];
        for (int i = 0; i < NV; ++i) fin[i] = fpost[upwind(nx, ny, nz, s, i, z, y, x)];
        or_collide(fin, tau, project, out + k * NV);
    }
}

/* ------------------------------------------------------------------ */
/* Isothermal nonideal fluid: BGK with a force (Sec. "Nonideal Fluids")  */
/* ------------------------------------------------------------------ */

/* One collision with a force density per node, on the pre-collision
 * (streamed) populations fpre, Eq. (multiphaseEvolution) with alpha = 2
 * (BGK): rho = sum_i f_i, u = sum_i f_i c_i / rho + g / 2 (the velocity of
 * the trapezoid-rule variables), f^eq = f^eq(rho, u, theta_0) (isothermal),
 * F_i = g . (c_i - u) / theta_0 f^eq_i, and
 *   f_i' = f_i + 2 beta (f^eq_i - f_i) + (1 - beta) F_i.
 * g[d][node] is the acceleration g^nid of each node (same layout as a
 * vector field).  fpost receives the post-collision populations. */
void or_collide_forced(int64_t nx, int64_t ny, int64_t nz, double tau, int project, const double *fpre,
                       const double *g, double *fpost, int nthreads) {
    init_lattice();
    set_threads(nthreads);
    const int64_t nn = 2 * nx * ny * nz;
    const double b2 = 2.0 * beta_of_tau(tau);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nn; ++q) {
        int64_t x = q % nx, r = q / nx;
        int64_t y = r % ny;
        r /= ny;
        int64_t z = r % nz;
        int s = (int)(r / nz);
        double fin[NV], feq[NV], rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NV; ++i) {
            fin[i] = fpre[pidx(nx, ny, nz, s, i, z, y, x)];
            rho += fin[i];
            for (int d = 0; d < 3; ++d) j[d] += fin[i] * CV[i][d];
        }
        double gq[3] = {g[q], g[nn + q], g[2 * nn + q]}, u[3];
        for (int d = 0; d < 3; ++d) u[d] = j[d] / rho + 0.5 * gq[d];
        equilibrium_of_kind(rho, u, THETA0, project, feq);
        for (int i = 0; i < NV; ++i) {
            double gc = 0.0;
            for (int d = 0; d < 3; ++d) gc += gq[d] * (CV[i][d] - u[d]);
            const double F = gc / THETA0 * feq[i];
            fpost[pidx(nx, ny, nz, s, i, z, y, x)] = fin[i] + b2 * (feq[i] - fin[i]) + (1.0 - 0.5 * b2) * F;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Kinetic (diffuse) walls normal to z                                 */
/* ------------------------------------------------------------------ */

/* Wall column of a doubled lateral coordinate q (periodic, n cells).  The bottom wall's
 * column x holds q in {2x, 2x + 1}, the top wall's {2x - 1, 2x}: the bottom wall faces the A
 * plane z = 0 and the top wall the B plane z = nz - 1, and the mirror that exchanges the walls
 * shifts x and y by half a cell, so it carries the one partition onto the other. */
static int64_t column_of(int64_t q, int64_t n, int side) {
    q += side;
    return mod(q >= 0 ? q / 2 : -((-q + 1) / 2), n);
}

/* n time steps with two kinetic walls normal to z instead of the periodic
 * wrap in z (x and y stay periodic).  In doubled coordinates the nodes occupy
 * z2 = 2z + s in [0, 2 nz); the bottom wall lies at z2 = -1/2 and the top
 * wall at z2 = 2 nz - 1/2, a quarter cell beyond the outermost node planes,
 * so the channel height is nz cells.  The paper applies the kinetic boundary
 * condition of Ansumali and Karlin (2002) without restating it; this is that
 * condition (diffuse reflection) written for the crystallographic lattice,
 * point by point along the wall, the wall being divided into the cell
 * columns (x, y) of the grid:
 *   - a post-collision population whose destination z2 + 2 c_iz lies beyond a
 *     wall is absorbed by the wall column that contains its destination's
 *     (x, y) (see column_of for how a wall is cut into columns);
 *   - a population whose upwind position z2 - 2 c_iz lies beyond a wall is
 *     emitted by the wall column that contains the upwind position's (x, y):
 *     f_i = rho_w f^eq_i(1, u_w, theta_w), the model's own equilibrium at that
 *     column's velocity and temperature;
 *   - rho_w of each column makes the mass it emits equal to the mass it
 *     absorbs, so no column creates or destroys mass.
 * wall[2][4][ny][nx]: {u_x, u_y, u_z, theta} of every column of the bottom
 * wall, then of the top wall (u_z must be 0).  wall_rho[nsteps][2][ny][nx]
 * receives the columns' rho_w per step if it is not NULL. */
void or_step_walls(int64_t nx, int64_t ny, int64_t nz, double tau, int project, int64_t nsteps, double *f,
                   double *work, const double *wall, double *wall_rho, int nthreads) {
    init_lattice();
    set_threads(nthreads);
    const int64_t ncol = nx * ny;
    double *e = (double *)malloc(sizeof(double) * (size_t)(2 * ncol * NV));  /* [side][col][i] */
    double *emitted = (double *)malloc(sizeof(double) * (size_t)(2 * ncol));
    double *absorbed = (double *)malloc(sizeof(double) * (size_t)(2 * ncol));
    double *rho_w = (double *)malloc(sizeof(double) * (size_t)(2 * ncol));
    for (int side = 0; side < 2; ++side)
        for (int64_t col = 0; col < ncol; ++col) {
            const double *w = wall + side * 4 * ncol;
            double u[3] = {w[col], w[ncol + col], w[2 * ncol + col]};
            equilibrium_of_kind(1.0, u, w[3 * ncol + col], project, e + (side * ncol + col) * NV);
        }
    for (int64_t t = 0; t < nsteps; ++t) {
        for (int64_t k = 0; k < 2 * ncol; ++k) absorbed[k] = emitted[k] = 0.0;
        for (int s = 0; s < 2; ++s)
            for (int i = 0; i < NV; ++i)
                for (int64_t z = 0; z < nz; ++z)
                    for (int64_t y = 0; y < ny; ++y)
                        for (int64_t x = 0; x < nx; ++x) {
                            int64_t z2 = 2 * z + s;
                            int64_t dest = z2 + C2[i][2], src = z2 - C2[i][2];
                            if (dest < 0 || dest >= 2 * nz) {
                                int side = dest < 0 ? 0 : 1;
                                int64_t col = column_of(2 * y + s + C2[i][1], ny, side) * nx +
                                              column_of(2 * x + s + C2[i][0], nx, side);
                                absorbed[side * ncol + col] += f[pidx(nx, ny, nz, s, i, z, y, x)];
                            }
                            if (src < 0 || src >= 2 * nz) {
                                int side = src < 0 ? 0 : 1;
                                int64_t col = column_of(2 * y + s - C2[i][1], ny, side) * nx +
                                              column_of(2 * x + s - C2[i][0], nx, side);
                                emitted[side * ncol + col] += e[(side * ncol + col) * NV + i];
                            }
                        }
        for (int64_t k = 0; k < 2 * ncol; ++k) rho_w[k] = absorbed[k] / emitted[k];
        if (wall_rho) memcpy(wall_rho + t * 2 * ncol, rho_w, sizeof(double) * (size_t)(2 * ncol));
#pragma omp parallel for collapse(3) schedule(static)
        for (int s = 0; s < 2; ++s)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        double fin[NV], fout[NV];
                        for (int i = 0; i < NV; ++i) {
                            int64_t src = 2 * z + s - C2[i][2];
                            if (src < 0 || src >= 2 * nz) {
                                int side = src < 0 ? 0 : 1;
                                int64_t col = column_of(2 * y + s - C2[i][1], ny, side) * nx +
                                              column_of(2 * x + s - C2[i][0], nx, side);
                                fin[i] = rho_w[side * ncol + col] * e[(side * ncol + col) * NV + i];
                            } else {
                                fin[i] = f[upwind(nx, ny, nz, s, i, z, y, x)];
                            }
                        }
                        or_collide(fin, tau, project, fout);
                        for (int i = 0; i < NV; ++i) work[pidx(nx, ny, nz, s, i, z, y, x)] = fout[i];
                    }
        memcpy(f, work, sizeof(double) * (size_t)(2 * NV * nx * ny * nz));
    }
    free(e);
    free(emitted);
    free(absorbed);
    free(rho_w);
}

/* Populations set to the equilibrium of the given fields (rho[s][z][y][x],
 * u[d][s][z][y][x], theta[s][z][y][x]); collision leaves f^eq unchanged, so
 * this is also the post-collision state at t = 0. */
void or_init_fields(int64_t nx, int64_t ny, int64_t nz, const double *rho, const double *u, const double *theta,
                    int project, double *f, int nthreads) {
    init_lattice();
    set_threads(nthreads);
    int64_t nn = 2 * nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nn; ++q) {
        double uu[3] = {u[q], u[nn + q], u[2 * nn + q]};
        double feq[NV];
        equilibrium_of_kind(rho[q], uu, theta[q], project, feq);
        int64_t x = q % nx, r = q / nx;
        int64_t y = r % ny;
        r /= ny;
        int64_t z = r % nz;
        int s = (int)(r / nz);
        for (int i = 0; i < NV; ++i) f[pidx(nx, ny, nz, s, i, z, y, x)] = feq[i];
    }
}

/* Node moments of a population array (collision invariants, so the moments
 * of the post-collision state equal those of the pre-collision state). */
void or_get_moments(int64_t nx, int64_t ny, int64_t nz, const double *f, double *rho, double *u, double *theta,
                    int nthreads) {
    init_lattice();
    set_threads(nthreads);
    int64_t nn = 2 * nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < nn; ++q) {
        int64_t x = q % nx, r = q / nx;
        int64_t y = r % ny;
        r /= ny;
        int64_t z = r % nz;
        int s = (int)(r / nz);
        double fin[NV], uu[3];
        for (int i = 0; i < NV; ++i) fin[i] = f[pidx(nx, ny, nz, s, i, z, y, x)];
        or_moments(fin, &rho[q], uu, &theta[q]);
        for (int d = 0; d < 3; ++d) u[d * nn + q] = uu[d];
    }
}

/* Global mass, momentum (3) and energy sum_x <f, c^2/2>, in FP64. */
void or_conserved(int64_t nx, int64_t ny, int64_t nz, const double *f, double out[5]) {
    init_lattice();
    double acc[5] = {0, 0, 0, 0, 0};
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < NV; ++i)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        double v = f[pidx(nx, ny, nz, s, i, z, y, x)];
                        acc[0] += v;
                        for (int d = 0; d < 3; ++d) acc[1 + d] += v * CV[i][d];
                        acc[4] += 0.5 * v * csq(i);
                    }
    for (int k = 0; k < 5; ++k) out[k] = acc[k];
}
