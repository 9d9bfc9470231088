"""Seeded synthetic initial fields for the RD3Q41 solver and its oracle.

This module only builds input fields (density, velocity, temperature) on the
bcc node positions; it holds none of the lattice Boltzmann arithmetic, so both
the CUDA path and the CPU oracle can take their inputs from it.  Temperatures
are produced relative to a reference temperature ``theta0`` that the caller
passes in.

Node positions of an ``nx x ny x nz`` grid (periodic, unit spacing): the A
sub-lattice sits at integer points ``(x, y, z)``, the B sub-lattice at
``(x + 1/2, y + 1/2, z + 1/2)`` (the bcc grid of two simple-cubic lattices,
Sec. IV).  Every field is evaluated at each node's own position.

Shapes: scalar fields ``[2][nz][ny][nx]`` (index 0 = A, 1 = B), velocity
``[3][2][nz][ny][nx]``; all float64.

Workloads (the shapes and amplitudes of the paper's periodic acoustic and
thermal tests, Secs. VI-VIII):
  * ``standing_wave``      density wave rho = 1 + A sin(2 pi m x / nx), u = 0,
                           theta = theta0
  * ``acoustic_thermal``   acoustic wave along x + transverse temperature wave
                           along y + seeded uniform density noise
  * ``thermoacoustic_pulse`` Gaussian pressure pulse at the centre + seeded
                           random temperature field from a 16^3 Fourier box
  * ``spherical_pulse``    the 3D acoustic pulse of Sec. VII: rho' = eps exp(-alpha r^2),
                           alpha = ln 2 / b^2, isentropic (all of it acoustic) or
                           isothermal
  * ``shear_wave``         transverse velocity wave u_y = U sin(2 pi x / nx)
  * ``batch_sweep``        per-simulation grid edges, tau and amplitudes
  * ``random_fields``      seeded smooth-ish random fields for parity tests
  * ``droplet_pair``       two liquid drops in their vapour approaching each other
                           (Sec. "Droplet Collision")
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

F64 = torch.float64


def node_positions(nx: int, ny: int, nz: int, device="cpu"):
    """Coordinates X, Y, Z of every node, each shaped [2][nz][ny][nx]."""
    x = torch.arange(nx, dtype=F64, device=device)
    y = torch.arange(ny, dtype=F64, device=device)
    z = torch.arange(nz, dtype=F64, device=device)
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    X = torch.stack([X, X + 0.5])
    Y = torch.stack([Y, Y + 0.5])
    Z = torch.stack([Z, Z + 0.5])
    return X, Y, Z


def _fields(rho, ux, uy, uz, theta):
    return {"rho": rho.contiguous(), "u": torch.stack([ux, uy, uz]).contiguous(), "theta": theta.contiguous()}


def standing_wave(nx, ny, nz, theta0, amplitude=1e-3, mode=1, device="cpu"):
    X, _, _ = node_positions(nx, ny, nz, device)
    rho = 1.0 + amplitude * torch.sin(2 * math.pi * mode * X / nx)
    zero = torch.zeros_like(rho)
    return _fields(rho, zero, zero, zero, torch.full_like(rho, theta0))


def shear_wave(nx, ny, nz, theta0, amplitude=1e-3, mode=1, device="cpu"):
    X, _, _ = node_positions(nx, ny, nz, device)
    uy = amplitude * torch.sin(2 * math.pi * mode * X / nx)
    one = torch.ones_like(uy)
    zero = torch.zeros_like(uy)
    return _fields(one, zero, uy, zero, torch.full_like(uy, theta0))


def isobaric_thermal_wave(nx, ny, nz, theta0, amplitude=1e-3, mode=1, device="cpu"):
    """theta = theta0 (1 + A cos(k x)) with rho theta constant (no pressure perturbation)."""
    X, _, _ = node_positions(nx, ny, nz, device)
    g = 1.0 + amplitude * torch.cos(2 * math.pi * mode * X / nx)
    zero = torch.zeros_like(g)
    return _fields(1.0 / g, zero, zero, zero, theta0 * g)


def acoustic_thermal(n, theta0, amplitude=1e-3, k_acoustic=4, theta_amplitude=1e-3, k_theta=2,
                     noise=1e-5, seed=2, device="cpu", nx=None, ny=None, nz=None):
    """Acoustic wave rho' = A sin(2 pi k_a x / n) plus a transverse temperature wave
    theta = theta0 (1 + A_t cos(2 pi k_t y / n)) plus uniform noise U(-noise, noise) on rho
    (drawn on the host from numpy's PCG64 with the given seed, in [s][z][y][x] order)."""
    nx = nx or n
    ny = ny or n
    nz = nz or n
    X, Y, _ = node_positions(nx, ny, nz, device)
    rng = np.random.default_rng(seed)
    eps = torch.from_numpy(rng.uniform(-noise, noise, size=(2, nz, ny, nx))).to(device)
    rho = 1.0 + amplitude * torch.sin(2 * math.pi * k_acoustic * X / nx) + eps
    theta = theta0 * (1.0 + theta_amplitude * torch.cos(2 * math.pi * k_theta * Y / ny))
    zero = torch.zeros_like(rho)
    return _fields(rho, zero, zero, zero, theta)


def fourier_box_field(nx, ny, nz, seed, kmax=8, device="cpu"):
    """Real random field sum_k (a_k cos(2 pi k.x/n) + b_k sin(2 pi k.x/n)) over the
    16^3 box k_i in [-kmax, kmax-1] without k = 0, a_k, b_k ~ N(0,1) from numpy's
    PCG64(seed); normalised to max |field| = 1 over both sub-lattices."""
    rng = np.random.default_rng(seed)
    nk = 2 * kmax
    a = rng.standard_normal((nk, nk, nk))
    b = rng.standard_normal((nk, nk, nk))
    ks = np.arange(-kmax, kmax)
    coef = torch.from_numpy(a - 1j * b).to(device)  # field = Re sum c_k e^{i k.x}
    coef[kmax, kmax, kmax] = 0
    k = torch.from_numpy(ks.astype(np.float64)).to(device)
    out = []

    def phase(n, shift):
        pos = torch.arange(n, dtype=F64, device=device) + shift
        return torch.exp(1j * (2 * math.pi / n) * k[:, None] * pos[None, :])  # complex128 [nk, n]

    for shift in (0.0, 0.5):
        ex, ey, ez = phase(nx, shift), phase(ny, shift), phase(nz, shift)
        # coef[kz, ky, kx] -> field[z, y, x]
        g = torch.einsum("abc,cx->abx", coef, ex)
        g = torch.einsum("abx,by->ayx", g, ey)
        g = torch.einsum("ayx,az->zyx", g, ez)
        out.append(g.real)
    f = torch.stack(out)
    return f / f.abs().max()


def thermoacoustic_pulse(n, theta0, amplitude=1e-2, sigma=8.0, theta_amplitude=1e-3, seed=3, kmax=8,
                         device="cpu", centre=None):
    """Gaussian pressure pulse about the centre, imposed as a density pulse at theta0
    (rho' = A exp(-r^2 / (2 sigma^2)), periodic minimum-image distance), plus a seeded
    random temperature perturbation theta = theta0 (1 + A_t g(x)) with g from a 16^3
    Fourier box normalised to max 1."""
    X, Y, Z = node_positions(n, n, n, device)
    c = n / 2.0 if centre is None else centre

    def d(P):
        r = P - c
        return r - n * torch.round(r / n)

    r2 = d(X) ** 2 + d(Y) ** 2 + d(Z) ** 2
    rho = 1.0 + amplitude * torch.exp(-r2 / (2 * sigma * sigma))
    g = fourier_box_field(n, n, n, seed, kmax=kmax, device=device)
    theta = theta0 * (1.0 + theta_amplitude * g)
    zero = torch.zeros_like(rho)
    return _fields(rho, zero, zero, zero, theta)


def spherical_pulse(n, theta0, b=4.0, eps=1e-3, isentropic=True, device="cpu"):
    """The 3D acoustic spherical pulse (Sec. VII): rho = 1 + eps exp(-alpha r^2) with
    alpha = ln 2 / b^2 (b is the half-width at half maximum, in sc cells), u = 0, centred in
    the periodic n^3 box (minimum-image distance).  With `isentropic` the temperature follows
    the density adiabatically for a monatomic gas, theta = theta0 rho^(2/3), so the whole
    pulse is an acoustic disturbance; otherwise theta = theta0 (the isothermal pulse, which
    also carries an entropy mode)."""
    X, Y, Z = node_positions(n, n, n, device)
    c = n / 2.0

    def d(P):
        r = P - c
        return r - n * torch.round(r / n)

    r2 = d(X) ** 2 + d(Y) ** 2 + d(Z) ** 2
    rho = 1.0 + eps * torch.exp(-(math.log(2.0) / (b * b)) * r2)
    theta = theta0 * rho ** (2.0 / 3.0) if isentropic else torch.full_like(rho, theta0)
    zero = torch.zeros_like(rho)
    return _fields(rho, zero, zero, zero, theta)


def pulse_radius(n, device="cpu"):
    """Distance of every node from the centre of the n^3 box used by `spherical_pulse`."""
    X, Y, Z = node_positions(n, n, n, device)
    c = n / 2.0

    def d(P):
        r = P - c
        return r - n * torch.round(r / n)

    return torch.sqrt(d(X) ** 2 + d(Y) ** 2 + d(Z) ** 2)


def gaussian_pulse_sample(n, theta0, seed, device="cpu"):
    """One seeded training sample: Gaussian density pulse of amplitude U[1e-3, 1e-2], random
    centre and width sigma U[3, 8], plus a Fourier-box temperature perturbation of max 1e-3."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(1e-3, 1e-2)
    centre = rng.uniform(0, n, size=3)
    sigma = rng.uniform(3.0, 8.0)
    X, Y, Z = node_positions(n, n, n, device)

    def d(P, c):
        r = P - c
        return r - n * torch.round(r / n)

    r2 = d(X, centre[0]) ** 2 + d(Y, centre[1]) ** 2 + d(Z, centre[2]) ** 2
    rho = 1.0 + amp * torch.exp(-r2 / (2 * sigma * sigma))
    g = fourier_box_field(n, n, n, seed + 1_000_003, kmax=4, device=device)
    theta = theta0 * (1.0 + 1e-3 * g)
    zero = torch.zeros_like(rho)
    return _fields(rho, zero, zero, zero, theta)


def random_fields(nx, ny, nz, theta0, seed, du=0.05, drho=0.05, dtheta=0.05, device="cpu"):
    """Uncorrelated seeded fields: rho = 1 + drho U(-1,1), u = du U(-1,1), theta = theta0 (1 + dtheta U(-1,1))."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + drho * rng.uniform(-1, 1, size=(2, nz, ny, nx))
    u = du * rng.uniform(-1, 1, size=(3, 2, nz, ny, nx))
    theta = theta0 * (1.0 + dtheta * rng.uniform(-1, 1, size=(2, nz, ny, nx)))
    t = lambda a: torch.from_numpy(a).to(device)
    return {"rho": t(rho).contiguous(), "u": t(u).contiguous(), "theta": t(theta).contiguous()}


def random_populations(nx, ny, nz, weights, seed, spread=0.1):
    """Seeded populations near the rest state: f_i = w_i (1 + spread U(-1,1)), shaped
    [2][41][nz][ny][nx] in the order of the given weight vector."""
    rng = np.random.default_rng(seed)
    w = np.asarray(weights, dtype=np.float64)
    f = w[None, :, None, None, None] * (1.0 + spread * rng.uniform(-1, 1, size=(2, len(w), nz, ny, nx)))
    return f


@dataclass
class BatchSim:
    n: int
    tau: float
    amplitude: float


def batch_sweep(count=64, seed=4, edges=(32, 48, 64, 96, 128), tau_range=(0.51, 1.0), amp_range=(1e-4, 1e-2)):
    """Per-simulation parameters of the batched sweep: cubic edge uniform over ``edges``,
    tau uniform in ``tau_range``, standing-wave amplitude log-uniform in ``amp_range``."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.asarray(edges), size=count)
    tau = rng.uniform(*tau_range, size=count)
    amp = np.exp(rng.uniform(math.log(amp_range[0]), math.log(amp_range[1]), size=count))
    return [BatchSim(int(a), float(b), float(c)) for a, b, c in zip(n, tau, amp)]


def droplet_pair(nx, ny, nz, theta0, rho_gas, rho_liquid, diameter=45.0, separation=30.0, width=5.0, u0=0.2,
                 offset=0.0, device="cpu"):
    """Two liquid drops in their vapour approaching each other along x (Sec. "Droplet
    Collision": a 160 x 200 x 200 box, diameter 45, interface width 5, separation 30, relative
    speed 0.2).  Drop k has the profile phi_k = (1 - tanh(2 (r_k - R) / width)) / 2 about its
    centre, the centres at the box centre -+ (diameter + separation) / 2 in x (separation is
    read as the gap between the drops' surfaces: their centres 30 apart would overlap drops of
    diameter 45), the second one shifted by `offset` in y (the impact parameter); distances
    are to the nearest periodic image.  Density
    rho_gas + (rho_liquid - rho_gas) max(phi_1, phi_2); velocity u_x = (u0 / 2)(phi_1 - phi_2),
    so the vapour starts at rest; theta = theta0."""
    X, Y, Z = node_positions(nx, ny, nz, device)
    R = 0.5 * diameter
    cx, cy, cz = nx / 2.0, ny / 2.0, nz / 2.0
    dx = 0.5 * (diameter + separation)

    def image(d, n):  # nearest periodic image of a displacement
        return torch.remainder(d + 0.5 * n, n) - 0.5 * n

    r1 = torch.sqrt(image(X - (cx - dx), nx) ** 2 + image(Y - cy, ny) ** 2 + image(Z - cz, nz) ** 2)
    r2 = torch.sqrt(image(X - (cx + dx), nx) ** 2 + image(Y - (cy + offset), ny) ** 2 + image(Z - cz, nz) ** 2)
    phi1 = 0.5 * (1 - torch.tanh(2 * (r1 - R) / width))
    phi2 = 0.5 * (1 - torch.tanh(2 * (r2 - R) / width))
    rho = rho_gas + (rho_liquid - rho_gas) * torch.maximum(phi1, phi2)
    ux = 0.5 * u0 * (phi1 - phi2)
    zero = torch.zeros_like(rho)
    return _fields(rho, ux, zero, zero.clone(), torch.full_like(rho, theta0))
