"""FP64 CPU oracle for the RD3Q41 lattice Boltzmann model (arXiv:1909.08406).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the library.  It shares no
code with the CUDA path.  See ``rd3q41_oracle.c`` for the paper's equations
this follows and for the readings taken where the paper is silent.

Arrays use the oracle's own velocity order (``velocities()``) and the layout
``f[s][i][z][y][x]`` (s = sub-lattice A/B), fields ``a[s][z][y][x]`` and
``u[d][s][z][y][x]``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
NV = 41

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_theta0.restype = ctypes.c_double
        L.or_nvel.restype = ctypes.c_int
        L.or_max_threads.restype = ctypes.c_int
        L.or_entropic_equilibrium.restype = ctypes.c_int
        L.or_path_length.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _kind(project):
    """Equilibrium used by collide/step/init_fields: project=True (series with the momentum
    projection), False (the series as printed), "entropic" (the exact entropic equilibrium,
    Eq. (discreteentropiceq), by Newton's method) or "entropic_path" (that equilibrium, and the
    relaxation alpha beta with the entropic path length alpha of path_length)."""
    if project == "entropic":
        return ctypes.c_int(2)
    if project == "entropic_path":
        return ctypes.c_int(3)
    return ctypes.c_int(1 if project else 0)


def _threads(n):
    return ctypes.c_int(0 if n is None else int(n))


def theta0():
    return lib().or_theta0()


def max_threads():
    return lib().or_max_threads()


def velocities():
    """(c, w, shell): c = [41,3] float velocities, w = [41] weights, shell = [41]."""
    c2 = np.zeros((NV, 3), dtype=np.int32)
    w = np.zeros(NV)
    sh = np.zeros(NV, dtype=np.int32)
    lib().or_velocities(c2.ctypes.data_as(_ip), _p(w), sh.ctypes.data_as(_ip))
    return c2.astype(np.float64) / 2.0, w, sh


def velocities_doubled():
    c2 = np.zeros((NV, 3), dtype=np.int32)
    lib().or_velocities(c2.ctypes.data_as(_ip), None, None)
    return c2


def weight_constraints(theta0_value=0.0):
    r = np.zeros(7)
    lib().or_weight_constraints(ctypes.c_double(theta0_value), _p(r))
    return r


def rest_equilibrium(rho, theta):
    out = np.zeros(NV)
    lib().or_rest_equilibrium(ctypes.c_double(rho), ctypes.c_double(theta), _p(out))
    return out


def m_terms(rho, theta):
    out = np.zeros(4)
    lib().or_m_terms(ctypes.c_double(rho), ctypes.c_double(theta), _p(out))
    return out


def equilibrium(rho, u, theta, project=True):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(NV)
    lib().or_equilibrium(ctypes.c_double(rho), _p(u), ctypes.c_double(theta), ctypes.c_int(int(project)), _p(out))
    return out


def path_length(f, feq):
    """Entropic path length alpha of one node (Sec. "Droplet Collision"): the nontrivial root of
    H(f + alpha (f^eq - f)) = H(f), H(f) = sum_i f_i ln(f_i / w_i); 2 when f = f^eq or no root
    lies below the positivity limit.  f, feq: [41] float64 in the oracle's velocity order."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    feq = np.ascontiguousarray(feq, dtype=np.float64)
    return lib().or_path_length(_p(f), _p(feq))


def entropic_equilibrium(rho, u, theta):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(NV)
    it = lib().or_entropic_equilibrium(ctypes.c_double(rho), _p(u), ctypes.c_double(theta), _p(out))
    if it < 0:
        raise RuntimeError("entropic Newton solve did not converge")
    return out


def moments(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = ctypes.c_double()
    th = ctypes.c_double()
    u = np.zeros(3)
    lib().or_moments(_p(f), ctypes.byref(rho), _p(u), ctypes.byref(th))
    return rho.value, u, th.value


def collide(f, tau, project=True):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(NV)
    lib().or_collide(_p(f), ctypes.c_double(tau), _kind(project), _p(out))
    return out


def stream(fpost, nthreads=None):
    fpost = np.ascontiguousarray(fpost, dtype=np.float64)
    _, _, nz, ny, nx = fpost.shape
    out = np.empty_like(fpost)
    lib().or_stream(_i64(nx), _i64(ny), _i64(nz), _p(fpost), _p(out), _threads(nthreads))
    return out


def step(f, tau, nsteps, project=True, nthreads=None):
    """Advance post-collision populations f[2][41][nz][ny][nx] by nsteps; returns a new array."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    _, _, nz, ny, nx = f.shape
    work = np.empty_like(f)
    lib().or_step(_i64(nx), _i64(ny), _i64(nz), ctypes.c_double(tau), _kind(project), _i64(nsteps),
                  _p(f), _p(work), _threads(nthreads))
    return f


def step_walls(f, tau, nsteps, bottom, top, project=True, nthreads=None, wall_rho=False):
    """Advance f by nsteps with kinetic (diffuse) walls normal to z (x, y periodic).
    bottom, top: (u_x, u_y, theta) of each wall, each a number (the same for every cell column
    of the wall) or an array [ny][nx]; the walls sit a quarter cell beyond the outermost node
    planes (channel height nz cells).  With wall_rho=True also returns the walls' densities per
    step and column, shape (nsteps, 2, ny, nx)."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    _, _, nz, ny, nx = f.shape
    work = np.empty_like(f)
    w = np.zeros((2, 4, ny, nx))
    for side, (ux, uy, th) in enumerate((bottom, top)):
        w[side, 0], w[side, 1], w[side, 3] = ux, uy, th
    w = np.ascontiguousarray(w)
    rho_w = np.zeros((int(nsteps), 2, ny, nx))
    lib().or_step_walls(_i64(nx), _i64(ny), _i64(nz), ctypes.c_double(tau), _kind(project), _i64(nsteps),
                        _p(f), _p(work), _p(w), _p(rho_w), _threads(nthreads))
    return (f, rho_w) if wall_rho else f


def step_nodes(fpost, tau, nodes, project=True, nthreads=None):
    """One update at the listed flat node indices ((s*nz+z)*ny+y)*nx+x; returns [n][41]."""
    fpost = np.ascontiguousarray(fpost, dtype=np.float64)
    _, _, nz, ny, nx = fpost.shape
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.zeros((len(nodes), NV))
    lib().or_step_nodes(_i64(nx), _i64(ny), _i64(nz), ctypes.c_double(tau), _kind(project), _p(fpost),
                        nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _i64(len(nodes)), _p(out),
                        _threads(nthreads))
    return out


def init_fields(rho, u, theta, project=True, nthreads=None):
    """Equilibrium populations for fields rho[2][nz][ny][nx], u[3][2][nz][ny][nx], theta[2][nz][ny][nx]."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    _, nz, ny, nx = rho.shape
    f = np.zeros((2, NV, nz, ny, nx))
    lib().or_init_fields(_i64(nx), _i64(ny), _i64(nz), _p(rho), _p(u), _p(theta), _kind(project), _p(f),
                         _threads(nthreads))
    return f


def get_moments(f, nthreads=None):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, _, nz, ny, nx = f.shape
    rho = np.zeros((2, nz, ny, nx))
    u = np.zeros((3, 2, nz, ny, nx))
    th = np.zeros((2, nz, ny, nx))
    lib().or_get_moments(_i64(nx), _i64(ny), _i64(nz), _p(f), _p(rho), _p(u), _p(th), _threads(nthreads))
    return rho, u, th


def conserved(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    _, _, nz, ny, nx = f.shape
    out = np.zeros(5)
    lib().or_conserved(_i64(nx), _i64(ny), _i64(nz), _p(f), _p(out))
    return out


def beta_of_tau(tau):
    return 0.0 if np.isinf(tau) else 1.0 / (2.0 * tau + 1.0)
