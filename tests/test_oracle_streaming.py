"""Brute-force pins of the oracle's streaming on the bcc grid (Sec. IV, Sec. II).

The brute force here works in real (fractional) node positions: a population
at the node at position p moves to p + c_i (mod the box); sub-lattice A has
integer positions, B has positions offset by (1/2, 1/2, 1/2).  The oracle
instead uses doubled integer coordinates, so the two are independent.
Streaming is a pure copy: results must be bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1909_08406_gb300 import workloads as wl


def _brute_force_stream(fpost, c):
    _, nv, nz, ny, nx = fpost.shape
    fpre = np.full_like(fpost, np.nan)
    dims = np.array([nx, ny, nz], dtype=np.float64)
    for s in range(2):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    p = np.array([x, y, z], dtype=np.float64) + 0.5 * s
                    for i in range(nv):
                        q = np.mod(p + c[i], dims)
                        frac = q - np.floor(q)
                        assert np.all(frac == frac[0]) and frac[0] in (0.0, 0.5)
                        sd = 1 if frac[0] == 0.5 else 0
                        qx, qy, qz = np.floor(q).astype(int)
                        fpre[sd, i, qz, qy, qx] = fpost[s, i, z, y, x]
    return fpre


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 7), (1, 2, 5)])
def test_stream_matches_brute_force(shape):
    nx, ny, nz = shape
    c, w, _ = oracle.velocities()
    f = wl.random_populations(nx, ny, nz, w, seed=11)
    got = oracle.stream(f)
    ref = _brute_force_stream(f, c)
    assert not np.isnan(ref).any()
    assert np.array_equal(got, ref)


def test_stream_is_a_permutation_per_plane():
    c, w, _ = oracle.velocities()
    f = wl.random_populations(5, 4, 3, w, seed=12)
    g = oracle.stream(f)
    for i in range(41):
        assert np.array_equal(np.sort(f[:, i].ravel()), np.sort(g[:, i].ravel()))


def test_free_streaming_step_is_pure_streaming():
    """With tau = inf (beta = 0) the BGK step is the identity on collision, so a step is a stream."""
    c, w, _ = oracle.velocities()
    f = wl.random_populations(4, 3, 5, w, seed=13)
    assert np.array_equal(oracle.step(f, np.inf, 1), oracle.stream(f))


def test_stream_round_trip():
    """Streaming with c and then the inverted set returns the start (inversion symmetry)."""
    c, w, _ = oracle.velocities()
    f = wl.random_populations(4, 4, 4, w, seed=14)
    g = oracle.stream(f)
    inv = [int(np.where((c == -c[i]).all(1))[0][0]) for i in range(41)]
    g2 = oracle.stream(g[:, inv])[:, inv]
    assert np.array_equal(g2, f)
