"""The seeded input generators: shapes, dtypes, determinism and the stated recipes."""
import math

import numpy as np
import pytest
import torch

from paper_1909_08406_gb300 import workloads as wl

TH0 = 0.2948964908710634


def _check(fl, nx, ny, nz):
    assert fl["rho"].shape == (2, nz, ny, nx) and fl["theta"].shape == (2, nz, ny, nx)
    assert fl["u"].shape == (3, 2, nz, ny, nx)
    for v in fl.values():
        assert v.dtype == torch.float64 and v.is_contiguous()


def test_node_positions_bcc():
    X, Y, Z = wl.node_positions(3, 4, 5)
    assert X.shape == (2, 5, 4, 3)
    assert X[0, 0, 0, 2] == 2.0 and X[1, 0, 0, 2] == 2.5
    assert Y[1, 0, 3, 0] == 3.5 and Z[1, 4, 0, 0] == 4.5


def test_generators_shapes_and_determinism():
    a = wl.acoustic_thermal(16, TH0, seed=2)
    b = wl.acoustic_thermal(16, TH0, seed=2)
    _check(a, 16, 16, 16)
    for k in a:
        assert torch.equal(a[k], b[k])
    assert (a["rho"] - 1).abs().max() <= 1e-3 + 1e-5 + 1e-15
    t = wl.thermoacoustic_pulse(24, TH0)
    _check(t, 24, 24, 24)
    assert (t["rho"] - 1).max() == pytest.approx(1e-2, rel=0.05)  # pulse peak near the centre
    assert (t["theta"] / TH0 - 1).abs().max() == pytest.approx(1e-3, rel=1e-12)
    r = wl.random_fields(5, 4, 3, TH0, seed=1)
    _check(r, 5, 4, 3)


def test_fourier_box_field_is_real_band_limited_and_normalised():
    g = wl.fourier_box_field(32, 32, 32, seed=3)
    assert g.abs().max() == pytest.approx(1.0, rel=1e-14)
    spec = np.fft.fftn(g[0].numpy())
    k = np.fft.fftfreq(32, 1 / 32)
    KZ, KY, KX = np.meshgrid(k, k, k, indexing="ij")
    outside = (np.abs(KX) > 8) | (np.abs(KY) > 8) | (np.abs(KZ) > 8)
    assert np.abs(spec[outside]).max() < 1e-9 * np.abs(spec).max()


def test_batch_sweep_ranges():
    sims = wl.batch_sweep()
    assert len(sims) == 64
    assert {s.n for s in sims} <= {32, 48, 64, 96, 128}
    assert all(0.51 <= s.tau <= 1.0 for s in sims)
    assert all(1e-4 <= s.amplitude <= 1e-2 for s in sims)
    assert [s.n for s in sims] == [s.n for s in wl.batch_sweep()]


def test_standing_wave_values():
    fl = wl.standing_wave(8, 1, 1, TH0, amplitude=1e-3)
    assert fl["rho"][1, 0, 0, 1].item() == pytest.approx(1 + 1e-3 * math.sin(2 * math.pi * 1.5 / 8))
    assert torch.all(fl["theta"] == TH0)


def test_droplet_pair():
    """Two drops approaching head-on: liquid at the centres moving at +-u0/2, vapour at rest, no
    net momentum (the pair is mirror-symmetric about the box centre, sub-lattices included), and
    the liquid volume of two spheres with the tanh profile's correction."""
    import math
    nx, ny, nz, d, sep, u0 = 48, 40, 40, 16.0, 8.0, 0.2
    f = wl.droplet_pair(nx, ny, nz, 0.3, 0.2, 2.4, diameter=d, separation=sep, width=3.0, u0=u0)
    rho, u = f["rho"], f["u"]
    assert rho.shape == (2, nz, ny, nx) and u.shape == (3, 2, nz, ny, nx)
    c1 = int(nx / 2 - (d + sep) / 2)  # centre of the left drop (an A node)
    c2 = int(nx / 2 + (d + sep) / 2)
    # at the centres tanh(-2R/width) = -1 + 1e-4
    assert float(rho[0, nz // 2, ny // 2, c1]) == pytest.approx(2.4, abs=2e-4)
    assert float(u[0, 0, nz // 2, ny // 2, c1]) == pytest.approx(u0 / 2, rel=1e-4)
    assert float(u[0, 0, nz // 2, ny // 2, c2]) == pytest.approx(-u0 / 2, rel=1e-4)
    assert float(rho[0, 0, 0, 0]) == pytest.approx(0.2, abs=1e-9) and abs(float(u[0, 0, 0, 0, 0])) <= 1e-9
    assert abs(float((rho * u[0]).sum())) <= 1e-12 * float((rho * u[0]).abs().sum())
    assert float(u[1:].abs().max()) == 0.0 and float((f["theta"] - 0.3).abs().max()) == 0.0
    # phi = 1 / (1 + exp((r - R) / T)), T = width / 4: by the Sommerfeld expansion each drop holds
    # (4 pi / 3)(R^3 + pi^2 T^2 R) of liquid
    volume = 0.5 * float(((rho - 0.2) / (2.4 - 0.2)).sum())
    R, T = d / 2, 3.0 / 4
    assert volume == pytest.approx(2 * 4 / 3 * math.pi * (R ** 3 + math.pi ** 2 * T ** 2 * R), rel=0.01)
