"""The seeded synthetic workloads follow the recipe the benchmark and the parity tests state for them
(the stand-ins for the paper's Sec. VI.A and VI.B experiments): grid, spacing, PML, medium
statistics, absorption, sensor geometry, time axis and phantom value ranges, and the same arrays
for the same seed."""
import numpy as np
import pytest

from paper_1603_02329_gb300 import synth


def test_disc_phantom_168():
    pb = synth.disc_phantom_2d(seed=1)
    assert pb.shape == (168, 168) and pb.spacing == (1e-4, 1e-4) and pb.pml == (20, 20)
    assert pb.pml_alpha == 2.0                      # Sec. VI.A: 2 Np per grid point
    assert np.all(pb.c == 1500.0) and np.all(pb.rho == 1000.0) and not pb.lossy
    assert pb.dt == pytest.approx(0.3 * 1e-4 / 1500.0) and pb.Nt == 600
    # 256 point sensors equispaced on a circle of radius 5.5 mm about the grid centre
    r = np.hypot(pb.sensor_pos[:, 0], pb.sensor_pos[:, 1])
    assert pb.Ns == 256 and np.allclose(r, 5.5e-3)
    ang = np.sort(np.mod(np.arctan2(pb.sensor_pos[:, 1], pb.sensor_pos[:, 0]), 2 * np.pi))
    assert np.allclose(np.diff(ang), 2 * np.pi / 256)
    # five binary discs of amplitude U[0.5, 1]: centres within 3.5 mm, radii up to 1.5 mm, so every
    # source point lies inside the sensor circle
    x = (np.arange(168) - 84) * 1e-4
    rr = np.hypot(*np.meshgrid(x, x, indexing="ij"))
    assert pb.p0.min() == 0.0 and 0.5 <= pb.p0.max() <= 5.0
    assert rr[pb.p0 > 0].max() <= 5.0e-3 + 1e-12


def test_vessel_phantom_512():
    pb = synth.vessel_phantom_2d(seed=2)
    assert pb.shape == (512, 512) and pb.spacing == (5e-5, 5e-5) and pb.pml == (20, 20)
    # c = 1500 + 100 n1, rho = 1000 (1 + 0.05 n2), n1 and n2 smoothed noise of zero mean, unit variance
    assert pb.c.mean() == pytest.approx(1500.0, abs=1e-9) and pb.c.std() == pytest.approx(100.0, rel=1e-9)
    assert pb.rho.mean() == pytest.approx(1000.0, abs=1e-9) and pb.rho.std() == pytest.approx(50.0, rel=1e-9)
    # smoothed with sigma = 8 px: neighbouring points are strongly correlated, distant ones are not
    n1 = (pb.c - 1500.0) / 100.0
    assert np.mean(n1 * np.roll(n1, 1, axis=1)) > 0.95
    assert abs(np.mean(n1 * np.roll(n1, 128, axis=1))) < 0.1
    assert np.all(pb.alpha0 == 0.75) and pb.y == 1.5
    assert pb.dt == pytest.approx(0.3 * 5e-5 / pb.c.max()) and pb.Nt == 2000
    # 512 on-grid sensors along row 20, the first row inside the PML
    assert np.array_equal(pb.sensor_index, 20 * 512 + np.arange(512))
    # vessels and discs of amplitude U[0.5, 1], overlaps take the maximum
    assert pb.p0.min() == 0.0 and 0.5 <= pb.p0.max() <= 1.0
    assert 0.01 < np.mean(pb.p0 > 0) < 0.2


def test_tube_phantom_128():
    pb = synth.tube_phantom_3d(seed=3)
    assert pb.shape == (128,) * 3 and pb.spacing == (6.25e-5,) * 3 and pb.pml == (10,) * 3
    assert pb.c.std() == pytest.approx(100.0, rel=1e-9) and pb.rho.std() == pytest.approx(50.0, rel=1e-9)
    assert np.all(pb.alpha0 == 0.75) and pb.y == 1.5 and pb.Nt == 1000
    # a 64 x 64 array at stride 2 on the face z = 10 (the first plane inside the PML)
    z, yy, xx = np.unravel_index(pb.sensor_index, pb.shape)
    assert pb.Ns == 64 * 64 and np.all(z == 10)
    assert np.array_equal(np.unique(yy), np.arange(0, 128, 2)) and np.array_equal(np.unique(xx), np.arange(0, 128, 2))
    # tubes of amplitude U[0.5, 1] (overlaps take the maximum) and three balls, which add where they
    # overlap
    assert pb.p0.min() == 0.0 and 0.5 <= pb.p0.max() <= 3.0


def test_awgn_snr():
    rng = np.random.default_rng(0)
    data = np.sin(np.linspace(0, 50, 200000))
    noisy = synth.awgn(rng, data, 40.0)
    snr = 10 * np.log10(np.mean(data**2) / np.mean((noisy - data) ** 2))
    assert snr == pytest.approx(40.0, abs=0.05)


def test_generators_are_seeded():
    a, b, c = synth.vessel_phantom_2d(seed=2, n=128), synth.vessel_phantom_2d(seed=2, n=128), \
        synth.vessel_phantom_2d(seed=3, n=128)
    for f in ("c", "rho", "p0"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
        assert not np.array_equal(getattr(a, f), getattr(c, f))
