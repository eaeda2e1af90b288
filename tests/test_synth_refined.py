"""The data generator that avoids the inverse crime (synth.refined_problem): a finer grid over the
same extent, with the sensors at the same physical positions, checked with the FP64 oracle.  Data
generated on it agree with the reconstruction grid's to discretization accuracy for a smooth
phantom. Contaminating the maps moves the data by a small but non-zero amount."""
import numpy as np

from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth


def _smooth_case():
    pb = synth.small_lossy_2d(shape=(48, 48), pml=6, Nt=80, n_sensors=16)
    g = np.meshgrid(*synth.coords(pb.shape, pb.spacing), indexing="ij")
    pb.p0 = np.exp(-(g[0] ** 2 + g[1] ** 2) / (2 * (0.4e-3) ** 2))
    return pb


def test_refined_geometry():
    pb = _smooth_case()
    pf = synth.refined_problem(pb, ratio=1.5, map_snr_db=None, seed=1)
    assert pf.shape == (72, 72) and pf.pml == (9, 9)
    for n, h, nf, hf in zip(pb.shape, pb.spacing, pf.shape, pf.spacing):
        assert abs(n * h - nf * hf) < 1e-15
    assert pf.dt == pb.dt and pf.Nt == pb.Nt
    assert np.array_equal(pf.sensor_pos, pb.sensor_pos)
    # on-grid sensors become their physical positions, (x, y) order
    pb3 = synth.small_lossy_3d(shape=(8, 10, 12), pml=2, Nt=10)
    pf3 = synth.refined_problem(pb3, ratio=1.5, map_snr_db=None)
    idx = np.unravel_index(pb3.sensor_index[5], pb3.shape)
    x = [(idx[a] - pb3.shape[a] // 2) * pb3.spacing[a] for a in range(3)][::-1]
    assert np.allclose(pf3.sensor_pos[5], x, rtol=0, atol=1e-18)
    assert all(synth.smooth_even_size(n) == n for n in pf3.shape)
    assert synth.smooth_even_size(738) == 750 and synth.smooth_even_size(472) == 480


def test_refined_data_match_the_reconstruction_grid():
    pb = _smooth_case()
    d_c = Operator.from_problem(pb).forward(pb.p0)
    pf = synth.refined_problem(pb, ratio=1.5, map_snr_db=None, seed=1)
    d_f = Operator.from_problem(pf).forward(pf.p0)
    e0 = np.linalg.norm(d_f - d_c) / np.linalg.norm(d_c)
    assert e0 < 1e-2
    pn = synth.refined_problem(pb, ratio=1.5, map_snr_db=35.0, seed=1)
    assert np.abs(pn.c - pf.c).max() > 1.0
    d_n = Operator.from_problem(pn).forward(pn.p0)
    e1 = np.linalg.norm(d_n - d_c) / np.linalg.norm(d_c)
    assert e1 < 2e-2 and np.linalg.norm(d_n - d_f) > 1e-4 * np.linalg.norm(d_f)
