"""Pins of the oracle's time-reversal reconstruction (oracle/pat_tr.py; Sec. II.B.1), readings T1-T5.

* Every node a sensor: the image is the enforced t = 0 frame, exactly (order of the reversal).
* Closed sensor surface, homogeneous lossless medium, data until the waves have left: TR recovers
  p0 (Huygens' principle in 3-D; in 2-D the wake has passed by the end of the record).
* Absorbing medium: reversing the absorption sign (band-limited, T5) undoes most of the loss that
  plain TR leaves, and keeping more of the band undoes more of it (noise-free data).
"""
import os

import numpy as np
import pytest

from oracle.pat_oracle import Operator
from oracle.pat_tr import time_reversal


def _box_nodes(shape, lo, hi):
    """Flat indices of the grid nodes on the surface of the box [lo, hi]^d."""
    idx = np.indices(shape).reshape(len(shape), -1).T
    inside = np.all((idx >= lo) & (idx <= hi), axis=1)
    return np.flatnonzero(inside & np.any((idx == lo) | (idx == hi), axis=1))


def _gaussians(shape, h, centres, widths, amps):
    ax = [(np.arange(n) - n // 2) * h for n in shape]
    X = np.meshgrid(*ax, indexing="ij")
    out = np.zeros(shape)
    for c, w, a in zip(centres, widths, amps):
        out += a * np.exp(-sum((X[i] - c[i] * h) ** 2 for i in range(len(shape))) / (2 * (w * h) ** 2))
    return out


def test_all_nodes_return_the_first_frame():
    shape, h = (20, 24), 1e-4
    rng = np.random.default_rng(1)
    op = Operator(shape, (h, h), (4, 4), 2.0, 1500.0, 1000.0, 0.75, 1.5, 0.3 * h / 1500.0, 12,
                  sensor_index=np.arange(20 * 24))
    data = rng.standard_normal((12, 20 * 24))
    assert np.array_equal(time_reversal(op, data).ravel(), data[0])
    with pytest.raises(ValueError):
        time_reversal(Operator(shape, (h, h), (4, 4), 2.0, 1500.0, 1000.0, 0.0, 1.5, 2e-8, 4,
                               sensor_pos=np.array([[0.5e-4, 0.0]])), np.zeros((4, 1)))
    with pytest.raises(ValueError):
        time_reversal(Operator(shape, (h, h), (4, 4), 2.0, 1500.0, 1000.0, 0.0, 1.5, 2e-8, 4,
                               sensor_index=[5, 5]), np.zeros((4, 2)))


def test_closed_surface_recovers_p0_3d():
    n, h, c = 48, 1e-4, 1500.0
    p0 = _gaussians((n,) * 3, h, [(0, -2, 3)], [2.5], [1.0])
    op = Operator((n,) * 3, (h,) * 3, (6,) * 3, 2.0, c, 1000.0, 0.0, 1.5, 0.3 * h / c, 150,
                  sensor_index=_box_nodes((n,) * 3, 8, n - 9))
    img = time_reversal(op, op.forward(p0))
    sl = (slice(9, n - 9),) * 3
    assert np.linalg.norm((img - p0)[sl]) / np.linalg.norm(p0[sl]) < 0.03


def _absorbing_2d(alpha0):
    n, h, c = 96, 1e-4, 1500.0
    p0 = _gaussians((n, n), h, [(-3, 5), (6, -8)], [2.5, 3.75], [1.0, 0.7])
    op = Operator((n, n), (h, h), (10, 10), 2.0, c, 1000.0, alpha0, 1.5, 0.3 * h / c, 600,
                  sensor_index=_box_nodes((n, n), 12, n - 13))
    sl = (slice(13, n - 13),) * 2
    return op, op.forward(p0), p0, sl


def test_closed_surface_recovers_p0_2d_and_compensation_is_neutral_without_loss():
    op, data, p0, sl = _absorbing_2d(0.0)
    img = time_reversal(op, data)
    assert np.linalg.norm((img - p0)[sl]) / np.linalg.norm(p0[sl]) < 0.02
    assert np.array_equal(img, time_reversal(op, data, compensate=False))


def test_reversed_absorption_compensates_the_loss():
    op, data, p0, sl = _absorbing_2d(5.0)
    re = lambda img: np.linalg.norm((img - p0)[sl]) / np.linalg.norm(p0[sl])
    plain = re(time_reversal(op, data, compensate=False))
    comp = [re(time_reversal(op, data, k_cut=kc)) for kc in (0.25, 0.5, 0.75)]
    assert plain > 0.2                    # the loss is real: plain TR is off by a fifth or more
    assert comp[1] < 0.35 * plain         # the default band undoes most of it
    assert comp[0] > comp[1] > comp[2]    # a wider band undoes more (noise-free data)


@pytest.mark.skipif(not os.environ.get("PAT_SLOW_ORACLE"), reason="about a minute of FP64 CPU work; set PAT_SLOW_ORACLE=1")
def test_time_reversal_warm_start_helps_fista():
    # Sec. II.B.1's TR image as FISTA's starting point (the paper's baseline, used as a warm start):
    # a 128^2 absorbing vessel workload seen by one line of sensors (limited view), 40 dB noise.
    # Measured: TR alone RE 0.77; FISTA from it reaches in 10 iterations the RE that FISTA from
    # zero reaches in 14.
    from oracle import pat_optim as po
    from paper_1603_02329_gb300 import synth

    pb = synth.vessel_phantom_2d(n=128, pml=10, Nt=500)
    op = Operator.from_problem(pb)
    phat = synth.awgn(np.random.default_rng(9), op.forward(pb.p0), 40.0)
    L = po.power_iteration(lambda v: op.adjoint(op.forward(v)), pb.shape, n_iter=15, seed=1)
    tr = np.maximum(time_reversal(op, phat), 0.0)
    re_tr = np.linalg.norm(tr - pb.p0) / np.linalg.norm(pb.p0)
    assert re_tr < 0.85
    opts = po.FistaOpts(variant=1, max_iter=14, eps_d=-1.0, recursion=False)
    _, cold = po.mg_fista(op, phat, np.zeros(pb.shape), L, opts, p_exact=pb.p0)
    _, warm = po.mg_fista(op, phat, tr, L, opts, p_exact=pb.p0)
    re_cold = np.array([r.RE for r in cold])
    re_warm = np.array([r.RE for r in warm])
    assert re_warm[0] < re_cold[0] - 0.15
    assert re_warm[9] <= re_cold[13]
