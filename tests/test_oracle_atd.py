"""Pins of the oracle's "adjoint-then-discretize" adjoint (oracle/pat_atd.py; Sec. III Eqs. (moma),
(massa), (statea), (adjj); Sec. VI) against the exact transpose.

The two are different discretisations of one continuous adjoint, so with the time interval [0, T]
fixed, dt * H^T h - ATD(h) must vanish as dt -> 0 at the scheme's order, on a heterogeneous
absorbing medium; a wrong sign, factor, operator order or source timing leaves an O(1) remainder.
Two deviations do not vanish and are stated (readings A4, A5): inside the PML layer, where the
split of the adjoint densities differs, and between the paper's gradient rho*(T) / rho0 and the
gradient of the forward map's own initial state, which differ by O(alpha0)."""
import os

import numpy as np
import pytest

from oracle.pat_atd import adjoint_then_discretize
from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth


def _family(alpha0, pml, levels=3, initial="R5", graded=False):
    """(whole-grid, interior) relative differences for dt, dt/2, ... over a fixed [0, T].  With
    ``graded`` the absorption varies from 0.1 to 1.9 times alpha0 across the grid, so that the
    order of tau, eta and the fractional Laplacians in Eq. (statea) matters."""
    pb = synth.small_lossy_2d(shape=(32, 36), pml=5, Nt=41, n_sensors=10, alpha0=alpha0)
    if graded:
        x = np.linspace(-1.0, 1.0, pb.shape[1])
        pb.alpha0 = alpha0 * (1.0 + 0.9 * np.sin(3.0 * x))[None, :] * np.ones(pb.shape)
    T = (pb.Nt - 1) * pb.dt
    rng = np.random.default_rng(3)
    amp, t0 = rng.standard_normal(10), rng.uniform(0.3 * T, 0.7 * T, 10)
    width, om = 0.1 * T, 2 * np.pi / (0.25 * T)
    whole, inner = [], []
    for k in range(levels):
        dt = pb.dt / 2**k
        Nt = (pb.Nt - 1) * 2**k + 1
        op = Operator(pb.shape, pb.spacing, (pml, pml), pb.pml_alpha, pb.c, pb.rho, pb.alpha0, pb.y, dt, Nt,
                      sensor_pos=pb.sensor_pos)
        t = np.arange(Nt)[:, None] * dt
        h = amp * np.exp(-((t - t0) / width) ** 2) * np.sin(om * (t - t0))   # smooth in time
        gt = dt * op.adjoint(h)
        ga = adjoint_then_discretize(op, h, initial)
        sl = (slice(pml, pb.shape[0] - pml), slice(pml, pb.shape[1] - pml))
        whole.append(np.linalg.norm(ga - gt) / np.linalg.norm(gt))
        inner.append(np.linalg.norm((ga - gt)[sl]) / np.linalg.norm(gt[sl]))
    return np.array(whole), np.array(inner)


@pytest.mark.parametrize("alpha0", [0.0, 0.75])
def test_atd_converges_to_the_transpose_at_first_order(alpha0):
    whole, _ = _family(alpha0, pml=0)
    ratios = whole[:-1] / whole[1:]
    assert np.all(ratios > 1.8), ratios
    assert whole[-1] < 1e-3


def test_atd_converges_with_graded_absorption():
    # tau and eta vary by a factor 19 across the grid: swapping them with the fractional
    # Laplacians in Eq. (statea) leaves a remainder that does not vanish with dt
    whole, _ = _family(1.5, pml=0, graded=True)
    assert np.all(whole[:-1] / whole[1:] > 1.8), whole
    assert whole[-1] < 3e-3


@pytest.mark.parametrize("alpha0", [0.0, 0.75])
def test_atd_with_pml_converges_outside_the_layer(alpha0):
    whole, inner = _family(alpha0, pml=5)
    assert np.all(inner[:-1] / inner[1:] > 1.8), inner
    assert inner[-1] < 1e-3
    # inside the layer the split adjoint densities differ (reading A4): no convergence there
    assert whole[-1] > 5e-3 and whole[-1] > 0.9 * whole[0]


def test_paper_gradient_differs_by_order_alpha0():
    # reading A5: rho*(T) / rho0 is the gradient for the paper's initial condition; against the
    # transpose of the forward map's own initial state the remainder does not vanish with dt and
    # scales with alpha0
    d_full, _ = _family(0.75, pml=0, levels=2, initial="paper")
    d_half, _ = _family(0.375, pml=0, levels=2, initial="paper")
    assert d_full[1] > 0.9 * d_full[0] and d_full[1] > 3e-3
    assert 1.6 < d_full[1] / d_half[1] < 2.4
    lossless, _ = _family(0.0, pml=0, levels=1, initial="paper")
    lossless_r5, _ = _family(0.0, pml=0, levels=1, initial="R5")
    assert lossless[0] == lossless_r5[0]


@pytest.mark.skipif(not os.environ.get("PAT_SLOW_ORACLE"), reason="about 6 minutes of FP64 CPU work; set PAT_SLOW_ORACLE=1")
def test_deviation_on_the_512_vessel_workload():
    # The paper's adjoint against the transpose on the 512^2 absorbing workload (Nt 2000, sensors
    # on the first row inside the 20-point PML), residual = the 40 dB data itself.  Measured:
    # 65 % over the whole grid (the PML layer, A4), 6.1 % inside it, dot-test mismatch 1.5 %
    # (transpose: 2e-16).
    pb = synth.vessel_phantom_2d()
    op = Operator.from_problem(pb)
    d = op.forward(pb.p0)
    h = d + 0.01 * np.sqrt(np.mean(d * d)) * np.random.default_rng(7).standard_normal(d.shape)
    gt = op.dt * op.adjoint(h)
    ga = adjoint_then_discretize(op, h)
    P = pb.pml[0]
    sl = (slice(P, pb.shape[0] - P), slice(P, pb.shape[1] - P))
    inner = np.linalg.norm((ga - gt)[sl]) / np.linalg.norm(gt[sl])
    lhs = float(np.sum(d * h))
    mismatch = abs(lhs - np.sum(pb.p0 * ga) / op.dt) / abs(lhs)
    assert 0.01 < inner < 0.1
    assert 1e-3 < mismatch < 0.05


def test_atd_converges_in_3d():
    # the source split 1/d and the 3-D derivative set: first order on a 3-D absorbing medium
    pb = synth.small_lossy_3d(shape=(12, 16, 20), pml=3, Nt=21)
    T = (pb.Nt - 1) * pb.dt
    rng = np.random.default_rng(4)
    Ns = len(pb.sensor_index)
    amp, t0 = rng.standard_normal(Ns), rng.uniform(0.3 * T, 0.7 * T, Ns)
    width, om = 0.12 * T, 2 * np.pi / (0.3 * T)
    diffs = []
    for k in range(3):
        dt = pb.dt / 2**k
        Nt = (pb.Nt - 1) * 2**k + 1
        op = Operator(pb.shape, pb.spacing, (0, 0, 0), pb.pml_alpha, pb.c, pb.rho, pb.alpha0, pb.y, dt, Nt,
                      sensor_index=pb.sensor_index)
        t = np.arange(Nt)[:, None] * dt
        h = amp * np.exp(-((t - t0) / width) ** 2) * np.sin(om * (t - t0))
        gt = dt * op.adjoint(h)
        diffs.append(np.linalg.norm(adjoint_then_discretize(op, h) - gt) / np.linalg.norm(gt))
    diffs = np.array(diffs)
    assert np.all(diffs[:-1] / diffs[1:] > 1.8), diffs
    assert diffs[-1] < 3e-3
