"""GPU parity of the checkpointed c0^2 gradient (pat_gradient_c2) against the FP64 oracle
(oracle/pat_medium.py, pinned by finite differences), through the C ABI.

FP64 plans agree to rounding (1e-10).  FP32 plans: g sums Nt-1 products p_bar^n q^n per point;
each factor carries the FP32 field error of the solve (~1e-6 relative), so 1e-5 relative L2 is
the stated bar, as for the other FP32 results.  The checkpoint interval only changes where the
forward states are recomputed from, never the operations: results for different K are bitwise
equal."""
import numpy as np
import pytest
import torch

from oracle import pat_medium as pm
from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


@pytest.fixture(scope="module")
def dev():
    from paper_1603_02329_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def _T(a, prec, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == "f64" else torch.float32, device=dev)


CASES = [
    ("2d_lossy_f64", lambda: synth.small_lossy_2d(shape=(40, 48), pml=6, Nt=61, n_sensors=16), "f64", (7, 1, 60)),
    ("2d_lossless_f64", lambda: synth.small_lossy_2d(shape=(32, 36), pml=4, Nt=40, n_sensors=12, alpha0=0.0),
     "f64", (5, 39)),
    ("2d_pow2_lossy_f32", lambda: synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=90, n_sensors=24), "f32", (10, 13)),
    ("3d_lossy_f64", lambda: synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=30), "f64", (4, 29)),
    ("3d_lossy_f32", lambda: synth.small_lossy_3d(shape=(16, 16, 16), pml=3, Nt=33), "f32", (8,)),
]


@pytest.mark.parametrize("name,make,prec,Ks", CASES, ids=[c[0] for c in CASES])
def test_gradient_c2_matches_oracle(dev, name, make, prec, Ks):
    from paper_1603_02329_gb300.api import PATOperator

    pb = make()
    ref = Operator.from_problem(pb)
    rng = np.random.default_rng(31)
    h = rng.standard_normal((pb.Nt, ref.Ns))
    g_ref, gp_ref = pm.sound_speed_gradient(ref, pb.p0, h, pb.y)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    tol = 1e-10 if prec == "f64" else 1e-5
    first = None
    for K in Ks:
        g, gp = op.gradient_c2(_T(pb.p0, prec, dev), _T(h, prec, dev), checkpoint_every=K, with_p0_grad=True)
        g, gp = g.cpu().numpy(), gp.cpu().numpy()
        assert rel(g, g_ref) <= tol, (K, rel(g, g_ref))
        assert rel(gp, gp_ref) <= tol, (K, rel(gp, gp_ref))
        if first is None:
            first = g
        else:
            assert np.array_equal(g, first)   # independent of the checkpoint interval
    # the p0 gradient from this sweep is the ordinary adjoint
    assert rel(op.adjoint(_T(h, prec, dev)).cpu().numpy(), gp_ref) <= tol


def test_gradient_c2_edge_cases(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import PATOperator

    # Nt = 1: no time step, no dependence on c0^2 (p^0 = p0 and no density is ever read)
    pb = synth.small_lossy_2d(shape=(24, 24), pml=3, Nt=1, n_sensors=6)
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    h = np.random.default_rng(2).standard_normal((1, op.Ns))
    g = op.gradient_c2(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=3)
    assert float(g.abs().max()) == 0.0
    # K larger than the time axis, Nt = 2: one segment holding one level
    pb = synth.small_lossy_2d(shape=(24, 24), pml=3, Nt=2, n_sensors=6)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(3).standard_normal((2, ref.Ns))
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    g = op.gradient_c2(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=50).cpu().numpy()
    assert rel(g, pm.sound_speed_gradient(ref, pb.p0, h, pb.y)[0]) <= 1e-10
    # invalid interval
    with pytest.raises(_lib.PatError):
        op.gradient_c2(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=0)


# Density gradient (pat_gradient_rho, readings D1-D3) against oracle/pat_medium.density_gradient,
# which is pinned by central finite differences and the scaling invariant <dJ/drho0, rho0> = 0.
# Intervals K below Nt - 1 make several segments, so the step at each segment's top comes from the
# segment above (the carried slot); x-lines of 48 / 36 points take the generic row kernels, 64 / 16
# the register-fused ones.
RHO_CASES = [
    ("2d_lossy_f64", lambda: synth.small_lossy_2d(shape=(40, 48), pml=6, Nt=61, n_sensors=16), "f64", (7, 1, 60)),
    ("2d_lossless_f64", lambda: synth.small_lossy_2d(shape=(32, 36), pml=4, Nt=40, n_sensors=12, alpha0=0.0),
     "f64", (5, 39)),
    ("2d_pow2_lossy_f64", lambda: synth.small_lossy_2d(shape=(32, 64), pml=6, Nt=45, n_sensors=16), "f64", (6, 44)),
    ("2d_pow2_lossless_f64", lambda: synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=33, n_sensors=12, alpha0=0.0),
     "f64", (4,)),
    ("2d_pow2_lossy_f32", lambda: synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=90, n_sensors=24), "f32", (10, 13)),
    ("3d_lossy_f64", lambda: synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=30), "f64", (4, 29)),
    ("3d_pow2_lossy_f64", lambda: synth.small_lossy_3d(shape=(16, 16, 16), pml=3, Nt=25), "f64", (3,)),
    ("3d_lossy_f32", lambda: synth.small_lossy_3d(shape=(16, 16, 16), pml=3, Nt=33), "f32", (8,)),
]


@pytest.mark.parametrize("name,make,prec,Ks", RHO_CASES, ids=[c[0] for c in RHO_CASES])
def test_gradient_rho_matches_oracle(dev, name, make, prec, Ks):
    from paper_1603_02329_gb300.api import PATOperator

    pb = make()
    ref = Operator.from_problem(pb)
    rng = np.random.default_rng(37)
    h = rng.standard_normal((pb.Nt, ref.Ns))
    g_ref = pm.density_gradient(ref, pb.p0, h)
    gp_ref = ref.adjoint(h)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    tol = 1e-10 if prec == "f64" else 1e-5
    first = None
    for K in Ks:
        g, gp = op.gradient_rho(_T(pb.p0, prec, dev), _T(h, prec, dev), checkpoint_every=K, with_p0_grad=True)
        g, gp = g.cpu().numpy(), gp.cpu().numpy()
        assert rel(g, g_ref) <= tol, (K, rel(g, g_ref))
        assert rel(gp, gp_ref) <= tol, (K, rel(gp, gp_ref))
        if first is None:
            first = g
        else:
            assert np.array_equal(g, first)   # independent of the checkpoint interval
    if prec == "f64":   # J(lambda rho0) = J(rho0): <dJ/drho0, rho0> = 0 (reading D3's invariant)
        assert abs(float(np.sum(first * pb.rho))) <= 1e-9 * float(np.sum(np.abs(first * pb.rho)))


@pytest.mark.parametrize("rowu1", ["1", "0"])
def test_gradient_medium_fp32_3d_on_the_fused_paths(dev, monkeypatch, rowu1):
    # FP32 3-D with 128-point x-lines: the checkpointed sweep's hooks in the one-component momentum
    # row kernels (default) and in k_row2 (PAT_ROWU1=0), c0^2 and rho0 gradients against the oracle
    from paper_1603_02329_gb300.api import PATOperator

    monkeypatch.setenv("PAT_ROWU1", rowu1)
    pb = synth.small_lossy_3d(shape=(12, 16, 128), pml=3, Nt=20)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(41).standard_normal((pb.Nt, ref.Ns))
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    assert op.info.rowu1 == (rowu1 == "1")
    gr, gc, gp = op.gradient_medium(_T(pb.p0, "f32", dev), _T(h, "f32", dev), checkpoint_every=6)
    gc_ref, gp_ref = pm.sound_speed_gradient(ref, pb.p0, h, pb.y)
    assert rel(gc.cpu().numpy(), gc_ref) <= 1e-5
    assert rel(gr.cpu().numpy(), pm.density_gradient(ref, pb.p0, h)) <= 1e-5
    assert rel(gp.cpu().numpy(), gp_ref) <= 1e-5


def test_gradient_medium_one_sweep_equals_separate_sweeps(dev):
    from paper_1603_02329_gb300.api import PATOperator

    pb = synth.small_lossy_2d(shape=(32, 64), pml=6, Nt=37, n_sensors=16)
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    h = _T(np.random.default_rng(5).standard_normal((pb.Nt, op.Ns)), "f64", dev)
    x = _T(pb.p0, "f64", dev)
    gr, gc, gp = op.gradient_medium(x, h, checkpoint_every=9)
    assert torch.equal(gr, op.gradient_rho(x, h, checkpoint_every=9))
    assert torch.equal(gc, op.gradient_c2(x, h, checkpoint_every=9))
    assert rel(gp.cpu().numpy(), op.adjoint(h).cpu().numpy()) <= 1e-12


def test_gradient_rho_edge_cases(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import PATOperator

    # Nt = 1: p^0 = p0 does not depend on rho0
    pb = synth.small_lossy_2d(shape=(24, 24), pml=3, Nt=1, n_sensors=6)
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    h = np.random.default_rng(2).standard_normal((1, op.Ns))
    g = op.gradient_rho(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=3)
    assert float(g.abs().max()) == 0.0
    # Nt = 2 with K beyond the time axis: one segment of one step
    pb = synth.small_lossy_2d(shape=(24, 24), pml=3, Nt=2, n_sensors=6)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(3).standard_normal((2, ref.Ns))
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    g = op.gradient_rho(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=50).cpu().numpy()
    assert rel(g, pm.density_gradient(ref, pb.p0, h)) <= 1e-10
    with pytest.raises(_lib.PatError):
        op.gradient_rho(_T(pb.p0, "f64", dev), _T(h, "f64", dev), checkpoint_every=0)
