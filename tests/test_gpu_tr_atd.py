"""GPU parity of the time-reversal image (pat_time_reversal; Sec. II.B.1, readings T1-T5) and of the
paper's adjoint-then-discretize adjoint (pat_adjoint_atd; Sec. VI with Sec. III Eqs. (moma), (massa),
(statea), (adjj); readings A1-A5) against the FP64 oracle modules oracle/pat_tr.py and
oracle/pat_atd.py, through the C ABI.  FP64 plans: relative L2 <= 1e-11; FP32: <= 1e-5.

Both run the forward-direction per-phase kernels with their time-reversal / adjoint-then-discretize
modes, so the cases cover x-lines of both kernel families (power-of-two lengths take the
register-fused row kernels, others the generic ones), lossy and lossless media, 2-D and 3-D."""
import numpy as np
import pytest
import torch

from oracle.pat_atd import adjoint_then_discretize
from oracle.pat_oracle import Operator
from oracle.pat_tr import time_reversal
from paper_1603_02329_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 1e-5}


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


# on-grid sensors: line arrays (2-D vessel cases, on the first row inside the PML) and planar arrays (3-D)
TR_CASES = [
    ("2d_pow2_lossy", lambda: synth.vessel_phantom_2d(n=64, pml=8, Nt=150, n_vessels=2, n_discs=2)),
    ("2d_pow2_lossless", lambda: synth.vessel_phantom_2d(n=64, pml=8, Nt=120, alpha0=0.0, n_vessels=2, n_discs=2)),
    ("2d_generic_lossy", lambda: synth.vessel_phantom_2d(n=60, pml=6, Nt=130, n_vessels=2, n_discs=2)),
    ("3d_lossy", lambda: synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=40)),
    ("3d_pow2_lossy", lambda: synth.small_lossy_3d(shape=(16, 16, 32), pml=3, Nt=36)),
    # 128-point z-lines: FP32 takes the 16-column z passes, whose absorption pass computes the windowed
    # multiplier inline
    ("3d_wide_z_lossy", lambda: synth.small_lossy_3d(shape=(128, 16, 32), pml=3, Nt=30)),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,make", TR_CASES, ids=[c[0] for c in TR_CASES])
def test_time_reversal_matches_oracle(dev, name, make, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = make()
    ref = Operator.from_problem(pb)
    data = ref.forward(pb.p0)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    for compensate, k_cut in ((True, 0.5), (False, 0.5), (True, 0.75)):
        img_ref = time_reversal(ref, data, compensate=compensate, k_cut=k_cut)
        img = op.time_reversal(_T(data, prec, dev), compensate=compensate, k_cut=k_cut).cpu().numpy()
        assert rel(img, img_ref) <= TOL[prec], (compensate, k_cut, rel(img, img_ref))
    # the solve leaves the plan's operators intact
    x = _T(pb.p0, prec, dev)
    assert rel(op.forward(x).cpu().numpy(), data) <= TOL[prec]


def test_time_reversal_edge_cases(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import PATOperator

    # Nt = 1: the image is the enforced first frame (zero elsewhere)
    pb = synth.vessel_phantom_2d(n=32, pml=4, Nt=1, n_vessels=1, n_discs=1)
    ref = Operator.from_problem(pb)
    data = np.random.default_rng(3).standard_normal((1, ref.Ns))
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    img = op.time_reversal(_T(data, "f64", dev)).cpu().numpy()
    assert np.array_equal(img, time_reversal(ref, data))
    # every node a sensor: the image is the t = 0 datum exactly (reading T3)
    n, h = 24, 1e-4
    pb_all = synth.small_lossy_2d(shape=(n, n), pml=3, Nt=10)
    op_all = PATOperator((n, n), (h, h), (3, 3), 2.0, pb_all.c, pb_all.rho, pb_all.alpha0, pb_all.y, pb_all.dt, 10,
                         sensor_index=np.arange(n * n), precision="f64", device=dev)
    d_all = np.random.default_rng(4).standard_normal((10, n * n))
    assert np.array_equal(op_all.time_reversal(_T(d_all, "f64", dev)).cpu().numpy().ravel(), d_all[0])
    # off-grid sensors are rejected (reading T2)
    pb_off = synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=20, n_sensors=8)
    op_off = PATOperator.from_problem(pb_off, precision="f64", device=dev)
    with pytest.raises(_lib.PatError):
        op_off.time_reversal(_T(np.zeros((20, op_off.Ns)), "f64", dev))
    with pytest.raises(_lib.PatError):   # k_cut outside (0, 1]
        op.time_reversal(_T(data, "f64", dev), k_cut=1.5)


ATD_CASES = [
    ("2d_generic_lossy", lambda: synth.small_lossy_2d(shape=(32, 36), pml=5, Nt=41, n_sensors=10)),
    ("2d_generic_lossless", lambda: synth.small_lossy_2d(shape=(32, 36), pml=5, Nt=41, n_sensors=10, alpha0=0.0)),
    ("2d_pow2_lossy", lambda: synth.small_lossy_2d(shape=(48, 64), pml=6, Nt=60, n_sensors=16)),
    ("2d_pow2_lossless", lambda: synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=33, n_sensors=12, alpha0=0.0)),
    ("3d_lossy", lambda: synth.small_lossy_3d(shape=(12, 16, 20), pml=3, Nt=21)),
    ("3d_pow2_lossy", lambda: synth.small_lossy_3d(shape=(16, 16, 16), pml=3, Nt=25)),
    ("3d_wide_z_lossy", lambda: synth.small_lossy_3d(shape=(128, 16, 32), pml=3, Nt=21)),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name,make", ATD_CASES, ids=[c[0] for c in ATD_CASES])
def test_adjoint_then_discretize_matches_oracle(dev, name, make, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = make()
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(21).standard_normal((pb.Nt, ref.Ns))
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    for initial in ("R5", "paper"):
        g_ref = adjoint_then_discretize(ref, h, initial=initial)
        g = op.adjoint_atd(_T(h, prec, dev), initial=initial).cpu().numpy()
        assert rel(g, g_ref) <= TOL[prec], (initial, rel(g, g_ref))
    # it is not the transpose: dt H^T h differs (by O(dt) and inside the PML, reading A3-A4)
    gt = op.adjoint(_T(h, prec, dev)).cpu().numpy() * pb.dt
    assert rel(gt, g_ref) > 1e-4


def test_adjoint_then_discretize_with_smoothing(dev):
    from paper_1603_02329_gb300.api import PATOperator

    pb = synth.small_lossy_2d(shape=(32, 64), pml=6, Nt=40, n_sensors=12)
    pb.smooth = True
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(22).standard_normal((pb.Nt, ref.Ns))
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    op.set_smoothing(True)
    g = op.adjoint_atd(_T(h, "f64", dev)).cpu().numpy()
    assert rel(g, adjoint_then_discretize(ref, h)) <= 1e-11


def test_time_reversal_and_atd_on_the_512_workload(dev):
    # the 2-D 512^2 absorbing workload at full size (Nt = 2000, 512 line sensors on the first row inside
    # the PML), FP32, against the oracle: the compensated time-reversal image of the noise-free data,
    # and the adjoint-then-discretize image of that data as the residual (about 35 s of oracle per solve)
    from paper_1603_02329_gb300.api import PATOperator

    pb = synth.vessel_phantom_2d()
    ref = Operator.from_problem(pb)
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    d_ref = ref.forward(pb.p0)           # the oracle's record is the input of both sides
    d = _T(d_ref, "f32", dev)
    img = op.time_reversal(d, compensate=True, k_cut=0.5).cpu().numpy()
    assert rel(img, time_reversal(ref, d_ref, compensate=True, k_cut=0.5)) <= 1e-5
    g = op.adjoint_atd(d).cpu().numpy()
    assert rel(g, adjoint_then_discretize(ref, d_ref)) <= 1e-5
