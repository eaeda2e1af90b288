"""GPU parity of the optional p0 smoothing S (Sec. VI.A; the oracle's reading R9) against the FP64
oracle, through the C ABI: S alone on 2-D and 3-D grids of power-of-two and mixed-radix sizes,
H S and S H^T on both 2-D paths and the 3-D path, the coarse level, the checkpointed gradient and
a batch.  Tolerances as for the unsmoothed operator: 1e-5 relative L2 in FP32, 1e-11 in FP64.
S alone is a handful of transforms: its error is bounded relative to the input, ||S x - ref|| <=
1e-6 ||x|| in FP32 and 1e-13 ||x|| in FP64 (relative to ||S x||, which the window shrinks to a
fraction of ||x|| for white noise, the FP32 error would read several times larger)."""
import numpy as np
import pytest
import torch

from oracle import pat_medium as pm
from oracle import pat_optim as po
from oracle.pat_oracle import Operator, smooth_image
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


def _smooth_problem(kind, **kw):
    pb = synth.small_lossy_3d(**kw) if kind == "3d" else synth.small_lossy_2d(**kw)
    pb.smooth = True
    return pb


S_CASES = [
    ("2d_64x64", "2d", dict(shape=(64, 64), pml=8, Nt=4, n_sensors=8)),
    ("2d_30x42_anisotropic", "2d", dict(shape=(30, 42), pml=5, Nt=4, n_sensors=8)),
    ("2d_512x512", "2d", dict(shape=(512, 512), pml=20, Nt=2, n_sensors=8)),
    ("3d_24x32x40", "3d", dict(shape=(24, 32, 40), pml=4, Nt=4)),
    ("3d_16x20x28", "3d", dict(shape=(16, 20, 28), pml=3, Nt=4)),
]


@pytest.mark.parametrize("name,kind,kw", S_CASES, ids=[c[0] for c in S_CASES])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smoothing_alone_matches_oracle(dev, name, kind, kw, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _smooth_problem(kind, **kw)
    if name == "2d_30x42_anisotropic":
        pb.spacing = (pb.spacing[0], 1.5 * pb.spacing[1])
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    x = np.random.default_rng(21).standard_normal(pb.shape)
    ref = smooth_image(x, pb.spacing)
    tol = 1e-13 if prec == "f64" else 1e-6
    y = op.smooth(_T(x, prec, dev)).cpu().numpy()
    assert np.linalg.norm(y - ref) <= tol * np.linalg.norm(x)
    # in place
    xt = _T(x, prec, dev)
    op.smooth(xt, out=xt)
    assert np.linalg.norm(xt.cpu().numpy() - ref) <= tol * np.linalg.norm(x)
    # W(0) = 1: a constant field is returned unchanged
    one = torch.ones(pb.shape, dtype=xt.dtype, device=dev)
    assert torch.max(torch.abs(op.smooth(one) - 1)).item() <= 2 * tol


H_CASES = [
    # 2-D power of two: the register-fused persistent kernel; 2-D ragged: the generic persistent
    # kernel; 3-D: the CUDA graph of per-phase kernels
    ("2d_pow2_persistent", "2d", dict(shape=(64, 64), pml=8, Nt=120, n_sensors=24)),
    ("2d_ragged", "2d", dict(shape=(48, 40), pml=6, Nt=100, n_sensors=16)),
    ("3d", "3d", dict(shape=(16, 20, 24), pml=3, Nt=30)),
]


@pytest.mark.parametrize("name,kind,kw", H_CASES, ids=[c[0] for c in H_CASES])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smoothed_forward_and_adjoint_match_oracle(dev, name, kind, kw, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _smooth_problem(kind, **kw)
    ref = Operator.from_problem(pb)
    assert ref.smooth
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    assert op.smoothing
    tol = 1e-11 if prec == "f64" else 1e-5
    h = np.random.default_rng(22).standard_normal((pb.Nt, ref.Ns))
    d = op.forward(_T(pb.p0, prec, dev)).cpu().numpy()
    g = op.adjoint(_T(h, prec, dev)).cpu().numpy()
    assert rel(d, ref.forward(pb.p0)) <= tol
    assert rel(g, ref.adjoint(h)) <= tol
    # the switch: off gives the plain operator, on again the smoothed one
    op.set_smoothing(False)
    pb_plain = synth.small_lossy_3d(**kw) if kind == "3d" else synth.small_lossy_2d(**kw)
    assert rel(op.forward(_T(pb.p0, prec, dev)).cpu().numpy(), Operator.from_problem(pb_plain).forward(pb.p0)) <= tol
    op.set_smoothing(True)
    assert rel(op.forward(_T(pb.p0, prec, dev)).cpu().numpy(), d) <= tol


def test_coarse_level_inherits_smoothing(dev):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _smooth_problem("2d", shape=(64, 64), pml=8, Nt=60, n_sensors=24)
    ref_c, _ = po.coarse_operator(pb)
    assert ref_c.smooth
    opc = PATOperator.from_problem(pb, precision="f64", device=dev).coarse()
    assert opc.smoothing
    x = np.random.default_rng(23).standard_normal(ref_c.shape)
    assert rel(opc.forward(_T(x, "f64", dev)).cpu().numpy(), ref_c.forward(x)) <= 1e-11
    h = np.random.default_rng(24).standard_normal((ref_c.Nt, ref_c.Ns))
    assert rel(opc.adjoint(_T(h, "f64", dev)).cpu().numpy(), ref_c.adjoint(h)) <= 1e-11


@pytest.mark.parametrize("kind,prec", [("2d", "f64"), ("3d", "f32")])
def test_checkpointed_gradient_with_smoothing(dev, kind, prec):
    from paper_1603_02329_gb300.api import PATOperator

    if kind == "2d":
        pb = _smooth_problem("2d", shape=(40, 48), pml=6, Nt=41, n_sensors=16)
    else:
        pb = _smooth_problem("3d", shape=(16, 16, 16), pml=3, Nt=25)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(25).standard_normal((pb.Nt, ref.Ns))
    g_ref, gp_ref = pm.sound_speed_gradient(ref, pb.p0, h, pb.y)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    g, gp = op.gradient_c2(_T(pb.p0, prec, dev), _T(h, prec, dev), checkpoint_every=7, with_p0_grad=True)
    tol = 1e-10 if prec == "f64" else 1e-5
    assert rel(g.cpu().numpy(), g_ref) <= tol
    assert rel(gp.cpu().numpy(), gp_ref) <= tol


def test_batch_with_a_smoothing_instance(dev):
    from paper_1603_02329_gb300.api import PATBatch, PATOperator

    pbs = [synth.small_lossy_2d(seed=60, shape=(48, 40), pml=5, Nt=50, n_sensors=10),
           synth.small_lossy_2d(seed=61, shape=(64, 64), pml=5, Nt=60, n_sensors=12)]
    pbs[1].smooth = True
    ops = [PATOperator.from_problem(pb, precision="f64", device=dev) for pb in pbs]
    batch = PATBatch(ops)
    rng = np.random.default_rng(26)
    xs = [_T(pb.p0, "f64", dev) for pb in pbs]
    hs = [_T(rng.standard_normal((pb.Nt, op.Ns)), "f64", dev) for pb, op in zip(pbs, ops)]
    ds = batch.forward(xs)
    gs = batch.adjoint(hs)
    for pb, h, d, g in zip(pbs, hs, ds, gs):
        ref = Operator.from_problem(pb)
        assert rel(d.cpu().numpy(), ref.forward(pb.p0)) <= 1e-11
        assert rel(g.cpu().numpy(), ref.adjoint(h.cpu().numpy())) <= 1e-11
    batch.close()


def test_smoothing_argument_checks(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import PATOperator

    pb = synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=10, n_sensors=8)
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    L = _lib.lib()
    assert L.pat_plan_set_smoothing(op._plan, 2) != 0
    assert L.pat_plan_set_smoothing(None, 1) != 0
    assert L.pat_plan_smooth(op._plan, None, None, None) != 0
