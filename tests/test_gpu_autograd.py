"""The autograd binding: the gradient of the data misfit f(p0) = 1/2 ||H p0 - p_hat||^2 through
torch.autograd equals the oracle gradient H^T (H p0 - p_hat) and central finite differences
(exact for a quadratic) on random directions; the batched form handles uneven instances."""
import numpy as np
import pytest
import torch

from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    from paper_1603_02329_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


# f is quadratic, so central differences are exact for any step; the FD tolerance only covers the
# rounding of f: ~1e-16 relative in FP64, ~1e-7 relative (amplified by 1/eps) in FP32.
@pytest.mark.parametrize("prec,tol_fd,tol_or", [("f64", 1e-9, 1e-11), ("f32", 2e-3, 1e-5)])
def test_autograd_gradient_3d_fd_16_directions(dev, prec, tol_fd, tol_or):
    from paper_1603_02329_gb300.api import PATOperator
    from paper_1603_02329_gb300.autograd import pat_apply

    dt = torch.float64 if prec == "f64" else torch.float32
    pb = synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=40)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    ref = Operator.from_problem(pb)
    rng = np.random.default_rng(21)
    phat = rng.standard_normal((pb.Nt, op.Ns))
    x = rng.standard_normal(pb.shape)
    xt = torch.tensor(x, dtype=dt, device=dev, requires_grad=True)
    ph = torch.tensor(phat, dtype=dt, device=dev)
    f = 0.5 * torch.sum((pat_apply(op, xt) - ph).double() ** 2)
    f.backward()
    g = xt.grad.double().cpu().numpy()
    g_ref = ref.gradient(x, phat)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= tol_or

    def fval(v):
        with torch.no_grad():
            d = op.forward(torch.tensor(v, dtype=dt, device=dev)).double() - ph.double()
            return 0.5 * float(torch.sum(d * d))

    for k in range(16):
        v = rng.standard_normal(pb.shape)
        eps = np.linalg.norm(x) / np.linalg.norm(v)
        fd = (fval(x + eps * v) - fval(x - eps * v)) / (2 * eps)
        scale = max(abs(fd), 1e-2 * np.linalg.norm(g) * np.linalg.norm(v))
        assert abs(fd - float(np.sum(g * v))) <= tol_fd * scale


def test_batched_uneven_instances(dev):
    from paper_1603_02329_gb300.api import PATOperator
    from paper_1603_02329_gb300.autograd import pat_apply_batch

    pbs = [synth.small_lossy_2d(seed=40 + i, shape=s, pml=6, Nt=50, n_sensors=16)
           for i, s in enumerate([(48, 48), (64, 56), (40, 72)])]
    ops = [PATOperator.from_problem(pb, precision="f64", device=dev) for pb in pbs]
    xs = [torch.tensor(pb.p0, dtype=torch.float64, device=dev, requires_grad=True) for pb in pbs]
    outs = pat_apply_batch(ops, xs)
    loss = sum(0.5 * torch.sum(o * o) for o in outs)
    loss.backward()
    for pb, x in zip(pbs, xs):
        ref = Operator.from_problem(pb)
        d = ref.forward(pb.p0)
        g_ref = ref.adjoint(d)
        g = x.grad.cpu().numpy()
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-11


def test_autograd_p0_gradient_on_the_128_workload(dev):
    # The 128^3 absorbing workload (Nt = 1000, 64 x 64 planar sensors, FP32): the gradient of the
    # data misfit through torch.autograd against central differences on 16 random directions (f is
    # quadratic: exact up to the rounding of f), and, for a misfit over the first K = 40 samples,
    # against the oracle gradient H^T r of that prefix.
    from paper_1603_02329_gb300.api import PATOperator
    from paper_1603_02329_gb300.autograd import pat_apply

    pb = synth.tube_phantom_3d(seed=3, n=128, pml=10, Nt=1000, sensors=64)
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    rng = np.random.default_rng(22)
    phat = torch.tensor(rng.standard_normal((pb.Nt, op.Ns)) * 0.1, dtype=torch.float32, device=dev)
    x = 0.5 * pb.p0
    xt = torch.tensor(x, dtype=torch.float32, device=dev, requires_grad=True)
    f = 0.5 * torch.sum((pat_apply(op, xt) - phat).double() ** 2)
    f.backward()
    g = xt.grad.double().cpu().numpy()

    def fval(v):
        with torch.no_grad():
            d = op.forward(torch.tensor(v, dtype=torch.float32, device=dev)).double() - phat.double()
            return 0.5 * float(torch.sum(d * d))

    for k in range(16):
        v = rng.standard_normal(pb.shape)
        eps = np.linalg.norm(x) / np.linalg.norm(v)
        fd = (fval(x + eps * v) - fval(x - eps * v)) / (2 * eps)
        scale = max(abs(fd), 1e-2 * np.linalg.norm(g) * np.linalg.norm(v))
        assert abs(fd - float(np.sum(g * v))) <= 2e-3 * scale, k
    K = 40
    xt.grad = None
    fK = 0.5 * torch.sum((pat_apply(op, xt)[:K] - phat[:K]).double() ** 2)
    fK.backward()
    ref = Operator.from_problem(pb, Nt=K)
    g_ref = ref.gradient(x, phat[:K].double().cpu().numpy())
    gK = xt.grad.double().cpu().numpy()
    assert np.linalg.norm(gK - g_ref) / np.linalg.norm(g_ref) <= 1e-5


def _perturbed_op(pb, c2, rho, dev, prec="f64"):
    from paper_1603_02329_gb300.api import PATOperator

    return PATOperator(pb.shape, pb.spacing, pb.pml, pb.pml_alpha, np.sqrt(c2), rho, pb.alpha0, pb.y, pb.dt, pb.Nt,
                       sensor_pos=pb.sensor_pos, sensor_index=pb.sensor_index, precision=prec, device=dev)


def test_autograd_medium_gradients_match_finite_differences(dev):
    # J = <H(c0^2, rho0) p0, h> through PATMediumFunction: d/dc0^2, d/drho0 and d/dp0 against central
    # differences of J with plans rebuilt for the perturbed medium (FP64, 3-D absorbing).  The
    # reference speed c_ref = max c0 (kappa, PML, dt) is held fixed as readings M1 / D1 state: the
    # c0^2 directions vanish within 3 points of the maximum of c0.
    from paper_1603_02329_gb300.autograd import pat_apply_medium

    pb = synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=30)
    c2 = pb.c ** 2
    op = _perturbed_op(pb, c2, pb.rho, dev)
    rng = np.random.default_rng(23)
    h = torch.tensor(rng.standard_normal((pb.Nt, op.Ns)), dtype=torch.float64, device=dev)
    p0 = torch.tensor(pb.p0, dtype=torch.float64, device=dev, requires_grad=True)
    c2t = torch.tensor(c2, dtype=torch.float64, device=dev, requires_grad=True)
    rt = torch.tensor(pb.rho, dtype=torch.float64, device=dev, requires_grad=True)
    J = torch.sum(pat_apply_medium(op, p0, c2t, rt, checkpoint_every=7) * h)
    J.backward()
    gc, gr, gp = c2t.grad.cpu().numpy(), rt.grad.cpu().numpy(), p0.grad.cpu().numpy()
    assert np.abs(gc).max() > 0 and np.abs(gr).max() > 0

    def Jof(c2v, rv):
        o = _perturbed_op(pb, c2v, rv, dev)
        out = float(torch.sum(o.forward(torch.tensor(pb.p0, dtype=torch.float64, device=dev)) * h))
        o.close()
        return out

    imax = np.unravel_index(np.argmax(pb.c), pb.shape)
    near = np.ones(pb.shape, bool)
    near[tuple(slice(max(i - 3, 0), i + 4) for i in imax)] = False
    for k in range(4):
        v = rng.standard_normal(pb.shape) * near
        eps = 1e-5 * c2.max() / np.abs(v).max()
        fd = (Jof(c2 + eps * v, pb.rho) - Jof(c2 - eps * v, pb.rho)) / (2 * eps)
        assert abs(fd - float(np.sum(gc * v))) <= 1e-6 * np.sum(np.abs(gc * v)), ("c2", k)
        w = rng.standard_normal(pb.shape)
        eps = 1e-5 * pb.rho.max() / np.abs(w).max()
        fd = (Jof(c2, pb.rho + eps * w) - Jof(c2, pb.rho - eps * w)) / (2 * eps)
        assert abs(fd - float(np.sum(gr * w))) <= 1e-6 * np.sum(np.abs(gr * w)), ("rho", k)
    # J is linear in p0: the p0 gradient is H^T h
    assert np.linalg.norm(gp - op.adjoint(h).cpu().numpy()) <= 1e-12 * np.linalg.norm(gp)


def test_autograd_medium_gradients_on_the_128_grid_match_oracle(dev):
    # the 128^3 workload's grid and medium on a short time axis (Nt = 12), FP32: the c0^2 and rho0
    # gradients through PATMediumFunction against the oracle's, and the sweep's device memory
    from oracle import pat_medium as pm
    from paper_1603_02329_gb300.api import PATOperator
    from paper_1603_02329_gb300.autograd import checkpoint_bytes, pat_apply_medium

    pb = synth.tube_phantom_3d(seed=3, n=128, pml=10, Nt=12, sensors=64)
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    rng = np.random.default_rng(24)
    h = rng.standard_normal((pb.Nt, op.Ns))
    p0 = torch.tensor(pb.p0, dtype=torch.float32, device=dev)
    c2t = torch.tensor(pb.c ** 2, dtype=torch.float32, device=dev, requires_grad=True)
    rt = torch.tensor(pb.rho, dtype=torch.float32, device=dev, requires_grad=True)
    torch.cuda.reset_peak_memory_stats(dev)
    J = torch.sum(pat_apply_medium(op, p0, c2t, rt, checkpoint_every=5).double() *
                  torch.tensor(h, dtype=torch.float64, device=dev))
    J.backward()
    ref = Operator.from_problem(pb)
    gc_ref, _ = pm.sound_speed_gradient(ref, pb.p0, h, pb.y)
    gr_ref = pm.density_gradient(ref, pb.p0, h)
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(c2t.grad.double().cpu().numpy(), gc_ref) <= 1e-5
    assert rel(rt.grad.double().cpu().numpy(), gr_ref) <= 1e-5
    mb = checkpoint_bytes(op, 5) / 2**20
    print(f"128^3, Nt = 12, K = 5: the checkpointed sweep allocates {mb:.0f} MiB")
    assert mb > 0
