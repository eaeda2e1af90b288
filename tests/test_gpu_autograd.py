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
