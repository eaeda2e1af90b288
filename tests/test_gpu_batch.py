"""Several independent instances of uneven size in one launch (pat_batch_*): the results equal
each plan's own calls and the oracle; the batched autograd form gives the oracle gradients.  One
instance is a power-of-two grid whose own calls take the persistent kernel: in a batch it runs
the per-phase kernels, and both agree with the oracle."""
import numpy as np
import pytest
import torch

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


def _problems():
    return [synth.small_lossy_2d(seed=50 + i, shape=s, pml=5, Nt=nt, n_sensors=ns, alpha0=a)
            for i, (s, nt, ns, a) in enumerate([((48, 40), 70, 12, 0.75), ((64, 64), 90, 20, 0.75),
                                                  ((36, 56), 60, 10, 0.0), ((40, 40), 50, 8, 0.75)])]


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_batch_matches_plans_and_oracle(dev, prec, tol):
    from paper_1603_02329_gb300.api import PATBatch, PATOperator

    dt = torch.float64 if prec == "f64" else torch.float32
    pbs = _problems()
    ops = [PATOperator.from_problem(pb, precision=prec, device=dev) for pb in pbs]
    assert any(op.info.path == 2 for op in ops)   # the 64^2 instance runs persistent on its own
    batch = PATBatch(ops)
    rng = np.random.default_rng(5)
    xs = [torch.tensor(pb.p0, dtype=dt, device=dev) for pb in pbs]
    hs = [torch.tensor(rng.standard_normal((pb.Nt, op.Ns)), dtype=dt, device=dev) for pb, op in zip(pbs, ops)]
    for rep in range(2):    # the second launch reuses the instantiated graphs
        ds = batch.forward(xs)
        gs = batch.adjoint(hs)
        for pb, op, x, h, d, g in zip(pbs, ops, xs, hs, ds, gs):
            ref = Operator.from_problem(pb)
            assert rel(d.cpu().numpy(), ref.forward(pb.p0)) <= tol
            assert rel(g.cpu().numpy(), ref.adjoint(h.cpu().numpy())) <= tol
            assert rel(d.cpu().numpy(), op.forward(x).cpu().numpy()) <= tol
            assert rel(g.cpu().numpy(), op.adjoint(h).cpu().numpy()) <= tol
    batch.close()


def test_batched_autograd_in_one_launch(dev):
    from paper_1603_02329_gb300.api import PATBatch, PATOperator
    from paper_1603_02329_gb300.autograd import pat_apply_batch

    pbs = _problems()
    ops = [PATOperator.from_problem(pb, precision="f64", device=dev) for pb in pbs]
    batch = PATBatch(ops)
    xs = [torch.tensor(pb.p0, dtype=torch.float64, device=dev, requires_grad=True) for pb in pbs]
    outs = pat_apply_batch(ops, xs, batch=batch)
    loss = sum(0.5 * torch.sum(o * o) for o in outs)
    loss.backward()
    for pb, x in zip(pbs, xs):
        ref = Operator.from_problem(pb)
        assert rel(x.grad.cpu().numpy(), ref.adjoint(ref.forward(pb.p0))) <= 1e-11
    batch.close()


def test_batch_argument_checks(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import PATBatch, PATOperator

    pb = _problems()[0]
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    with pytest.raises(_lib.PatError):
        PATBatch([op, op])            # the same plan twice
