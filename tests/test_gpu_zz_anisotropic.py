"""GPU parity of H and H^T on anisotropic grids (different dx per axis) against the FP64 oracle,
through the C ABI.  Every per-axis table (wavenumbers, staggered shifts, PML profiles scaled by
c_ref / dx, sensor interpolation) then differs between axes, on each execution path: the
register-fused persistent kernel (power-of-two 2-D), the generic persistent kernel (other 2-D
sizes) and the per-phase graph (3-D).  Tolerances as elsewhere: 1e-5 relative L2 in FP32, 1e-11
in FP64."""
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


def _T(a, prec, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == "f64" else torch.float32, device=dev)


def _anisotropic(kind, factors):
    if kind == "3d":
        pb = synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=30)
    elif kind == "2d_pow2":
        pb = synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=100, n_sensors=24)
    else:
        pb = synth.small_lossy_2d(shape=(48, 40), pml=6, Nt=90, n_sensors=16)
    pb.spacing = tuple(h * f for h, f in zip(pb.spacing, factors))
    # the time step follows the finest spacing (CFL 0.3 on the smallest dx)
    pb.dt = 0.3 * min(pb.spacing) / float(np.max(pb.c))
    return pb


CASES = [
    ("2d_pow2_persistent", "2d_pow2", (1.0, 1.5)),
    ("2d_ragged_persistent", "2d_ragged", (1.25, 1.0)),
    ("3d_graph", "3d", (1.0, 1.25, 1.5)),
]


@pytest.mark.parametrize("name,kind,factors", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_anisotropic_grid_matches_oracle(dev, name, kind, factors, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _anisotropic(kind, factors)
    ref = Operator.from_problem(pb)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    tol = 1e-11 if prec == "f64" else 1e-5
    h = np.random.default_rng(41).standard_normal((pb.Nt, ref.Ns))
    assert rel(op.forward(_T(pb.p0, prec, dev)).cpu().numpy(), ref.forward(pb.p0)) <= tol
    assert rel(op.adjoint(_T(h, prec, dev)).cpu().numpy(), ref.adjoint(h)) <= tol
