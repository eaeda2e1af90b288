"""GPU parity of the optimisation shell (TV prox, smoothed TV, transfer operators, restricted
bound, FP64 reductions, power method, coarse level, ISTA / FISTA / MG-FISTA) against the FP64
oracle, through the C ABI.  FP64 plans are compared tightly, FP32 within its rounding."""
import numpy as np
import pytest
import torch

from oracle import pat_optim as po
from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def dev():
    from paper_1603_02329_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def T(a, dev, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)


@pytest.mark.parametrize("shape", [(20, 24), (8, 10, 12)])
def test_tv_prox_and_tv_values(dev, shape):
    from paper_1603_02329_gb300 import api

    rng = np.random.default_rng(1)
    z = rng.standard_normal(shape) + 0.3
    for lam, nin in ((0.2, 20), (0.05, 7), (0.0, 20)):
        ref = po.tv_prox(z, lam, nin, nonneg=True)
        out = api.tv_prox(T(z, dev), lam, nin, nonneg=True).cpu().numpy()
        assert rel(out, ref) <= 1e-12
        out32 = api.tv_prox(T(z, dev, torch.float32), lam, nin).cpu().numpy()
        assert rel(out32, ref) <= 2e-6
    ref_free = po.tv_prox(z, 0.15, 20, nonneg=False)
    assert rel(api.tv_prox(T(z, dev), 0.15, 20, nonneg=False).cpu().numpy(), ref_free) <= 1e-12
    assert abs(api.tv(T(z, dev)) - po.tv(z)) <= 1e-12 * po.tv(z)
    assert abs(api.tv(T(z, dev), rho=0.03) - po.tv_smooth(z, 0.03)) <= 1e-12 * po.tv_smooth(z, 0.03)
    g = api.tv_smooth_grad(T(z, dev), 0.03).cpu().numpy()
    assert rel(g, po.tv_smooth_grad(z, 0.03)) <= 1e-12


@pytest.mark.parametrize("shape_c", [(6, 10), (4, 6, 8)])
def test_transfer_and_bound(dev, shape_c):
    from paper_1603_02329_gb300 import api

    rng = np.random.default_rng(2)
    shape_f = tuple(2 * n for n in shape_c)
    xf = rng.standard_normal(shape_f)
    xc = rng.standard_normal(shape_c)
    assert rel(api.restrict(T(xf, dev)).cpu().numpy(), po.restrict(xf)) <= 1e-14
    assert rel(api.prolong(T(xc, dev)).cpu().numpy(), po.prolong(xc)) <= 1e-14
    assert rel(api.coarse_bound(T(xf, dev)).cpu().numpy(), po.coarse_lower_bound(xf)) <= 1e-14
    a, b = rng.standard_normal(1000), rng.standard_normal(1000)
    assert abs(api.dot(T(a, dev), T(b, dev)) - float(a @ b)) <= 1e-12 * np.abs(a) @ np.abs(b)


def _small(prec="f64", shape=(32, 32), Nt=40):
    pb = synth.small_lossy_2d(shape=shape, pml=4, Nt=Nt, n_sensors=24, sensor_radius_frac=0.3)
    return pb


def test_power_iteration_and_coarse_level(dev):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _small()
    ref = Operator.from_problem(pb)
    op = PATOperator.from_problem(pb, precision="f64", device=dev)
    v0 = np.random.default_rng(1).standard_normal(pb.shape)
    L_ref = po.power_iteration(lambda v: ref.adjoint(ref.forward(v)), pb.shape, n_iter=15, seed=1)
    assert abs(op.power_iteration(T(v0, dev), 15) / L_ref - 1) <= 1e-12
    # coarse level: same operator as the oracle's coarse level
    ref_c, Ntc = po.coarse_operator(pb)
    opc = op.coarse()
    assert opc.shape == ref_c.shape and opc.Nt == Ntc and opc.Ns == ref_c.Ns
    xc = np.random.default_rng(3).standard_normal(ref_c.shape)
    assert rel(opc.forward(T(xc, dev)).cpu().numpy(), ref_c.forward(xc)) <= 1e-11


def _mg_setup(dev, prec):
    from paper_1603_02329_gb300.api import PATOperator

    pb = _small()
    ref = Operator.from_problem(pb)
    phat = ref.forward(pb.p0)
    L = po.power_iteration(lambda v: ref.adjoint(ref.forward(v)), pb.shape, n_iter=15, seed=1)
    ref_c, Ntc = po.coarse_operator(pb)
    Lc = po.power_iteration(lambda v: ref_c.adjoint(ref_c.forward(v)), ref_c.shape, n_iter=15, seed=2)
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    opc = op.coarse()
    return pb, ref, phat, L, (ref_c, phat[::2][:Ntc], Lc), op, opc


@pytest.mark.parametrize("variant,recursion,iters", [(0, False, 3), (1, False, 4), (1, True, 6)])
def test_mg_fista_matches_oracle_f64(dev, variant, recursion, iters):
    from paper_1603_02329_gb300.api import mg_fista

    pb, ref, phat, L, coarse, op, opc = _mg_setup(dev, "f64")
    kw = dict(variant=variant, step_scale=2.0 if variant == 0 else 1.0, max_iter=iters, eps_d=-1.0,
              recursion=recursion, kappa=0.25)
    oo = po.FistaOpts(variant=variant, step_scale=kw["step_scale"], max_iter=iters, eps_d=-1.0, recursion=recursion)
    x_ref, recs = po.mg_fista(ref, phat, np.zeros(pb.shape), L, oo, coarse=coarse if recursion else None,
                              p_exact=pb.p0)
    x, rep, grecs = mg_fista(op, opc if recursion else None, T(phat, dev), T(np.zeros(pb.shape), dev), L,
                             L_coarse=coarse[2], p_exact=T(pb.p0, dev), **kw)
    assert [r["branch"] for r in grecs] == [r.branch for r in recs]
    if recursion:
        assert any(r.branch == "recursive" for r in recs)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-9
    for a, b in zip(grecs, recs):
        assert abs(a["F"] - b.F) <= 1e-9 * abs(b.F)
        assert abs(a["RE"] - b.RE) <= 1e-9
    assert x.cpu().numpy().min() >= -1e-12


@pytest.mark.parametrize("recursion", [False, True])
def test_mg_fista_f32_iterates_match_oracle(dev, recursion):
    # FP32 fields with FP64 scalars: every iterate x_1 .. x_5 of FISTA and of two-level MG-FISTA within
    # 1e-5 relative L2 of the FP64 oracle's, with the same branch sequence
    from paper_1603_02329_gb300.api import mg_fista

    pb, ref, phat, L, coarse, op, opc = _mg_setup(dev, "f32")
    errs = []
    for k in range(1, 6):
        oo = po.FistaOpts(variant=1, max_iter=k, eps_d=-1.0, recursion=recursion)
        x_ref, recs = po.mg_fista(ref, phat, np.zeros(pb.shape), L, oo, coarse=coarse if recursion else None,
                                  p_exact=pb.p0)
        x, rep, grecs = mg_fista(op, opc if recursion else None, T(phat, dev, torch.float32),
                                 T(np.zeros(pb.shape), dev, torch.float32), L, L_coarse=coarse[2], max_iter=k,
                                 eps_d=-1.0, recursion=recursion, p_exact=T(pb.p0, dev, torch.float32))
        assert [r["branch"] for r in grecs] == [r.branch for r in recs]
        assert rep["iters"] == k
        errs.append(rel(x.cpu().numpy(), x_ref))
        for a, b in zip(grecs, recs):
            assert abs(a["F"] - b.F) <= 1e-5 * abs(b.F)
    print("FP32 iterate error vs FP64 oracle (recursion=%s):" % recursion, ["%.2e" % e for e in errs])
    if recursion:
        assert any(r.branch == "recursive" for r in recs)
    assert max(errs) <= 1e-5, errs


def test_mg_fista_unweighted_coarse_term_matches_oracle_f64(dev):
    # the coarse objective exactly as Eq. (Fourteen) prints it: data term weight 1 (coarse_weight = 1)
    # instead of reading O11's 2^(1-d)
    from paper_1603_02329_gb300.api import mg_fista

    pb, ref, phat, L, coarse, op, opc = _mg_setup(dev, "f64")
    oo = po.FistaOpts(variant=1, max_iter=6, eps_d=-1.0, coarse_weight=1.0, kappa=0.25)
    x_ref, recs = po.mg_fista(ref, phat, np.zeros(pb.shape), L, oo, coarse=coarse, p_exact=pb.p0)
    x, rep, grecs = mg_fista(op, opc, T(phat, dev), T(np.zeros(pb.shape), dev), L, L_coarse=coarse[2],
                             p_exact=T(pb.p0, dev), max_iter=6, eps_d=-1.0, coarse_weight=1.0, kappa=0.25)
    assert [r["branch"] for r in grecs] == [r.branch for r in recs]
    assert any(r.branch == "recursive" for r in recs)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-9
    for a, b in zip(grecs, recs):
        assert abs(a["F"] - b.F) <= 1e-9 * abs(b.F)
    # and it is a different run from the default weight's
    x_w, _, _ = mg_fista(op, opc, T(phat, dev), T(np.zeros(pb.shape), dev), L, L_coarse=coarse[2],
                         p_exact=T(pb.p0, dev), max_iter=6, eps_d=-1.0, kappa=0.25)
    assert rel(x_w.cpu().numpy(), x.cpu().numpy()) > 1e-6


@pytest.mark.parametrize("q_c", [8, 1])
def test_mg_fista_three_levels_match_oracle_f64(dev, q_c):
    # pat_mg_fista_levels on three levels (reading O12) against the oracle, iterate by iterate; with
    # q_c = 1 the middle level never recurses and the run equals the two-level one
    from paper_1603_02329_gb300.api import mg_fista

    pb, ref, phat, L, lev1, op, opc = _mg_setup(dev, "f64")
    p1 = po.coarse_problem(pb)
    ref2, Nt2 = po.coarse_operator(p1)
    L2 = po.power_iteration(lambda v: ref2.adjoint(ref2.forward(v)), ref2.shape, n_iter=15, seed=3)
    lev2 = (ref2, lev1[1][::2][:Nt2], L2)
    opc2 = opc.coarse()
    assert opc2.shape == ref2.shape and opc2.Nt == Nt2
    oo = po.FistaOpts(variant=1, max_iter=6, eps_d=-1.0, q_c=q_c, kappa=0.25)
    x_ref, recs = po.mg_fista(ref, phat, np.zeros(pb.shape), L, oo, coarse=[lev1, lev2], p_exact=pb.p0)
    x, rep, grecs = mg_fista(op, [opc, opc2], T(phat, dev), T(np.zeros(pb.shape), dev), L,
                             L_coarse=[lev1[2], L2], p_exact=T(pb.p0, dev), max_iter=6, eps_d=-1.0, q_c=q_c,
                             kappa=0.25)
    assert [r["branch"] for r in grecs] == [r.branch for r in recs]
    assert any(r.branch == "recursive" for r in recs)
    assert rel(x.cpu().numpy(), x_ref) <= 1e-9
    for a, b in zip(grecs, recs):
        assert abs(a["F"] - b.F) <= 1e-9 * abs(b.F)
    assert x.cpu().numpy().min() >= -1e-12
    if q_c == 1:
        x2, _, _ = mg_fista(op, opc, T(phat, dev), T(np.zeros(pb.shape), dev), L, L_coarse=lev1[2],
                            p_exact=T(pb.p0, dev), max_iter=6, eps_d=-1.0, q_c=1, kappa=0.25)
        assert torch.equal(x, x2)


def test_mg_fista_levels_argument_checks(dev):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import mg_fista

    pb, ref, phat, L, lev1, op, opc = _mg_setup(dev, "f64")
    with pytest.raises(Exception):   # a level that is not the coarse level of the one above
        mg_fista(op, [opc, opc], T(phat, dev), T(np.zeros(pb.shape), dev), L, L_coarse=[1.0, 1.0], max_iter=2)
    with pytest.raises(Exception):   # L of a level the recursion uses
        mg_fista(op, [opc, opc.coarse()], T(phat, dev), T(np.zeros(pb.shape), dev), L, L_coarse=[1.0, 0.0],
                 max_iter=2)
    assert _lib.lib().pat_mg_fista_levels(None, 0, None, None, None, None, None, None, _lib.ITER_CB(0), None,
                                          None) != 0


def test_coarse_plan_with_edge_line_sensors(dev):
    from paper_1603_02329_gb300.api import PATOperator

    pb = synth.vessel_phantom_2d(n=64, pml=8, Nt=40, n_vessels=2, n_discs=2)
    ref_c, Ntc = po.coarse_operator(pb)
    opc = PATOperator.from_problem(pb, precision="f64", device=dev).coarse()
    xc = np.random.default_rng(4).standard_normal(ref_c.shape)
    assert rel(opc.forward(T(xc, dev)).cpu().numpy(), ref_c.forward(xc)) <= 1e-11
