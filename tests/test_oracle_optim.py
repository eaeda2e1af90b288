"""Pins of the FP64 oracle's optimisation shell (TV, FGP prox, grid transfer, constraint
restriction, ISTA / FISTA / MG-FISTA, power method) against what the mathematics fixes."""
import json
import math
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import pat_optim as po
from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_tv_difference_operator_transpose():
    rng = np.random.default_rng(0)
    for shape in [(5, 7), (3, 4, 6)]:
        x = rng.standard_normal(shape)
        q = [rng.standard_normal(shape) for _ in shape]
        lhs = sum(np.sum(g * qa) for g, qa in zip(po.grad_fwd(x), q))
        rhs = np.sum(x * po.grad_fwd_T(q))
        assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
    # D of a constant is zero; TV of a step edge of height s across a full column is s * rows
    assert po.tv(np.full((4, 5), 3.0)) == 0.0
    img = np.zeros((4, 6))
    img[:, 3:] = 2.0
    assert abs(po.tv(img) - 2.0 * 4) < 1e-14


def test_tv_prox_special_cases():
    rng = np.random.default_rng(1)
    z = rng.standard_normal((6, 7))
    # lam' = 0 reduces to the projection on x >= 0
    assert np.array_equal(po.tv_prox(z, 0.0, 20), np.maximum(z, 0.0))
    # a constant non-negative image is a fixed point for every lam'
    cst = np.full((5, 6), 0.7)
    assert np.max(np.abs(po.tv_prox(cst, 0.3, 20) - cst)) < 1e-14
    # without the constraint, the prox keeps the mean (D^T q sums to zero)
    x = po.tv_prox(z, 0.2, 50, nonneg=False)
    assert abs(x.mean() - z.mean()) < 1e-12


@pytest.mark.parametrize("shape", [(4, 4), (3, 3, 3)])
def test_tv_prox_matches_direct_minimisation(shape):
    # FGP after many inner iterations: (i) the duality gap certificate -> 0, (ii) agreement with
    # a generic bound-constrained minimiser on a finely smoothed copy of the same objective.
    rng = np.random.default_rng(2)
    z = rng.standard_normal(shape) + 0.5
    lam = 0.15
    x, q = po.tv_prox(z, lam, 3000, nonneg=True, return_dual=True)
    gap = po.tv_prox_gap(z, lam, x, q)
    assert -1e-12 < gap < 1e-7

    eps = 1e-9

    def obj(v):
        v = v.reshape(shape)
        g = po.grad_fwd(v)
        nrm = np.sqrt(sum(ga * ga for ga in g) + eps * eps)
        val = 0.5 * np.sum((v - z) ** 2) + lam * np.sum(nrm)
        grad = (v - z) + lam * po.grad_fwd_T([ga / nrm for ga in g])
        return val, grad.ravel()

    res = minimize(obj, np.maximum(z, 0).ravel(), jac=True, method="L-BFGS-B",
                   bounds=[(0, None)] * z.size, options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12})
    assert np.max(np.abs(res.x.reshape(shape) - x)) < 5e-4
    f_fgp = 0.5 * np.sum((x - z) ** 2) + lam * po.tv(x)
    f_ref = 0.5 * np.sum((res.x.reshape(shape) - z) ** 2) + lam * po.tv(res.x.reshape(shape))
    assert f_fgp <= f_ref + 1e-8


def test_tv_prox_gap_detects_a_wrong_transpose():
    # the certificate is not vacuous: with D^T replaced by -D^T the iteration does not converge
    rng = np.random.default_rng(3)
    z = rng.standard_normal((4, 4))
    lam = 0.2
    x, q = po.tv_prox(z, lam, 500, return_dual=True)
    assert po.tv_prox_gap(z, lam, x, q) < 1e-6
    bad_x = np.maximum(z + lam * po.grad_fwd_T(q), 0)
    assert po.tv_prox_gap(z, lam, bad_x, q) > 1e-3


def test_smoothed_tv_gradient_and_limit():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((6, 5))
    rho = 0.05
    g = po.tv_smooth_grad(x, rho)
    v = rng.standard_normal(x.shape)
    e = 1e-6
    fd = (po.tv_smooth(x + e * v, rho) - po.tv_smooth(x - e * v, rho)) / (2 * e)
    assert abs(fd - np.sum(g * v)) < 1e-6 * (1 + abs(fd))
    assert abs(po.tv_smooth(x, 1e-12) - po.tv(x)) < 1e-9
    assert po.tv_smooth(np.ones((3, 3)), 0.1) == 0.0


def test_transfer_operators():
    rng = np.random.default_rng(5)
    for shape_c in [(5, 6), (3, 4, 5)]:
        d = len(shape_c)
        shape_f = tuple(2 * n for n in shape_c)
        xc = rng.standard_normal(shape_c)
        xf = rng.standard_normal(shape_f)
        # R = 2^-d P^T
        lhs = np.sum(po.restrict(xf) * xc)
        rhs = np.sum(xf * po.prolong(xc)) / 2**d
        assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
        # P reproduces constants and (away from the clamped last index) linear functions
        assert np.allclose(po.prolong(np.ones(shape_c)), 1.0)
        grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape_c], indexing="ij")
        lin = sum((a + 1.0) * g for a, g in enumerate(grids))
        pf = po.prolong(lin)
        gf = np.meshgrid(*[np.arange(n, dtype=float) / 2 for n in shape_f], indexing="ij")
        ref = sum((a + 1.0) * g for a, g in enumerate(gf))
        inner = tuple(slice(0, n - 1) for n in shape_f)
        assert np.max(np.abs(pf[inner] - ref[inner])) < 1e-12
        # full weighting keeps constants away from the boundary
        rc = po.restrict(np.ones(shape_f))
        inner_c = tuple(slice(1, n - 1) for n in shape_c)
        assert np.allclose(rc[inner_c], 1.0)


def test_coarse_bound_keeps_feasibility():
    # x = y + P(x_c - R y) >= 0 whenever x_c >= phi = R y - min_nbr(y)   (Sec. V.C)
    rng = np.random.default_rng(6)
    for shape in [(8, 10), (6, 4, 8)]:
        for _ in range(20):
            y = rng.standard_normal(shape)
            phi = po.coarse_lower_bound(y)
            xc = phi + np.abs(rng.standard_normal(phi.shape)) * rng.integers(0, 2, phi.shape)
            x = y + po.prolong(xc - po.restrict(y))
            assert x.min() >= -1e-12
        # and the bound is tight somewhere: at x_c = phi some fine value touches zero
        x = y + po.prolong(phi - po.restrict(y))
        assert x.min() >= -1e-12 and x.min() < 1e-12


def _tiny_problem():
    pb = synth.small_lossy_2d(shape=(16, 16), pml=3, Nt=24, n_sensors=10, sensor_radius_frac=0.3)
    return pb, Operator.from_problem(pb)


def test_power_iteration_matches_dense_eigenvalue():
    # Dense H (N forward solves) on a tiny grid: the power method's estimate lies below the
    # largest eigenvalue of H^T H and within the textbook convergence bound of it.
    pb, op = _tiny_problem()
    N = pb.N
    cols = [op.forward(np.eye(N)[i].reshape(pb.shape)).ravel() for i in range(N)]
    H = np.stack(cols, axis=1)
    w, V = np.linalg.eigh(H.T @ H)
    lmax, l2 = w[-1], w[-2]
    n_iter = 300
    L = po.power_iteration(lambda v: op.adjoint(op.forward(v)), pb.shape, n_iter=n_iter, seed=1)
    v0 = np.random.default_rng(1).standard_normal(pb.shape).ravel()
    c1 = abs(V[:, -1] @ v0) / np.linalg.norm(v0)
    # ||A^n v|| / ||A^(n-1) v|| >= lmax (1 - tan^2(angle) (l2/lmax)^(2n-2))
    bound = (1 - c1**2) / c1**2 * (l2 / lmax) ** (2 * n_iter - 2)
    assert L <= lmax * (1 + 1e-12)
    assert (lmax - L) / lmax <= bound + 1e-12
    assert abs(L / lmax - 1) < 1e-4


def _mg_setup():
    pb = synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=40, n_sensors=24, sensor_radius_frac=0.3)
    op = Operator.from_problem(pb)
    phat = op.forward(pb.p0)
    L = po.power_iteration(lambda v: op.adjoint(op.forward(v)), pb.shape, n_iter=15, seed=1)
    op_c, Nt_c = po.coarse_operator(pb)
    Lc = po.power_iteration(lambda v: op_c.adjoint(op_c.forward(v)), op_c.shape, n_iter=15, seed=2)
    return pb, op, phat, L, (op_c, phat[::2][:Nt_c], Lc)


def test_fista_theta_zero_is_ista_and_no_recursion_is_fista():
    pb, op, phat, L, coarse = _mg_setup()
    x0 = np.zeros(pb.shape)
    o_ista = po.FistaOpts(variant=0, step_scale=2.0, max_iter=3, eps_d=-1.0)
    xa, ra = po.mg_fista(op, phat, x0, L, o_ista, coarse=None, p_exact=pb.p0)
    # Alg. 1 written out directly
    x = x0.copy()
    for _ in range(3):
        g = op.adjoint(op.forward(x) - phat)
        x = po.tv_prox(x - (2.0 / L) * g, (2.0 / L) * o_ista.lam, o_ista.n_tv)
    assert np.max(np.abs(xa - x)) < 1e-12 * (1 + np.abs(x).max())
    # recursion disabled == plain FISTA, whatever the coarse level
    o_f = po.FistaOpts(variant=1, max_iter=4, eps_d=-1.0)
    x1, r1 = po.mg_fista(op, phat, x0, L, o_f, coarse=None)
    o_nr = po.FistaOpts(variant=1, max_iter=4, eps_d=-1.0, recursion=False)
    x2, r2 = po.mg_fista(op, phat, x0, L, o_nr, coarse=coarse)
    assert np.array_equal(x1, x2)
    assert all(r.branch == "direct" for r in r2)


def test_first_order_coherence():
    # grad phi_{h-1}(x_{h-1,0}) = R grad F_h(y)   (Sec. V.A, Eqs. (fourteen)-(Fourteen))
    pb, op, phat, L, (op_c, phat_c, Lc) = _mg_setup()
    rng = np.random.default_rng(7)
    y = np.abs(rng.standard_normal(pb.shape))
    lam, rho = 1e-2, 1e-2
    gF = op.adjoint(op.forward(y) - phat) + lam * po.tv_smooth_grad(y, rho)
    xc0 = po.restrict(y)
    gFc = op_c.adjoint(op_c.forward(xc0) - phat_c) + lam * po.tv_smooth_grad(xc0, rho)
    v = po.restrict(gF) - gFc
    gphi = op_c.adjoint(op_c.forward(xc0) - phat_c) + lam * po.tv_smooth_grad(xc0, rho) + v
    assert np.max(np.abs(gphi - po.restrict(gF))) < 1e-12 * np.abs(gF).max()


def test_mg_fista_runs_recursive_branch_and_stays_feasible():
    pb, op, phat, L, coarse = _mg_setup()
    opts = po.FistaOpts(variant=1, max_iter=6, eps_d=-1.0, kappa=0.25)
    xs = []
    x, recs = po.mg_fista(op, phat, np.zeros(pb.shape), L, opts, coarse=coarse, p_exact=pb.p0,
                          callback=lambda r: xs.append(r))
    assert recs[0].branch == "direct"
    assert any(r.branch == "recursive" for r in recs)
    assert x.min() >= -1e-12   # x = y + P(x_c - R y) >= 0 holds up to rounding
    # the objective comes down from F(x0)
    F0 = 0.5 * np.sum(phat**2)
    assert recs[-1].F < 0.5 * F0


def _mg3_setup():
    # three levels: 32^2 -> 16^2 -> 8^2 (O12)
    pb, op, phat, L, lev1 = _mg_setup()
    p1 = po.coarse_problem(pb)
    op2, Nt2 = po.coarse_operator(p1)
    L2 = po.power_iteration(lambda v: op2.adjoint(op2.forward(v)), op2.shape, n_iter=15, seed=3)
    lev2 = (op2, lev1[1][::2][:Nt2], L2)
    return pb, op, phat, L, lev1, lev2


def test_restricted_bound_keeps_a_nonzero_fine_bound():
    # O12: with b_c = R y - min_{neighbourhood}(y - b), every x_c >= b_c gives y + P(x_c - R y) >= b
    rng = np.random.default_rng(21)
    for shape in [(16, 12), (8, 6, 10)]:
        y = rng.standard_normal(shape)
        b = y - np.abs(rng.standard_normal(shape))          # y is feasible for b
        bc = po.coarse_lower_bound(y, b)
        xc = bc + np.abs(rng.standard_normal(bc.shape)) * rng.integers(0, 2, bc.shape)   # some active
        x = y + po.prolong(xc - po.restrict(y))
        assert (x - b).min() >= -1e-12
    # b = 0 is Eq. (constraint) as before
    y = np.abs(rng.standard_normal((12, 10)))
    assert np.array_equal(po.coarse_lower_bound(y, np.zeros_like(y)), po.coarse_lower_bound(y))


def test_second_level_first_order_coherence():
    # O12: grad phi_2(x_{2,0}) = R grad phi_1(y) for the coarse model phi_1 of a fine iterate
    pb, op, phat, L, (op1, p1, L1), (op2, p2, L2) = _mg3_setup()
    rng = np.random.default_rng(8)
    lam, rho, w1 = 1e-2, 1e-2, 0.5
    y = np.abs(rng.standard_normal(op1.shape))
    v1 = rng.standard_normal(op1.shape)
    g1 = w1 * op1.adjoint(op1.forward(y) - p1) + lam * po.tv_smooth_grad(y, rho) + v1
    x20 = po.restrict(y)
    w2 = w1 * 0.5
    v2 = po.restrict(g1) - (w2 * op2.adjoint(op2.forward(x20) - p2) + lam * po.tv_smooth_grad(x20, rho))
    g2 = w2 * op2.adjoint(op2.forward(x20) - p2) + lam * po.tv_smooth_grad(x20, rho) + v2
    assert np.max(np.abs(g2 - po.restrict(g1))) < 1e-12 * np.abs(g1).max()


def test_three_levels_reduce_to_two_with_one_coarse_iteration():
    # the level-1 solve recurses only from its second iteration on (O12), so with q_c = 1 the
    # three-level run is the two-level run, operation for operation
    pb, op, phat, L, lev1, lev2 = _mg3_setup()
    opts = po.FistaOpts(variant=1, max_iter=5, eps_d=-1.0, q_c=1)
    x2, r2 = po.mg_fista(op, phat, np.zeros(pb.shape), L, opts, coarse=lev1)
    x3, r3 = po.mg_fista(op, phat, np.zeros(pb.shape), L, opts, coarse=[lev1, lev2])
    assert any(r.branch == "recursive" for r in r2)
    assert np.array_equal(x2, x3)
    assert [r.F for r in r2] == [r.F for r in r3]


def test_three_levels_recurse_at_the_middle_level_and_stay_feasible():
    pb, op, phat, L, (op1, p1, L1), lev2 = _mg3_setup()
    rng = np.random.default_rng(9)
    lam, rho, w1 = 1e-2, 1e-2, 0.5
    y = np.abs(rng.standard_normal(pb.shape))
    x10 = po.restrict(y)
    g = op.adjoint(op.forward(y) - phat) + lam * po.tv_smooth_grad(y, rho)
    v1 = po.restrict(g) - (w1 * op1.adjoint(op1.forward(x10) - p1) + lam * po.tv_smooth_grad(x10, rho))
    b1 = po.coarse_lower_bound(y)
    L1c = w1 * L1 + lam * 8.0 / rho
    opts = po.FistaOpts(variant=1, q_c=8, eps_c=-1.0, kappa=0.25)
    xa, ka, _, _, nra = po.fista_coarse(op1, p1, x10, v1, b1, lam, rho, L1c, opts, w=w1)
    xb, kb, _, _, nrb = po.fista_coarse(op1, p1, x10, v1, b1, lam, rho, L1c, opts, w=w1, deeper=[lev2])
    assert nra == 0 and nrb >= 1 and ka == kb == 8
    assert (xb - b1).min() >= -1e-12

    def phi(x):
        r = op1.forward(x) - p1
        return 0.5 * w1 * np.sum(r * r) + lam * po.tv_smooth(x, rho) + np.sum(v1 * x)

    assert phi(xb) < phi(x10) and phi(xa) < phi(x10)


def test_paper_parameters_golden():
    # The algorithm parameters printed in Sec. VI.A / VI.B are the FistaOpts defaults (2-D).
    with open(os.path.join(GOLDEN, "paper_parameters.json")) as f:
        g = json.load(f)
    o = po.FistaOpts()
    assert o.lam == g["lambda"]["value"]
    assert o.kappa == g["kappa_2d"]["value"]
    assert o.vartheta == g["vartheta"]["value"]
    assert o.q_d == g["q_d"]["value"] and o.q_c == g["q_c"]["value"]
    assert o.eps_d == g["eps_d"]["value"] and o.eps_c == g["eps_c"]["value"]
    assert o.tv_rho == g["rho_tv_2d"]["value"]


def test_coarse_level_clamps_edge_sensors():
    # a line of on-grid sensors spanning the whole row: the one on the last fine column lies beyond
    # the last coarse node and is clamped onto it (weight 1), the even ones land on coarse nodes
    pb = synth.vessel_phantom_2d(n=32, pml=4, Nt=10, n_vessels=1, n_discs=1)
    op_c, Nt_c = po.coarse_operator(pb)
    M = op_c.M.toarray()
    assert np.allclose(M.sum(axis=1), 1.0)
    row = pb.pml[0] // 2
    last = row * 16 + 15
    assert M[31, last] == 1.0          # fine x = 31 -> clamped onto coarse x = 15
    assert M[30, last] == 1.0          # fine x = 30 -> coarse node 15
    assert M[29, last - 1] == 0.5 and M[29, last] == 0.5


def test_forward_operator_is_linear():
    # the cost-saving identity (O9) rests on H being linear, smoothing and absorption included
    pb = synth.small_lossy_2d(shape=(24, 28), pml=5, Nt=25, n_sensors=8)
    pb.smooth = True
    op = Operator.from_problem(pb)
    rng = np.random.default_rng(41)
    x, z = rng.standard_normal(pb.shape), rng.standard_normal(pb.shape)
    a, b = 1.7, -0.4
    lhs = op.forward(a * x + b * z)
    rhs = a * op.forward(x) + b * op.forward(z)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def test_data_space_momentum_equals_direct_forward():
    # O9: FISTA forms H y_{k+1} = (1 + theta_k) H x_k - theta_k H x_{k-1} in data space.  Record
    # what the solver hands to H and H^T, rebuild y_3 = x_2 + theta_2 (x_2 - x_1) with the
    # momentum of Beck and Teboulle's t-rule (t_1 = 1, t_2 = (1 + sqrt 5) / 2, theta_2 =
    # (t_2 - 1) / t_3 = 0.28175...), and compare the residual the solver used at iteration 3 with
    # a direct forward solve of y_3.
    pb, op, phat, L, _ = _mg_setup()

    class Recorder:
        def __init__(self, inner):
            self.inner, self.fwd_in, self.adj_in = inner, [], []

        def forward(self, x):
            self.fwd_in.append(np.array(x))
            return self.inner.forward(x)

        def adjoint(self, r):
            self.adj_in.append(np.array(r))
            return self.inner.adjoint(r)

    rec = Recorder(op)
    po.mg_fista(rec, phat, np.zeros(pb.shape), L, po.FistaOpts(variant=1, max_iter=4, eps_d=-1.0))
    x1, x2 = rec.fwd_in[1], rec.fwd_in[2]            # forward inputs: x_0, x_1, x_2, ...
    t2 = (1 + math.sqrt(5)) / 2
    t3 = (1 + math.sqrt(1 + 4 * t2 * t2)) / 2
    theta2 = (t2 - 1) / t3
    assert abs(theta2 - 0.2817529) < 1e-6
    y3 = x2 + theta2 * (x2 - x1)
    Hy3_used = rec.adj_in[2] + phat                  # adjoint inputs: H y_k - p_hat, k = 1, 2, 3
    Hy3 = op.forward(y3)
    assert np.max(np.abs(Hy3_used - Hy3)) <= 1e-12 * np.max(np.abs(Hy3))
    # iteration 2 has theta_1 = 0: y_2 = x_1 exactly
    assert np.max(np.abs(rec.adj_in[1] + phat - op.forward(x1))) <= 1e-12 * np.max(np.abs(Hy3))
