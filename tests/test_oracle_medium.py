"""Pins of the oracle's medium gradients (oracle/pat_medium.py).  c0^2 (readings M1-M3): central
finite differences of J(c0^2) = <H p0, h> with the reference speed held fixed, on heterogeneous
media with PML (absorbing and lossless, 2-D and 3-D), and a closed form for a homogeneous lossless
periodic medium under a uniform perturbation.  rho0 (readings D1-D3): central finite differences
in 2-D and 3-D, and the scaling invariant <dJ/drho0, rho0> = 0."""
import numpy as np
import pytest

from oracle import pat_medium as pm
from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth


def _fd_check(pb, ndir, seed, tol):
    rng = np.random.default_rng(seed)
    op = Operator.from_problem(pb)
    h = rng.standard_normal((pb.Nt, op.Ns))
    g, gp0 = pm.sound_speed_gradient(op, pb.p0, h, pb.y)
    # the same sweep also gives the ordinary adjoint
    assert np.allclose(gp0, op.adjoint(h), rtol=0, atol=1e-12 * np.abs(gp0).max())
    c2 = np.asarray(pb.c, float) ** 2
    for _ in range(ndir):
        v = rng.standard_normal(pb.shape) * c2
        eps = 1e-5
        jp = pm.objective(pb, c2 + eps * v, h, op.c_ref)
        jm = pm.objective(pb, c2 - eps * v, h, op.c_ref)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * v))
        assert abs(fd - an) <= tol * max(abs(an), 1e-30), (fd, an)
    return g


@pytest.mark.parametrize("alpha0", [0.75, 0.0])
def test_c2_gradient_matches_central_differences_2d(alpha0):
    pb = synth.small_lossy_2d(shape=(20, 24), pml=4, Nt=36, n_sensors=10, alpha0=alpha0)
    _fd_check(pb, 4, 5, 1e-6)


def test_c2_gradient_matches_central_differences_3d():
    pb = synth.small_lossy_3d(shape=(8, 10, 12), pml=2, Nt=20)
    _fd_check(pb, 3, 6, 1e-6)


def test_c2_gradient_uniform_closed_form():
    # homogeneous lossless, no PML, periodic: <g, 1> = d/dc0^2 sum_n <h_n, M p^n> in closed form
    shape, h, c0 = (16, 20), (1e-4, 1e-4), 1500.0
    dt = 0.3 * h[0] / c0
    Nt = 30
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(shape)
    op = Operator(shape, h, (0, 0), 2.0, c0, 1000.0, 0.0, 1.5, dt, Nt,
                  sensor_index=np.arange(0, 16 * 20, 7, dtype=np.int64))
    hh = rng.standard_normal((Nt, op.Ns))
    g, _ = pm.sound_speed_gradient(op, p0, hh, 1.5)
    weights = np.stack([op.scatter(hh[n]) for n in range(Nt)])
    closed = pm.homogeneous_uniform_derivative(shape, h, c0, dt, Nt, p0, weights)
    # The whole discrete scheme (density initialised as p0/(2 c0^2), reading M3, included) has the
    # exact solution p^n = F^-1{cos(n w) F p0} here, so <g, 1> equals the closed form's derivative.
    assert abs(float(np.sum(g)) - closed) <= 1e-8 * abs(closed)


# ---- the density gradient (readings D1-D3) ----

def _rho_fd_check(pb, ndir, seed, tol):
    rng = np.random.default_rng(seed)
    op = Operator.from_problem(pb)
    h = rng.standard_normal((pb.Nt, op.Ns))
    g = pm.density_gradient(op, pb.p0, h)
    rho = np.broadcast_to(np.asarray(pb.rho, float), pb.shape).copy()
    for _ in range(ndir):
        v = rng.standard_normal(pb.shape) * rho * 1e-2
        eps = 1e-3
        fd = (pm.density_objective(pb, rho + eps * v, h) - pm.density_objective(pb, rho - eps * v, h)) / (2 * eps)
        an = float(np.sum(g * v))
        assert abs(fd - an) <= tol * max(abs(an), 1e-30), (fd, an)
    return g, rho


@pytest.mark.parametrize("alpha0", [0.75, 0.0])
def test_density_gradient_matches_central_differences_2d(alpha0):
    pb = synth.small_lossy_2d(shape=(20, 24), pml=4, Nt=36, n_sensors=10, alpha0=alpha0)
    _rho_fd_check(pb, 4, 7, 1e-6)


def test_density_gradient_matches_central_differences_3d():
    pb = synth.small_lossy_3d(shape=(8, 10, 12), pml=2, Nt=20)
    _rho_fd_check(pb, 3, 8, 1e-6)


def test_density_gradient_scaling_invariant():
    # J(lambda rho0) = J(rho0): with b = 1/rho0 the velocity scales as 1/lambda and the density
    # update -dt rho0 D- u, the absorption term rho0 sum D- u and the pressure do not move, so the
    # directional derivative along rho0 itself vanishes, for any heterogeneous medium
    pb = synth.small_lossy_2d(shape=(22, 20), pml=3, Nt=30, n_sensors=8)
    op = Operator.from_problem(pb)
    h = np.random.default_rng(9).standard_normal((pb.Nt, op.Ns))
    g = pm.density_gradient(op, pb.p0, h)
    rho = np.broadcast_to(np.asarray(pb.rho, float), pb.shape)
    assert np.abs(rho - rho.mean()).max() > 1.0           # heterogeneous density
    scale = float(np.sum(np.abs(g) * rho))
    assert scale > 0
    assert abs(float(np.sum(g * rho))) <= 1e-12 * scale
    # the invariance itself, on the forward map
    J0 = float(np.sum(op.forward(pb.p0) * h))
    J1 = pm.density_objective(pb, 1.7 * rho, h)
    assert abs(J1 - J0) <= 1e-12 * abs(J0)
