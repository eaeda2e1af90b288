"""Pins of the FP64 oracle's forward operator and adjoint against what the mathematics fixes.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or
shift, a transposed operand, a wrong unit conversion) fails at least one of them:

* exact discrete solution p^n = F^-1 cos(n c |k| dt) F p0 (homogeneous, lossless, periodic),
* the leapfrog energy invariant on a heterogeneous medium,
* the transpose identities (D-)^T = -D+ and <Hx, h> = <x, H^T h>,
* the staggered derivative of a sine,
* the physical decay rate and dispersion sign of a plane mode under power-law absorption,
* linear interpolation reproduces linear fields; an on-node sensor reads the node value,
* finite differences of the quadratic data misfit,
* the smoothing of p0: window values on chosen Fourier modes, symmetry, the dot test with it on,
* the continuum solution of a smooth radial pulse (d'Alembert in 3-D, Hankel quadrature in 2-D).
"""
import numpy as np
import pytest
from numpy.fft import irfftn, rfftn

from oracle.pat_oracle import Operator, sensor_matrix, smooth_image
from paper_1603_02329_gb300 import synth


def _all_points(shape):
    return np.arange(int(np.prod(shape)))


@pytest.mark.parametrize("shape", [(24, 30), (12, 14, 10)])
def test_exact_periodic_solution(shape):
    # Homogeneous lossless medium without PML: the kappa-corrected leapfrog is exact in time,
    # P^{n+1} - 2 cos(w) P^n + P^{n-1} = 0 with w = c |k| dt and P^1 = cos(w) P^0.
    rng = np.random.default_rng(1)
    h = 1e-4
    c = 1500.0
    dt = 0.3 * h / c
    Nt = 25
    op = Operator(shape, (h,) * len(shape), (0,) * len(shape), 2.0, c, 1000.0, 0.0, 1.5, dt, Nt,
                  sensor_index=_all_points(shape))
    p0 = rng.standard_normal(shape)
    data = op.forward(p0)
    kx = [2 * np.pi * np.fft.fftfreq(n, h) for n in shape]
    kk = np.meshgrid(*kx, indexing="ij")
    w = c * np.sqrt(sum(k * k for k in kk)) * dt
    for n in (1, 2, 7, Nt - 1):
        ref = np.real(np.fft.ifftn(np.cos(n * w) * np.fft.fftn(p0)))
        assert np.max(np.abs(data[n] - ref.ravel())) < 1e-12 * np.max(np.abs(p0)) * 10


def test_energy_invariant_heterogeneous():
    # E^n = 1/2 sum p^2/(rho0 c0^2) + 1/2 sum_xi u^(n-1/2) u^(n+1/2) / b_xi is conserved by the
    # leapfrog when (D-)^T = -D+, with PML and absorption off and a heterogeneous medium.
    rng = np.random.default_rng(2)
    shape = (32, 36)
    h = 1e-4
    c, rho = synth.heterogeneous_medium(rng, shape, sigma_px=3.0)
    dt = 0.3 * h / c.max()
    Nt = 60
    op = Operator(shape, (h, h), (0, 0), 2.0, c, rho, 0.0, 1.5, dt, Nt, sensor_index=[0])
    p0 = synth.discs(rng, shape, (h, h), 3, 1e-3, (2e-4, 6e-4), (0.5, 1.0))
    _, ps, us = op.forward(p0, keep_fields=True)
    E = []
    for n in range(Nt - 1):
        ep = 0.5 * np.sum(ps[n] ** 2 / (rho * c * c))
        eu = 0.5 * sum(np.sum(us[n][a] * us[n + 1][a] / op.b[a]) for a in range(2))
        E.append(ep + eu)
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) / E[0] < 1e-12
    # the pressure part alone is not conserved: the check is not vacuous
    ep_only = [0.5 * np.sum(ps[n] ** 2 / (rho * c * c)) for n in range(Nt - 1)]
    assert np.ptp(ep_only) / ep_only[0] > 1e-3


def test_derivative_transpose_and_sine():
    rng = np.random.default_rng(3)
    shape = (16, 20)
    h = (1e-4, 2e-4)
    op = Operator(shape, h, (0, 0), 2.0, 1500.0, 1000.0, 0.0, 1.5, 1e-8, 2, sensor_index=[0])
    f = rng.standard_normal(shape)
    g = rng.standard_normal(shape)
    for a in range(2):
        lhs = np.sum(op.Dminus(a, f) * g)
        rhs = -np.sum(f * op.Dplus(a, g))
        assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(f) * np.linalg.norm(g) * 1e3
    # D+_x sin(k0 x) = k0 kappa(k0) cos(k0 (x + h/2)), a single-mode identity
    nx = shape[1]
    x = (np.arange(nx) - nx // 2) * h[1]
    k0 = 2 * np.pi * 3 / (nx * h[1])
    s = np.broadcast_to(np.sin(k0 * x), shape)
    zk = 1500.0 * k0 * 1e-8 / 2
    kappa = np.sin(zk) / zk
    ref = k0 * kappa * np.cos(k0 * (x + h[1] / 2))
    assert np.max(np.abs(op.Dplus(1, s) - ref[None, :])) < 1e-9 * k0


@pytest.mark.parametrize("case", ["lossy2d_offgrid", "lossy3d_ongrid", "lossless2d", "smooth2d", "smooth3d"])
def test_adjoint_dot_product(case):
    if case in ("lossy2d_offgrid", "smooth2d"):
        pb = synth.small_lossy_2d(shape=(32, 40), pml=6, Nt=40, n_sensors=12)
    elif case in ("lossy3d_ongrid", "smooth3d"):
        pb = synth.small_lossy_3d(shape=(12, 16, 20), pml=3, Nt=20)
    else:
        pb = synth.disc_phantom_2d(interior=24, pml=6, Nt=40, n_sensors=10, sensor_radius=1e-3)
    pb.smooth = case.startswith("smooth")
    op = Operator.from_problem(pb)
    assert op.smooth == pb.smooth
    rng = np.random.default_rng(4)
    x = rng.standard_normal(pb.shape)
    hh = rng.standard_normal((pb.Nt, op.Ns))
    Hx = op.forward(x)
    HTh = op.adjoint(hh)
    lhs, rhs = np.sum(Hx * hh), np.sum(x * HTh)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Hx) * np.linalg.norm(hh)
    assert np.linalg.norm(Hx) > 0 and np.linalg.norm(HTh) > 0


def test_finite_difference_gradient():
    # f is quadratic, so the central difference equals <grad f, v> for any step
    pb = synth.small_lossy_2d(shape=(24, 28), pml=5, Nt=30, n_sensors=10)
    op = Operator.from_problem(pb)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(pb.shape)
    phat = rng.standard_normal((pb.Nt, op.Ns))
    g = op.gradient(x, phat)
    for _ in range(3):
        v = rng.standard_normal(pb.shape)
        eps = np.linalg.norm(x) / np.linalg.norm(v)
        fd = (op.data_misfit(x + eps * v, phat) - op.data_misfit(x - eps * v, phat)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) <= 1e-9 * abs(fd) + 1e-12


def test_absorption_decay_and_dispersion():
    # A single plane mode on a homogeneous periodic grid without PML: the pressure coefficient
    # follows a two-term recurrence (state = (rho, u)), so a least-squares fit of
    # P_{n+1} = a1 P_n + a2 P_{n-1} recovers the damping exactly. Physical law (Sec. II.A):
    # spatial attenuation alpha0 f_MHz^y dB/cm, temporal decay ~ c * attenuation.
    nx, ny = 64, 4
    h = 0.1e-3
    c = 1500.0
    y = 1.5
    a0 = 5.0
    dt = 0.3 * h / c
    m = 4
    k0 = 2 * np.pi * m / (nx * h)
    Nt = 400
    op = Operator((ny, nx), (h, h), (0, 0), 2.0, c, 1000.0, a0, y, dt, Nt,
                  sensor_index=np.arange(nx * ny))
    x = (np.arange(nx) - nx // 2) * h
    p0 = np.broadcast_to(np.cos(k0 * x), (ny, nx))
    data = op.forward(p0).reshape(Nt, ny, nx)
    P = np.array([np.fft.rfft(d[0])[m] for d in data]).real
    # P^0 = p0 is imposed (not produced by the recurrence from rho^0, u^(-1/2)): fit from n = 1
    A = np.stack([P[2:-1], P[1:-2]], axis=1)
    coef, *_ = np.linalg.lstsq(A, P[3:], rcond=None)
    assert np.max(np.abs(A @ coef - P[3:])) < 1e-10
    r = np.sqrt(-coef[1])
    gamma = -np.log(r) / dt
    omega = np.arccos(coef[0] / (2 * r)) / dt
    f_mhz = c * k0 / (2 * np.pi) / 1e6
    atten_np_per_m = a0 * f_mhz**y * 100.0 / (20 * np.log10(np.e))
    gamma_ref = c * atten_np_per_m
    assert abs(gamma / gamma_ref - 1) < 0.02
    # dispersion: y = 1.5 gives eta < 0, so the mode runs faster than c (sound speed rises with
    # frequency) by the (1 - eta k^(y-1)) factor of Eq. (state)
    assert omega > c * k0
    assert np.max(np.abs(P[-50:])) < 0.7 * np.max(np.abs(P[:50]))


def test_sensor_interpolation():
    shape = (10, 12)
    h = (1e-4, 1e-4)
    # exactly on a node: weight 1 on that node
    pos = np.array([[(7 - 6) * 1e-4, (3 - 5) * 1e-4]])
    M = sensor_matrix(shape, h, pos=pos)
    assert M.nnz == 1 and M[0, 3 * 12 + 7] == 1.0
    # linear fields are reproduced exactly by the multilinear weights
    rng = np.random.default_rng(6)
    pos = rng.uniform(-3e-4, 3e-4, size=(20, 2))
    M = sensor_matrix(shape, h, pos=pos)
    yy, xx = np.meshgrid((np.arange(10) - 5) * 1e-4, (np.arange(12) - 6) * 1e-4, indexing="ij")
    f = 2.0 + 3.0 * xx / 1e-4 - 1.5 * yy / 1e-4
    ref = 2.0 + 3.0 * pos[:, 0] / 1e-4 - 1.5 * pos[:, 1] / 1e-4
    assert np.max(np.abs(M @ f.ravel() - ref)) < 1e-10
    assert np.allclose(np.asarray(M.sum(axis=1)).ravel(), 1.0)
    with pytest.raises(ValueError):
        sensor_matrix(shape, h, pos=np.array([[1.0, 0.0]]))


def test_pml_damps_outgoing_energy():
    # With the PML on, an outgoing pulse loses almost all of its energy after crossing the
    # boundary, while without it the periodic grid keeps it.
    shape = (48, 48)
    h = 1e-4
    c = 1500.0
    dt = 0.3 * h / c
    Nt = 300
    p0 = synth.discs(np.random.default_rng(7), shape, (h, h), 1, 1e-4, (3e-4, 3e-4), (1.0, 1.0))
    idx = np.arange(48 * 48)
    with_pml = Operator(shape, (h, h), (8, 8), 2.0, c, 1000.0, 0.0, 1.5, dt, Nt, sensor_index=idx)
    no_pml = Operator(shape, (h, h), (0, 0), 2.0, c, 1000.0, 0.0, 1.5, dt, Nt, sensor_index=idx)
    e_pml = np.sum(with_pml.forward(p0)[-1] ** 2)
    e_per = np.sum(no_pml.forward(p0)[-1] ** 2)
    assert e_pml < 1e-2 * e_per


# PML pins (reading R3; Sec. VI.A fixes the thickness, 20 points, and the maximum, 2 Np per grid
# point).  (1) One step from a constant field: D+ of a constant is zero, so u stays zero and each
# split density only decays, rho_x^1 = exp(-sigma dt) rho_x^0, while rho_y^1 = rho_y^0; in 2-D
# p^1 = p0 (1 + exp(-sigma dt)) / 2 in closed form.  From the recorded p^1 the damping rate per grid
# point of travel, sigma h / c_ref, is read back at every node of a 64-point x axis: the paper's
# 2 Np at the outer node of each side, alpha (depth / P)^4 inside the layer, and exactly P damped
# nodes per side (a shifted depth or a wrong c_ref / h scaling moves the edge value).
def test_pml_damping_rate_from_one_step_closed_form():
    nx, ny, P, alpha = 64, 4, 20, 2.0
    h, c = 1e-4, 1500.0
    dt = 0.3 * h / c
    idx = np.arange(nx)                       # row y = 0, every x
    op = Operator((ny, nx), (h, h), (0, P), alpha, c, 1000.0, 0.0, 1.5, dt, 2, sensor_index=idx)
    s1 = op.forward(np.ones((ny, nx)))[1]
    rate = -np.log(2.0 * s1 - 1.0) * h / (c * dt)     # sigma h / c_ref [Np per grid point]
    assert abs(rate[0] - 2.0) < 1e-9 and abs(rate[-1] - 2.0) < 1e-9
    depth = np.maximum(np.maximum(P - idx, idx - (nx - 1 - P)), 0)
    assert np.allclose(rate, alpha * (depth / P) ** 4, atol=1e-9)
    assert np.count_nonzero(rate[: nx // 2] > 1e-12) == P and np.count_nonzero(rate[nx // 2:] > 1e-12) == P


# (2) A plane pulse crossing the layer.  A Gaussian pulse (width 6 h, uniform in y) splits into two
# halves that run through the x layers on both sides of the periodic grid and meet again at the
# centre after one period, attenuated by exp(-G) with G = int sigma / c dx over both layers.  For
# the quartic profile the continuum integral is 2 alpha P / 5 (alpha in Np per point, P points); the
# sampled profile adds an edge term that does not depend on P, so thickening the layer from P to 2P
# adds exactly 2 alpha P / 5.  Measured with alpha = 0.05 and P = 20, 40: 0.399 against 0.4.  A
# profile exponent m would add 2 alpha P / (m + 1); a c_ref / h slip scales it.  With the paper's
# 2 Np per point the pulse is absorbed and what returns from the layer's inner edge is below 1e-5.
def _pml_pulse(alpha, P, nx=512, ny=4, h=1e-4, c=1500.0):
    dt = 0.3 * h / c
    n_period = int(round(nx * h / (c * dt)))
    x = np.arange(nx)
    p0 = np.repeat(np.exp(-0.5 * ((x - nx // 2) / 6.0) ** 2)[None, :], ny, axis=0)
    op = Operator((ny, nx), (h, h), (0, P), alpha, c, 1000.0, 0.0, 1.5, dt, n_period + 40,
                  sensor_index=np.array([nx // 2]))
    s = op.forward(p0)[:, 0]
    n_refl = int(round(2 * (nx // 2 - P) * h / (c * dt)))
    return s[n_period - 30:n_period + 30].max(), np.abs(s[n_refl - 40:n_refl + 40]).max()


def test_pml_attenuation_grows_by_the_continuum_integral():
    alpha = 0.05
    t20, _ = _pml_pulse(alpha, 20)
    t40, _ = _pml_pulse(alpha, 40)
    extra = np.log(t20) - np.log(t40)
    assert abs(extra - 2 * alpha * 20 / 5) < 0.01 * (2 * alpha * 20 / 5)
    assert 0.5 < t20 < 0.8                            # it does cross the layer
    t_paper, refl = _pml_pulse(2.0, 20)
    assert t_paper < 1e-6 and refl < 1e-5


# Blackman window B(q) at the radii where it has a short closed form: B(0) = 1,
# B(1/3) = 0.42 + 0.5/2 - 0.08/2 = 0.63, B(1/2) = 0.42 - 0.08 = 0.34, B(q >= 1) = 0.
# Grid (Ny, Nx) = (24, 32) with spacing (1e-4, 2e-4): the cut-off radius is the Nyquist
# wavenumber of the coarser x axis, pi / 2e-4, so a mode (my, mx) sits at
# q = sqrt((mx / 16)^2 + (my / 6)^2).  A y mode with my = 6 is cut although it lies at half the
# y axis' own Nyquist wavenumber; a window cut at the finer axis would keep 0.34 of it.
@pytest.mark.parametrize("my,mx,gain", [(0, 0, 1.0), (0, 8, 0.34), (3, 0, 0.34), (2, 0, 0.63), (6, 0, 0.0),
                                        (0, 16, 0.0), (12, 0, 0.0), (3, 16, 0.0), (5, 10, 0.0)])
def test_smoothing_window_on_fourier_modes(my, mx, gain):
    ny, nx = 24, 32
    spacing = (1e-4, 2e-4)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    f = np.cos(2 * np.pi * (mx * ii / nx + my * jj / ny) + 0.3)
    assert np.max(np.abs(smooth_image(f, spacing) - gain * f)) < 1e-13


def test_smoothing_window_3d_mode_and_symmetry():
    # 3-D: a z mode at half the (common) Nyquist radius keeps 0.34 of its amplitude
    shape = (8, 12, 16)
    h = 1e-4
    kk = np.arange(8)[:, None, None] * np.ones(shape)
    f = np.sin(2 * np.pi * 2 * kk / 8 + 0.1)
    assert np.max(np.abs(smooth_image(f, (h, h, h)) - 0.34 * f)) < 1e-13
    # S is symmetric and non-expansive (0 <= W <= 1), on anisotropic 2-D and 3-D grids
    rng = np.random.default_rng(11)
    for shape, sp in (((20, 28), (1e-4, 1.5e-4)), ((8, 10, 12), (1e-4, 2e-4, 1e-4))):
        x, y = rng.standard_normal(shape), rng.standard_normal(shape)
        Sx, Sy = smooth_image(x, sp), smooth_image(y, sp)
        assert abs(np.sum(Sx * y) - np.sum(x * Sy)) < 1e-13 * np.linalg.norm(x) * np.linalg.norm(y)
        assert np.linalg.norm(Sx) < np.linalg.norm(x)
        assert np.sum(x * Sx) >= 0.0


def test_smoothing_enters_forward_and_adjoint():
    # H S p0 = H (S p0): the smoothed operator's record equals the plain one's on S p0, and its
    # adjoint ends with S
    pb = synth.small_lossy_2d(shape=(24, 28), pml=5, Nt=20, n_sensors=8)
    plain = Operator.from_problem(pb)
    pb.smooth = True
    op = Operator.from_problem(pb)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(pb.shape)
    Sx = smooth_image(x, pb.spacing)
    assert np.max(np.abs(op.forward(x) - plain.forward(Sx))) <= 1e-13 * np.max(np.abs(plain.forward(Sx)))
    hh = rng.standard_normal((pb.Nt, op.Ns))
    ref = smooth_image(plain.adjoint(hh), pb.spacing)
    assert np.max(np.abs(op.adjoint(hh) - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_continuum_radial_pulse_3d():
    # Homogeneous lossless medium, periodic grid without PML, a Gaussian p0 of width s = 2.5 h:
    # the continuum solution is r p(r, t) = [(r - ct) P(r - ct) + (r + ct) P(r + ct)] / 2
    # (P the radial profile, even).  The k-space scheme is exact in time for this medium and
    # the pulse is band-limited to ~1e-13 on the grid, so the discrete record matches the
    # continuum solution until the wave reaches a periodic image.
    n = 48
    h = 1e-4
    c = 1500.0
    dt = 0.3 * h / c
    s = 2.5 * h
    Nt = 41                       # c t = 12 h at the last sample
    ax = (np.arange(n) - n // 2) * h
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.sqrt(xx**2 + yy**2 + zz**2)
    prof = lambda q: np.exp(-q * q / (2 * s * s))
    sel = (r > 0.5 * h) & (r < 16 * h)
    idx = np.flatnonzero(sel.ravel())
    op = Operator((n, n, n), (h, h, h), (0, 0, 0), 2.0, c, 1000.0, 0.0, 1.5, dt, Nt, sensor_index=idx)
    data = op.forward(prof(r))
    rs = r.ravel()[idx]
    for m in (10, 25, Nt - 1):
        ct = c * m * dt
        ref = ((rs - ct) * prof(rs - ct) + (rs + ct) * prof(rs + ct)) / (2 * rs)
        assert np.max(np.abs(data[m] - ref)) < 1e-11    # a 0.1 % error in c gives ~1e-3


def test_continuum_radial_pulse_2d():
    # 2-D counterpart: p(r, t) = int_0^inf k P^(k) J0(k r) cos(c k t) dk with the Hankel
    # transform P^(k) = s^2 exp(-k^2 s^2 / 2) of the Gaussian profile, by quadrature.
    from scipy import integrate, special

    n = 96
    h = 1e-4
    c = 1500.0
    dt = 0.3 * h / c
    s = 2.5 * h
    Nt = 61                       # c t = 18 h at the last sample
    ax = (np.arange(n) - n // 2) * h
    yy, xx = np.meshgrid(ax, ax, indexing="ij")
    r = np.sqrt(xx**2 + yy**2)
    # sensors along the +x half line through the centre, out to 24 h
    idx = (n // 2) * n + n // 2 + np.arange(0, 25)
    op = Operator((n, n), (h, h), (0, 0), 2.0, c, 1000.0, 0.0, 1.5, dt, Nt, sensor_index=idx)
    data = op.forward(np.exp(-r * r / (2 * s * s)))
    rs = np.arange(0, 25) * h
    kmax = 12.0 / s
    for m in (20, Nt - 1):
        ct = c * m * dt
        ref = [integrate.quad(lambda k: k * s * s * np.exp(-(k * s) ** 2 / 2) * special.j0(k * q) * np.cos(k * ct),
                              0.0, kmax, limit=400, epsabs=1e-13)[0] for q in rs]
        assert np.max(np.abs(data[m] - np.array(ref))) < 1e-10    # a 0.1 % error in c gives ~1e-3


def _dft_all_axes(f, inverse=False):
    """Multi-dimensional DFT by its definition, one O(n^2) matrix product per axis."""
    out = np.asarray(f, dtype=complex)
    for a, n in enumerate(out.shape):
        j = np.arange(n)
        F = np.exp((2j if inverse else -2j) * np.pi * np.outer(j, j) / n)
        if inverse:
            F = F / n
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, a, 0), axes=(1, 0)), 0, a)
    return out


@pytest.mark.parametrize("shape", [(6, 7), (12, 10), (8, 9, 10), (6, 5, 14)])
def test_spectral_operators_match_brute_force_dft(shape):
    # D+, D-, the fractional Laplacians and the smoothing window, computed by the oracle through
    # rfftn / irfftn on the half-spectrum layout, against full complex DFTs by definition with the
    # symbols written on the whole grid (radices 2, 3, 5, 7; odd and even lengths)
    rng = np.random.default_rng(13)
    d = len(shape)
    h = tuple(1e-4 * (1 + 0.25 * a) for a in range(d))
    c, dt, y = 1500.0, 2e-8, 1.5
    op = Operator(shape, h, (0,) * d, 2.0, c, 1000.0, 0.75, y, dt, 2, sensor_index=[0])
    f = rng.standard_normal(shape)
    grids = np.meshgrid(*[2 * np.pi * np.where(np.arange(n) > n // 2, np.arange(n) - n, np.arange(n)) / (n * h[a])
                          for a, n in enumerate(shape)], indexing="ij")
    kmag = np.sqrt(sum(k * k for k in grids))
    z = c * kmag * dt / 2
    kappa = np.where(z > 0, np.sin(z) / np.where(z > 0, z, 1.0), 1.0)
    Ff = _dft_all_axes(f)

    def brute(symbol):
        return np.real(_dft_all_axes(symbol * Ff, inverse=True))

    for a in range(d):
        k = grids[a]
        assert np.max(np.abs(op.Dplus(a, f) - brute(1j * k * kappa * np.exp(0.5j * k * h[a])))) < 1e-12 * np.abs(k).max()
        assert np.max(np.abs(op.Dminus(a, f) - brute(1j * k * kappa * np.exp(-0.5j * k * h[a])))) < 1e-12 * np.abs(k).max()
    for s in (y - 2.0, y - 1.0):
        sym = np.where(kmag > 0, np.where(kmag > 0, kmag, 1.0) ** s, 0.0)
        assert np.max(np.abs(op.ks.apply(op.Ly2 if s < -0.1 else op.Ly1, f) - brute(sym))) < 1e-12 * sym.max()
    q = kmag / min(np.pi / hh for hh in h)
    W = np.where(q < 1, 0.42 + 0.5 * np.cos(np.pi * q) + 0.08 * np.cos(2 * np.pi * q), 0.0)
    assert np.max(np.abs(smooth_image(f, h) - brute(W))) < 1e-13
