"""FP64 CPU oracle for the photoacoustic forward operator H and its adjoint H*.

TEST INFRASTRUCTURE ONLY. This module is the slow, plain reference that the CUDA path is
checked against. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (``cpu_baseline`` / ``--impl reference``) may import it. The product path never calls it
and shares no code with it; the two meet only in the seeded input generators.

Method: Javaherian & Holman, "A Multi-Grid Iterative Method for Photoacoustic Tomography"
(arXiv:1603.02329).

* Sec. II.A, Eqs. (mom), (mass), (estate), (initial): first-order acoustic system
  du/dt = -grad p / rho0, drho/dt = -rho0 div u, with p(0) = p0, u(0) = 0.
* Sec. II.A, Eqs. (state), (Twelve): power-law absorption and dispersion,
  p = c0^2 {1 - tau d/dt (-lap)^(y/2-1) - eta (-lap)^((y-1)/2)} rho,
  tau = -2 alpha0 c0^(y-1), eta = 2 alpha0 c0^y tan(pi y / 2).
* Sec. III: H = M w P (sensor sampling of the pressure field) and its adjoint.
* Sec. VI.A: 20-point PML at 2 Np per grid point; linear interpolation onto point sensors.

The paper solves the system with the k-space pseudospectral method (Sec. I, Sec. II.A,
Sec. VI) without printing the discrete scheme. The readings taken here (all in one place):

R1  grid-centred coordinates x_i = (i - n/2) h; periodic FFTs, the PML absorbs wrap-around;
    k = 2 pi m / (n h) with the Nyquist bin (m = n/2, n even) taken positive.
R2  staggered spectral derivatives D+/- f = Re F^-1{ i k kappa exp(+/- i k h/2) F f },
    kappa = sinc(c_ref |k| dt / 2), c_ref = max c0.  (D-)^T = -D+ exactly.
R3  PML: sigma(delta) = alpha_pml (c_ref / h) (delta / P)^4, delta = depth into the layer in
    grid units (staggered points at i + 1/2); damping factors a = exp(-sigma dt / 2) applied
    as a (a f - dt * rhs) on each split component (u_xi and rho_xi damped along xi only).
R4  alpha0 in dB MHz^-y cm^-1 is converted to Np m^-1 (rad/s)^-y (the paper's "angular
    frequency in MHz" is read as ordinary frequency in MHz, omega in rad/s);
    1/rho0 at a staggered point uses the mean of the two neighbouring rho0 values.
R5  initial state: p^0 = p0, rho_xi^0 = p0 / (d c0^2), u_xi^(-1/2) = +(dt/2) b_xi D+_xi p0;
    the record includes t = 0, so s^0 = M p0 and Nt samples are t = 0 .. (Nt-1) dt.
R6  one time step n -> n+1 (n = 0 .. Nt-2):
        g = D+_xi p;  u_xi <- au (au u_xi - dt b_xi g)
        e_xi = D-_xi u_xi;  rho_xi <- a (a rho_xi - dt rho0 e_xi)
        dd = rho0 sum e_xi (= -drho/dt);  r = sum rho_xi
        p = c0^2 (r + tau L_{y-2} dd - eta L_{y-1} r),  L_s = F^-1 |k|^s F, |k|^s(0) = 0
        s^{n+1} = M p
R7  the adjoint is the exact transpose of R5-R6 (so <Hx, h> = <x, H^T h> to rounding); it
    runs in reverse time with the residual entering as a source, the discrete counterpart of
    Sec. III Eqs. (moma), (massa), (statea), (adjj). The paper's own "adjoint-then-discretize"
    variant (Sec. VI) differs from the transpose by O(dt) and is not what is computed here.
R8  off-grid sensors: multilinear interpolation weights from the physical position; on-grid
    sensors: weight 1 at the given flat index.
R9  optional smoothing of the initial pressure (Sec. VI.A: the high frequencies of p0 are
    filtered by a self-adjoint operator before every forward solve, and the filter is part of
    the adjoint).  The paper names no filter.  Reading: S = F^-1 diag(W) F with the radial
    Blackman window W(k) = B(|k| / k_c), B(q) = 0.42 + 0.5 cos(pi q) + 0.08 cos(2 pi q) for
    q < 1 and 0 for q >= 1, k_c = min over axes of the Nyquist wavenumber pi / h.  W is real,
    even in k and in [0, 1], so S is real, symmetric and non-expansive; the smoothed operator
    is H S and its transpose S H^T.
"""
from __future__ import annotations

import numpy as np
from numpy.fft import irfftn, rfftn
from scipy import sparse

# 1 Np = 20 log10(e) dB
DB_PER_NEPER = 20.0 * np.log10(np.e)


# ---------------------------------------------------------------------------------------------
# Grid, wavenumbers and spectral operators (R1, R2)
# ---------------------------------------------------------------------------------------------

def axis_wavenumbers(n, h, half=False):
    """Wavenumbers of one axis in FFT order (R1). ``half`` gives the rfft layout 0..n/2."""
    m = np.arange(n // 2 + 1) if half else np.arange(n)
    m = np.where(m > n // 2, m - n, m)
    return 2.0 * np.pi * m / (n * h)


class KSpace:
    """Per-axis wavenumbers, |k|, kappa and the staggered derivative symbols on the rfftn
    layout (last numpy axis halved).  Sec. I / Sec. II.A (k-space method), readings R1-R2."""

    def __init__(self, shape, spacing, c_ref, dt):
        self.shape = tuple(shape)
        d = len(shape)
        ks = []
        for a in range(d):
            k1 = axis_wavenumbers(shape[a], spacing[a], half=(a == d - 1))
            bshape = [1] * d
            bshape[a] = -1
            ks.append(k1.reshape(bshape))
        self.k = ks
        self.kmag = np.sqrt(sum(k * k for k in ks))
        # np.sinc(x) = sin(pi x) / (pi x); kappa = sin(z)/z with z = c_ref |k| dt / 2
        self.kappa = np.sinc(c_ref * self.kmag * dt / (2.0 * np.pi))
        self.dplus = [1j * ks[a] * self.kappa * np.exp(+0.5j * ks[a] * spacing[a]) for a in range(d)]
        self.dminus = [1j * ks[a] * self.kappa * np.exp(-0.5j * ks[a] * spacing[a]) for a in range(d)]

    def kpow(self, s):
        """Symbol |k|^s of (-lap)^(s/2), set to 0 at k = 0 (Sec. II.A Eq. (state))."""
        out = np.zeros_like(self.kmag)
        nz = self.kmag > 0
        out[nz] = self.kmag[nz] ** s
        return out

    def apply(self, symbol, f):
        return irfftn(symbol * rfftn(f), s=self.shape, axes=tuple(range(len(self.shape))))


def smoothing_window(shape, spacing):
    """W(k) of reading R9 on the rfftn layout: the radial Blackman window in |k| / k_c."""
    d = len(shape)
    ks = []
    for a in range(d):
        k1 = axis_wavenumbers(shape[a], spacing[a], half=(a == d - 1))
        bshape = [1] * d
        bshape[a] = -1
        ks.append(k1.reshape(bshape))
    k_c = min(np.pi / h for h in spacing)
    q = np.sqrt(sum(k * k for k in ks)) / k_c
    w = 0.42 + 0.5 * np.cos(np.pi * q) + 0.08 * np.cos(2.0 * np.pi * q)
    return np.where(q < 1.0, w, 0.0)


def smooth_image(x, spacing):
    """S x of reading R9 (Sec. VI.A)."""
    shape = np.shape(x)
    W = smoothing_window(shape, spacing)
    return irfftn(W * rfftn(x), s=shape, axes=tuple(range(len(shape))))


# ---------------------------------------------------------------------------------------------
# Medium, PML, sensors (R3, R4, R8)
# ---------------------------------------------------------------------------------------------

def alpha_db_to_neper(alpha0_db, y):
    """dB MHz^-y cm^-1  ->  Np m^-1 (rad/s)^-y  (R4; Sec. II.A power law alpha = alpha0 w^y)."""
    return 100.0 * np.asarray(alpha0_db, dtype=float) / DB_PER_NEPER * (2.0 * np.pi * 1e6) ** (-y)


def absorption_coefficients(c, alpha0_db, y):
    """tau, eta of Sec. II.A Eq. (Twelve)."""
    a = alpha_db_to_neper(alpha0_db, y)
    tau = -2.0 * a * c ** (y - 1.0)
    eta = 2.0 * a * c**y * np.tan(np.pi * y / 2.0)
    return tau, eta


def staggered_inverse_density(rho, axis):
    """b_xi = 1/rho0 at r + h_xi/2, rho0 there = mean of the two neighbours, periodic (R4)."""
    return 2.0 / (rho + np.roll(rho, -1, axis=axis))


def pml_factors(n, P, alpha_pml, c_ref, h, dt):
    """Damping factors exp(-sigma dt/2) at normal points i and staggered points i + 1/2 (R3;
    Sec. VI.A: P points, maximum alpha_pml Np per grid point)."""
    if P <= 0:
        return np.ones(n), np.ones(n)

    def sigma(pos):
        depth = np.maximum(np.maximum(P - pos, pos - (n - 1 - P)), 0.0)
        return alpha_pml * (c_ref / h) * (depth / P) ** 4

    i = np.arange(n, dtype=float)
    return np.exp(-sigma(i) * dt / 2.0), np.exp(-sigma(i + 0.5) * dt / 2.0)


def sensor_matrix(shape, spacing, pos=None, index=None):
    """Sparse M [Ns x N]: s = M p (Sec. III, operator M w; Sec. VI.A linear interpolation; R8).

    ``pos`` is [Ns][d] in (x, y[, z]) order (grid-centred metres); ``index`` is [Ns] flat
    C-order indices of on-grid sensors."""
    N = int(np.prod(shape))
    if index is not None:
        index = np.asarray(index, dtype=np.int64)
        Ns = len(index)
        return sparse.csr_matrix((np.ones(Ns), (np.arange(Ns), index)), shape=(Ns, N))
    pos = np.asarray(pos, dtype=float)
    d = len(shape)
    rows, cols, vals = [], [], []
    for j in range(pos.shape[0]):
        corners = [([], [])]  # list of (indices per axis, weight)
        per_axis = []
        for a in range(d):  # numpy axis a <-> physical component d-1-a
            f = pos[j, d - 1 - a] / spacing[a] + shape[a] // 2
            i0 = int(np.floor(f))
            t = f - i0
            opts = [(i0, 1.0 - t)]
            if t != 0.0:
                opts.append((i0 + 1, t))
            for ii, _ in opts:
                if ii < 0 or ii >= shape[a]:
                    raise ValueError(f"sensor {j} lies outside the grid")
            per_axis.append(opts)
        corners = [((), 1.0)]
        for opts in per_axis:
            corners = [(idx + (ii,), w * wi) for idx, w in corners for ii, wi in opts]
        for idx, w in corners:
            if w != 0.0:
                rows.append(j)
                cols.append(int(np.ravel_multi_index(idx, shape)))
                vals.append(w)
    return sparse.csr_matrix((vals, (rows, cols)), shape=(pos.shape[0], N))


# ---------------------------------------------------------------------------------------------
# The discrete forward operator and its exact transpose (R5-R7)
# ---------------------------------------------------------------------------------------------

class Operator:
    """H: p0 -> s[Nt][Ns] and its transpose, in FP64 (Sec. III; readings R1-R8)."""

    def __init__(self, shape, spacing, pml, pml_alpha, c, rho, alpha0, y, dt, Nt,
                 sensor_pos=None, sensor_index=None, smooth=False):
        self.shape = tuple(int(n) for n in shape)
        self.smooth = bool(smooth)
        self.d = len(self.shape)
        self.spacing = tuple(float(h) for h in spacing)
        self.dt = float(dt)
        self.Nt = int(Nt)
        c = np.broadcast_to(np.asarray(c, dtype=float), self.shape)
        rho = np.broadcast_to(np.asarray(rho, dtype=float), self.shape)
        alpha0 = np.broadcast_to(np.asarray(alpha0, dtype=float), self.shape)
        self.c_ref = float(c.max())
        self.c2 = c * c
        self.rho0 = np.array(rho)
        self.b = [staggered_inverse_density(self.rho0, a) for a in range(self.d)]
        tau, eta = absorption_coefficients(c, alpha0, y)
        self.c2tau = self.c2 * tau
        self.c2eta = self.c2 * eta
        self.lossy = bool(np.any(alpha0 != 0.0))
        self.ks = KSpace(self.shape, self.spacing, self.c_ref, self.dt)
        self.Ly2 = self.ks.kpow(y - 2.0)
        self.Ly1 = self.ks.kpow(y - 1.0)
        self.a, self.au = [], []
        for a in range(self.d):
            fa, fau = pml_factors(self.shape[a], int(pml[a]), pml_alpha, self.c_ref, self.spacing[a], self.dt)
            bshape = [1] * self.d
            bshape[a] = -1
            self.a.append(fa.reshape(bshape))
            self.au.append(fau.reshape(bshape))
        self.M = sensor_matrix(self.shape, self.spacing, sensor_pos, sensor_index)
        self.Ns = self.M.shape[0]

    @classmethod
    def from_problem(cls, pb, Nt=None):
        return cls(pb.shape, pb.spacing, pb.pml, pb.pml_alpha, pb.c, pb.rho, pb.alpha0, pb.y, pb.dt,
                   pb.Nt if Nt is None else Nt, sensor_pos=pb.sensor_pos, sensor_index=pb.sensor_index,
                   smooth=getattr(pb, "smooth", False))

    def initial_pressure(self, p0):
        """p^0 of R5: p0 itself, or S p0 when the smoothing of R9 is on."""
        return smooth_image(p0, self.spacing) if self.smooth else np.array(p0, dtype=float)

    # -- building blocks -------------------------------------------------------------------
    def Dplus(self, a, f):
        return self.ks.apply(self.ks.dplus[a], f)

    def Dminus(self, a, f):
        return self.ks.apply(self.ks.dminus[a], f)

    def gather(self, p):
        return self.M @ p.ravel()

    def scatter(self, h_row):
        return (self.M.T @ h_row).reshape(self.shape)

    def pressure(self, r, dd):
        """Eq. (state) with drho/dt = -rho0 div u substituted (R6)."""
        p = self.c2 * r
        if self.lossy:
            p = p + self.c2tau * self.ks.apply(self.Ly2, dd) - self.c2eta * self.ks.apply(self.Ly1, r)
        return p

    # -- H ----------------------------------------------------------------------------------
    def forward(self, p0, keep_fields=False):
        """Returns data [Nt][Ns]; with ``keep_fields`` also the lists p^n (n = 0..Nt-1) and
        u^(n-1/2) (n = 0..Nt-1, i.e. u^(-1/2) .. u^(Nt-3/2)) for invariant checks."""
        d, dt = self.d, self.dt
        p = self.initial_pressure(p0)
        data = np.zeros((self.Nt, self.Ns))
        rho = [p / (d * self.c2) for _ in range(d)]
        g = [self.Dplus(a, p) for a in range(d)]
        u = [0.5 * dt * self.b[a] * g[a] for a in range(d)]
        data[0] = self.gather(p)
        ps, us = ([p.copy()], [[x.copy() for x in u]]) if keep_fields else (None, None)
        for n in range(self.Nt - 1):
            if n > 0:
                g = [self.Dplus(a, p) for a in range(d)]
            u = [self.au[a] * (self.au[a] * u[a] - dt * self.b[a] * g[a]) for a in range(d)]
            e = [self.Dminus(a, u[a]) for a in range(d)]
            rho = [self.a[a] * (self.a[a] * rho[a] - dt * self.rho0 * e[a]) for a in range(d)]
            dd = self.rho0 * sum(e)
            r = sum(rho)
            p = self.pressure(r, dd)
            data[n + 1] = self.gather(p)
            if keep_fields:
                ps.append(p.copy())
                us.append([x.copy() for x in u])
        if keep_fields:
            return data, ps, us
        return data

    # -- H^T ----------------------------------------------------------------------------------
    def adjoint(self, h):
        """Exact transpose of ``forward`` (R7): image-space gradient of <H x, h>."""
        d, dt = self.d, self.dt
        h = np.asarray(h, dtype=float).reshape(self.Nt, self.Ns)
        pbar = self.scatter(h[self.Nt - 1])
        ubar = [np.zeros(self.shape) for _ in range(d)]
        rhobar = [np.zeros(self.shape) for _ in range(d)]
        for n in range(self.Nt - 2, -1, -1):
            # p^{n+1} = c2 r + c2tau L_{y-2} dd - c2eta L_{y-1} r
            rbar = self.c2 * pbar
            ddbar = np.zeros(self.shape)
            if self.lossy:
                rbar = rbar - self.ks.apply(self.Ly1, self.c2eta * pbar)
                ddbar = self.ks.apply(self.Ly2, self.c2tau * pbar)
            # r = sum rho_xi ; dd = rho0 sum e_xi ; rho_xi <- a (a rho_xi - dt rho0 e_xi)
            ebar = []
            for a in range(d):
                rhobar[a] = rhobar[a] + rbar
                ebar.append(self.rho0 * ddbar - dt * self.rho0 * self.a[a] * rhobar[a])
                rhobar[a] = self.a[a] ** 2 * rhobar[a]
            # e_xi = D-_xi u_xi, (D-)^T = -D+
            gbar = []
            for a in range(d):
                ubar[a] = ubar[a] - self.Dplus(a, ebar[a])
                # u_xi <- au (au u_xi - dt b_xi g_xi)
                gbar.append(-dt * self.b[a] * self.au[a] * ubar[a])
                ubar[a] = self.au[a] ** 2 * ubar[a]
            # g_xi = D+_xi p^n, (D+)^T = -D-
            pbar = -sum(self.Dminus(a, gbar[a]) for a in range(d)) + self.scatter(h[n])
        # initial state R5: p^0 = p0, rho^0 = p0/(d c2), u^(-1/2) = dt/2 b D+ p0
        grad = pbar + sum(rhobar) / (d * self.c2)
        grad = grad - sum(self.Dminus(a, 0.5 * dt * self.b[a] * ubar[a]) for a in range(d))
        # R9: (H S)^T = S^T H^T = S H^T
        return smooth_image(grad, self.spacing) if self.smooth else grad

    # -- objective pieces (Sec. IV, Eqs. (two), (Six)) ------------------------------------------
    def data_misfit(self, x, p_hat):
        """f(x) = 1/2 ||H x - p_hat||^2 (Sec. IV)."""
        r = self.forward(x) - p_hat
        return 0.5 * float(np.sum(r * r))

    def gradient(self, x, p_hat):
        """grad f(x) = H^T (H x - p_hat) (Sec. IV, Eq. (Six))."""
        return self.adjoint(self.forward(x) - p_hat)
