"""Seeded synthetic inputs for the photoacoustic forward/adjoint path.

This module only draws and rasterises inputs: initial-pressure phantoms, medium maps,
sensor positions and the time axis. It holds none of the method's arithmetic (no
wavenumbers, no PML, no absorption coefficients, no interpolation weights); both the
FP64 oracle and the CUDA path derive those themselves from what is generated here.

The paper's phantoms and medium maps exist only as figures (Sec. VI.A, Figs. 1-2;
Sec. VI.B, Figs. 6-7), so every workload here is a synthetic stand-in with the shape,
spacing, sensor geometry and value distribution of the paper's experiments:

* 2-D vessel-like phantoms with sharp discs (Sec. VI.A: vessels, maximum amplitude 2),
* heterogeneous smooth sound-speed and density maps around water values (Sec. VI.A),
* power-law absorption alpha0 = 0.75 dB MHz^-y cm^-1, y = 1.5 (Sec. VI.A),
* point sensors on a circle / on a line / on a planar face (Sec. VI.A, VI.B),
* PML of 20 points at 2 Np per point (Sec. VI.A).

Array conventions: numpy order (Ny, Nx) or (Nz, Ny, Nx), x fastest. Physical
coordinates are grid-centred, x_i = (i - n/2) * h. Sensor positions are stored as
[Ns][d] in (x, y[, z]) component order, matching the C ABI.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One forward/adjoint workload: grid, medium, sensors, time axis and a phantom."""

    name: str
    shape: tuple            # numpy order, e.g. (Ny, Nx)
    spacing: tuple          # metres, numpy order
    pml: tuple              # PML thickness in points per axis, numpy order
    pml_alpha: float        # Np per grid point at the outer edge
    c: np.ndarray           # sound speed [m/s], shape
    rho: np.ndarray         # ambient density [kg/m^3], shape
    alpha0: np.ndarray      # absorption coefficient [dB MHz^-y cm^-1], shape (zeros = lossless)
    y: float                # power-law exponent
    dt: float               # time step [s]
    Nt: int                 # number of recorded samples (t = 0 .. (Nt-1) dt)
    p0: np.ndarray          # initial pressure (ground truth phantom)
    sensor_pos: Optional[np.ndarray] = None    # [Ns][d] (x,y[,z]) metres, off-grid (linear interpolation)
    sensor_index: Optional[np.ndarray] = None  # [Ns] flat C-order indices, on-grid sensors
    seed: int = 0
    smooth: bool = False    # filter p0 with the plan's self-adjoint smoothing before each solve

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def N(self) -> int:
        return int(np.prod(self.shape))

    @property
    def Ns(self) -> int:
        if self.sensor_index is not None:
            return int(len(self.sensor_index))
        return int(len(self.sensor_pos))

    @property
    def lossy(self) -> bool:
        return bool(np.any(np.asarray(self.alpha0) != 0.0))


# --------------------------------------------------------------------------------------
# Raw random fields and shapes
# --------------------------------------------------------------------------------------

def coords(shape, spacing):
    """Grid-centred coordinate vectors per numpy axis: (i - n/2) * h."""
    return [(np.arange(n) - n // 2) * h for n, h in zip(shape, spacing)]


def smooth_unit_noise(rng, shape, sigma_px):
    """White N(0,1) noise, Gaussian-smoothed (periodic), renormalised to unit variance."""
    from scipy.ndimage import gaussian_filter

    w = rng.standard_normal(shape)
    s = gaussian_filter(w, sigma=sigma_px, mode="wrap")
    s = s - s.mean()
    return s / s.std()


def discs(rng, shape, spacing, count, r_center_max, radius_range, amp_range):
    """Sum of binary discs/balls with random centre (|centre| < r_center_max), radius and amplitude."""
    d = len(shape)
    grids = np.meshgrid(*coords(shape, spacing), indexing="ij")
    out = np.zeros(shape)
    for _ in range(count):
        # uniform in a disc/ball of radius r_center_max (rejection sampling)
        while True:
            ctr = rng.uniform(-r_center_max, r_center_max, size=d)
            if np.sum(ctr**2) < r_center_max**2:
                break
        rad = rng.uniform(*radius_range)
        amp = rng.uniform(*amp_range)
        dist2 = sum((g - c0) ** 2 for g, c0 in zip(grids, ctr))
        out += amp * (dist2 <= rad**2)
    return out


def vessels_2d(rng, shape, count, width_px_choices=(2, 3, 4), amp_range=(0.5, 1.0), margin_px=40):
    """Vessel-like curves: cubic splines through 5 random control points, rasterised with
    a random width (pixels) and amplitude. Overlaps take the maximum amplitude."""
    from scipy.interpolate import CubicSpline

    ny, nx = shape
    out = np.zeros(shape)
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for _ in range(count):
        pts = np.stack([rng.uniform(margin_px, ny - margin_px, 5),
                        rng.uniform(margin_px, nx - margin_px, 5)], axis=1)
        tpar = np.linspace(0.0, 1.0, 5)
        cs = CubicSpline(tpar, pts, axis=0)
        curve = cs(np.linspace(0.0, 1.0, 400))
        curve[:, 0] = np.clip(curve[:, 0], margin_px / 2, ny - 1 - margin_px / 2)
        curve[:, 1] = np.clip(curve[:, 1], margin_px / 2, nx - 1 - margin_px / 2)
        width = float(rng.choice(width_px_choices))
        amp = rng.uniform(*amp_range)
        mask = np.zeros(shape, dtype=bool)
        half = width / 2.0
        for cy, cx in curve:
            y0, y1 = int(max(cy - half - 1, 0)), int(min(cy + half + 2, ny))
            x0, x1 = int(max(cx - half - 1, 0)), int(min(cx + half + 2, nx))
            sub = (yy[y0:y1, x0:x1] - cy) ** 2 + (xx[y0:y1, x0:x1] - cx) ** 2 <= half**2
            mask[y0:y1, x0:x1] |= sub
        out = np.maximum(out, amp * mask)
    return out


def tubes_3d(rng, shape, count, radius_px_range=(1.0, 2.0), amp_range=(0.5, 1.0), margin_px=12):
    """3-D tube phantoms: splines through 5 random control points swept with a radius."""
    from scipy.interpolate import CubicSpline

    out = np.zeros(shape)
    zz, yy, xx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    for _ in range(count):
        pts = np.stack([rng.uniform(margin_px, n - margin_px, 5) for n in shape], axis=1)
        cs = CubicSpline(np.linspace(0, 1, 5), pts, axis=0)
        curve = cs(np.linspace(0, 1, 200))
        for ax, n in enumerate(shape):
            curve[:, ax] = np.clip(curve[:, ax], margin_px / 2, n - 1 - margin_px / 2)
        rad = rng.uniform(*radius_px_range)
        amp = rng.uniform(*amp_range)
        mask = np.zeros(shape, dtype=bool)
        for cz, cy, cx in curve:
            lo = [int(max(v - rad - 1, 0)) for v in (cz, cy, cx)]
            hi = [int(min(v + rad + 2, n)) for v, n in zip((cz, cy, cx), shape)]
            sl = tuple(slice(a, b) for a, b in zip(lo, hi))
            sub = (zz[sl] - cz) ** 2 + (yy[sl] - cy) ** 2 + (xx[sl] - cx) ** 2 <= rad**2
            mask[sl] |= sub
        out = np.maximum(out, amp * mask)
    return out


def circle_sensors(count, radius, arc=2 * np.pi, start=0.0):
    """Equispaced point sensors on a circle (or an arc) about the grid centre, (x, y) order."""
    th = start + arc * np.arange(count) / (count if abs(arc - 2 * np.pi) < 1e-12 else max(count - 1, 1))
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


def awgn(rng, data, snr_db):
    """Additive white Gaussian noise at a global SNR: sigma = rms(data) * 10^(-snr/20)."""
    sigma = np.sqrt(np.mean(data**2)) * 10 ** (-snr_db / 20.0)
    return data + sigma * rng.standard_normal(data.shape)


# --------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------

def heterogeneous_medium(rng, shape, c_mean=1500.0, c_dev=100.0, rho_mean=1000.0, rho_rel=0.05,
                         sigma_px=8.0):
    """c = c_mean + c_dev * n1, rho = rho_mean * (1 + rho_rel * n2), with n1, n2 smoothed unit noise."""
    n1 = smooth_unit_noise(rng, shape, sigma_px)
    n2 = smooth_unit_noise(rng, shape, sigma_px)
    return c_mean + c_dev * n1, rho_mean * (1.0 + rho_rel * n2)


def disc_phantom_2d(seed=1, interior=128, pml=20, h=0.1e-3, Nt=600, n_sensors=256,
                    sensor_radius=5.5e-3, cfl=0.3):
    """2-D homogeneous lossless disc phantom: 128^2 interior at 0.1 mm plus a 20-point PML
    added outside (168^2 total), 256 sensors on a 5.5 mm circle, CFL 0.3, Nt = 600,
    five random discs (radius 0.3-1.5 mm, amplitude U[0.5, 1], centres within 3.5 mm)."""
    rng = np.random.default_rng(seed)
    n = interior + 2 * pml
    shape = (n, n)
    spacing = (h, h)
    c = np.full(shape, 1500.0)
    rho = np.full(shape, 1000.0)
    p0 = discs(rng, shape, spacing, 5, 3.5e-3, (0.3e-3, 1.5e-3), (0.5, 1.0))
    dt = cfl * h / c.max()
    return Problem("disc2d_168", shape, spacing, (pml, pml), 2.0, c, rho, np.zeros(shape), 1.5,
                   dt, Nt, p0, sensor_pos=circle_sensors(n_sensors, sensor_radius), seed=seed)


def vessel_phantom_2d(seed=2, n=512, pml=20, h=0.05e-3, Nt=2000, alpha0=0.75, y=1.5, cfl=0.3,
                      sensor_row=None, n_vessels=6, n_discs=5):
    """2-D heterogeneous absorbing workload: n^2 grid with an internal 20-point PML, smoothed
    random c (1500 +/- 100 m/s) and rho (1000 +/- 5%), alpha0 = 0.75 dB MHz^-1.5 cm^-1, y = 1.5,
    a line of on-grid sensors along the first row inside the PML, vessels plus discs."""
    rng = np.random.default_rng(seed)
    shape = (n, n)
    spacing = (h, h)
    c, rho = heterogeneous_medium(rng, shape)
    a0 = np.full(shape, float(alpha0))
    ves = vessels_2d(rng, shape, n_vessels, margin_px=max(pml + 8, n // 8))
    r_ctr = 0.3 * n * h
    sc = min(1.0, n / 512)
    dsk = discs(rng, shape, spacing, n_discs, r_ctr, (0.3e-3 * sc, 1.5e-3 * sc), (0.5, 1.0))
    p0 = np.maximum(ves, dsk)
    dt = cfl * h / c.max()
    row = pml if sensor_row is None else sensor_row
    idx = row * n + np.arange(n)
    return Problem(f"vessel2d_{n}", shape, spacing, (pml, pml), 2.0, c, rho, a0, y, dt, Nt, p0,
                   sensor_index=idx.astype(np.int64), seed=seed)


def small_lossy_2d(seed=7, shape=(64, 64), pml=8, h=0.1e-3, Nt=120, n_sensors=48, alpha0=0.75,
                   y=1.5, cfl=0.3, sensor_radius_frac=0.3):
    """Small heterogeneous absorbing 2-D case with off-grid circular sensors (for parity tests)."""
    rng = np.random.default_rng(seed)
    spacing = (h, h)
    c, rho = heterogeneous_medium(rng, shape, sigma_px=3.0)
    a0 = np.full(shape, float(alpha0))
    L = min(shape) * h
    p0 = discs(rng, shape, spacing, 4, 0.2 * L, (0.05 * L, 0.12 * L), (0.5, 1.0))
    p0 += 0.1 * rng.standard_normal(shape)  # broadband content exercises every wavenumber
    dt = cfl * h / c.max()
    sens = circle_sensors(n_sensors, sensor_radius_frac * L)
    return Problem(f"small2d_{shape[0]}x{shape[1]}", tuple(shape), spacing, (pml, pml), 2.0, c, rho, a0,
                   y, dt, Nt, p0, sensor_pos=sens, seed=seed)


def small_lossy_3d(seed=8, shape=(24, 32, 40), pml=4, h=0.0625e-3, Nt=60, alpha0=0.75, y=1.5, cfl=0.3,
                   stride=2, plane=None):
    """Small heterogeneous absorbing 3-D case with an on-grid planar sensor array on one face."""
    rng = np.random.default_rng(seed)
    spacing = (h, h, h)
    c, rho = heterogeneous_medium(rng, shape, sigma_px=2.0)
    a0 = np.full(shape, float(alpha0))
    L = min(shape) * h
    p0 = discs(rng, shape, spacing, 3, 0.2 * L, (0.1 * L, 0.2 * L), (0.5, 1.0))
    p0 += 0.1 * rng.standard_normal(shape)
    dt = cfl * h / c.max()
    z = pml if plane is None else plane
    nz, ny, nx = shape
    ys = np.arange(pml, ny - pml, stride)
    xs = np.arange(pml, nx - pml, stride)
    idx = (z * ny + ys[:, None]) * nx + xs[None, :]
    return Problem(f"small3d_{nz}x{ny}x{nx}", tuple(shape), spacing, (pml,) * 3, 2.0, c, rho, a0, y,
                   dt, Nt, p0, sensor_index=idx.ravel().astype(np.int64), seed=seed)


def tube_phantom_3d(seed=3, n=128, pml=10, h=0.0625e-3, Nt=1000, alpha0=0.75, y=1.5, cfl=0.3,
                    sensors=64, stride=2):
    """3-D heterogeneous absorbing workload: n^3, internal PML, tubes plus balls, a planar
    sensors x sensors on-grid array at stride 2 on the face z = pml."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    spacing = (h, h, h)
    c, rho = heterogeneous_medium(rng, shape)
    a0 = np.full(shape, float(alpha0))
    p0 = np.maximum(tubes_3d(rng, shape, 4, margin_px=pml + 6),
                    discs(rng, shape, spacing, 3, 0.25 * n * h, (0.2e-3, 0.6e-3), (0.5, 1.0)))
    dt = cfl * h / c.max()
    lo = (n - stride * sensors) // 2
    ys = lo + stride * np.arange(sensors)
    xs = lo + stride * np.arange(sensors)
    idx = (pml * n + ys[:, None]) * n + xs[None, :]
    return Problem(f"tube3d_{n}", shape, spacing, (pml,) * 3, 2.0, c, rho, a0, y, dt, Nt, p0,
                   sensor_index=idx.ravel().astype(np.int64), seed=seed)


def smooth_even_size(n):
    """The smallest even size >= n whose prime factors are 2, 3, 5 and 7 (the FFT radices)."""
    m = int(n) + (int(n) % 2)
    while True:
        k = m
        for f in (2, 3, 5, 7):
            while k % f == 0:
                k //= f
        if k == 1:
            return m
        m += 2


def refined_problem(pb, ratio=1.44, map_snr_db=35.0, seed=0):
    """Data-generation problem for the reconstruction problem ``pb`` that avoids the inverse crime,
    a stand-in for the data grid of Sec. VI.A (data on 472^2 for a 328^2 reconstruction, maps
    contaminated with 35 dB AWGN):
      - about ``ratio`` times as many points per axis over the same physical extent (even sizes with
        factors 2, 3, 5, 7);
      - the PML scaled by the ratio;
      - sound speed, density, alpha0 and p0 linearly interpolated onto the finer grid (clamped at the
        ends);
      - the sound-speed and density maps contaminated with AWGN at ``map_snr_db`` (None: none);
      - the sensors at the same physical positions (off-grid points);
      - the same dt and Nt, so the data are directly comparable."""
    rng = np.random.default_rng(seed)
    d = pb.ndim
    shape_f = tuple(smooth_even_size(round(n * ratio)) for n in pb.shape)
    spacing_f = tuple(n * h / nf for n, h, nf in zip(pb.shape, pb.spacing, shape_f))
    pml_f = tuple(int(round(p * nf / n)) for p, n, nf in zip(pb.pml, pb.shape, shape_f))
    xc = coords(pb.shape, pb.spacing)
    xf = coords(shape_f, spacing_f)

    def interp(a):
        a = np.broadcast_to(np.asarray(a, dtype=float), pb.shape)
        for ax in range(d):
            a = np.apply_along_axis(lambda v: np.interp(xf[ax], xc[ax], v), ax, a)
        return np.ascontiguousarray(a)

    c_f, rho_f = interp(pb.c), interp(pb.rho)
    if map_snr_db is not None:
        c_f = awgn(rng, c_f, map_snr_db)
        rho_f = awgn(rng, rho_f, map_snr_db)
    if pb.sensor_pos is not None:
        pos = np.array(pb.sensor_pos, dtype=float)
    else:
        idx = np.unravel_index(np.asarray(pb.sensor_index), pb.shape)
        pos = np.stack([xc[a][idx[a]] for a in range(d)][::-1], axis=1)   # (x, y[, z]) order
    return Problem(f"{pb.name}_refined_{'x'.join(map(str, shape_f))}", shape_f, spacing_f, pml_f, pb.pml_alpha,
                   c_f, rho_f, interp(pb.alpha0), pb.y, pb.dt, pb.Nt, interp(pb.p0), sensor_pos=pos, seed=seed)


def random_residual(seed, Nt, Ns):
    """A seeded random data-space vector (adjoint input for dot tests)."""
    return np.random.default_rng(seed).standard_normal((Nt, Ns))


def random_image(seed, shape):
    """A seeded random image-space vector."""
    return np.random.default_rng(seed).standard_normal(shape)
