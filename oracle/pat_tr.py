"""FP64 CPU oracle of time-reversal (TR) reconstruction (Sec. II.B.1), the paper's comparison
baseline and a warm start for the iterative methods.

TEST INFRASTRUCTURE ONLY (as ``pat_oracle``): imported by ``tests/`` alone.

Sec. II.B.1 enforces the measured pressure as a Dirichlet condition at the sensors in reversed
time, p_tr(r_s, t) = p_m(r_s, T - t), runs the acoustic system from a zero state and reads the
image at the end; to compensate absorption, the sign of the absorption term of Eq. (state) is
reversed and the dispersion term kept.  Readings (T1-T4):

T1  The scheme is the forward one (readings R1-R6 of ``pat_oracle``) with tau replaced by -tau
    (eta unchanged), on the same grid, PML, time step and reference speed.
T2  Sensors must lie on grid nodes (the Dirichlet condition needs nodes): on-grid sensor indices;
    off-grid positions are rejected.
T3  Start: p^0 = 0 except p^0 = p_m^{Nt-1} at the sensors, rho_xi^0 = p^0 / (d c0^2), u^{-1/2} = 0.
    Step n (n = 0 .. Nt-2): the updates of R6; then at the sensor nodes the split densities are
    reset to p_m^{Nt-2-n} / (d c0^2) and the pressure to p_m^{Nt-2-n}, so the enforced value holds
    exactly whatever the absorption terms give there.
T4  The image is p after the last step (reversed time T, original time 0).  Each node carries
    one sensor: repeated nodes are rejected.
T5  With the sign reversed, the absorption term amplifies each mode at the rate the forward
    model damped it, and that rate grows like |k|^y: rounding noise at high |k| grows without
    bound over a run (measured: 1e5 times the image at alpha0 = 5 dB MHz^-y cm^-1 on a 96^2 grid).
    The paper gives no remedy.  Reading: the reversed absorption term is band-limited by the
    radial Blackman window of reading R9 with its cut-off at ``k_cut`` (default one half) of
    the Nyquist radius; above it the modes propagate without absorption.
"""
from __future__ import annotations

import numpy as np

from .pat_oracle import Operator


def time_reversal(op: Operator, data, compensate=True, k_cut=0.5):
    """TR image from data [Nt][Ns] recorded at on-grid sensors (readings T1-T5).  With
    ``compensate`` False the absorption keeps its forward sign (for comparison)."""
    d, dt = op.d, op.dt
    data = np.asarray(data, dtype=float).reshape(op.Nt, op.Ns)
    M = op.M.tocsr()
    if not (np.all(M.getnnz(axis=1) == 1) and np.allclose(M.data, 1.0)):
        raise ValueError("time reversal needs sensors on grid nodes")
    nodes = M.indices.copy()                         # flat node index of each sensor
    if len(np.unique(nodes)) != len(nodes):
        raise ValueError("time reversal needs one sensor per node")
    Ly2 = op.Ly2
    if compensate:
        q = op.ks.kmag / (k_cut * min(np.pi / hh for hh in op.spacing))
        window = np.where(q < 1.0, 0.42 + 0.5 * np.cos(np.pi * q) + 0.08 * np.cos(2.0 * np.pi * q), 0.0)
        Ly2 = -op.Ly2 * window                        # reversed sign, band-limited (T1, T5)

    def enforce(p, rho, row):
        pf = p.reshape(-1)
        pf[nodes] = row
        for a in range(d):
            rf = rho[a].reshape(-1)
            rf[nodes] = row / (d * op.c2.reshape(-1)[nodes])

    p = np.zeros(op.shape)
    rho = [np.zeros(op.shape) for _ in range(d)]
    u = [np.zeros(op.shape) for _ in range(d)]
    enforce(p, rho, data[op.Nt - 1])
    for n in range(op.Nt - 1):
        g = [op.Dplus(a, p) for a in range(d)]
        u = [op.au[a] * (op.au[a] * u[a] - dt * op.b[a] * g[a]) for a in range(d)]
        e = [op.Dminus(a, u[a]) for a in range(d)]
        rho = [op.a[a] * (op.a[a] * rho[a] - dt * op.rho0 * e[a]) for a in range(d)]
        dd = op.rho0 * sum(e)
        r = sum(rho)
        p = op.c2 * r
        if op.lossy:
            p = p + op.c2tau * op.ks.apply(Ly2, dd) - op.c2eta * op.ks.apply(op.Ly1, r)
        enforce(p, rho, data[op.Nt - 2 - n])
    return p
