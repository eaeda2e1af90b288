"""FP64 CPU oracle of the paper's own adjoint: "adjoint-then-discretize" (Sec. VI), i.e. the
continuous adjoint system of Sec. III, Eqs. (moma), (massa), (statea), (initial2), (adjj),
discretised with the same k-space staggered scheme as the forward operator.

TEST INFRASTRUCTURE ONLY (as ``pat_oracle``): imported by ``tests/`` alone; the product path never
calls it.

The library's adjoint is the exact transpose of the discrete forward map (reading R7 of
``pat_oracle``).  The paper instead discretised the continuous adjoint; this module computes that
alternative so that its deviation from the transpose can be stated and measured.

Readings (A1-A4):

A1  Continuous system, forward in the adjoint time t (data reversed, h~(t) = h(T - t)):
        du*/dt = -(1/rho0) grad p*,
        drho*/dt = rho0 (-div u* + w h~),
        p* = rho0 {q - (-lap)^(y/2-1) tau dq/dt - (-lap)^((y-1)/2) eta q},  q = c0^2 rho* / rho0,
    zero initial state, and P*[h] = rho*(T) / rho0.  In the state equation tau and eta act before
    the fractional Laplacians (the reverse of the forward Eq. (state)); dq/dt is taken from the
    mass equation, dq/dt = c0^2 (-div u* + w h~).
A2  Discretisation: the leapfrog of reading R6 with split fields and the same PML factors,
        u*^{n+1/2} = au (au u*^{n-1/2} - dt b D+ p*^n),  e* = D- u*^{n+1/2},
        rho*_xi^{n+1} = a (a rho*_xi^n - dt rho0 e*_xi + dt rho0 s / d),
        s = M^T (h~^n + h~^{n+1}) / 2     (the source at the half step, shared equally by the d
                                           split components),
        p*^{n+1} = rho0 [q - L_{y-2}(tau c0^2 (-sum e* + s)) - L_{y-1}(eta q)],  q = c0^2 sum rho* / rho0,
    for n = 0 .. Nt-2 with h~^n = h^{Nt-1-n}; the result is sum_xi rho*_xi^{Nt-1} / rho0.
A3  Scaling: the data inner product is a plain sum over samples and sensors (reading C9), so
    <H x, h> = (1/dt) int P[x] h dt + O(dt) and the transpose satisfies dt H^T h -> P*[h] (with
    the point sensors' w as the grid weights M^T, image sums on both sides).  The comparison is
    therefore between ``adjoint_then_discretize(op, h)`` and dt * op.adjoint(h).
A4  PML: the damping is symmetric in space and time-independent, so the adjoint system is damped
    by the same split-field factors.  The split differs from the transpose's inside the layer: in
    the transpose every split density adjoint receives the whole divergence (the adjoint of
    p = c0^2 sum rho_xi), here each receives its own component, as in the forward system.  Outside
    the layer the split components stay equal and the two coincide.
A5  Initial state.  P*[h] = rho*(T) / rho0 (Eq. (adjj)) is the gradient for the initial condition
    of Sec. III, c0^2 {1 - eta (-lap)^((y-1)/2)} rho(0) = p0.  The forward operator instead takes
    rho^0 = p0 / (d c0^2) (reading R5), whose gradient is lambda(T) / c0^2 with
    lambda = q - (-lap)^((y-1)/2) (eta q) at T; the two differ by O(alpha0).  ``initial="paper"``
    returns the former, ``initial="R5"`` (the default) the latter, which is the continuous limit
    of the transpose.
"""
from __future__ import annotations

import numpy as np

from .pat_oracle import Operator, smooth_image


def adjoint_then_discretize(op: Operator, h, initial="R5"):
    """The discretised continuous adjoint (readings A1-A5), image shape."""
    if initial not in ("R5", "paper"):
        raise ValueError("initial must be 'R5' or 'paper'")
    d, dt = op.d, op.dt
    h = np.asarray(h, dtype=float).reshape(op.Nt, op.Ns)
    ht = h[::-1]                                   # h~^n = h^{Nt-1-n}
    tau = op.c2tau / op.c2                         # tau and eta of Eq. (Twelve)
    eta = op.c2eta / op.c2
    u = [np.zeros(op.shape) for _ in range(d)]
    rho = [np.zeros(op.shape) for _ in range(d)]
    p = np.zeros(op.shape)
    for n in range(op.Nt - 1):
        u = [op.au[a] * (op.au[a] * u[a] - dt * op.b[a] * op.Dplus(a, p)) for a in range(d)]
        e = [op.Dminus(a, u[a]) for a in range(d)]
        s = op.scatter(0.5 * (ht[n] + ht[n + 1]))
        rho = [op.a[a] * (op.a[a] * rho[a] - dt * op.rho0 * e[a] + dt * op.rho0 * s / d) for a in range(d)]
        q = op.c2 * sum(rho) / op.rho0
        p = q
        if op.lossy:
            qdot = op.c2 * (s - sum(e))
            p = q - op.ks.apply(op.Ly2, tau * qdot) - op.ks.apply(op.Ly1, eta * q)
        p = op.rho0 * p
    g = sum(rho) / op.rho0                                       # Eq. (adjj)
    if initial == "R5" and op.lossy:
        q = op.c2 * g
        g = (q - op.ks.apply(op.Ly1, eta * q)) / op.c2              # reading A5
    return smooth_image(g, op.spacing) if op.smooth else g   # (H S)^T = S H^T (reading R9)
