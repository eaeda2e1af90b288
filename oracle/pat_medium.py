"""Oracle: gradients of the forward map with respect to the squared sound speed c0^2 and the
ambient density rho0 (FP64, CPU).

TEST INFRASTRUCTURE.  Like the rest of ``oracle/``, this module is imported only by the tests,
by the smoke check and by the CPU-baseline leg of the benchmark; the library never calls it.

What it computes (the medium-sensitivity extension of Sec. III's adjoint, in the setting of the
joint sound-speed reconstruction that Sec. VII motivates): for J(c0^2) = <H_{c0^2} p0, h>, the
exact derivative of the DISCRETE forward map of ``pat_oracle.Operator`` with respect to c0^2 at
every grid point.  Readings (the paper gives no medium gradient):

M1  Held fixed: alpha0 (the power-law prefactor of Eq. (Twelve)), y, rho0, the reference speed
    c_ref (so kappa, the PML profile and dt do not move) and p0.
M2  tau and eta follow c0 through Eq. (Twelve): c0^2 tau ~ (c0^2)^((y+1)/2) and
    c0^2 eta ~ (c0^2)^((y+2)/2), so the explicit derivative of the equation of state
        p = c0^2 r + c0^2 tau L_{y-2} dd - c0^2 eta L_{y-1} r
    at a time level is
        q = r + (y+1)/2 tau L_{y-2} dd - (y+2)/2 eta L_{y-1} r       (q = r when lossless).
M3  The initial density rho_xi^0 = p0 / (d c0^2) (reading R5) contributes
        -p0 / (d c0^4) * sum_xi rho_bar_xi
    with rho_bar_xi the adjoint of rho_xi^0.

Adjoint-state form: g = sum_{n=1}^{Nt-1} p_bar^n * q^n + M3's term, where p_bar^n is the total
adjoint of p^n -- the value ``Operator.adjoint`` holds after processing time level n.  This
module stores every q^n (no checkpointing: plain and slow); the library recomputes them from
checkpoints.

Pins (tests/test_oracle_medium.py): central finite differences of J on heterogeneous absorbing
and lossless media with PML, 2-D and 3-D; and a closed form for the uniform perturbation of a
homogeneous lossless periodic medium, where p^n = F^-1{cos(n w_k) F p0} with
2 - 2 cos w_k = (c0 dt kappa |k|)^2.
"""
import numpy as np

from .pat_oracle import Operator, smooth_image


def operator_with_c_ref(pb, c, c_ref):
    """``Operator.from_problem(pb)`` with sound speed ``c`` but the reference speed (kappa, PML,
    dt) of the unperturbed medium (reading M1); used to difference J in c0^2."""
    from .pat_oracle import KSpace, pml_factors

    op = Operator(pb.shape, pb.spacing, pb.pml, pb.pml_alpha, c, pb.rho, pb.alpha0, pb.y, pb.dt, pb.Nt,
                  sensor_pos=pb.sensor_pos, sensor_index=pb.sensor_index, smooth=getattr(pb, "smooth", False))
    # rebuild the pieces that depend on the reference speed with the fixed one

    op.c_ref = float(c_ref)
    op.ks = KSpace(op.shape, op.spacing, op.c_ref, op.dt)
    op.Ly2 = op.ks.kpow(pb.y - 2.0)
    op.Ly1 = op.ks.kpow(pb.y - 1.0)
    op.a, op.au = [], []
    for a in range(op.d):
        fa, fau = pml_factors(op.shape[a], int(pb.pml[a]), pb.pml_alpha, op.c_ref, op.spacing[a], op.dt)
        bshape = [1] * op.d
        bshape[a] = -1
        op.a.append(fa.reshape(bshape))
        op.au.append(fau.reshape(bshape))
    return op


def forward_with_q(op: Operator, p0, y):
    """Forward solve of ``op`` returning (data, q) with q[n] = d p^n / d c0^2 (explicit, M2),
    q[0] = 0 (p^0 = p0)."""
    d, dt = op.d, op.dt
    c2 = op.c2
    tau = op.c2tau / c2
    eta = op.c2eta / c2
    p = np.array(p0, dtype=float)
    data = np.zeros((op.Nt, op.Ns))
    q = np.zeros((op.Nt,) + op.shape)
    rho = [p / (d * c2) for _ in range(d)]
    u = [0.5 * dt * op.b[a] * op.Dplus(a, p) for a in range(d)]
    data[0] = op.gather(p)
    for n in range(op.Nt - 1):
        g = [op.Dplus(a, p) for a in range(d)]
        u = [op.au[a] * (op.au[a] * u[a] - dt * op.b[a] * g[a]) for a in range(d)]
        e = [op.Dminus(a, u[a]) for a in range(d)]
        rho = [op.a[a] * (op.a[a] * rho[a] - dt * op.rho0 * e[a]) for a in range(d)]
        dd = op.rho0 * sum(e)
        r = sum(rho)
        p = op.pressure(r, dd)
        qn = np.array(r)
        if op.lossy:
            qn = qn + 0.5 * (y + 1.0) * tau * op.ks.apply(op.Ly2, dd) - 0.5 * (y + 2.0) * eta * op.ks.apply(op.Ly1, r)
        q[n + 1] = qn
        data[n + 1] = op.gather(p)
    return data, q


def sound_speed_gradient(op: Operator, p0, h, y):
    """g = dJ/d(c0^2), J = <H p0, h> (readings M1-M3).  Returns (g, grad_p0) where grad_p0 is
    the ordinary adjoint H^T h (the same sweep)."""
    d, dt = op.d, op.dt
    h = np.asarray(h, dtype=float).reshape(op.Nt, op.Ns)
    p0 = op.initial_pressure(p0)      # S p0 when the smoothing of R9 is on (S does not depend on c0)
    _, q = forward_with_q(op, p0, y)
    g = np.zeros(op.shape)
    pbar = op.scatter(h[op.Nt - 1])
    if op.Nt > 1:
        g += pbar * q[op.Nt - 1]
    ubar = [np.zeros(op.shape) for _ in range(d)]
    rhobar = [np.zeros(op.shape) for _ in range(d)]
    for n in range(op.Nt - 2, -1, -1):
        rbar = op.c2 * pbar
        ddbar = np.zeros(op.shape)
        if op.lossy:
            rbar = rbar - op.ks.apply(op.Ly1, op.c2eta * pbar)
            ddbar = op.ks.apply(op.Ly2, op.c2tau * pbar)
        ebar = []
        for a in range(d):
            rhobar[a] = rhobar[a] + rbar
            ebar.append(op.rho0 * ddbar - dt * op.rho0 * op.a[a] * rhobar[a])
            rhobar[a] = op.a[a] ** 2 * rhobar[a]
        gbar = []
        for a in range(d):
            ubar[a] = ubar[a] - op.Dplus(a, ebar[a])
            gbar.append(-dt * op.b[a] * op.au[a] * ubar[a])
            ubar[a] = op.au[a] ** 2 * ubar[a]
        pbar = -sum(op.Dminus(a, gbar[a]) for a in range(d)) + op.scatter(h[n])
        if n >= 1:
            g += pbar * q[n]      # p_bar^n: total adjoint of p^n
    g += -np.asarray(p0, float) / (d * op.c2 * op.c2) * sum(rhobar)     # M3
    grad_p0 = pbar + sum(rhobar) / (d * op.c2)
    grad_p0 = grad_p0 - sum(op.Dminus(a, 0.5 * dt * op.b[a] * ubar[a]) for a in range(d))
    if op.smooth:
        grad_p0 = smooth_image(grad_p0, op.spacing)
    return g, grad_p0


def objective(pb, c2, h, c_ref):
    """J(c0^2) = <H_{c0^2} p0, h> with the reference speed held at ``c_ref`` (M1)."""
    op = operator_with_c_ref(pb, np.sqrt(c2), c_ref)
    return float(np.sum(op.forward(pb.p0) * h))


def homogeneous_uniform_derivative(shape, spacing, c0, dt, Nt, p0, weights):
    """Closed form of d/dc0^2 (uniform) of sum_n <weights[n], p^n> for a homogeneous lossless
    periodic medium without PML: p^n = F^-1{cos(n w) F p0}, cos w = 1 - (c0^2 dt^2 kappa^2 |k|^2)/2,
    kappa = sinc(c0 |k| dt / 2) with c_ref = c0 fixed, so dw/dc0^2 = (dt^2 kappa^2 |k|^2 / 2) / sin w
    and d p^n / dc0^2 = F^-1{-n sin(n w) dw/dc0^2 F p0} (w = 0 at k = 0 contributes nothing)."""
    d = len(shape)
    ks = [2.0 * np.pi * np.fft.fftfreq(n, h) for n, h in zip(shape, spacing)]
    grids = np.meshgrid(*ks, indexing="ij")
    k2 = sum(g * g for g in grids)
    km = np.sqrt(k2)
    kappa = np.sinc(c0 * km * dt / (2.0 * np.pi))
    s2 = (c0 * dt * kappa * km) ** 2
    w = np.arccos(1.0 - 0.5 * s2)
    sw = np.sin(w)
    dw = np.where(sw > 0, 0.5 * dt * dt * kappa * kappa * k2 / np.where(sw > 0, sw, 1.0), 0.0)
    P0 = np.fft.fftn(p0)
    total = 0.0
    for n in range(Nt):
        dpn = np.real(np.fft.ifftn(-n * np.sin(n * w) * dw * P0))
        total += float(np.sum(weights[n] * dpn))
    return total


# ---------------------------------------------------------------------------------------------
# Gradient with respect to the ambient density rho0 (readings D1-D3)
# ---------------------------------------------------------------------------------------------
# D1  Held fixed: c0, alpha0, y, the reference speed (kappa, PML, dt) and p0; tau and eta depend on
#     c0 and alpha0 only (Eq. (Twelve)), so the equation of state does not move.
# D2  rho0 enters the discrete step in three places: b_xi = 2 / (rho0 + rho0 shifted by one point
#     along xi) in the u update and in u^(-1/2) = dt/2 b D+ p0 (readings R4, R5); -dt rho0 e_xi in the
#     density update; and dd = rho0 sum e_xi in the absorption term (Sec. II.A).
# D3  Adjoint-state form, with the adjoint variables of Operator.adjoint: per step n,
#         dJ/db_xi   += u_bar_xi^{n+1/2} (-dt au_xi g_xi^n),  g^n = D+ p^n,
#         dJ/drho0   += sum_xi e_xi^n (dd_bar - dt a_xi rho_bar_xi^{n+1}),  e^n = D- u^{n+1/2},
#     plus dJ/db_xi += u_bar_xi^{-1/2} dt/2 D+_xi p0 for the initial state; then through b_xi,
#     db_xi[j] / drho0[j] = db_xi[j] / drho0[j+1] = -b_xi[j]^2 / 2.
# Pins (tests/test_oracle_medium.py): central finite differences of J in random directions of
# rho0 (2-D absorbing with PML, 2-D lossless, 3-D), and the scaling invariant: J(lambda rho0) =
# J(rho0) for every lambda > 0 (u scales as 1/lambda, the density and the pressure do not move),
# hence <dJ/drho0, rho0> = 0 for every medium.


def forward_with_fields(op: Operator, p0):
    """Forward solve of ``op`` returning (data, g, e) with g[n][xi] = D+_xi p^n and
    e[n][xi] = D-_xi u_xi^{n+1/2} for the steps n = 0 .. Nt-2 (D3)."""
    d, dt = op.d, op.dt
    p = np.array(p0, dtype=float)
    data = np.zeros((op.Nt, op.Ns))
    G, E = [], []
    rho = [p / (d * op.c2) for _ in range(d)]
    u = [0.5 * dt * op.b[a] * op.Dplus(a, p) for a in range(d)]
    data[0] = op.gather(p)
    for n in range(op.Nt - 1):
        g = [op.Dplus(a, p) for a in range(d)]
        u = [op.au[a] * (op.au[a] * u[a] - dt * op.b[a] * g[a]) for a in range(d)]
        e = [op.Dminus(a, u[a]) for a in range(d)]
        rho = [op.a[a] * (op.a[a] * rho[a] - dt * op.rho0 * e[a]) for a in range(d)]
        dd = op.rho0 * sum(e)
        p = op.pressure(sum(rho), dd)
        G.append(g)
        E.append(e)
        data[n + 1] = op.gather(p)
    return data, G, E


def density_gradient(op: Operator, p0, h):
    """g = dJ/drho0, J = <H p0, h> (readings D1-D3)."""
    d, dt = op.d, op.dt
    h = np.asarray(h, dtype=float).reshape(op.Nt, op.Ns)
    p0 = op.initial_pressure(p0)      # S p0 when the smoothing of R9 is on (S does not depend on rho0)
    _, G, E = forward_with_fields(op, p0)
    g_rho = np.zeros(op.shape)
    g_b = [np.zeros(op.shape) for _ in range(d)]
    pbar = op.scatter(h[op.Nt - 1])
    ubar = [np.zeros(op.shape) for _ in range(d)]
    rhobar = [np.zeros(op.shape) for _ in range(d)]
    for n in range(op.Nt - 2, -1, -1):
        rbar = op.c2 * pbar
        ddbar = np.zeros(op.shape)
        if op.lossy:
            rbar = rbar - op.ks.apply(op.Ly1, op.c2eta * pbar)
            ddbar = op.ks.apply(op.Ly2, op.c2tau * pbar)
        ebar = []
        for a in range(d):
            rhobar[a] = rhobar[a] + rbar          # adjoint of rho_xi^{n+1}
            g_rho += E[n][a] * (ddbar - dt * op.a[a] * rhobar[a])
            ebar.append(op.rho0 * ddbar - dt * op.rho0 * op.a[a] * rhobar[a])
            rhobar[a] = op.a[a] ** 2 * rhobar[a]
        gbar = []
        for a in range(d):
            ubar[a] = ubar[a] - op.Dplus(a, ebar[a])   # adjoint of u_xi^{n+1/2}
            g_b[a] += ubar[a] * (-dt * op.au[a] * G[n][a])
            gbar.append(-dt * op.b[a] * op.au[a] * ubar[a])
            ubar[a] = op.au[a] ** 2 * ubar[a]
        pbar = -sum(op.Dminus(a, gbar[a]) for a in range(d)) + op.scatter(h[n])
    for a in range(d):
        g_b[a] += ubar[a] * (0.5 * dt * op.Dplus(a, p0))    # u^(-1/2) = dt/2 b D+ p0
        B = g_b[a] * (-0.5 * op.b[a] ** 2)
        g_rho += B + np.roll(B, 1, axis=a)                   # b_xi[j] depends on rho0[j], rho0[j+1]
    return g_rho


def density_objective(pb, rho, h):
    """J(rho0) = <H_{rho0} p0, h> with everything else of ``pb`` fixed (D1)."""
    op = Operator(pb.shape, pb.spacing, pb.pml, pb.pml_alpha, pb.c, rho, pb.alpha0, pb.y, pb.dt, pb.Nt,
                  sensor_pos=pb.sensor_pos, sensor_index=pb.sensor_index, smooth=getattr(pb, "smooth", False))
    return float(np.sum(op.forward(pb.p0) * h))
