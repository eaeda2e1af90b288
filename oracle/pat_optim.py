"""FP64 CPU oracle for the optimisation shell around H: TV, its proximal map, smoothed TV,
grid transfer, bound-constraint restriction, ISTA / FISTA and the line-search multi-grid
FISTA of Javaherian & Holman (arXiv:1603.02329), Sec. IV and Sec. V.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg, never by the product path.

Readings where the paper is silent (all listed here):

O1  TV is isotropic with forward differences and a zero difference at the last index
    (Neumann): TV(x) = sum_i sqrt(sum_xi (D_xi x)_i^2)  (Sec. II.B "total variation").
O2  The TV proximal map of Sec. IV Eq. (proxmal) with g = lambda TV + indicator(x >= 0) is
    computed by the dual fast-gradient-projection approach cited there: dual variable q with
    |q_i| <= 1, x(q) = max(0, z - lam' D^T q), lam' = alpha lambda, projected ascent step
    1 / (4 d lam') with Nesterov momentum, zero warm start, a fixed inner count n_tv.
O3  Smoothed TV, Sec. V.B Eq. (Thirty-two): J_rho(y) = sum_i (sqrt(|D y|_i^2 + rho^2) - rho),
    the "- rho" taken per point, so J_rho -> TV as rho -> 0; gradient per Eq. (Twentyone):
    D^T (D y / sqrt(|D y|^2 + rho^2)).
O4  Prolongation P (coarse -> fine) is tensor-product linear interpolation: fine 2i <- coarse i,
    fine 2i+1 <- (coarse i + coarse i+1)/2, the last fine index clamps to the last coarse value;
    restriction R = 2^-d P^T (full weighting).  Sec. V.A names I_h^{h-1}, I_{h-1}^h only.
O5  Bound restriction, Sec. V.C Eq. (constraint): phi_i = (R y)_i - min_{j in {2i-1,2i,2i+1}^d} y_j
    (indices clamped), evaluated at y_{h,k} (where the transfer happens, Sec. V.C last sentence).
O6  Coarse level: n/2 points, spacing 2h, PML/2 points, dt_c = 2 dt, Nt_c = ceil(Nt/2)
    (Sec. V: the time step follows the spacing), medium decimated (c_c = c[::2, ::2]), sensors at
    the same physical positions, data decimated in time (p_hat_c = p_hat[::2]).  A position
    beyond the first or last coarse node (a fine sensor on the last fine index) is clamped onto
    that node, as P clamps at the last index.  When the fine operator smooths p0 (reading R9 of
    the forward oracle), the coarse one applies its own window, cut at its own Nyquist radius.
O7  Coarse iteration: FISTA (or ISTA) on phi_{h-1} with projection on {x >= phi} (Sec. V.E),
    step 1 / L_c, L_c = w L(H_c^T H_c) + lambda 4 d / rho (w of O11); its own t-sequence from 1; stop when
    (phi_k - phi_{k+1}) / max(|phi_k|, |phi_{k+1}|) < eps_c or after q_c iterations (the paper's
    denominator carries F_h subscripts and phi may be negative: absolute coarse values are used).
O8  Momentum: theta follows the FISTA t-rule every fine iteration whatever the branch; ISTA has
    theta = 0 (Sec. IV, Alg. 2 remark).  Fine stop (Sec. V.E): (F_k - F_{k+1}) / max(F_k, F_{k+1})
    < eps_d, or max_iter, or RE <= target_re (benchmark mode).
O9  Cost-saving identity: H y_{k+1} = (1 + theta) H x_k - theta H x_{k-1} (H linear), so each fine
    iteration runs one forward (for F(x_k)) and one adjoint (for grad f(y_k)).
O10 Power iteration (Sec. IV, Sec. VI.A): v <- H^T H v / ||H^T H v|| from a seeded N(0,1) start;
    L = ||H^T H v|| at the last iteration (30 by default).
O11 Weight of the coarse data term (Eq. (Fourteen) writes the coarse objective with the same
    1/2 ||H x - p||^2 as the fine one; the weight of the coarse copy is not discussed):
    phi_{h-1} = w/2 ||H_c x - p_c||^2 + lambda J_rho + <v, x> with w = 2^(1-d).  Reason: with
    R = 2^-d P^T (O4) the Galerkin model of the fine data term is R (H^T H) P = 2^-d P^T H^T H P,
    while H_c ~ (decimate in time) H P gives H_c^T H_c ~ 1/2 P^T H^T H P, i.e. 2^(d-1) times stiffer;
    unweighted, the coarse minimiser under-shoots the correction by that factor.  v (first-order
    coherence) and L_c use the same w.  On a 128^2 line-array case (40 dB noise), MG-FISTA with
    w = 1 gains a few iterations at the start only; with w = 1/2 it reaches in 3 iterations the RE
    that FISTA reaches in 10.
O12 More than two levels (the paper states Alg. 3 for two grids; Sec. V.E).  A coarse level l >= 1
    minimises phi_l = w_l/2 ||H_l x - p_l||^2 + lambda J_rho(x) + <v_l, x> on {x >= b_l} by the
    projected FISTA of O7, and when a level l + 1 exists, an iteration k > 1 of it takes a
    recursive direction under the test of Sec. V.D applied to phi_l (its own y~, K_r, K_d):
    x_{l+1,0} = R y, v_{l+1} = R grad phi_l(y) - grad(w_{l+1}/2 ||H_{l+1} x - p_{l+1}||^2 +
    lambda J_rho)(x_{l+1,0}) (first-order coherence with phi_l), the bound restricted from b_l as
    b_{l+1} = R y - min_{j in the fine neighbourhood} (y - b_l)_j (Eq. (constraint) for a bound
    b_l in place of 0, so that y + P(x_{l+1} - x_{l+1,0}) >= b_l whenever x_{l+1} >= b_{l+1}),
    and x = y + P(x_{l+1,*} - x_{l+1,0}).  Data decimate by 2 in time per level (O6); the data
    weight compounds, w_l = (2^(1-d))^l (O11 per level step); L_l = w_l L(H_l^T H_l) +
    lambda 4 d / rho.  With one coarse level this is O7 exactly.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

from .pat_oracle import Operator


# ---------------------------------------------------------------------------------------------
# TV pieces (O1-O3)
# ---------------------------------------------------------------------------------------------

def grad_fwd(x):
    """D x: forward differences per numpy axis, zero at the last index (O1)."""
    out = []
    for a in range(x.ndim):
        g = np.zeros_like(x)
        sl_lo = [slice(None)] * x.ndim
        sl_hi = [slice(None)] * x.ndim
        sl_lo[a] = slice(0, -1)
        sl_hi[a] = slice(1, None)
        g[tuple(sl_lo)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
        out.append(g)
    return out


def grad_fwd_T(q):
    """D^T q (= -div q), the exact transpose of ``grad_fwd``."""
    x = np.zeros_like(q[0])
    nd = x.ndim
    for a in range(nd):
        sl_lo = [slice(None)] * nd
        sl_hi = [slice(None)] * nd
        sl_lo[a] = slice(0, -1)
        sl_hi[a] = slice(1, None)
        qa = q[a]
        # <D x, q> = sum_{i<n-1} (x[i+1] - x[i]) q[i]
        x[tuple(sl_hi)] += qa[tuple(sl_lo)]
        x[tuple(sl_lo)] -= qa[tuple(sl_lo)]
    return x


def tv(x):
    """Isotropic TV (O1)."""
    g = grad_fwd(x)
    return float(np.sum(np.sqrt(sum(ga * ga for ga in g))))


def tv_smooth(x, rho):
    """J_rho of Sec. V.B Eq. (Thirty-two) (O3)."""
    g = grad_fwd(x)
    return float(np.sum(np.sqrt(sum(ga * ga for ga in g) + rho * rho) - rho))


def tv_smooth_grad(x, rho):
    """Gradient of J_rho: D^T (D x / sqrt(|D x|^2 + rho^2)) (Sec. V.B Eq. (Twentyone)) (O3)."""
    g = grad_fwd(x)
    nrm = np.sqrt(sum(ga * ga for ga in g) + rho * rho)
    return grad_fwd_T([ga / nrm for ga in g])


def project_unit_ball(q):
    """Pointwise projection of the dual field onto |q_i| <= 1 (isotropic)."""
    nrm = np.sqrt(sum(qa * qa for qa in q))
    s = 1.0 / np.maximum(1.0, nrm)
    return [qa * s for qa in q]


def tv_prox(z, lam_eff, n_inner=20, nonneg=True, return_dual=False):
    """argmin_x lam_eff TV(x) + indicator(x >= 0) + 1/2 ||x - z||^2 by FGP (Sec. IV Eq. (proxmal); O2).

    ``lam_eff`` = alpha * lambda.  Returns x (and the final dual q if ``return_dual``)."""
    z = np.asarray(z, dtype=float)
    d = z.ndim
    proj = (lambda v: np.maximum(v, 0.0)) if nonneg else (lambda v: v)
    if lam_eff <= 0.0:
        x = proj(z)
        return (x, [np.zeros_like(z) for _ in range(d)]) if return_dual else x
    step = 1.0 / (4.0 * d * lam_eff)
    q_prev = [np.zeros_like(z) for _ in range(d)]
    r = [np.zeros_like(z) for _ in range(d)]
    t = 1.0
    for _ in range(n_inner):
        x = proj(z - lam_eff * grad_fwd_T(r))
        gx = grad_fwd(x)
        q = project_unit_ball([ra + step * ga for ra, ga in zip(r, gx)])
        t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        w = (t - 1.0) / t_next
        r = [qa + w * (qa - qp) for qa, qp in zip(q, q_prev)]
        q_prev, t = q, t_next
    x = proj(z - lam_eff * grad_fwd_T(q_prev))
    return (x, q_prev) if return_dual else x


def tv_prox_gap(z, lam_eff, x, q):
    """Duality gap certificate of the prox problem at the primal-dual pair (x(q), q):
    lam_eff * (TV(x) - <q, D x>) >= 0, zero exactly at the optimum (O2)."""
    gx = grad_fwd(x)
    return lam_eff * (tv(x) - float(sum(np.sum(qa * ga) for qa, ga in zip(q, gx))))


# ---------------------------------------------------------------------------------------------
# Grid transfer and constraint restriction (O4, O5)
# ---------------------------------------------------------------------------------------------

def _prolong_axis(xc, a):
    nc = xc.shape[a]
    nf = 2 * nc
    shp = list(xc.shape)
    shp[a] = nf
    xf = np.zeros(shp)
    take = lambda arr, idx: np.take(arr, idx, axis=a)
    ic = np.arange(nc)
    nxt = np.minimum(ic + 1, nc - 1)
    even = [slice(None)] * xc.ndim
    odd = [slice(None)] * xc.ndim
    even[a] = slice(0, nf, 2)
    odd[a] = slice(1, nf, 2)
    xf[tuple(even)] = xc
    xf[tuple(odd)] = 0.5 * (xc + take(xc, nxt))
    return xf


def prolong(xc):
    """I_{h-1}^h: tensor-product linear interpolation (O4)."""
    xf = np.asarray(xc, dtype=float)
    for a in range(xf.ndim):
        xf = _prolong_axis(xf, a)
    return xf


def _prolong_axis_T(xf, a):
    nf = xf.shape[a]
    nc = nf // 2
    even = [slice(None)] * xf.ndim
    odd = [slice(None)] * xf.ndim
    even[a] = slice(0, nf, 2)
    odd[a] = slice(1, nf, 2)
    fe = xf[tuple(even)]
    fo = xf[tuple(odd)]
    xc = fe + 0.5 * fo
    # the odd fine point 2i+1 also feeds coarse i+1 (clamped at the last coarse index)
    hi = [slice(None)] * xf.ndim
    lo = [slice(None)] * xf.ndim
    hi[a] = slice(1, nc)
    lo[a] = slice(0, nc - 1)
    xc[tuple(hi)] += 0.5 * fo[tuple(lo)]
    last = [slice(None)] * xf.ndim
    last[a] = slice(nc - 1, nc)
    xc[tuple(last)] += 0.5 * fo[tuple(last)]
    return xc


def restrict(xf):
    """I_h^{h-1} = 2^-d P^T (full weighting) (O4)."""
    xc = np.asarray(xf, dtype=float)
    for a in range(xc.ndim):
        xc = _prolong_axis_T(xc, a)
    return xc / (2.0 ** xc.ndim)


def neighbourhood_min(yf):
    """min_{j in {2i-1, 2i, 2i+1}^d} y_j for every coarse index i (clamped) (O5)."""
    m = np.asarray(yf, dtype=float)
    for a in range(m.ndim):
        n = m.shape[a]
        nc = n // 2
        ic = np.arange(nc)
        cand = [np.take(m, np.clip(2 * ic + o, 0, n - 1), axis=a) for o in (-1, 0, 1)]
        m = np.minimum(np.minimum(cand[0], cand[1]), cand[2])
    return m


def coarse_lower_bound(y_fine, lower_fine=None):
    """phi_{h-1} = R y - min over the fine neighbourhood of y (Sec. V.C Eq. (constraint); O5), or of
    y - b for a fine bound b (O12)."""
    if lower_fine is None:
        return restrict(y_fine) - neighbourhood_min(y_fine)
    return restrict(y_fine) - neighbourhood_min(np.asarray(y_fine, dtype=float) - lower_fine)


# ---------------------------------------------------------------------------------------------
# Levels (O6) and the power method (O10)
# ---------------------------------------------------------------------------------------------

def coarse_problem(pb):
    """The coarse level's problem description (O6), in the fields Operator.from_problem reads; a
    coarse problem can itself be coarsened (O12)."""
    import types

    d = pb.ndim if hasattr(pb, "ndim") else len(pb.shape)
    shape_c = tuple(n // 2 for n in pb.shape)
    spacing_c = tuple(2.0 * h for h in pb.spacing)
    pml_c = tuple(p // 2 for p in pb.pml)
    sl = tuple(slice(0, None, 2) for _ in range(d))
    c_c = np.broadcast_to(np.asarray(pb.c, dtype=float), pb.shape)[sl]
    rho_c = np.broadcast_to(np.asarray(pb.rho, dtype=float), pb.shape)[sl]
    a_c = np.broadcast_to(np.asarray(pb.alpha0, dtype=float), pb.shape)[sl]
    Nt_c = (pb.Nt + 1) // 2
    if pb.sensor_index is not None:
        # on-grid sensors become points at the same physical position
        idx = np.unravel_index(np.asarray(pb.sensor_index), pb.shape)
        pos = np.stack([(idx[a] - pb.shape[a] // 2) * pb.spacing[a] for a in range(d)][::-1], axis=1)
    else:
        pos = np.asarray(pb.sensor_pos, dtype=float)
    pos = np.array(pos, dtype=float)
    for a in range(d):  # numpy axis a <-> position component d-1-a
        lo = (0 - shape_c[a] // 2) * spacing_c[a]
        hi = (shape_c[a] - 1 - shape_c[a] // 2) * spacing_c[a]
        pos[:, d - 1 - a] = np.clip(pos[:, d - 1 - a], lo, hi)
    return types.SimpleNamespace(ndim=d, shape=shape_c, spacing=spacing_c, pml=pml_c, pml_alpha=pb.pml_alpha,
                                 c=c_c, rho=rho_c, alpha0=a_c, y=pb.y, dt=2.0 * pb.dt, Nt=Nt_c,
                                 sensor_pos=pos, sensor_index=None, smooth=getattr(pb, "smooth", False))


def coarse_operator(pb):
    """Coarse-level operator for a Problem (O6).  Returns (Operator, Nt_c)."""
    pc = coarse_problem(pb)
    return Operator.from_problem(pc), pc.Nt


def power_iteration(apply_HtH: Callable[[np.ndarray], np.ndarray], shape, n_iter=30, seed=0):
    """L_f = sigma_max(H^T H) by the power method (Sec. IV; O10)."""
    v = np.random.default_rng(seed).standard_normal(shape)
    v /= np.linalg.norm(v)
    L = 0.0
    for _ in range(n_iter):
        w = apply_HtH(v)
        L = float(np.linalg.norm(w))
        v = w / L
    return L


# ---------------------------------------------------------------------------------------------
# ISTA / FISTA / MG-FISTA (Alg. 1-3; O7-O9)
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass
class FistaOpts:
    variant: int = 1            # 0 = ISTA, 1 = FISTA
    lam: float = 1e-2           # lambda (Sec. VI.A)
    step_scale: float = 1.0     # alpha = step_scale / L (2 for ISTA, 1 for FISTA; Sec. VI.A)
    kappa: float = 0.25         # 1/4 in 2-D, 1/8 in 3-D (Sec. VI.A, VI.B)
    vartheta: float = 0.1
    q_d: int = 3
    q_c: int = 8
    eps_d: float = 1e-3
    eps_c: float = 1e-2
    tv_rho: float = 1e-2        # smoothing of Eq. (Thirty-two): 1e-2 (2-D), 3e-2 (3-D)
    n_tv: int = 20              # inner FGP iterations (O2)
    max_iter: int = 50
    target_re: float = 0.0      # stop when RE <= target (0 = off)
    recursion: bool = True      # False: never take the coarse branch (plain FISTA / ISTA)
    coarse_weight: float = 0.0  # weight of the coarse data term; <= 0: 2^(1-d) (O11)


@dataclasses.dataclass
class IterRecord:
    k: int
    branch: str        # "direct" | "recursive"
    F: float
    RES: float
    RE: float
    fwd: int
    adj: int


def fista_coarse(op_c, phat_c, x0, v, lower, lam, rho, L_c, opts: FistaOpts, w=1.0, deeper=(), w_step=None):
    """Coarse-level FISTA/ISTA on phi = w/2||H_c x - p_c||^2 + lam J_rho(x) + <v, x> with the
    projection on {x >= lower} (Sec. V.E; O7, O11).  ``deeper`` = [(op, phat, L_data), ...] are the
    next coarser levels: with one or more, an iteration k > 1 may take a recursive direction (O12);
    ``w_step`` is the weight factor per level step (2^(1-d) by default).  Returns (x_*, number of
    iterations, fwd, adj, recursive iterations at this level and below)."""
    alpha = 1.0 / L_c
    d = x0.ndim
    ws = w_step if w_step is not None else 2.0 ** (1 - d)

    def phi(x, Hx):
        r = Hx - phat_c
        return 0.5 * w * float(np.sum(r * r)) + lam * tv_smooth(x, rho) + float(np.sum(v * x))

    x_prev = x0.copy()
    Hx_prev = op_c.forward(x_prev)
    fwd, adj, nrec = 1, 0, 0
    y, Hy = x_prev.copy(), Hx_prev.copy()
    phi_prev = phi(x_prev, Hx_prev)
    t = 1.0
    K_d, K_r = 0, 0
    y_tilde = None
    k = 0
    while True:
        k += 1
        grad = w * op_c.adjoint(Hy - phat_c) + lam * tv_smooth_grad(y, rho) + v
        adj += 1
        recursive = False
        if deeper and opts.recursion and k > 1:
            Rg = restrict(grad)
            c1 = np.linalg.norm(Rg) > opts.kappa * np.linalg.norm(grad)
            far = (y_tilde is not None) and (np.linalg.norm(y - y_tilde) > opts.vartheta * np.linalg.norm(y_tilde))
            recursive = bool(c1 and (far or K_r == 0 or K_d > opts.q_d))
        if recursive:
            K_d, K_r = 0, K_r + 1
            y_tilde = y.copy()
            op_n, phat_n, Ld_n = deeper[0]
            w_n = w * ws
            x_n0 = restrict(y)
            g_n = w_n * op_n.adjoint(op_n.forward(x_n0) - phat_n) + lam * tv_smooth_grad(x_n0, rho)
            fwd += 1
            adj += 1
            v_n = Rg - g_n                                       # coherence with phi (O12)
            lower_n = coarse_lower_bound(y, lower)               # restricted bound (O12)
            L_n = w_n * Ld_n + lam * 4.0 * d / rho
            x_ns, _, cf, ca, cr = fista_coarse(op_n, phat_n, x_n0, v_n, lower_n, lam, rho, L_n, opts, w=w_n,
                                               deeper=deeper[1:], w_step=ws)
            fwd += cf
            adj += ca
            nrec += 1 + cr
            x = y + prolong(x_ns - x_n0)
        else:
            K_d += 1
            x = np.maximum(y - alpha * grad, lower)
        Hx = op_c.forward(x)
        fwd += 1
        phi_x = phi(x, Hx)
        if opts.variant == 1:
            t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            theta = (t - 1.0) / t_next
            t = t_next
        else:
            theta = 0.0
        y = x + theta * (x - x_prev)
        Hy = (1.0 + theta) * Hx - theta * Hx_prev
        dec = (phi_prev - phi_x) / max(abs(phi_prev), abs(phi_x), 1e-300)
        x_prev, Hx_prev, phi_prev = x, Hx, phi_x
        if dec < opts.eps_c or k >= opts.q_c:
            return x, k, fwd, adj, nrec


def mg_fista(op, phat, x0, L, opts: FistaOpts, coarse=None, p_exact=None,
             callback: Optional[Callable[[IterRecord], None]] = None):
    """Alg. 3 (Sec. V.E) on two levels, or on more (O12); with ``coarse`` None or
    ``opts.recursion`` False it is Alg. 2 (FISTA) or Alg. 1 (ISTA, variant 0).

    ``coarse`` = (op_c, phat_c, L_c_data) for two levels, or a list of such tuples from the first
    coarse level down.  Returns (x, list of IterRecord)."""
    levels = [] if coarse is None else ([coarse] if isinstance(coarse, tuple) else list(coarse))
    lam, rho = opts.lam, opts.tv_rho
    d = x0.ndim
    alpha = opts.step_scale / L
    nrm_exact = float(np.linalg.norm(p_exact)) if p_exact is not None else 0.0

    def F_of(x, Hx):
        r = Hx - phat
        return 0.5 * float(np.sum(r * r)) + lam * tv(x), float(np.linalg.norm(r))

    x_prev = np.array(x0, dtype=float)
    Hx_prev = op.forward(x_prev)
    fwd, adj = 1, 0
    F_prev, _ = F_of(x_prev, Hx_prev)
    y, Hy = x_prev.copy(), Hx_prev.copy()
    t = 1.0
    K_d, K_r = 0, 0
    y_tilde = None
    records = []
    for k in range(1, opts.max_iter + 1):
        gf = op.adjoint(Hy - phat)   # grad f(y_k) = H^T (H y_k - p_hat), Eq. (Six)
        adj += 1
        recursive = False
        if levels and opts.recursion and k > 1:
            gF = gf + lam * tv_smooth_grad(y, rho)   # Eq. (Twentyone)
            Rg = restrict(gF)
            c1 = np.linalg.norm(Rg) > opts.kappa * np.linalg.norm(gF)
            far = (y_tilde is not None) and (np.linalg.norm(y - y_tilde) > opts.vartheta * np.linalg.norm(y_tilde))
            c2 = far or K_r == 0 or K_d > opts.q_d
            recursive = bool(c1 and c2)
        if recursive:
            K_d, K_r = 0, K_r + 1
            y_tilde = y.copy()
            op_c, phat_c, L_c_data = levels[0]
            x_c0 = restrict(y)
            w_c = opts.coarse_weight if opts.coarse_weight > 0 else 2.0 ** (1 - d)   # O11
            gc = w_c * op_c.adjoint(op_c.forward(x_c0) - phat_c) + lam * tv_smooth_grad(x_c0, rho)
            fwd += 1
            adj += 1
            v = Rg - gc                                   # Eq. (Fourteen)
            lower = coarse_lower_bound(y)                 # Eq. (constraint) at y (O5)
            L_c = w_c * L_c_data + lam * 4.0 * d / rho
            x_cs, _, cf, ca, _ = fista_coarse(op_c, phat_c, x_c0, v, lower, lam, rho, L_c, opts, w=w_c,
                                              deeper=levels[1:], w_step=w_c)
            fwd += cf
            adj += ca
            x = y + prolong(x_cs - x_c0)
            branch = "recursive"
        else:
            K_d += 1
            x = tv_prox(y - alpha * gf, alpha * lam, opts.n_tv, nonneg=True)
            branch = "direct"
        Hx = op.forward(x)
        fwd += 1
        F_x, RES = F_of(x, Hx)
        RE = float(np.linalg.norm(x - p_exact)) / nrm_exact if p_exact is not None else float("nan")
        rec = IterRecord(k, branch, F_x, RES, RE, fwd, adj)
        records.append(rec)
        if callback is not None:
            callback(rec)
        if opts.variant == 1:
            t_next = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
            theta = (t - 1.0) / t_next
            t = t_next
        else:
            theta = 0.0
        y = x + theta * (x - x_prev)
        Hy = (1.0 + theta) * Hx - theta * Hx_prev
        dec = (F_prev - F_x) / max(F_prev, F_x)
        x_prev, Hx_prev, F_prev = x, Hx, F_x
        if dec < opts.eps_d:
            break
        if opts.target_re > 0.0 and p_exact is not None and RE <= opts.target_re:
            break
    return x_prev, records
