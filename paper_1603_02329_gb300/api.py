"""Python binding of the C ABI: argument marshalling around ``libpat_gb300.so``.

PyTorch provides device memory and streams; every step of the forward operator H and its
transpose H^T (Sec. III of Javaherian & Holman, arXiv:1603.02329) runs in the library's own
CUDA kernels.  Names follow the C calls of ``include/pat.h``.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import PAT_F32, PAT_F64, check, lib

_DTYPES = {PAT_F32: torch.float32, PAT_F64: torch.float64}


def _as_f64(a, N, name):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if arr.size not in (1, N):
        raise ValueError(f"{name} must have 1 or {N} values, got {arr.size}")
    return arr


def make_grid(shape, spacing, pml, pml_alpha=2.0) -> _lib.pat_grid:
    """numpy-order shape/spacing/pml ((Ny, Nx) or (Nz, Ny, Nx)) -> pat_grid (x first)."""
    d = len(shape)
    g = _lib.pat_grid()
    g.ndim = d
    for a in range(3):
        g.n[a] = int(shape[d - 1 - a]) if a < d else 1
        g.dx[a] = float(spacing[d - 1 - a]) if a < d else 1.0
        g.pml[a] = int(pml[d - 1 - a]) if a < d else 0
    g.pml_alpha = float(pml_alpha)
    return g


def _stream_ptr(stream, device):
    if stream is None:
        if device is None or device.type != "cuda":
            return None
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


class PATOperator:
    """Plan of the forward operator H and its exact transpose (``pat_plan_*`` calls).

    Fields are numpy-ordered (``shape`` = (Ny, Nx) or (Nz, Ny, Nx)); data are [Nt][Ns].
    ``forward`` / ``adjoint`` accept CUDA or CPU tensors of the plan's dtype and return a tensor
    on the same device (CPU tensors go through the library's host-pointer path)."""

    def __init__(self, shape, spacing, pml, pml_alpha, c, rho, alpha0, y, dt, Nt,
                 sensor_pos=None, sensor_index=None, precision="f32", device=None, smooth=False):
        self.shape = tuple(int(n) for n in shape)
        self.N = int(np.prod(self.shape))
        self.Nt = int(Nt)
        self.prec = PAT_F64 if precision in ("f64", "float64", torch.float64, PAT_F64) else PAT_F32
        self.dtype = _DTYPES[self.prec]
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._grid = make_grid(self.shape, spacing, pml, pml_alpha)
        self._c = _as_f64(c, self.N, "c")
        self._rho = _as_f64(rho, self.N, "rho")
        if self._c.size == 1:
            self._c = np.full(self.N, self._c[0])
        if self._rho.size == 1:
            self._rho = np.full(self.N, self._rho[0])
        self._a0 = _as_f64(alpha0, self.N, "alpha0")
        sens = _lib.pat_sensors()
        if sensor_index is not None:
            self._sidx = np.ascontiguousarray(np.asarray(sensor_index, dtype=np.int64).reshape(-1))
            sens.count = int(self._sidx.size)
            sens.index = self._sidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            sens.pos = None
        else:
            self._spos = np.ascontiguousarray(np.asarray(sensor_pos, dtype=np.float64))
            sens.count = int(self._spos.shape[0])
            sens.pos = self._spos.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            sens.index = None
        self.Ns = sens.count
        self._plan = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        with torch.cuda.device(self.device):
            check(lib().pat_plan_create(ctypes.byref(self._grid), self._c.ctypes.data_as(dp),
                                        self._rho.ctypes.data_as(dp), self._a0.ctypes.data_as(dp),
                                        int(self._a0.size == 1), float(y), ctypes.byref(sens), float(dt),
                                        self.Nt, self.prec, ctypes.byref(self._plan)))
        info = _lib.pat_plan_info_t()
        check(lib().pat_plan_get_info(self._plan, ctypes.byref(info)))
        self.info = info
        self.lossy = bool(info.lossy)
        self.smoothing = False
        if smooth:
            self.set_smoothing(True)

    @classmethod
    def from_problem(cls, pb, precision="f32", Nt=None, device=None):
        return cls(pb.shape, pb.spacing, pb.pml, pb.pml_alpha, pb.c, pb.rho, pb.alpha0, pb.y, pb.dt,
                   pb.Nt if Nt is None else Nt, sensor_pos=pb.sensor_pos, sensor_index=pb.sensor_index,
                   precision=precision, device=device, smooth=getattr(pb, "smooth", False))

    def set_smoothing(self, enable: bool):
        """pat_plan_set_smoothing: H becomes H S and its transpose S H^T (Sec. VI.A)."""
        check(lib().pat_plan_set_smoothing(self._plan, int(bool(enable))))
        self.smoothing = bool(enable)

    def smooth(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """pat_plan_smooth: S x with the plan's window (device tensors)."""
        self._check_in(x, self.N, "x")
        if x.device.type != "cuda":
            raise ValueError("smooth takes a CUDA tensor")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=x.device)
        self._check_in(out, self.N, "out")
        with torch.cuda.device(self.device):
            check(lib().pat_plan_smooth(self._plan, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        _stream_ptr(stream, self.device)))
        return out

    # -- calls ---------------------------------------------------------------------------------
    def _check_in(self, t, n, name):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}, got {t.dtype}")
        if t.numel() != n:
            raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")

    def forward(self, p0: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """pat_forward_plan: data[Nt][Ns] = H p0."""
        self._check_in(p0, self.N, "p0")
        if out is None:
            out = torch.empty((self.Nt, self.Ns), dtype=self.dtype, device=p0.device)
        self._check_in(out, self.Nt * self.Ns, "out")
        with torch.cuda.device(self.device):
            check(lib().pat_forward_plan(self._plan, ctypes.c_void_p(p0.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         _stream_ptr(stream, self.device)))
        return out

    def adjoint(self, residual: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """pat_adjoint: grad = H^T residual, shaped like the grid."""
        self._check_in(residual, self.Nt * self.Ns, "residual")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=residual.device)
        self._check_in(out, self.N, "out")
        with torch.cuda.device(self.device):
            check(lib().pat_adjoint(self._plan, ctypes.c_void_p(residual.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    _stream_ptr(stream, self.device)))
        return out

    def gradient_c2(self, p0: torch.Tensor, residual: torch.Tensor, checkpoint_every: int = 50,
                    with_p0_grad: bool = False, stream=None):
        """pat_gradient_c2: d<H p0, h>/d(c0^2) per grid point with forward checkpoints every
        ``checkpoint_every`` time levels (and H^T h when ``with_p0_grad``)."""
        self._check_in(p0, self.N, "p0")
        self._check_in(residual, self.Nt * self.Ns, "residual")
        g = torch.empty(self.shape, dtype=self.dtype, device=p0.device)
        gp = torch.empty(self.shape, dtype=self.dtype, device=p0.device) if with_p0_grad else None
        with torch.cuda.device(self.device):
            check(lib().pat_gradient_c2(self._plan, ctypes.c_void_p(p0.data_ptr()),
                                        ctypes.c_void_p(residual.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                        ctypes.c_void_p(gp.data_ptr()) if gp is not None else None,
                                        int(checkpoint_every), _stream_ptr(stream, self.device)))
        return (g, gp) if with_p0_grad else g

    def gradient_rho(self, p0: torch.Tensor, residual: torch.Tensor, checkpoint_every: int = 50,
                     with_p0_grad: bool = False, stream=None):
        """pat_gradient_rho: d<H p0, h>/d(rho0) per grid point with forward checkpoints every
        ``checkpoint_every`` time levels (and H^T h when ``with_p0_grad``)."""
        g, _, gp = self.gradient_medium(p0, residual, checkpoint_every, want=("rho", "p0") if with_p0_grad else ("rho",),
                                        stream=stream)
        return (g, gp) if with_p0_grad else g

    def gradient_medium(self, p0: torch.Tensor, residual: torch.Tensor, checkpoint_every: int = 50,
                        want=("c2", "rho", "p0"), stream=None):
        """pat_gradient_medium: (d<H p0, h>/d rho0, d<H p0, h>/d c0^2, H^T h) from one checkpointed sweep;
        the entries not in ``want`` are None.  Returns (grad_rho, grad_c2, grad_p0)."""
        self._check_in(p0, self.N, "p0")
        self._check_in(residual, self.Nt * self.Ns, "residual")
        mk = lambda key: torch.empty(self.shape, dtype=self.dtype, device=p0.device) if key in want else None
        gr, gc, gp = mk("rho"), mk("c2"), mk("p0")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        with torch.cuda.device(self.device):
            if gc is None and gr is not None:
                check(lib().pat_gradient_rho(self._plan, ptr(p0), ptr(residual), ptr(gr), ptr(gp),
                                             int(checkpoint_every), _stream_ptr(stream, self.device)))
            else:
                check(lib().pat_gradient_medium(self._plan, ptr(p0), ptr(residual), ptr(gc), ptr(gr), ptr(gp),
                                                int(checkpoint_every), _stream_ptr(stream, self.device)))
        return gr, gc, gp

    def time_reversal(self, data: torch.Tensor, compensate: bool = True, k_cut: float = 0.5,
                      out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """pat_time_reversal: the time-reversal image of data [Nt][Ns] (Sec. II.B.1; on-grid sensors),
        with the band-limited absorption compensation when ``compensate``."""
        self._check_in(data, self.Nt * self.Ns, "data")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=data.device)
        self._check_in(out, self.N, "out")
        with torch.cuda.device(self.device):
            check(lib().pat_time_reversal(self._plan, ctypes.c_void_p(data.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          int(bool(compensate)), float(k_cut), _stream_ptr(stream, self.device)))
        return out

    def adjoint_atd(self, residual: torch.Tensor, initial: str = "R5", out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
        """pat_adjoint_atd: the paper's adjoint-then-discretize image of residual [Nt][Ns] (Sec. VI);
        ``initial`` "R5" (the forward map's initial state) or "paper" (Eq. (adjj))."""
        if initial not in ("R5", "paper"):
            raise ValueError("initial must be 'R5' or 'paper'")
        self._check_in(residual, self.Nt * self.Ns, "residual")
        if out is None:
            out = torch.empty(self.shape, dtype=self.dtype, device=residual.device)
        self._check_in(out, self.N, "out")
        with torch.cuda.device(self.device):
            check(lib().pat_adjoint_atd(self._plan, ctypes.c_void_p(residual.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), int(initial == "paper"),
                                        _stream_ptr(stream, self.device)))
        return out

    # -- optimisation shell ---------------------------------------------------------------------
    def power_iteration(self, v0: torch.Tensor, n_iter: int = 30, stream=None) -> float:
        """pat_power_iteration: sigma_max(H^T H) from the start vector v0 (device, plan dtype)."""
        self._check_in(v0, self.N, "v0")
        L = ctypes.c_double()
        with torch.cuda.device(self.device):
            check(lib().pat_power_iteration(self._plan, ctypes.c_void_p(v0.data_ptr()), int(n_iter), ctypes.byref(L),
                                            _stream_ptr(stream, self.device)))
        return L.value

    def coarse(self) -> "PATOperator":
        """pat_plan_create_coarse: the next coarser level (half the points, twice dx and dt)."""
        op = PATOperator.__new__(PATOperator)
        op._plan = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().pat_plan_create_coarse(self._plan, ctypes.byref(op._plan)))
        info = _lib.pat_plan_info_t()
        check(lib().pat_plan_get_info(op._plan, ctypes.byref(info)))
        d = info.ndim
        op.info = info
        op.shape = tuple(int(info.n[d - 1 - a]) for a in range(d))
        op.N = int(info.N)
        op.Nt = int(info.Nt)
        op.Ns = int(info.Ns)
        op.prec = self.prec
        op.dtype = self.dtype
        op.device = self.device
        op.lossy = bool(info.lossy)
        op.smoothing = self.smoothing   # pat_plan_create_coarse carries the switch over
        return op

    # -- kernel-timing probe ------------------------------------------------------------------------
    def set_probe(self, stride: int):
        """pat_plan_set_probe: bracket the launches of every `stride`-th step with CUDA events."""
        check(lib().pat_plan_set_probe(self._plan, int(stride)))

    def probe(self, adjoint: bool):
        """pat_plan_probe_read for every slot: list of (kernel name, mean ms, samples) of the last solve."""
        out = []
        n = lib().pat_plan_probe_slots(self._plan, int(adjoint))
        for k in range(n):
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            cnt = ctypes.c_int()
            check(lib().pat_plan_probe_read(self._plan, int(adjoint), k, ctypes.byref(name), ctypes.byref(ms),
                                            ctypes.byref(cnt)))
            out.append((name.value.decode(), ms.value, cnt.value))
        return out

    # -- phase-timeline trace (persistent path) -------------------------------------------------
    def set_trace(self, k0: int, nk: int):
        """pat_plan_set_trace: record barrier entry/exit times for barriers k0 .. k0 + nk - 1."""
        check(lib().pat_plan_set_trace(self._plan, int(k0), int(nk)))
        self._trace_nk = int(nk)

    def read_trace(self):
        """pat_plan_read_trace: uint64 array [grid][nk][8] (barrier entry, exit, sub-phase marks) in ns."""
        nk = getattr(self, "_trace_nk", 0)
        if nk == 0:
            return None
        cap = 4096 * nk * 8
        buf = np.zeros(cap, dtype=np.uint64)
        grid = ctypes.c_int()
        check(lib().pat_plan_read_trace(self._plan, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap,
                                        ctypes.byref(grid)))
        if grid.value == 0:
            return None
        return buf[: grid.value * nk * 8].reshape(grid.value, nk, 8)

    def close(self):
        if getattr(self, "_plan", None) is not None and self._plan.value:
            lib().pat_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pat_forward(p0: torch.Tensor, c, rho, alpha0, y, shape, spacing, pml, pml_alpha, sensor_pos=None,
                sensor_index=None, dt=None, Nt=None, precision="f32", stream=None) -> torch.Tensor:
    """One-shot ``pat_forward`` (builds and frees a plan inside the library)."""
    prec = PAT_F64 if precision in ("f64", "float64", torch.float64) else PAT_F32
    dtype = _DTYPES[prec]
    if p0.dtype != dtype or not p0.is_contiguous():
        raise TypeError("p0 must be a contiguous tensor of the requested precision")
    N = int(np.prod(shape))
    grid = make_grid(shape, spacing, pml, pml_alpha)
    cc = np.ascontiguousarray(np.broadcast_to(np.asarray(c, np.float64), (N,)) if np.size(c) == 1 else np.asarray(c, np.float64).reshape(-1))
    rr = np.ascontiguousarray(np.broadcast_to(np.asarray(rho, np.float64), (N,)) if np.size(rho) == 1 else np.asarray(rho, np.float64).reshape(-1))
    aa = np.ascontiguousarray(np.asarray(alpha0, np.float64).reshape(-1))
    sens = _lib.pat_sensors()
    if sensor_index is not None:
        sidx = np.ascontiguousarray(np.asarray(sensor_index, np.int64).reshape(-1))
        sens.count, sens.index, sens.pos = int(sidx.size), sidx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), None
    else:
        spos = np.ascontiguousarray(np.asarray(sensor_pos, np.float64))
        sens.count, sens.pos, sens.index = int(spos.shape[0]), spos.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None
    out = torch.empty((int(Nt), sens.count), dtype=dtype, device=p0.device)
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().pat_forward(ctypes.c_void_p(p0.data_ptr()), cc.ctypes.data_as(dp), rr.ctypes.data_as(dp),
                            aa.ctypes.data_as(dp), int(aa.size == 1), float(y), ctypes.byref(grid), ctypes.byref(sens),
                            float(dt), int(Nt), prec, ctypes.c_void_p(out.data_ptr()),
                            _stream_ptr(stream, p0.device)))
    return out


# ---------------------------------------------------------------------------------------------
# image-space operators of the optimisation shell (Sec. IV, Sec. V)
# ---------------------------------------------------------------------------------------------
def _prec_of(t: torch.Tensor):
    if t.dtype == torch.float32:
        return PAT_F32
    if t.dtype == torch.float64:
        return PAT_F64
    raise TypeError("float32 or float64 tensor expected")


def _img_grid(shape):
    return make_grid(tuple(shape), (1.0,) * len(shape), (0,) * len(shape), 0.0)


def _dev_stream(t, stream):
    return _stream_ptr(stream, t.device)


def tv_prox(z: torch.Tensor, weight: float, n_inner: int = 20, nonneg: bool = True, stream=None) -> torch.Tensor:
    """pat_tv_prox: argmin weight TV(x) + [x >= 0] + 1/2 ||x - z||^2 (dual FGP, n_inner steps)."""
    x = torch.empty_like(z)
    g = _img_grid(z.shape)
    check(lib().pat_tv_prox(ctypes.byref(g), ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                            float(weight), int(n_inner), int(bool(nonneg)), _prec_of(z), _dev_stream(z, stream)))
    return x


def tv(x: torch.Tensor, rho: float = 0.0, stream=None) -> float:
    """pat_tv: TV(x) (rho = 0) or J_rho(x) (rho > 0), FP64 accumulation."""
    v = ctypes.c_double()
    g = _img_grid(x.shape)
    check(lib().pat_tv(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), float(rho), ctypes.byref(v), _prec_of(x),
                       _dev_stream(x, stream)))
    return v.value


def tv_smooth_grad(y: torch.Tensor, rho: float, stream=None) -> torch.Tensor:
    """pat_tv_smooth_grad: gradient of J_rho."""
    out = torch.empty_like(y)
    g = _img_grid(y.shape)
    check(lib().pat_tv_smooth_grad(ctypes.byref(g), ctypes.c_void_p(y.data_ptr()), float(rho),
                                   ctypes.c_void_p(out.data_ptr()), _prec_of(y), _dev_stream(y, stream)))
    return out


def restrict(xf: torch.Tensor, stream=None) -> torch.Tensor:
    """pat_restrict: R = 2^-d P^T onto half the points per axis."""
    xc = torch.empty(tuple(n // 2 for n in xf.shape), dtype=xf.dtype, device=xf.device)
    g = _img_grid(xf.shape)
    check(lib().pat_restrict(ctypes.byref(g), ctypes.c_void_p(xf.data_ptr()), ctypes.c_void_p(xc.data_ptr()),
                             _prec_of(xf), _dev_stream(xf, stream)))
    return xc


def prolong(xc: torch.Tensor, stream=None) -> torch.Tensor:
    """pat_prolong: linear interpolation onto twice the points per axis."""
    fine = tuple(2 * n for n in xc.shape)
    xf = torch.empty(fine, dtype=xc.dtype, device=xc.device)
    g = _img_grid(fine)
    check(lib().pat_prolong(ctypes.byref(g), ctypes.c_void_p(xc.data_ptr()), ctypes.c_void_p(xf.data_ptr()),
                            _prec_of(xc), _dev_stream(xc, stream)))
    return xf


def coarse_bound(y: torch.Tensor, stream=None) -> torch.Tensor:
    """pat_coarse_bound: phi = R y - min over the fine neighbourhood."""
    phi = torch.empty(tuple(n // 2 for n in y.shape), dtype=y.dtype, device=y.device)
    g = _img_grid(y.shape)
    check(lib().pat_coarse_bound(ctypes.byref(g), ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                 _prec_of(y), _dev_stream(y, stream)))
    return phi


def dot(a: torch.Tensor, b: torch.Tensor, stream=None) -> float:
    """pat_dot: FP64-accumulated inner product."""
    v = ctypes.c_double()
    check(lib().pat_dot(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), a.numel(), _prec_of(a),
                        ctypes.byref(v), _dev_stream(a, stream)))
    return v.value


FISTA_DEFAULTS = dict(variant=1, lam=1e-2, step_scale=1.0, kappa=0.25, vartheta=0.1, q_d=3, q_c=8, eps_d=1e-3,
                      eps_c=1e-2, tv_rho=1e-2, n_tv=20, max_iter=50, recursion=True, target_re=0.0)


def probe_fp32_peak(device=None) -> float:
    """pat_probe_fp32_peak: measured FP32 FMA throughput of the device [TFLOP/s]."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    v = ctypes.c_double()
    with torch.cuda.device(dev):
        check(lib().pat_probe_fp32_peak(ctypes.byref(v), _stream_ptr(None, dev)))
    return v.value


def mg_fista(fine: "PATOperator", coarse: Optional["PATOperator"], data: torch.Tensor, x0: torch.Tensor, L: float,
             L_coarse: float = 0.0, p_exact: Optional[torch.Tensor] = None, callback=None, stream=None, **opts):
    """pat_mg_fista: Alg. 3 (two levels) or Alg. 2 / Alg. 1.  Returns (x, report dict, records).

    ``coarse`` may also be a list of operators, each the coarse level of the one before
    (``PATOperator.coarse()``), with ``L_coarse`` the list of their sigma_max(H^T H): the call is
    then pat_mg_fista_levels on 1 + len(coarse) levels."""
    o = dict(FISTA_DEFAULTS)
    o.update(opts)
    po = _lib.pat_fista_opts()
    po.variant = int(o["variant"])
    po.lambda_ = float(o["lam"])
    po.step_scale = float(o["step_scale"])
    po.kappa = float(o["kappa"])
    po.vartheta = float(o["vartheta"])
    po.q_d = int(o["q_d"])
    po.q_c = int(o["q_c"])
    po.eps_d = float(o["eps_d"])
    po.eps_c = float(o["eps_c"])
    po.tv_rho = float(o["tv_rho"])
    po.n_tv = int(o["n_tv"])
    po.max_iter = int(o["max_iter"])
    po.recursion = int(bool(o["recursion"]))
    po.L = float(L)
    po.L_coarse = float(L_coarse[0] if isinstance(L_coarse, (list, tuple)) else L_coarse)
    po.target_re = float(o["target_re"])
    po.p_exact = ctypes.c_void_p(p_exact.data_ptr()) if p_exact is not None else None
    po.coarse_weight = float(o.get("coarse_weight", 0.0))
    records = []

    def _cb(ctx, k, rec, F, RES, RE, nf, na):
        records.append(dict(k=k, branch="recursive" if rec else "direct", F=F, RES=RES, RE=RE, fwd=nf, adj=na))
        if callback is not None:
            callback(records[-1])

    cb = _lib.ITER_CB(_cb)
    rep = _lib.pat_fista_report()
    x = torch.empty_like(x0)
    if isinstance(coarse, (list, tuple)):
        ops = [fine] + list(coarse)
        Ls = [float(L)] + [float(v) for v in (L_coarse if isinstance(L_coarse, (list, tuple)) else [L_coarse])]
        if len(Ls) != len(ops):
            raise ValueError("L_coarse needs one value per coarse level")
        plans = (ctypes.c_void_p * len(ops))(*[op._plan.value for op in ops])
        larr = (ctypes.c_double * len(Ls))(*Ls)
        po.L_coarse = Ls[1] if len(Ls) > 1 else 0.0
        with torch.cuda.device(fine.device):
            check(lib().pat_mg_fista_levels(plans, len(ops), larr, ctypes.c_void_p(data.data_ptr()),
                                            ctypes.c_void_p(x0.data_ptr()), ctypes.byref(po),
                                            ctypes.c_void_p(x.data_ptr()), ctypes.byref(rep), cb, None,
                                            _stream_ptr(stream, fine.device)))
    else:
        cplan = coarse._plan if coarse is not None else None
        with torch.cuda.device(fine.device):
            check(lib().pat_mg_fista(fine._plan, cplan, ctypes.c_void_p(data.data_ptr()),
                                     ctypes.c_void_p(x0.data_ptr()), ctypes.byref(po), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.byref(rep), cb, None, _stream_ptr(stream, fine.device)))
    report = dict(iters=rep.iters, recursive_iters=rep.recursive_iters, fwd_solves=rep.fwd_solves,
                  adj_solves=rep.adj_solves, F=rep.F, RES=rep.RES, RE=rep.RE)
    return x, report, records


class PATBatch:
    """pat_batch_*: several independent instances (uneven grids) as one graph launch per call."""

    def __init__(self, ops):
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[op._plan.value for op in self.ops])
        self._b = ctypes.c_void_p()
        self.device = self.ops[0].device
        with torch.cuda.device(self.device):
            check(lib().pat_batch_create(arr, len(self.ops), ctypes.byref(self._b)))

    def _run(self, fn, xs, shapes, stream):
        if len(xs) != len(self.ops):
            raise ValueError("one tensor per instance")
        outs = [torch.empty(sh, dtype=op.dtype, device=x.device) for sh, op, x in zip(shapes, self.ops, xs)]
        ins = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        ous = (ctypes.c_void_p * len(xs))(*[o.data_ptr() for o in outs])
        with torch.cuda.device(self.device):
            check(fn(self._b, ins, ous, _stream_ptr(stream, self.device)))
        return outs

    def forward(self, p0s, stream=None):
        for op, x in zip(self.ops, p0s):
            op._check_in(x, op.N, "p0")
        return self._run(lib().pat_batch_forward, p0s, [(op.Nt, op.Ns) for op in self.ops], stream)

    def adjoint(self, residuals, stream=None):
        for op, r in zip(self.ops, residuals):
            op._check_in(r, op.Nt * op.Ns, "residual")
        return self._run(lib().pat_batch_adjoint, residuals, [op.shape for op in self.ops], stream)

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            lib().pat_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
