"""pat_forward_static: the forward operator for callers that cannot allocate device memory.

Such callers (an application whose own pool allocator owns all device memory, a service that
must not allocate once running) cannot use pat_forward, which builds a plan with cudaMalloc.
pat_forward_static computes the same data inside the library's fixed device scratch array.
This test calls both entry points through the C ABI and checks that two calls in a row of the
allocation-free one agree with the allocating one within the parity tolerances of the other GPU
tests; it also checks that an oversized request is rejected before any device work.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _args(pb, dev, dtype):
    from paper_1603_02329_gb300 import _lib
    from paper_1603_02329_gb300.api import make_grid

    keep = {}
    keep["grid"] = make_grid(pb.shape, pb.spacing, pb.pml, pb.pml_alpha)
    keep["c"] = np.ascontiguousarray(pb.c, dtype=np.float64).ravel()
    keep["rho"] = np.ascontiguousarray(pb.rho, dtype=np.float64).ravel()
    keep["a0"] = np.ascontiguousarray(pb.alpha0, dtype=np.float64).ravel()
    s = _lib.pat_sensors()
    if pb.sensor_index is not None:
        keep["idx"] = np.ascontiguousarray(pb.sensor_index, dtype=np.int64)
        s.count, s.index = keep["idx"].size, keep["idx"].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    else:
        keep["pos"] = np.ascontiguousarray(pb.sensor_pos, dtype=np.float64)
        s.count, s.pos = keep["pos"].shape[0], keep["pos"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    keep["sens"] = s
    keep["p0"] = torch.tensor(pb.p0, dtype=dtype, device=dev).contiguous()
    return keep


def _call(fn, k, pb, prec, dev, dtype, stream=None):
    dp = ctypes.POINTER(ctypes.c_double)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(s):
        out = torch.full((pb.Nt, k["sens"].count), float("nan"), dtype=dtype, device=dev)
    st = fn(ctypes.c_void_p(k["p0"].data_ptr()), k["c"].ctypes.data_as(dp), k["rho"].ctypes.data_as(dp),
            k["a0"].ctypes.data_as(dp), 0, float(pb.y), ctypes.byref(k["grid"]), ctypes.byref(k["sens"]),
            float(pb.dt), int(pb.Nt), prec, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize(dev)
    return st, out


def _problem(kind):
    from paper_1603_02329_gb300 import synth

    if kind == "2d":
        return synth.small_lossy_2d(shape=(64, 72), pml=8, Nt=150, n_sensors=24)
    # 3-D: x-lines of 32 points (the register-fused row kernels), an on-grid planar array
    return synth.small_lossy_3d(shape=(28, 24, 32), pml=4, Nt=40)


# "nonblocking": the caller's stream does not order after the legacy default stream, on which the
# plan's tables are written; the entry point must wait for them itself
@pytest.mark.parametrize("stream_kind", ["default", "nonblocking"])
@pytest.mark.parametrize("kind", ["2d", "3d"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_forward_matches_allocating_forward(prec, kind, stream_kind):
    from paper_1603_02329_gb300 import build, _lib

    build.build()
    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    dtype = torch.float64 if prec == "f64" else torch.float32
    code = _lib.PAT_F64 if prec == "f64" else _lib.PAT_F32
    tol = 1e-11 if prec == "f64" else 1e-5
    pb = _problem(kind)
    k = _args(pb, dev, dtype)
    st, ref = _call(L.pat_forward, k, pb, code, dev, dtype)
    assert st == 0, L.pat_last_error()
    assert torch.isfinite(ref).all() and ref.abs().max() > 0
    stream = torch.cuda.Stream(dev) if stream_kind == "nonblocking" else None
    for _ in range(2):  # two calls in a row share (and reuse) the scratch array
        st, out = _call(L.pat_forward_static, k, pb, code, dev, dtype, stream=stream)
        assert st == 0, L.pat_last_error()
        err = (torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert err <= tol


def test_static_forward_rejects_oversized_problem():
    from paper_1603_02329_gb300 import build, _lib
    from paper_1603_02329_gb300 import synth

    build.build()
    L = _lib.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    # 768^2 FP64 with a long record needs far more than the 32 MiB scratch
    pb = synth.small_lossy_2d(shape=(768, 768), pml=8, Nt=4000, n_sensors=16, sensor_radius_frac=0.3)
    pb.p0 = np.zeros(pb.shape)
    k = _args(pb, dev, torch.float64)
    st, out = _call(L.pat_forward_static, k, pb, _lib.PAT_F64, dev, torch.float64)
    assert st == _lib.PAT_EINVAL
    assert b"static scratch" in L.pat_last_error()
    assert torch.isnan(out).all()   # nothing was written
