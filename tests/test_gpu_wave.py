"""GPU parity of the forward operator H and its transpose against the FP64 oracle, through the C ABI.

Tolerances: relative L2 <= 1e-5 for FP32 fields (data and gradients), <= 1e-11 for FP64 plans.
Full-size workloads are checked on what the oracle can compute in seconds: the first time
samples (a causal prefix) and the adjoint of a residual supported on that prefix, plus the
dot-product identity, which holds at any size.
"""
import numpy as np
import pytest
import torch

from oracle.pat_oracle import Operator
from paper_1603_02329_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-11


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


@pytest.fixture(scope="module")
def dev():
    from paper_1603_02329_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def _gpu_op(pb, prec, dev, Nt=None):
    from paper_1603_02329_gb300.api import PATOperator

    return PATOperator.from_problem(pb, precision=prec, device=dev, Nt=Nt)


def _t(a, prec, dev):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32 if prec == "f32" else torch.float64, device=dev)


CASES_2D = [
    # name, factory kwargs
    ("lossy_48x40_offgrid", dict(shape=(48, 40), pml=6, Nt=120, n_sensors=20)),
    ("lossy_30x42_ragged", dict(shape=(30, 42), pml=5, Nt=80, n_sensors=12, sensor_radius_frac=0.25)),
    ("lossy_64x64", dict(shape=(64, 64), pml=8, Nt=200, n_sensors=48)),
    ("lossy_96x112", dict(shape=(96, 112), pml=10, Nt=150, n_sensors=32)),
]


@pytest.mark.parametrize("name,kw", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_forward_adjoint_parity_2d_f32(dev, name, kw):
    pb = synth.small_lossy_2d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(3).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f32", dev)
    d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
    g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
    assert rel(d, ref.forward(pb.p0)) <= TOL32
    assert rel(g, ref.adjoint(h)) <= TOL32


def test_forward_adjoint_parity_2d_f64_lossless(dev):
    pb = synth.disc_phantom_2d(interior=40, pml=8, Nt=150, n_sensors=24, sensor_radius=1.6e-3)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(4).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f64", dev)
    d = op.forward(_t(pb.p0, "f64", dev)).cpu().numpy()
    g = op.adjoint(_t(h, "f64", dev)).cpu().numpy()
    assert rel(d, ref.forward(pb.p0)) <= TOL64
    assert rel(g, ref.adjoint(h)) <= TOL64


def test_forward_adjoint_parity_2d_f64_lossy(dev):
    pb = synth.small_lossy_2d(shape=(40, 48), pml=6, Nt=90, n_sensors=16)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(5).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f64", dev)
    assert rel(op.forward(_t(pb.p0, "f64", dev)).cpu().numpy(), ref.forward(pb.p0)) <= TOL64
    assert rel(op.adjoint(_t(h, "f64", dev)).cpu().numpy(), ref.adjoint(h)) <= TOL64


@pytest.mark.parametrize("shape", [(24, 32, 40), (16, 20, 28)])
def test_forward_adjoint_parity_3d_f32(dev, shape):
    pb = synth.small_lossy_3d(shape=shape, pml=4, Nt=50)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(6).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f32", dev)
    assert rel(op.forward(_t(pb.p0, "f32", dev)).cpu().numpy(), ref.forward(pb.p0)) <= TOL32
    assert rel(op.adjoint(_t(h, "f32", dev)).cpu().numpy(), ref.adjoint(h)) <= TOL32


def test_forward_adjoint_parity_3d_f64_offgrid(dev):
    rng = np.random.default_rng(9)
    pb = synth.small_lossy_3d(shape=(16, 20, 24), pml=3, Nt=30)
    pos = rng.uniform(-0.3, 0.3, size=(15, 3)) * np.array([24, 20, 16]) * pb.spacing[0]
    pb.sensor_index = None
    pb.sensor_pos = pos
    ref = Operator.from_problem(pb)
    h = rng.standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f64", dev)
    assert rel(op.forward(_t(pb.p0, "f64", dev)).cpu().numpy(), ref.forward(pb.p0)) <= TOL64
    assert rel(op.adjoint(_t(h, "f64", dev)).cpu().numpy(), ref.adjoint(h)) <= TOL64


@pytest.mark.parametrize("Nt", [1, 2, 3])
def test_short_time_axes(dev, Nt):
    pb = synth.small_lossy_2d(shape=(32, 32), pml=4, Nt=Nt, n_sensors=8)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(7).standard_normal((Nt, ref.Ns))
    op = _gpu_op(pb, "f64", dev)
    assert rel(op.forward(_t(pb.p0, "f64", dev)).cpu().numpy(), ref.forward(pb.p0)) <= TOL64
    assert rel(op.adjoint(_t(h, "f64", dev)).cpu().numpy(), ref.adjoint(h)) <= TOL64


def test_coincident_and_corner_sensors(dev):
    # two sensors at the same point, one exactly on a node, one on a cell corner of the PML
    pb = synth.small_lossy_2d(shape=(32, 36), pml=4, Nt=40, n_sensors=6)
    h = pb.spacing[0]
    extra = np.array([[0.37 * h, -1.25 * h], [0.37 * h, -1.25 * h], [3 * h, 2 * h], [-18 * h, -16 * h]])
    pb.sensor_pos = np.concatenate([pb.sensor_pos, extra])
    ref = Operator.from_problem(pb)
    hh = np.random.default_rng(8).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f64", dev)
    d = op.forward(_t(pb.p0, "f64", dev)).cpu().numpy()
    assert rel(d, ref.forward(pb.p0)) <= TOL64
    assert np.array_equal(d[:, -3], d[:, -4])
    assert rel(op.adjoint(_t(hh, "f64", dev)).cpu().numpy(), ref.adjoint(hh)) <= TOL64


def test_dot_product_f32(dev):
    pb = synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=150, n_sensors=32)
    op = _gpu_op(pb, "f32", dev)
    rng = np.random.default_rng(10)
    x = _t(rng.standard_normal(pb.shape), "f32", dev)
    h = _t(rng.standard_normal((pb.Nt, op.Ns)), "f32", dev)
    Hx = op.forward(x).double()
    HTh = op.adjoint(h).double()
    lhs = torch.sum(Hx * h.double()).item()
    rhs = torch.sum(x.double() * HTh).item()
    assert abs(lhs - rhs) <= 1e-5 * Hx.norm().item() * h.double().norm().item()


def test_host_pointer_path_and_determinism(dev):
    pb = synth.small_lossy_2d(shape=(48, 48), pml=6, Nt=60, n_sensors=16)
    op = _gpu_op(pb, "f32", dev)
    x = _t(pb.p0, "f32", dev)
    d1 = op.forward(x).cpu()
    d2 = op.forward(x).cpu()
    d_host = op.forward(x.cpu())
    assert torch.equal(d1, d2) and torch.equal(d1, d_host)
    g1 = op.adjoint(d1.to(dev)).cpu()
    g_host = op.adjoint(d1)
    assert torch.equal(g1, g_host)


def test_one_shot_pat_forward(dev):
    from paper_1603_02329_gb300.api import pat_forward

    pb = synth.small_lossy_2d(shape=(32, 40), pml=4, Nt=30, n_sensors=10)
    ref = Operator.from_problem(pb)
    d = pat_forward(_t(pb.p0, "f64", dev), pb.c, pb.rho, pb.alpha0, pb.y, pb.shape, pb.spacing, pb.pml, pb.pml_alpha,
                    sensor_pos=pb.sensor_pos, dt=pb.dt, Nt=pb.Nt, precision="f64")
    assert rel(d.cpu().numpy(), ref.forward(pb.p0)) <= TOL64


def test_disc_phantom_168_f64_full_size(dev):
    # 128^2 interior + 20-point outer PML, 256 sensors on a 5.5 mm circle, Nt = 600, FP64
    pb = synth.disc_phantom_2d()
    ref = Operator.from_problem(pb)
    op = _gpu_op(pb, "f64", dev)
    d = op.forward(_t(pb.p0, "f64", dev)).cpu().numpy()
    d_ref = ref.forward(pb.p0)
    assert rel(d, d_ref) <= TOL64
    g = op.adjoint(_t(d_ref, "f64", dev)).cpu().numpy()
    assert rel(g, ref.adjoint(d_ref)) <= TOL64


def test_vessel_512_full_size_and_dot(dev):
    # 512^2 heterogeneous absorbing medium, Nt = 2000, 512 line sensors: the launch configuration
    # the benchmark times, compared with the oracle over the whole record (all 2000 samples, about
    # 35 s of oracle per solve): the forward data, the adjoint of a residual over all 2000 samples,
    # and the dot identity.  The late part of the record (after the first arrival near step 300:
    # the phantom starts 76 px away, ~4 steps per px) is also compared on its own.
    pb = synth.vessel_phantom_2d()
    ref = Operator.from_problem(pb)
    op = _gpu_op(pb, "f32", dev)
    d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
    assert d.shape == (2000, 512)
    d_ref = ref.forward(pb.p0)
    assert rel(d, d_ref) <= TOL32
    assert rel(d[1000:], d_ref[1000:]) <= TOL32
    rng = np.random.default_rng(12)
    h = rng.standard_normal((pb.Nt, op.Ns))
    g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
    assert rel(g, ref.adjoint(h)) <= TOL32
    x = _t(rng.standard_normal(pb.shape), "f32", dev)
    hh = _t(rng.standard_normal((pb.Nt, op.Ns)), "f32", dev)
    Hx = op.forward(x).double()
    HTh = op.adjoint(hh).double()
    lhs = torch.sum(Hx * hh.double()).item()
    rhs = torch.sum(x.double() * HTh).item()
    assert abs(lhs - rhs) <= 1e-5 * Hx.norm().item() * hh.double().norm().item()
    assert np.isfinite(d).all() and np.abs(d).max() > 0


def test_tube_128_full_size_prefix_and_dot(dev):
    # 128^3 heterogeneous absorbing medium, Nt = 1000, 64 x 64 sensors: the launch configuration the
    # benchmark times (per-phase graph, tuned layout, the kernels compiled for 128-point lines).
    # Prefix of K samples vs the oracle (causality), adjoint of a residual supported on that prefix
    # vs the oracle, and the dot identity over all 1000 samples.  The tubes start 6 px beyond the
    # sensor plane (about 3.3 steps per px at CFL 0.3), so K = 40 holds arrived signal.
    pb = synth.tube_phantom_3d(seed=3, n=128, pml=10, Nt=1000, sensors=64)
    K = 40
    ref = Operator.from_problem(pb, Nt=K)
    op = _gpu_op(pb, "f32", dev)
    assert op.info.path == 0
    d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
    assert d.shape == (1000, 64 * 64)
    d_ref = ref.forward(pb.p0)
    assert np.abs(d_ref[K - 10:]).max() > 1e-2 * np.abs(pb.p0).max()
    assert rel(d[:K], d_ref) <= TOL32
    rng = np.random.default_rng(13)
    h = np.zeros((pb.Nt, op.Ns))
    h[:K] = rng.standard_normal((K, op.Ns))
    g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
    assert rel(g, ref.adjoint(h[:K])) <= TOL32
    x = _t(rng.standard_normal(pb.shape), "f32", dev)
    hh = _t(rng.standard_normal((pb.Nt, op.Ns)), "f32", dev)
    Hx = op.forward(x).double()
    HTh = op.adjoint(hh).double()
    lhs = torch.sum(Hx * hh.double()).item()
    rhs = torch.sum(x.double() * HTh).item()
    assert abs(lhs - rhs) <= 1e-5 * Hx.norm().item() * hh.double().norm().item()


def test_tube_256_full_size_prefix_adjoint_and_dot(dev):
    # 256^3, Nt = 1500, 128 x 128 sensors: the benchmark's default configuration (about 2.5 GB of
    # device state, the kernels compiled for 256-point lines).  The oracle at this size manages a
    # few dozen steps: the first KF = 24 samples of the forward record, the adjoint of a residual
    # supported on the first K = 3 samples (the adjoint wave spreads from the sensor plane for 3
    # steps) vs the oracle, and the dot identity over all 1500 samples.  The phantom's tubes start
    # 6 px beyond the sensor plane (about 3.3 steps per px), so over the first 24 samples most of its
    # record is the pre-arrival floor, ~1e-6 of the field, where FP32 rounding of the field decides
    # the error; the forward prefix therefore adds a smooth ball 5 px from the plane, whose wave
    # reaches the sensors within the prefix.
    pb = synth.tube_phantom_3d(seed=3, n=256, pml=20, Nt=1500, sensors=128)
    KF = 24
    op = _gpu_op(pb, "f32", dev)
    assert op.info.path == 0
    zz, yy, xx = np.meshgrid(*[np.arange(256)] * 3, indexing="ij")
    x0 = pb.p0 + np.exp(-((zz - 25.0) ** 2 + (yy - 128.0) ** 2 + (xx - 128.0) ** 2) / (2 * 2.0 ** 2))
    d = op.forward(_t(x0, "f32", dev)).cpu().numpy()
    d_ref = Operator.from_problem(pb, Nt=KF).forward(x0)
    assert np.abs(d_ref[KF - 4:]).max() > 5e-2 * np.abs(x0).max()
    assert rel(d[:KF], d_ref) <= TOL32
    K = 3
    ref = Operator.from_problem(pb, Nt=K)
    rng = np.random.default_rng(14)
    h = np.zeros((pb.Nt, op.Ns))
    h[:K] = rng.standard_normal((K, op.Ns))
    g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
    g_ref = ref.adjoint(h[:K])
    assert np.abs(g_ref).max() > 0
    assert rel(g, g_ref) <= TOL32
    x = _t(rng.standard_normal(pb.shape), "f32", dev)
    hh = _t(rng.standard_normal((pb.Nt, op.Ns)), "f32", dev)
    Hx = op.forward(x).double()
    HTh = op.adjoint(hh).double()
    lhs = torch.sum(Hx * hh.double()).item()
    rhs = torch.sum(x.double() * HTh).item()
    assert abs(lhs - rhs) <= 1e-5 * Hx.norm().item() * hh.double().norm().item()


def test_both_2d_paths_agree_with_oracle(dev, monkeypatch):
    # 2-D plans use the persistent single-kernel path when the per-CTA state fits in shared
    # memory; PAT_PERSIST=0 forces the per-phase CUDA-graph path.  Both must match the oracle.
    pb = synth.small_lossy_2d(shape=(64, 80), pml=8, Nt=120, n_sensors=24)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(13).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    for flag, path, width in (("1", 1, "0"), ("1", 1, "2"), ("0", 0, "0")):
        monkeypatch.setenv("PAT_PERSIST", flag)
        monkeypatch.setenv("PAT_PERSIST_W", width)   # 0: automatic layout; 2: two columns per CTA
        for prec, tol in (("f32", TOL32), ("f64", TOL64)):
            op = _gpu_op(pb, prec, dev)
            assert op.info.path == path
            assert rel(op.forward(_t(pb.p0, prec, dev)).cpu().numpy(), d_ref) <= tol
            assert rel(op.adjoint(_t(h, prec, dev)).cpu().numpy(), g_ref) <= tol
            op.close()


# Power-of-two 2-D grids take the persistent kernel with register-fused transforms (path 2); the
# cases cover every radix schedule it uses: r0 = 2, 4, 8 and two to four stages per axis
# (16 = 2.8, 32 = 4.8, 64 = 8.8, 128 = 2.8.8, 256 = 4.8.8, 1024 = 2.8.8.8), non-square grids in both
# orientations, lossless and absorbing media, FP32 and FP64.  PAT_P2=0 selects the generic
# persistent kernel on the same plan, which must agree too.
P2_CASES = [
    ("16x16_lossless_f64", dict(shape=(16, 16), pml=2, Nt=30, n_sensors=6, alpha0=0.0), "f64"),
    ("32x64_lossy_f64", dict(shape=(32, 64), pml=4, Nt=60, n_sensors=12), "f64"),
    ("64x32_lossless_f32", dict(shape=(64, 32), pml=4, Nt=70, n_sensors=12, alpha0=0.0), "f32"),
    ("128x128_lossy_f32", dict(shape=(128, 128), pml=10, Nt=150, n_sensors=40), "f32"),
    ("256x32_lossy_f64", dict(shape=(256, 32), pml=4, Nt=50, n_sensors=16), "f64"),
    ("16x1024_lossy_f32", dict(shape=(16, 1024), pml=2, Nt=40, n_sensors=8, sensor_radius_frac=0.3), "f32"),
    ("1024x16_lossless_f32", dict(shape=(1024, 16), pml=2, Nt=40, n_sensors=8, alpha0=0.0), "f32"),
]


@pytest.mark.parametrize("name,kw,prec", P2_CASES, ids=[c[0] for c in P2_CASES])
def test_pow2_persistent_kernel_matches_oracle(dev, monkeypatch, name, kw, prec):
    pb = synth.small_lossy_2d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(17).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    tol = TOL32 if prec == "f32" else TOL64
    out = {}
    for flag, paths in (("1", (2,)), ("0", (1, 0))):
        # without the fused kernel the plan takes the generic persistent kernel, or the graph path
        # where the generic kernel's column buffers do not fit (ny = 1024 with four columns per CTA)
        monkeypatch.setenv("PAT_P2", flag)
        op = _gpu_op(pb, prec, dev)
        assert op.info.path in paths
        path = paths[0]
        d = op.forward(_t(pb.p0, prec, dev)).cpu().numpy()
        g = op.adjoint(_t(h, prec, dev)).cpu().numpy()
        assert rel(d, d_ref) <= tol, (path, rel(d, d_ref))
        assert rel(g, g_ref) <= tol, (path, rel(g, g_ref))
        out[path] = (d, g)
        op.close()
    assert rel(out[2][0], out[1][0]) <= tol and rel(out[2][1], out[1][1]) <= tol


def test_persistent_status_word_ok(dev):
    from paper_1603_02329_gb300 import _lib

    pb = synth.small_lossy_2d(shape=(48, 48), pml=6, Nt=30, n_sensors=8)
    op = _gpu_op(pb, "f32", dev)
    op.forward(_t(pb.p0, "f32", dev))
    assert _lib.lib().pat_plan_status(op._plan) == 0


@pytest.mark.parametrize("persist", ["1", "0"])
def test_autotuned_layout_gives_the_same_results(dev, monkeypatch, persist):
    # plan creation times the feasible launch layouts (PAT_AUTOTUNE=0: the first feasible one);
    # the layout changes how lines are grouped into CTAs, not the arithmetic of any line
    pb = synth.small_lossy_2d(shape=(64, 80), pml=8, Nt=60, n_sensors=24)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(23).standard_normal((pb.Nt, ref.Ns))
    monkeypatch.setenv("PAT_PERSIST", persist)
    out = {}
    for tune in ("1", "0"):
        monkeypatch.setenv("PAT_AUTOTUNE", tune)
        op = _gpu_op(pb, "f64", dev)
        assert op.info.tuned == (1 if tune == "1" else 0)
        assert op.info.layout[0] >= 1 and op.info.layout[1] >= 1
        out[tune] = (op.forward(_t(pb.p0, "f64", dev)).cpu().numpy(), op.adjoint(_t(h, "f64", dev)).cpu().numpy())
        assert rel(out[tune][0], ref.forward(pb.p0)) <= TOL64
        op.close()
    assert rel(out["1"][0], out["0"][0]) <= 1e-13 and rel(out["1"][1], out["0"][1]) <= 1e-13


@pytest.mark.parametrize("p2", ["1", "0"])
def test_persistent_barrier_timeout_is_reported_and_recovers(dev, monkeypatch, p2):
    # Failure detection without a GPU fault: pat_plan_set_fault makes every grid barrier wait for an
    # arrival that never comes; the bounded wait (0.2 s here) runs out, the kernel records
    # PAT_ETIMEOUT and returns, the host reads it, and the context stays usable.
    import time

    from paper_1603_02329_gb300 import _lib

    monkeypatch.setenv("PAT_P2", p2)
    pb = synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=30, n_sensors=12)
    op = _gpu_op(pb, "f32", dev)
    assert op.info.path == (2 if p2 == "1" else 1)
    L = _lib.lib()
    x = _t(pb.p0, "f32", dev)
    good = op.forward(x).cpu().numpy()
    assert L.pat_plan_set_fault(op._plan, 1, 0.2) == 0
    t0 = time.perf_counter()
    op.forward(x)
    st = L.pat_plan_status(op._plan)
    waited = time.perf_counter() - t0
    assert st == 5                          # PAT_ETIMEOUT
    assert waited < 5.0                     # bounded: ~0.2 s, not a hang
    assert L.pat_plan_set_fault(op._plan, 0, 2.0) == 0
    again = op.forward(x).cpu().numpy()
    assert L.pat_plan_status(op._plan) == 0
    assert np.array_equal(again, good)
    assert L.pat_plan_set_fault(op._plan, 2, 1.0) != 0      # invalid arguments are rejected


# Kernels compiled for fixed line lengths (float fields): the 2-D persistent kernel for 256^2 and
# 512^2 grids, the 3-D spectral kernels for y / z lines and the 3-D row kernels for x-lines of 64,
# 128 and 256 points.  Their arithmetic is that of the kernels for any length (only the index
# arithmetic is resolved at compile time), which PAT_P2SPEC=0 selects: both must match the
# oracle, and each other.
FIXED_CASES = [
    ("2d_256x256_lossy", "2d", dict(shape=(256, 256), pml=12, Nt=80, n_sensors=32)),
    ("2d_512x512_lossless", "2d", dict(shape=(512, 512), pml=20, Nt=40, n_sensors=32, alpha0=0.0)),
    ("3d_16x128x64_lossy", "3d", dict(shape=(16, 128, 64), pml=3, Nt=24)),        # y 128, x 64
    ("3d_16x256x128_lossy", "3d", dict(shape=(16, 256, 128), pml=3, Nt=20)),      # y 256, x 128
    ("3d_256x16x256_lossless", "3d", dict(shape=(256, 16, 256), pml=3, Nt=16, alpha0=0.0)),   # z 256, x 256
]


@pytest.mark.parametrize("name,kind,kw", FIXED_CASES, ids=[c[0] for c in FIXED_CASES])
def test_fixed_length_kernels_match_generic_and_oracle(dev, monkeypatch, name, kind, kw):
    pb = synth.small_lossy_3d(**kw) if kind == "3d" else synth.small_lossy_2d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(31).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_P2SPEC", flag)
        op = _gpu_op(pb, "f32", dev)
        assert op.info.path == (2 if kind == "2d" else 0)
        d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
        g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
        assert rel(d, d_ref) <= TOL32, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= TOL32, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    assert rel(out[0][0], out[1][0]) <= 1e-6 and rel(out[0][1], out[1][1]) <= 1e-6


# 3-D lines of 128 and 256 points: the plain y transforms take the two-stage spectral schedule
# (k_spec16: radices n/16 and 16); PAT_SPEC16=2 puts the fused multiply passes on it as well, 0
# none (the fixed-length k_spec2, radices r0, 8, 8).  All against the oracle and each other.
SPEC16_CASES = [
    ("3d_128x32x16_lossy", dict(shape=(128, 32, 16), pml=3, Nt=24)),       # z 128 (8 x 16), y 32
    ("3d_16x256x32_lossless", dict(shape=(16, 256, 32), pml=3, Nt=20, alpha0=0.0)),   # y 256 (16 x 16)
]


@pytest.mark.parametrize("name,kw", SPEC16_CASES, ids=[c[0] for c in SPEC16_CASES])
def test_two_stage_spectral_schedule_matches_oracle(dev, monkeypatch, name, kw):
    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(37).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    out = []
    for flag in ("2", "3", "1", "0"):   # every pass / plain + field-wise multiply passes / plain / none
        monkeypatch.setenv("PAT_SPEC16", flag)
        op = _gpu_op(pb, "f32", dev)
        d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
        g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
        assert rel(d, d_ref) <= TOL32, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= TOL32, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    for a in out[:3]:
        assert rel(a[0], out[3][0]) <= 1e-6 and rel(a[1], out[3][1]) <= 1e-6


@pytest.mark.parametrize("name,kw", SPEC16_CASES, ids=[c[0] for c in SPEC16_CASES])
def test_autotuned_radix_schedule_matches_oracle(dev, monkeypatch, name, kw):
    # without PAT_SPEC16 the plan-time tuner times the three radix schedules with the launch layouts
    # and keeps the fastest; whichever it picks, the solve matches the oracle
    monkeypatch.delenv("PAT_SPEC16", raising=False)
    monkeypatch.delenv("PAT_AUTOTUNE", raising=False)
    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(38).standard_normal((pb.Nt, ref.Ns))
    op = _gpu_op(pb, "f32", dev)
    assert op.info.path == 0 and op.info.tuned == 1
    assert op.info.schedule in (0, 1, 2, 3)
    assert rel(op.forward(_t(pb.p0, "f32", dev)).cpu().numpy(), ref.forward(pb.p0)) <= TOL32
    assert rel(op.adjoint(_t(h, "f32", dev)).cpu().numpy(), ref.adjoint(h)) <= TOL32
    monkeypatch.setenv("PAT_SPEC16", "2")
    assert _gpu_op(pb, "f32", dev).info.schedule == 2


@pytest.mark.parametrize("chunks", ["2", "3", "64"])
def test_chunked_spectral_passes_are_bitwise_equal(dev, monkeypatch, chunks):
    # a 3-D spectral operation run chunk by chunk over its column tiles does the same arithmetic per
    # tile: the solves are bitwise equal to the unchunked ones and match the oracle (64 chunks: more
    # than there are tiles, so one tile per chunk)
    pb = synth.small_lossy_3d(shape=(16, 32, 64), pml=3, Nt=20)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(39).standard_normal((pb.Nt, ref.Ns))
    outs = []
    monkeypatch.setenv("PAT_AUTOTUNE", "0")   # the same layout and radix schedule for both plans
    for c in ("1", chunks):
        monkeypatch.setenv("PAT_SPEC_CHUNKS", c)
        op = _gpu_op(pb, "f32", dev)
        outs.append((op.forward(_t(pb.p0, "f32", dev)), op.adjoint(_t(h, "f32", dev)), op.info.spec_chunks))
        op.close()
    assert outs[0][2] == 1 and outs[1][2] > 1
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert rel(outs[1][0].cpu().numpy(), ref.forward(pb.p0)) <= TOL32


@pytest.mark.parametrize("shape", [(16, 32, 64), (32, 64, 40), (64, 16, 32)])
def test_tensor_copy_staging_is_bitwise_equal(dev, monkeypatch, shape):
    from paper_1603_02329_gb300 import _lib

    # the 3-D spectral passes stage their 8-column tiles with tensor copies (cp.async.bulk.tensor) by
    # default, or with cp.async under PAT_TMA=0; the staged data and so the solves are identical
    pb = synth.small_lossy_3d(shape=shape, pml=3, Nt=16)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(41).standard_normal((pb.Nt, ref.Ns))
    monkeypatch.setenv("PAT_AUTOTUNE", "0")
    monkeypatch.setenv("PAT_COL_W", "8")
    outs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_TMA", flag)
        op = _gpu_op(pb, "f32", dev)
        outs.append((op.forward(_t(pb.p0, "f32", dev)), op.adjoint(_t(h, "f32", dev)), op.info.tma))
        assert _lib.lib().pat_plan_status(op._plan) == 0
        op.close()
    assert outs[0][2] == 1 and outs[1][2] == 0
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert rel(outs[0][0].cpu().numpy(), ref.forward(pb.p0)) <= TOL32
    assert rel(outs[0][1].cpu().numpy(), ref.adjoint(h)) <= TOL32


@pytest.mark.parametrize("name,kw", [("256x16x32_lossy", dict(shape=(256, 16, 32), pml=3, Nt=18)),
                                     ("256x32x16_lossless", dict(shape=(256, 32, 16), pml=3, Nt=16, alpha0=0.0)),
                                     ("256x16x48_lossy_generic_x", dict(shape=(256, 16, 48), pml=3, Nt=14))])
def test_register_z_passes_match_oracle(dev, monkeypatch, name, kw):
    # the z passes with the multiply on 256-point z-lines held in registers (16 x 16 transform per
    # half-warp, tiles by tensor copies under the 64-byte swizzle; the default for the D- passes,
    # PAT_ZREG=2 for every multiply pass) against the oracle and against the shared-memory z passes
    # (different rounding order: within 1e-6)
    from paper_1603_02329_gb300 import _lib

    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(43).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    monkeypatch.setenv("PAT_AUTOTUNE", "0")
    monkeypatch.setenv("PAT_COL_W", "8")
    monkeypatch.setenv("PAT_ZWIDE", "0")   # the 16-column field-wise z passes would take DIV and DIVT
    out = []
    for flag in ("2", "1", "0"):   # every multiply pass / the D- passes / none
        monkeypatch.setenv("PAT_ZREG", flag)
        op = _gpu_op(pb, "f32", dev)
        assert op.info.zreg == (flag != "0")
        d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
        g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
        assert _lib.lib().pat_plan_status(op._plan) == 0
        assert rel(d, d_ref) <= TOL32, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= TOL32, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    for a in out[:2]:
        assert rel(a[0], out[2][0]) <= 1e-6 and rel(a[1], out[2][1]) <= 1e-6


# shapes are (nz, ny, nx); nxh = nx / 2 + 1 half-spectrum columns make ceil(nxh / 16) tiles of 16.
# The tensor-copy staging (and so the 16-column passes) needs power-of-two y- and z-lines of 16 to 256
# points.
@pytest.mark.parametrize("name,kw", [("16x256x48_lossy", dict(shape=(16, 256, 48), pml=3, Nt=16)),
                                     ("16x128x64_lossless", dict(shape=(16, 128, 64), pml=3, Nt=16, alpha0=0.0)),
                                     ("16x256x256_lossy", dict(shape=(16, 256, 256), pml=3, Nt=8)),
                                     ("32x256x12_lossy", dict(shape=(32, 256, 12), pml=3, Nt=16))])
def test_wide_y_passes_match_oracle(dev, monkeypatch, name, kw):
    # the plain y transforms of 128- and 256-point y-lines on 16-column tiles, one field per CTA, in
    # place in the tile staged by one tensor copy (the default), against the oracle and against the
    # 8-column k_spec16 passes of the same two-stage schedule (PAT_YWIDE=0); nxh = 25, 33, 129, 7:
    # 2, 3, 9 and 1 tiles, the last one partly valid
    from paper_1603_02329_gb300 import _lib

    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(44).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    monkeypatch.setenv("PAT_AUTOTUNE", "0")
    monkeypatch.setenv("PAT_COL_W", "8")
    monkeypatch.setenv("PAT_SPEC16", "1")
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_YWIDE", flag)
        op = _gpu_op(pb, "f32", dev)
        assert op.info.ywide == (flag == "1")
        d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
        g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
        assert _lib.lib().pat_plan_status(op._plan) == 0
        assert rel(d, d_ref) <= TOL32, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= TOL32, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    print(f"{name}: wide against 8-column y passes: forward {rel(out[0][0], out[1][0]):.2e}, "
          f"adjoint {rel(out[0][1], out[1][1]):.2e}")
    assert rel(out[0][0], out[1][0]) <= 1e-6 and rel(out[0][1], out[1][1]) <= 1e-6


@pytest.mark.parametrize("name,kw", [("256x16x48_lossy", dict(shape=(256, 16, 48), pml=3, Nt=16)),
                                     ("128x16x64_lossy", dict(shape=(128, 16, 64), pml=3, Nt=16)),
                                     ("128x32x32_lossless", dict(shape=(128, 32, 32), pml=3, Nt=16, alpha0=0.0)),
                                     ("256x16x256_lossy", dict(shape=(256, 16, 256), pml=3, Nt=8))])
def test_wide_z_passes_match_oracle(dev, monkeypatch, name, kw):
    # the z passes with the multiply (D+, D-, their transposes, the absorption pass) of 128- and
    # 256-point z-lines on 16-column tiles, the multipliers from the plan's tables (the default),
    # against the oracle and against the 8-column z passes (PAT_ZWIDE=0: k_zreg for D- and its
    # transpose on 256-point lines, k_spec2 otherwise); shapes (nz, ny, nx), 2, 3, 2 and 9 tiles
    from paper_1603_02329_gb300 import _lib

    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(45).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    monkeypatch.setenv("PAT_AUTOTUNE", "0")
    monkeypatch.setenv("PAT_COL_W", "8")
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_ZWIDE", flag)
        op = _gpu_op(pb, "f32", dev)
        assert op.info.zwide == (flag == "1")
        d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
        g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
        assert _lib.lib().pat_plan_status(op._plan) == 0
        assert rel(d, d_ref) <= TOL32, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= TOL32, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    print(f"{name}: wide against 8-column z passes: forward {rel(out[0][0], out[1][0]):.2e}, "
          f"adjoint {rel(out[0][1], out[1][1]):.2e}")
    assert rel(out[0][0], out[1][0]) <= 1e-6 and rel(out[0][1], out[1][1]) <= 1e-6


@pytest.mark.parametrize("name,kw", [("12x16x128_lossy", dict(shape=(12, 16, 128), pml=3, Nt=18)),
                                     ("8x12x256_lossless", dict(shape=(8, 12, 256), pml=2, Nt=14, alpha0=0.0)),
                                     ("16x16x256_lossy", dict(shape=(16, 16, 256), pml=3, Nt=14))])
def test_one_component_momentum_rows_match_oracle(dev, monkeypatch, name, kw):
    # the u update and its transpose with one velocity component per CTA (the default for FP32 3-D
    # x-lines of 128 and 256 points) against the oracle and against k_row2's three components per
    # CTA (PAT_ROWU1=0), for 2 to 32 x-lines per CTA of the one-component kernels (32: more than
    # 8 x 12 x 256 has in a multiple, so its default of 16 runs)
    pb = synth.small_lossy_3d(**kw)
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(46).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    monkeypatch.setenv("PAT_AUTOTUNE", "0")
    monkeypatch.setenv("PAT_ROW_LINES", "8")
    for lines in ("16", "8", "2", "32"):
        monkeypatch.setenv("PAT_ROWU1_LINES", lines)
        out = []
        for flag in ("1", "0"):
            monkeypatch.setenv("PAT_ROWU1", flag)
            op = _gpu_op(pb, "f32", dev)
            assert op.info.rowu1 == (flag == "1") and op.info.layout[1] == 8
            d = op.forward(_t(pb.p0, "f32", dev)).cpu().numpy()
            g = op.adjoint(_t(h, "f32", dev)).cpu().numpy()
            assert rel(d, d_ref) <= TOL32, (lines, flag, rel(d, d_ref))
            assert rel(g, g_ref) <= TOL32, (lines, flag, rel(g, g_ref))
            out.append((d, g))
            op.close()
        assert rel(out[0][0], out[1][0]) <= 1e-6 and rel(out[0][1], out[1][1]) <= 1e-6


@pytest.mark.parametrize("persist", ["1", "0"])
def test_non_finite_output_is_reported(dev, monkeypatch, persist):
    # Failure detection on the host side of a solve: a NaN in p0 (forward) or in the residual
    # (adjoint) spreads through the transforms; the device-side scan of the output records
    # PAT_ENONFINITE, pat_plan_status reports it, and the next clean solve clears it.  NaN arithmetic
    # changes no control flow in the kernels.
    from paper_1603_02329_gb300 import _lib

    monkeypatch.setenv("PAT_PERSIST", persist)
    pb = synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=30, n_sensors=12)
    op = _gpu_op(pb, "f32", dev)
    assert op.info.path == (2 if persist == "1" else 0)
    L = _lib.lib()
    x = np.array(pb.p0)
    d = op.forward(_t(x, "f32", dev))
    assert L.pat_plan_status(op._plan) == 0
    x[20, 30] = np.nan
    op.forward(_t(x, "f32", dev))
    assert L.pat_plan_status(op._plan) == _lib.PAT_ENONFINITE
    assert "NaN" in L.pat_last_error().decode()
    d2 = op.forward(_t(pb.p0, "f32", dev))
    assert L.pat_plan_status(op._plan) == 0
    assert torch.equal(d, d2)
    h = np.random.default_rng(3).standard_normal((pb.Nt, op.Ns))
    h[5, 2] = np.inf
    op.adjoint(_t(h, "f32", dev))
    assert L.pat_plan_status(op._plan) == _lib.PAT_ENONFINITE
    h[5, 2] = 0.0
    op.adjoint(_t(h, "f32", dev))
    assert L.pat_plan_status(op._plan) == 0
    op.close()


# Power-of-two y (and z) axes take the register-fused spectral kernel of the per-phase path
# (k_spec2); PAT_SPEC2=0 selects the generic one.  3-D grids (always the per-phase path) and a
# 2-D grid forced onto it; radix schedules 16 = 2.8, 32 = 4.8, 64 = 8.8, 128 = 2.8.8.
SPEC2_CASES = [
    ("3d_16x32x64_lossy_f32", "3d", dict(shape=(16, 32, 64), pml=3, Nt=30), "f32"),
    ("3d_32x16x24_lossy_f64", "3d", dict(shape=(32, 16, 24), pml=3, Nt=24), "f64"),
    ("3d_64x64x32_lossless_f32", "3d", dict(shape=(64, 64, 32), pml=4, Nt=30, alpha0=0.0), "f32"),
    ("2d_graph_128x64_lossy_f64", "2d", dict(shape=(128, 64), pml=6, Nt=40, n_sensors=16), "f64"),
]


@pytest.mark.parametrize("name,kind,kw,prec", SPEC2_CASES, ids=[c[0] for c in SPEC2_CASES])
def test_pow2_spectral_kernel_matches_oracle(dev, monkeypatch, name, kind, kw, prec):
    pb = synth.small_lossy_3d(**kw) if kind == "3d" else synth.small_lossy_2d(**kw)
    if kind == "2d":
        monkeypatch.setenv("PAT_PERSIST", "0")
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(19).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    tol = TOL32 if prec == "f32" else TOL64
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_SPEC2", flag)
        op = _gpu_op(pb, prec, dev)
        assert op.info.path == 0
        d = op.forward(_t(pb.p0, prec, dev)).cpu().numpy()
        g = op.adjoint(_t(h, prec, dev)).cpu().numpy()
        assert rel(d, d_ref) <= tol, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= tol, (flag, rel(g, g_ref))
        out.append((d, g))
        op.close()
    assert rel(out[0][0], out[1][0]) <= tol and rel(out[0][1], out[1][1]) <= tol


# Power-of-two x-lines take the register-fused row kernels of the per-phase path (k_row2);
# PAT_ROW2=0 selects the generic ones.  Forward, adjoint and the checkpointed c0^2 gradient (whose
# hooks live in the row kernels) against the oracle, both kernels.
ROW2_CASES = [
    ("3d_16x32x64_lossy_f32", "3d", dict(shape=(16, 32, 64), pml=3, Nt=30), "f32"),
    ("3d_24x20x32_lossy_f64", "3d", dict(shape=(24, 20, 32), pml=3, Nt=22), "f64"),
    ("3d_32x32x16_lossless_f64", "3d", dict(shape=(32, 32, 16), pml=3, Nt=25, alpha0=0.0), "f64"),
    ("2d_graph_64x128_lossy_f32", "2d", dict(shape=(64, 128), pml=6, Nt=40, n_sensors=16), "f32"),
    ("2d_graph_96x64_lossless_f64", "2d", dict(shape=(96, 64), pml=6, Nt=30, n_sensors=12, alpha0=0.0), "f64"),
]


@pytest.mark.parametrize("name,kind,kw,prec", ROW2_CASES, ids=[c[0] for c in ROW2_CASES])
def test_pow2_row_kernels_match_oracle(dev, monkeypatch, name, kind, kw, prec):
    from oracle import pat_medium as pm

    pb = synth.small_lossy_3d(**kw) if kind == "3d" else synth.small_lossy_2d(**kw)
    if kind == "2d":
        monkeypatch.setenv("PAT_PERSIST", "0")
    ref = Operator.from_problem(pb)
    h = np.random.default_rng(29).standard_normal((pb.Nt, ref.Ns))
    d_ref, g_ref = ref.forward(pb.p0), ref.adjoint(h)
    c2_ref, _ = pm.sound_speed_gradient(ref, pb.p0, h, pb.y)
    tol = TOL32 if prec == "f32" else TOL64
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("PAT_ROW2", flag)
        op = _gpu_op(pb, prec, dev)
        assert op.info.path == 0
        d = op.forward(_t(pb.p0, prec, dev)).cpu().numpy()
        g = op.adjoint(_t(h, prec, dev)).cpu().numpy()
        gc2 = op.gradient_c2(_t(pb.p0, prec, dev), _t(h, prec, dev), checkpoint_every=7).cpu().numpy()
        assert rel(d, d_ref) <= tol, (flag, rel(d, d_ref))
        assert rel(g, g_ref) <= tol, (flag, rel(g, g_ref))
        assert rel(gc2, c2_ref) <= (tol if prec == "f32" else 1e-10), (flag, rel(gc2, c2_ref))
        out.append((d, g))
        op.close()
    assert rel(out[0][0], out[1][0]) <= tol and rel(out[0][1], out[1][1]) <= tol
