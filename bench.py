"""Benchmark of the forward + adjoint solve pair (one H^T H product) on GB300.

Workload (default): 3-D 256^3 heterogeneous absorbing medium (c = 1500 +/- 100 m/s, rho = 1000
+/- 5 %, alpha0 = 0.75 dB MHz^-1.5 cm^-1, y = 1.5), 20-point PML, a 128 x 128 on-grid planar
sensor array at stride 2, Nt = 1500, FP32 fields (about 1 GB of state: larger than L2).  One step =
pat_forward_plan + pat_adjoint through the C ABI: 2 N Nt grid-point-steps.  value = grid-point-steps
per second over all ranks (Gpt-steps/s).

The default run adds these records to the JSON line:
  - "vessel2d_512": the same measurement on the 2-D 512^2 absorbing workload (Nt = 2000, 512 line
    sensors), whose state stays in shared memory (one persistent kernel per solve), with the
    time-reversal image, FISTA warm-started from it, the adjoint-then-discretize deviation, and the
    oracle's bounded sample timed on one core and as one replica per host core;
  - "mg_vs_fista": wall time of 3-level MG-FISTA (256^3 / 128^3 / 64^3) and of single-grid FISTA to
    the same relative error on 40 dB data, 12 iterations of FISTA at most;
  - "mg_precision": relative L2 distance of the FP32 iterates from the FP64 iterates of the same
    MG-FISTA and FISTA runs on a small 2-D case, per iteration;
  - "mg_vs_fista_refined_2d": 2-level MG-FISTA vs FISTA at 512^2 on data generated on a finer grid
    from contaminated maps (no inverse crime);
  - "batch": eight uneven 2-D instances as one batched launch vs one at a time.

Multi-GPU: one independent instance per rank (weak scaling, no collective on the data path).

``--impl reference`` times the FP64 CPU oracle (the test oracle under ``oracle/``) on a bounded
sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adj Gpt-steps/s (%HBM roofline); MG-FISTA vs FISTA time to target RE"
UNIT = "Gpt-steps/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="tube3d_256",
                    choices=["vessel2d_512", "disc2d_168", "tube3d_128", "tube3d_256"])
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the 2-D 512^2 record that the default 256^3 run adds")
    ap.add_argument("--no-mg", action="store_true",
                    help="skip the MG-FISTA vs FISTA and FP32-vs-FP64 records of the default 256^3 run")
    ap.add_argument("--nt", type=int, default=0,
                    help="override the workload's time axis (small cases for profiler captures only)")
    ap.add_argument("--probe-stride", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mg", action="store_true", help="also time MG-FISTA vs FISTA to a target RE")
    ap.add_argument("--mg-iters", type=int, default=0,
                    help="FISTA iterations of the MG comparison (0: 12 at 256^3, else 20)")
    ap.add_argument("--mg-levels", type=int, default=0, help="levels of MG-FISTA (0: 3 at 256^3, else 2)")
    ap.add_argument("--mg-data", default="same", choices=["same", "refined"],
                    help="MG comparison data: from the reconstruction grid (inverse crime, stated) or from "
                         "a 1.44x finer grid with 35 dB-contaminated maps (synth.refined_problem)")
    ap.add_argument("--batch", action="store_true",
                    help="also time 8 uneven 2-D instances as one batched launch vs one at a time")
    ap.add_argument("--trace", type=int, default=0,
                    help="persistent path: after the timed steps, record the phase timeline of N grid barriers "
                         "in the middle of one forward solve (pat_plan_set_trace) and report its medians")
    ap.add_argument("--c2grad", type=int, default=0,
                    help="also time the checkpointed c0^2 gradient with this checkpoint interval")
    a = ap.parse_args()
    big = a.workload == "tube3d_256"
    if a.mg_iters <= 0:
        a.mg_iters = 12 if big else 20
    if a.mg_levels <= 0:
        a.mg_levels = 3 if big else 2
    a.mg_default = big and not a.no_mg
    return a


def workload(name, rank):
    from paper_1603_02329_gb300 import synth

    if name == "vessel2d_512":
        pb = synth.vessel_phantom_2d(seed=2 + rank)
        prec = "f32"
        desc = {"workload": "2-D 512^2 heterogeneous absorbing medium (alpha0=0.75, y=1.5), 20-pt PML, "
                            "512 on-grid line sensors, Nt=2000, vessel+disc phantom",
                "grid": [512, 512], "Nt": 2000, "Ns": 512, "pml": 20, "dx_m": 5e-5, "cfl": 0.3}
    elif name.startswith("tube3d_"):
        n = int(name.split("_")[1])
        pml, Nt, ns = (10, 1000, 64) if n == 128 else (20, 1500, 128)
        pb = synth.tube_phantom_3d(seed=3 + rank, n=n, pml=pml, Nt=Nt, sensors=ns)
        prec = "f32"
        desc = {"workload": f"3-D {n}^3 heterogeneous absorbing medium (alpha0=0.75, y=1.5), {pml}-pt PML, "
                            f"{ns}x{ns} planar on-grid sensors at stride 2, Nt={Nt}, tube+ball phantom",
                "grid": [n, n, n], "Nt": Nt, "Ns": ns * ns, "pml": pml, "dx_m": 6.25e-5, "cfl": 0.3}
    else:
        pb = synth.disc_phantom_2d(seed=1 + rank)
        prec = "f64"
        desc = {"workload": "2-D 168^2 homogeneous lossless (128^2 + 20-pt outer PML), 256 circle sensors, "
                            "Nt=600, disc phantom, FP64",
                "grid": [168, 168], "Nt": 600, "Ns": 256, "pml": 20, "dx_m": 1e-4, "cfl": 0.3}
    return pb, prec, desc


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# algorithmic bytes per launch of each kernel (operands read + written once; 2-D, lossy or not)
def kernel_bytes(name, N, Nh, w, D=2, lossy=True):
    Hs = Nh * 2 * w      # one half spectrum
    F = N * w            # one real field
    table = {
        "spec_grad": (1 + D) * Hs,
        "spec_div": 2 * D * Hs,
        "spec_divt": 2 * D * Hs,
        "spec_abs": 4 * Hs,
        "spec_gradt": (D + 1) * Hs,
        "fwd_u": 2 * D * Hs + 3 * D * F,
        "fwd_rho": ((D + 2) * Hs + (2 * D + 2) * F) if lossy else ((D + 1) * Hs + (2 * D + 2) * F),
        "fwd_p": 3 * Hs + 4 * F,
        "adj_rho": (2 + D) * Hs + (3 + 2 * D) * F,
        "adj_u": 2 * D * Hs + 3 * D * F,
        "adj_p": (3 * Hs + 3 * F) if lossy else ((1 + D) * Hs + (2 + 2 * D) * F),
    }
    return table.get(name)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel, from
# ncu captures of the same command with the time axis cut to Nt = 20 (and, for an earlier build of
# the kernel, Nt = 40: the two agreed, forward 8.25 / 8.26 MB, adjoint 6.60 / 6.72 MB; the state
# stays in shared memory, so the traffic is the set-up loads of the medium and tables), so the
# figure is taken as the full-length launch's.  Valid for the kernel version the captures were
# taken of (the 512^2 fixed-size k_persist2 with the one-load barrier poll).
MEASURED_TRAFFIC = {
    ("vessel2d_512", "k_persist2_adj", "k_persist2_adj"): 6.570e6,
    ("vessel2d_512", "k_persist2_fwd", "k_persist2_fwd"): 8.250e6,
    # the y forward transform at 256^3 on 8-column tiles (k_spec16 mode 0, tiles staged with tensor
    # copies; PAT_YWIDE=0), from a capture of the three launches of one forward step (1, 3 and 2 fields:
    # 682.8 MB over 12 field transfers) scaled to the mean launch of a forward + adjoint step (28 field
    # transfers over 6 launches)
    ("tube3d_256", "y_fwd", "k_spec16"): 682.8e6 / 12 * 28 / 6,
    # the y transforms at 256^3 on 16-column tiles (k_ywide, the default), from a capture of the six
    # launches of one forward step: forward 674.3 MB over 12 field transfers, inverse 954.1 MB over 16,
    # scaled to the mean launch of each direction in a forward + adjoint step (28 transfers, 6 launches)
    ("tube3d_256", "y_fwd", "k_ywide"): 674.3e6 / 12 * 28 / 6,
    ("tube3d_256", "y_inv", "k_ywide"): 954.1e6 / 16 * 28 / 6,
}


def measured_traffic(workload, kernel, version):
    """DRAM bytes per launch of `kernel` from an ncu capture of that kernel version, or None."""
    return MEASURED_TRAFFIC.get((workload, kernel, version))


def kernel_version(op, fam):
    """Which compiled kernel runs family `fam` on this plan (the captures above are per version)."""
    if fam.startswith("k_persist"):
        return fam
    if fam in ("y_fwd", "y_inv"):
        return "k_ywide" if int(getattr(op.info, "ywide", 0)) else "k_spec16"
    return None


def solve_bytes(N, Nt, w, D=2, lossy=True):
    # one whole solve (persistent kernel): state (u_xi, rho_xi, p) read + written once and the
    # medium read once per grid-point-step
    return (2 * (2 * D + 1) + (4 if lossy else 2)) * w * N * Nt


def step_schedule(D, lossy):
    """The per-phase launches of one forward and one adjoint step, in order: (graph, probe name,
    compiled-kernel family, spectral fields in, spectral fields out).  In 3-D a spectral operation is
    a y pass, the z pass with the multiply and a y pass back; the y passes of every operation share
    one kernel each way."""
    ops_f = [("spec_grad", 1, D), ("spec_div", D, D)] + ([("spec_abs", 2, 2)] if lossy else [])
    rows_f = ["fwd_u", "fwd_rho"] + (["fwd_p"] if lossy else [])
    ops_a = ([("spec_abs", 2, 2)] if lossy else []) + [("spec_divt", D, D), ("spec_gradt", D, 1)]
    rows_a = (["adj_rho"] if lossy else []) + ["adj_u", "adj_p"]
    out = []
    for g, ops, rows in (("fwd", ops_f, rows_f), ("adj", ops_a, rows_a)):
        for (mode, fi, fo), row in zip(ops, rows):
            if D == 3:
                out += [(g, "spec_y_fwd", "y_fwd", fi, fi), (g, mode, mode, fi, fo), (g, "spec_y_inv", "y_inv", fo, fo)]
            else:
                out.append((g, mode, mode, fi, fo))
            out.append((g, row, row, 0, 0))
    return out


def family_totals(kernels, N, Nh, w, D, lossy, chunks=1):
    """Per compiled-kernel family: launches, probed time [ms] and algorithmic bytes in one forward +
    adjoint step (chunks: each 3-D spectral launch covers 1 / chunks of the column tiles)."""
    Hs = Nh * 2 * w
    fams = {}
    for g, pname, fam, fi, fo in step_schedule(D, lossy):
        spec = pname.startswith("spec")
        n = chunks if (spec and D == 3) else 1
        b = (fi + fo) * Hs if spec else kernel_bytes(pname, N, Nh, w, D=D, lossy=lossy)
        f = fams.setdefault(fam, {"launches": 0, "ms": 0.0, "bytes": 0.0})
        f["launches"] += n
        f["ms"] += n * kernels.get(f"{g}:{pname}", 0.0)
        f["bytes"] += b
    return fams


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock, the maximum clock and the throttle reasons seen Active in the sampled
        csv lines (index, clocks.sm, clocks.max.sm, power, active mask, then the four reasons)."""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    """(world size, rank, local rank) from the launcher's environment (torchrun sets all three)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x, world, dev=None):
    """The largest x over all ranks (the slowest rank's time), by an all-reduce MAX; x itself on one
    rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gpts(pt_steps_per_rank, world, total_s):
    """Whole-job throughput: the grid-point-steps every rank processed (the same fixed work per rank,
    weak scaling) over the slowest rank's time, in Gpt-steps/s."""
    return pt_steps_per_rank * world / total_s / 1e9


def run_reference(args):
    """FP64 CPU oracle, timed as it stands on the host cores, on a bounded sample of the workload."""
    _, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.pat_oracle import Operator

    pb, prec, desc = workload(args.workload, 0)
    Nt_s = {"vessel2d_512": 50, "disc2d_168": 150, "tube3d_128": 6, "tube3d_256": 2}[args.workload]
    op = Operator.from_problem(pb, Nt=Nt_s)
    h = np.random.default_rng(0).standard_normal((Nt_s, op.Ns))
    for _ in range(args.warmup):
        op.adjoint(op.forward(pb.p0))
        break
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        op.adjoint(op.forward(pb.p0))
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    v = 2.0 * pb.N * Nt_s / t / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": desc,
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"forward+adjoint over the first {Nt_s} of {pb.Nt} time steps of the same grid"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(args, pb):
    """Oracle timed on a bounded sample (same grid, first Nt_s steps), single-threaded numpy."""
    from oracle.pat_oracle import Operator

    Nt_s = {"vessel2d_512": 200, "disc2d_168": 600, "tube3d_128": 20, "tube3d_256": 4}[args.workload]
    op = Operator.from_problem(pb, Nt=min(Nt_s, pb.Nt))
    t0 = time.perf_counter()
    op.adjoint(op.forward(pb.p0))
    t = time.perf_counter() - t0
    return {"value": 2.0 * pb.N * Nt_s / t / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one forward+adjoint over the first {Nt_s} of {pb.Nt} time steps of the same grid "
                      f"({t:.1f} s), FP64 numpy"}


def _oracle_replica(name, Nt_s, barrier, results, wait_s=120.0):
    """One replica of the bounded oracle sample, in its own spawned process on one core: build the
    workload's problem, wait for every replica to be ready, time one forward+adjoint over the first
    Nt_s steps.  perf_counter is the system-wide monotonic clock on Linux, so the start and end
    stamps of different replicas compare."""
    from oracle.pat_oracle import Operator

    pb, _, _ = workload(name, 0)
    op = Operator.from_problem(pb, Nt=min(Nt_s, pb.Nt))
    barrier.wait(timeout=wait_s)   # a replica that failed to start breaks the barrier for the others
    t0 = time.perf_counter()
    op.adjoint(op.forward(pb.p0))
    results.put((t0, time.perf_counter(), pb.N, min(Nt_s, pb.Nt)))


def cpu_baseline_all_cores(name, Nt_s, cores=0, timeout_s=180.0):
    """The bounded oracle sample of cpu_baseline on every host core at once.  One solve does not split
    across cores (its time steps are sequential and numpy's FFT runs one thread), so each core runs
    an independent replica of the same sample; value = the grid-point-steps of all replicas over the
    span from the first replica's start to the last one's end.  The replicas are spawned processes
    (no fork of a process that holds a CUDA context) with one thread each.  A replica that fails ends
    the measurement with an error at once; the whole leg is bounded by timeout_s."""
    import multiprocessing as mp
    import queue

    C = cores if cores > 0 else min(len(os.sched_getaffinity(0)), 32)   # at most 32 replicas on a shared host
    ctx = mp.get_context("spawn")
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    barrier, results = ctx.Barrier(C), ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(name, Nt_s, barrier, results, timeout_s)) for _ in range(C)]
    try:
        for p in procs:
            p.start()
        got = []
        deadline = time.perf_counter() + timeout_s
        while len(got) < C:
            try:
                got.append(results.get(timeout=1.0))
            except queue.Empty:
                if any(p.exitcode not in (None, 0) for p in procs):
                    raise RuntimeError("an oracle replica exited with an error")
                if time.perf_counter() > deadline:
                    raise TimeoutError(f"oracle replicas unfinished after {timeout_s:.0f} s")
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
        for p in procs:
            p.join(timeout=10.0)
            if p.is_alive():
                p.terminate()
                p.join()
    span = max(g[1] for g in got) - min(g[0] for g in got)
    N, nt = got[0][2], got[0][3]
    return {"value": 2.0 * N * nt * C / span / 1e9, "unit": UNIT, "cores": C, "kind": "oracle", "span_s": span,
            "sample": f"{C} independent replicas, one per core, each one forward+adjoint over the first {nt} "
                      f"time steps of the same grid ({span:.1f} s from the first start to the last end; one "
                      f"replica alone: see cpu_baseline), FP64 numpy"}


def batch_vs_sequential(dev):
    """Eight independent 2-D instances of uneven size (192^2 .. 384^2, 0.05 mm, 20-pt PML inside,
    own heterogeneous absorbing medium each, a 256-sensor circle of radius 0.4 x the interior
    width, Nt = 1200, FP32): forward + adjoint of all of them as one graph launch per direction
    (pat_batch_*) vs each plan's own calls one after the other."""
    import torch

    from paper_1603_02329_gb300 import synth
    from paper_1603_02329_gb300.api import PATBatch, PATOperator

    sizes = [192, 224, 256, 256, 288, 320, 320, 384]
    pbs = [synth.small_lossy_2d(seed=40 + i, shape=(n, n), pml=20, h=0.05e-3, Nt=1200, n_sensors=256,
                                sensor_radius_frac=0.4 * (n - 40) / n) for i, n in enumerate(sizes)]
    ops = [PATOperator.from_problem(pb, precision="f32", device=dev) for pb in pbs]
    xs = [torch.tensor(pb.p0, dtype=torch.float32, device=dev) for pb in pbs]
    hs = [torch.ones((op.Nt, op.Ns), dtype=torch.float32, device=dev) for op in ops]
    batch = PATBatch(ops)
    units = 2.0 * sum(pb.N * pb.Nt for pb in pbs)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    def one_at_a_time():
        for op, x, h in zip(ops, xs, hs):
            op.forward(x)
            op.adjoint(h)

    t_seq = timed(one_at_a_time)
    t_bat = timed(lambda: (batch.forward(xs), batch.adjoint(hs)))
    batch.close()
    return {"instances": sizes, "Nt": 1200, "paths_alone": [int(op.info.path) for op in ops],
            "sequential_s": t_seq, "batched_s": t_bat, "sequential_gpts": units / t_seq / 1e9,
            "batched_gpts": units / t_bat / 1e9, "speedup": t_seq / t_bat,
            "note": "best of 3 after one untimed run; a batch runs every instance on the per-phase path"}


def phase_trace(op, x, data, stream, nk):
    """Timeline of nk grid barriers in the middle of one forward solve of the persistent kernel:
    per barrier, the median over CTAs of the wait (entry to exit) and of the next phase's time to
    each of its sub-phase marks and to the next barrier, in microseconds."""
    import torch

    nph = op.Nt * (6 if op.lossy else 4)
    k0 = max(0, nph // 2 - nk // 2)
    op.set_trace(k0, nk)
    op.forward(x, out=data, stream=stream)
    torch.cuda.synchronize()
    tr = op.read_trace()
    op.set_trace(0, 0)
    if tr is None:
        return None
    tr = tr.astype(np.int64)
    ent, ext = tr[:, :, 0], tr[:, :, 1]
    rows = []
    for k in range(nk - 1):
        nxt = ent[:, k + 1]
        marks = []
        for j in range(6):
            m = tr[:, k + 1, 2 + j]    # a phase's marks share the slot of the barrier that ends it
            ok = (m > 0) & (m >= ext[:, k]) & (m <= nxt)
            marks.append(round(float(np.median(m[ok] - ext[ok, k])) / 1e3, 3) if ok.any() else None)
        rows.append({"barrier": int(k0 + k), "wait_us": round(float(np.median(ext[:, k] - ent[:, k])) / 1e3, 3),
                     "phase_us": round(float(np.median(nxt - ext[:, k])) / 1e3, 3), "marks_us": marks})
    return {"first_barrier": int(k0), "ctas": int(tr.shape[0]), "barriers": rows,
            "note": "marks: time from the barrier exit to sub-phase marks 0..5 of the next phase "
                    "(row phase: staged, inverse stage 0, inverse middle, fused, forward middle, stored; "
                    "column phase: staged, stage 0, middle, fused, inverse middle, stored)"}


def c2_gradient_timing(op, pb, K, dev, dtype):
    """Checkpointed c0^2 gradient (pat_gradient_c2, interval K) and the c0^2 + rho0 + p0 gradients of one
    sweep (pat_gradient_medium), each against one forward + adjoint."""
    import torch

    x = torch.tensor(pb.p0, dtype=dtype, device=dev)
    h = torch.ones((op.Nt, op.Ns), dtype=dtype, device=dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_fa = timed(lambda: op.adjoint(op.forward(x)))
    t_g = timed(lambda: op.gradient_c2(x, h, checkpoint_every=K))
    # the c0^2, rho0 and p0 gradients from one sweep (pat_gradient_medium)
    t_m = timed(lambda: op.gradient_medium(x, h, checkpoint_every=K, want=("c2", "rho", "p0")))
    w = 4 if dtype == torch.float32 else 8
    nseg = (pb.Nt - 2) // K + 1
    nh = int(np.prod(pb.shape[:-1])) * ((pb.shape[-1] // 2 + 1 + 7) // 8 * 8)
    d = len(pb.shape)
    return {"K": K, "fwd_adj_s": t_fa, "gradient_s": t_g, "ratio": t_g / t_fa,
            "checkpoint_bytes": nseg * (2 * d * pb.N + 2 * nh) * w, "q_bytes": min(K, pb.Nt) * pb.N * w,
            "medium_gradient_s": t_m, "medium_ratio": t_m / t_fa,
            # the density gradient also stores D+p and D-u (2 d fields) per level of a segment
            "medium_extra_bytes": (min(K, pb.Nt) + 1) * 2 * d * pb.N * w}


def mg_vs_fista(args, dev, pb):
    """Wall time of two-level MG-FISTA and of single-grid FISTA to the same relative error (Sec. VI.A
    compares the methods by RE and F against time) on the benchmark's workload.  Target: 1.05 x the
    best RE that FISTA reaches in --mg-iters iterations.  L estimation (power method, 30 iterations
    per level) is setup and is reported separately.  Parameters: Sec. VI.A (2-D) and Sec. VI.B
    (3-D: kappa = 1/8, rho = 3e-2)."""
    import torch

    from paper_1603_02329_gb300 import synth
    from paper_1603_02329_gb300.api import PATOperator, mg_fista

    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    opc = op.coarse()
    opc2 = opc.coarse() if args.mg_levels >= 3 else None
    x_true = torch.tensor(pb.p0, dtype=torch.float32, device=dev)
    if args.mg_data == "refined":
        # data from a finer grid with perturbed maps, sensors at the same positions (no inverse crime)
        pf = synth.refined_problem(pb, ratio=1.44, map_snr_db=35.0, seed=5)
        opf = PATOperator.from_problem(pf, precision="f32", device=dev)
        clean = opf.forward(torch.tensor(pf.p0, dtype=torch.float32, device=dev)).cpu().numpy()
        data_desc = (f"forward of the phantom on a {'x'.join(map(str, pf.shape))} grid with 35 dB-contaminated "
                     "sound-speed and density maps, sensors at the same positions, + 40 dB AWGN")
        opf.close()
    else:
        clean = op.forward(x_true).cpu().numpy()
        data_desc = "forward of the phantom on the same grid + 40 dB AWGN (inverse crime, stated)"
    noisy = synth.awgn(np.random.default_rng(2), clean, 40.0)
    data = torch.tensor(noisy, dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    L = op.power_iteration(torch.tensor(synth.random_image(11, pb.shape), dtype=torch.float32, device=dev), 30)
    Lc = opc.power_iteration(torch.tensor(synth.random_image(12, opc.shape), dtype=torch.float32, device=dev), 30)
    Lc2 = (opc2.power_iteration(torch.tensor(synth.random_image(13, opc2.shape), dtype=torch.float32, device=dev), 30)
           if opc2 is not None else None)
    setup_s = time.perf_counter() - t0
    x0 = torch.zeros_like(x_true)
    d = len(pb.shape)
    common = dict(variant=1, lam=1e-2, step_scale=1.0, kappa=0.25 if d == 2 else 0.125, vartheta=0.1, q_d=3,
                  q_c=8, eps_d=-1.0, eps_c=1e-2, tv_rho=1e-2 if d == 2 else 3e-2, n_tv=20)

    def timed(coarse, recursion, max_iter, target, coarse_weight=0.0):
        stamps = []
        t_start = time.perf_counter()
        Lco = Lc
        if coarse is not None and opc2 is not None:
            coarse, Lco = [opc, opc2], [Lc, Lc2]
        _, rep, recs = mg_fista(op, coarse, data, x0, L, L_coarse=Lco, p_exact=x_true, recursion=recursion,
                                max_iter=max_iter, target_re=target, coarse_weight=coarse_weight,
                                callback=lambda r: stamps.append(time.perf_counter() - t_start), **common)
        for r, ts in zip(recs, stamps):
            r["t"] = ts
        return rep, recs

    rep_f, recs_f = timed(None, False, args.mg_iters, 0.0)
    best = min(r["RE"] for r in recs_f)
    target = 1.05 * best
    t_f = next(r["t"] for r in recs_f if r["RE"] <= target)
    it_f = next(r["k"] for r in recs_f if r["RE"] <= target)
    rep_m, recs_m = timed(opc, True, args.mg_iters, target)
    hit = [r for r in recs_m if r["RE"] <= target]
    t_m = hit[0]["t"] if hit else None
    # the coarse data term as Eq. (Fourteen) prints it (weight 1) instead of reading O11's 2^(1-d)
    _, recs_u = timed(opc, True, min(args.mg_iters, it_f + 1), target, coarse_weight=1.0)   # capped: past FISTA's count it cannot win
    hit_u = [r for r in recs_u if r["RE"] <= target]

    def pair_s(o):   # one forward + one adjoint solve of a level (the cost unit of both methods)
        xx = torch.zeros(o.shape, dtype=torch.float32, device=dev)
        o.adjoint(o.forward(xx))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o.adjoint(o.forward(xx))
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    fine_pair, coarse_pair = pair_s(op), pair_s(opc)
    coarse2_pair = pair_s(opc2) if opc2 is not None else None
    curve = lambda recs: [(r["k"], r["branch"][0], round(r["RE"], 4), round(r["t"], 3)) for r in recs]
    return {"workload": pb.name, "target_re": target, "fista_best_re": best, "fista_s": t_f, "fista_iters": it_f,
            "levels": args.mg_levels,
            "fwd_adj_pair_s": {"fine": fine_pair, "coarse": coarse_pair, "ratio": coarse_pair / fine_pair,
                               "coarse2": coarse2_pair},
            "fista_curve": curve(recs_f), "mgfista_curve": curve(recs_m),
            "mgfista_s": t_m, "mgfista_iters": hit[0]["k"] if hit else None,
            "mgfista_recursive_iters": sum(1 for r in recs_m if r["branch"] == "recursive"),
            "speedup": (t_f / t_m) if t_m else None, "setup_s_power_method": setup_s,
            "unweighted_coarse_term": {"mgfista_curve": curve(recs_u), "mgfista_s": hit_u[0]["t"] if hit_u else None,
                                       "speedup": (t_f / hit_u[0]["t"]) if hit_u else None},
            "data": data_desc,
            "params": dict(common, lam=1e-2, L=L, L_coarse=Lc, L_coarse2=Lc2)}


def mg_precision(dev, iters=5):
    """FP32 against FP64 for the optimisation results: the relative L2 distance of the FP32 iterate
    x_k from the FP64 iterate x_k (k = 1 .. iters) of single-grid FISTA and of two-level MG-FISTA, run
    through the C ABI on a small 2-D absorbing case (64^2, 8-pt PML, 48 off-grid circle sensors,
    Nt = 120, 40 dB data; Sec. VI.A parameters).  The FP64 GPU path itself matches the FP64 CPU oracle
    iterate by iterate to 1e-9 (tests/test_gpu_optim.py), so this is the error of the FP32 results
    against the FP64 oracle up to that."""
    import torch

    from paper_1603_02329_gb300 import synth
    from paper_1603_02329_gb300.api import PATOperator, mg_fista

    pb = synth.small_lossy_2d(shape=(64, 64), pml=8, Nt=120, n_sensors=48)
    ops = {p: PATOperator.from_problem(pb, precision=p, device=dev) for p in ("f64", "f32")}
    opc = {p: ops[p].coarse() for p in ops}
    dts = {"f64": torch.float64, "f32": torch.float32}
    clean = ops["f64"].forward(torch.tensor(pb.p0, dtype=torch.float64, device=dev)).cpu().numpy()
    noisy = synth.awgn(np.random.default_rng(2), clean, 40.0)
    L = ops["f64"].power_iteration(torch.tensor(synth.random_image(11, pb.shape), device=dev), 30)
    Lc = opc["f64"].power_iteration(torch.tensor(synth.random_image(12, opc["f64"].shape), device=dev), 30)
    out = {"case": "2-D 64^2 absorbing, 8-pt PML, 48 circle sensors, Nt=120, 40 dB AWGN; lambda=1e-2, n_tv=20",
           "reference": "FP64 GPU iterates (equal to the FP64 oracle's to 1e-9)"}
    for label, rec in (("fista", False), ("mgfista", True)):
        errs, branches = [], []
        for k in range(1, iters + 1):
            xs = {}
            for p in ("f64", "f32"):
                d = torch.tensor(noisy, dtype=dts[p], device=dev)
                x0 = torch.zeros(pb.shape, dtype=dts[p], device=dev)
                x, _, recs = mg_fista(ops[p], opc[p] if rec else None, d, x0, L, L_coarse=Lc, recursion=rec,
                                      max_iter=k, eps_d=-1.0, variant=1, lam=1e-2, step_scale=1.0, kappa=0.25)
                xs[p] = x.double()
                if p == "f64" and k == iters:
                    branches = [r["branch"] for r in recs]
            errs.append(float(torch.linalg.norm(xs["f32"] - xs["f64"]) / torch.linalg.norm(xs["f64"])))
        out[label] = {"rel_l2_per_iter": errs, "branches": branches}
    for o in list(ops.values()) + list(opc.values()):
        o.close()
    return out


def tr_atd_record(dev, fista_iters=10):
    """The two comparison solves on the 2-D 512^2 absorbing workload with 40 dB data: the
    time-reversal image (Sec. II.B.1; pat_time_reversal, band-limited compensation at half the Nyquist
    radius, and plain) with its relative error, FISTA started from it against FISTA started from zero
    (Sec. VI.A parameters), and the paper's adjoint-then-discretize adjoint (pat_adjoint_atd) against
    dt times the exact transpose for the same residual (the data), over the whole grid and outside the
    PML layer."""
    import torch

    from paper_1603_02329_gb300 import synth
    from paper_1603_02329_gb300.api import PATOperator, mg_fista

    pb = synth.vessel_phantom_2d()
    op = PATOperator.from_problem(pb, precision="f32", device=dev)
    x_true = torch.tensor(pb.p0, dtype=torch.float32, device=dev)
    clean = op.forward(x_true).cpu().numpy()
    data = torch.tensor(synth.awgn(np.random.default_rng(2), clean, 40.0), dtype=torch.float32, device=dev)
    re = lambda x: float(torch.linalg.norm(x.double() - x_true.double()) / torch.linalg.norm(x_true.double()))

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    tr, t_tr = timed(lambda: op.time_reversal(data, compensate=True, k_cut=0.5))
    tr0 = op.time_reversal(data, compensate=False)
    L = op.power_iteration(torch.tensor(synth.random_image(11, pb.shape), dtype=torch.float32, device=dev), 30)
    common = dict(variant=1, lam=1e-2, step_scale=1.0, recursion=False, max_iter=fista_iters, eps_d=-1.0)
    _, _, r_zero = mg_fista(op, None, data, torch.zeros_like(x_true), L, p_exact=x_true, **common)
    _, _, r_tr = mg_fista(op, None, data, tr.clamp(min=0), L, p_exact=x_true, **common)
    target = r_zero[-1]["RE"]
    hit = next((r["k"] for r in r_tr if r["RE"] <= target), None)
    atd, t_atd = timed(lambda: op.adjoint_atd(data))
    tp = op.adjoint(data) * pb.dt
    P = pb.pml[0]
    inner = (slice(P, pb.shape[0] - P), slice(P, pb.shape[1] - P))
    dev_all = float(torch.linalg.norm((atd - tp).double()) / torch.linalg.norm(tp.double()))
    dev_in = float(torch.linalg.norm((atd - tp)[inner].double()) / torch.linalg.norm(tp[inner].double()))
    cos = float(torch.sum(atd.double() * tp.double()) / (torch.linalg.norm(atd.double()) * torch.linalg.norm(tp.double())))
    op.close()
    return {"workload": "2-D 512^2 absorbing, 512 line sensors on the first row inside the PML, Nt=2000, 40 dB AWGN",
            "time_reversal": {"re_compensated": re(tr), "re_plain": re(tr0), "k_cut": 0.5, "solve_s": t_tr},
            "fista_warm_start": {"iters": fista_iters, "re_from_zero": [round(r["RE"], 4) for r in r_zero],
                                 "re_from_tr": [round(r["RE"], 4) for r in r_tr],
                                 "iters_from_tr_to_zero_start_final_re": hit},
            "adjoint_then_discretize": {"rel_dev_from_dt_transpose": dev_all, "rel_dev_outside_pml": dev_in,
                                        "cosine": cos, "solve_s": t_atd}}


PATH_NAMES = {0: "CUDA graph of per-phase kernels", 1: "persistent kernel per solve",
              2: "persistent kernel per solve, register-fused power-of-two transforms"}


def measure(args, name, dev, world, rank, local, with_e2e=True):
    """Time args.steps forward + adjoint pairs of workload ``name`` after args.warmup untimed ones
    (CUDA events on the launching stream, L2 flushed between timed steps, clocks sampled), with the
    dominant kernel's roofline and the end-to-end variant through host buffers.  Returns
    (record, operator, problem)."""
    import torch
    import torch.distributed as dist

    from paper_1603_02329_gb300.api import PATOperator

    pb, prec, desc = workload(name, rank)
    if args.nt > 0:
        pb.Nt = args.nt
        desc = dict(desc, Nt=args.nt, workload=desc["workload"] + f" [time axis cut to Nt={args.nt}]")
    dtype = torch.float32 if prec == "f32" else torch.float64
    w = 4 if prec == "f32" else 8
    op = PATOperator.from_problem(pb, precision=prec, device=dev)
    if args.probe_stride > 0:
        op.set_probe(args.probe_stride)
    x = torch.tensor(pb.p0, dtype=dtype, device=dev)
    data = torch.empty((pb.Nt, op.Ns), dtype=dtype, device=dev)
    grad = torch.empty(pb.shape, dtype=dtype, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(args.warmup, 1)):
        op.forward(x, out=data, stream=stream)
        op.adjoint(data, out=grad, stream=stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    probe_acc = {}
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                       # evict L2 between timed steps (outside the events)
        ev[k][0].record(stream)
        op.forward(x, out=data, stream=stream)
        op.adjoint(data, out=grad, stream=stream)
        ev[k][1].record(stream)
        torch.cuda.synchronize()
        if args.probe_stride > 0:
            # the probe events of both graphs are final once the step has completed
            for g, tag in ((0, "fwd"), (1, "adj")):
                for kname, ms, cnt in op.probe(bool(g)):
                    acc = probe_acc.setdefault((tag, kname), [0.0, 0])
                    acc[0] += ms * cnt
                    acc[1] += cnt
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, world, dev)
    units_rank = 2.0 * pb.N * pb.Nt * args.steps
    value = aggregate_gpts(units_rank, world, total_s)

    # e2e: the same step through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if with_e2e and not args.no_e2e:
        xh = torch.tensor(pb.p0, dtype=dtype).pin_memory()
        dh = torch.empty((pb.Nt, op.Ns), dtype=dtype).pin_memory()
        gh = torch.empty(pb.shape, dtype=dtype).pin_memory()
        op.forward(xh, out=dh, stream=stream)
        op.adjoint(dh, out=gh, stream=stream)
        torch.cuda.synchronize()
        t_e2e = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            op.forward(xh, out=dh, stream=stream)
            op.adjoint(dh, out=gh, stream=stream)
            torch.cuda.synchronize()
            t_e2e += time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, world, dev)
        nb_in = pb.N * w + pb.Nt * op.Ns * w       # p0 for H, residual for H^T
        nb_out = pb.Nt * op.Ns * w + pb.N * w      # data from H, gradient from H^T
        e2e = {"value": aggregate_gpts(units_rank, world, t_e2e), "unit": UNIT, "h2d_bytes_per_step": nb_in,
               "d2h_bytes_per_step": nb_out}
    del flush

    # roofline of the dominant kernel: the compiled kernel with the largest share of the probed step
    # time (the y passes of all three spectral operations are one kernel each way), its algorithmic
    # bytes summed over its launches in one forward + adjoint step
    peak, peak_kind = measured_peaks()
    nxh = pb.shape[-1] // 2 + 1
    Nh = nxh * int(np.prod(pb.shape[:-1]))
    roof = None
    kernels = {}
    if probe_acc:
        for (tag, kname), (sm, cnt) in probe_acc.items():
            kernels[f"{tag}:{kname}"] = sm / max(cnt, 1)
        if int(op.info.path) >= 1:   # one persistent launch per solve
            dom = max(kernels, key=lambda k: kernels[k])
            ms = kernels[dom]
            b = solve_bytes(pb.N, pb.Nt, w, D=len(pb.shape), lossy=op.lossy)
            fam, launches, share = dom.split(":")[1], 1, ms / sum(kernels.values())
        else:
            fams = family_totals(kernels, pb.N, Nh, w, len(pb.shape), op.lossy, int(op.info.spec_chunks))
            fam = max(fams, key=lambda f: fams[f]["ms"])
            tot_ms = sum(f["ms"] for f in fams.values())
            ms = fams[fam]["ms"] / fams[fam]["launches"]
            b = fams[fam]["bytes"] / fams[fam]["launches"]
            launches, share = fams[fam]["launches"], fams[fam]["ms"] / tot_ms
        ach = b / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": measured_traffic(name, fam, kernel_version(op, fam)) if not args.nt else None,
                "kernel": fam, "kernel_ms": ms, "algorithmic_bytes": b, "launches_per_step": launches,
                "share_of_step": share, "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "note": ("one persistent launch per solve keeps the state in shared memory (DRAM traffic: "
                         "the set-up loads); the fraction is effective bandwidth of the algorithmic bytes"
                         if fam.startswith("k_persist") else
                         "per launch: mean algorithmic bytes (operands read and written once) and mean duration "
                         "over this kernel's launches in one forward + adjoint step")}
    # whole-step roofline by the per-point-step algorithmic bytes (state once + medium once)
    B_pt = (2 * (2 * len(pb.shape) + 1) + (4 if op.lossy else 2)) * w
    step_roof = {"bytes_per_pt_step": B_pt, "achieved_gbs": value * 1e9 * B_pt / 1e9 / world,
                 "frac": value * B_pt / world / peak, "peak": peak, "unit": "GB/s"}
    # whole-step FP32 roofline: algorithmic flops per grid-point-step of the packed transforms, about
    # 5.5 (2-D lossy) or 7 (3-D lossy) complex-transform equivalents of 5 log2 N flops each, against
    # the FMA throughput measured by the library's probe
    alu = None
    if prec == "f32" and op.lossy:
        from paper_1603_02329_gb300.api import probe_fp32_peak

        flops_pt = (7.0 if len(pb.shape) == 3 else 5.5) * 5.0 * np.log2(pb.N)
        fpeak = probe_fp32_peak(dev)
        ach = value / world * flops_pt / 1e3
        alu = {"bound": "alu", "flops_per_pt_step": flops_pt, "achieved": ach, "peak": fpeak, "unit": "TFLOP/s",
               "frac": ach / fpeak, "peak_source": "pat_probe_fp32_peak (measured FP32 FMA throughput)"}

    # per time step of the graph path: (3 or 2) spectral operations of 1 (2-D) or 3 (3-D: y, z, y)
    # launches, and as many row kernels
    nops = 3 if op.lossy else 2
    slots_f = nops * (3 * int(op.info.spec_chunks) if len(pb.shape) == 3 else 1) + nops
    persistent = int(op.info.path) >= 1
    # per solve: the persistent kernel or the graph's kernels, and the non-finite scan of the output
    launches = args.steps * 2 * ((1 if persistent else (1 + (pb.Nt - 1) * slots_f)) + 1)
    rec = {"value": value, "unit": UNIT, "ms_per_step": total_s * 1e3 / args.steps, "dtype": prec,
           "config": dict(desc, l2="flushed between timed steps (512 MB write)", instances_per_gpu=1,
                          layout=list(op.info.layout), layout_tuned=int(op.info.tuned),
                          radix_schedule=int(op.info.schedule), spec_chunks=int(op.info.spec_chunks),
                          parallelism=f"replicas x{world}", path=PATH_NAMES[int(op.info.path)],
                          kernels={"y_passes_16col": int(op.info.ywide), "z_passes_16col": int(op.info.zwide),
                                   "u_rows_per_component": int(op.info.rowu1), "tensor_copies": int(op.info.tma)}),
           "roofline": roof, "step_roofline": step_roof, "fp32_roofline": alu, "kernel_ms": kernels, "e2e": e2e,
           "gpu_launches": launches, "clocks": clk}
    return rec, op, pb


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1603_02329_gb300 import build

    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    rec, op, pb = measure(args, args.workload, dev, world, rank, local)
    out = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": rec["dtype"], "data": "synthetic"}
    out.update({k: rec[k] for k in ("config", "roofline", "step_roofline", "fp32_roofline", "kernel_ms", "e2e",
                                    "gpu_launches", "clocks")})
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(args, pb)
    x = None
    if args.trace > 0 and rank == 0 and int(op.info.path) >= 1:
        import torch as _t

        dtype = _t.float32 if rec["dtype"] == "f32" else _t.float64
        x = _t.tensor(pb.p0, dtype=dtype, device=dev)
        data = _t.empty((pb.Nt, op.Ns), dtype=dtype, device=dev)
        out["phase_trace"] = phase_trace(op, x, data, _t.cuda.current_stream(dev), args.trace)
    if args.c2grad > 0 and rank == 0:
        out["c2_gradient"] = c2_gradient_timing(op, pb, args.c2grad, dev,
                                                torch.float32 if rec["dtype"] == "f32" else torch.float64)
    op.close()
    del op
    torch.cuda.empty_cache()
    if rank == 0 and args.workload == "tube3d_256" and not args.no_secondary and not args.nt:
        rec2, op2, pb2 = measure(args, "vessel2d_512", dev, 1, 0, local, with_e2e=True)
        op2.close()
        rec2["steps"], rec2["warmup"] = args.steps, args.warmup
        if not args.no_cpu:
            a2 = argparse.Namespace(**vars(args))
            a2.workload = "vessel2d_512"
            rec2["cpu_baseline"] = cpu_baseline(a2, pb2)
            try:
                rec2["cpu_baseline_all_cores"] = cpu_baseline_all_cores("vessel2d_512", 200)
            except Exception as e:   # the record is context: its failure must not cost the bench line
                rec2["cpu_baseline_all_cores"] = {"error": f"{type(e).__name__}: {e}"}
        rec2["tr_atd"] = tr_atd_record(dev)
        out["vessel2d_512"] = rec2
    if (args.mg or args.mg_default) and rank == 0:
        out["mg_vs_fista"] = mg_vs_fista(args, dev, pb)
        out["mg_precision"] = mg_precision(dev)
    if args.mg_default and rank == 0:
        # the 2-D comparison on data without the inverse crime: generated on a 1.44x finer grid from
        # 35 dB-contaminated maps (Sec. VI.A's set-up), 2 levels, 20 FISTA iterations
        from paper_1603_02329_gb300 import synth

        a2 = argparse.Namespace(**vars(args))
        a2.mg_levels, a2.mg_iters, a2.mg_data = 2, 20, "refined"
        out["mg_vs_fista_refined_2d"] = mg_vs_fista(a2, dev, synth.vessel_phantom_2d(seed=2))
    if (args.batch or args.mg_default) and rank == 0:
        out["batch"] = batch_vs_sequential(dev)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
