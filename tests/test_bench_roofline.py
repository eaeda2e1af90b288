"""Host logic of the benchmark: the roofline's algorithmic bytes, which it divides by the measured
kernel times, checked against sums written out by hand from the operands each kernel reads and
writes once (real fields of N values, half spectra of Ny Nz (Nx/2 + 1) complex values); and the
summary of the clocks sampled during the timed region."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

MB = 1e6


def _sizes(shape, w=4):
    N = 1
    for s in shape:
        N *= s
    Nh = (shape[-1] // 2 + 1) * (N // shape[-1])
    return N, Nh, N * w, Nh * 2 * w   # N, Nh, one real field F, one half spectrum Hs


def test_bytes_per_grid_point_step():
    # (2 (2d + 1) state fields read and written + m medium fields) x w: u_xi, rho_xi (d each), p;
    # medium c0^2, rho0 (+ tau, eta when lossy)
    assert bench.solve_bytes(1, 1, 4, D=3, lossy=True) == 72
    assert bench.solve_bytes(1, 1, 4, D=2, lossy=True) == 56
    assert bench.solve_bytes(1, 1, 8, D=2, lossy=False) == 96
    # one 2000-step 512^2 solve of the persistent kernel
    assert bench.solve_bytes(512 * 512, 2000, 4, D=2, lossy=True) == pytest.approx(29.36e9, rel=1e-3)


def test_row_kernel_bytes_at_256_cubed():
    N, Nh, F, Hs = _sizes((256, 256, 256))
    # u update: D spectra of D+ p in, D spectra of u out; b_xi, u_xi read, u_xi written
    assert bench.kernel_bytes("fwd_u", N, Nh, 4, D=3) == 6 * Hs + 9 * F
    assert bench.kernel_bytes("fwd_u", N, Nh, 4, D=3) / MB == pytest.approx(1009.8, abs=0.1)
    # density update (lossy): D spectra of D- u in, 2 out (dd, r); rho0, rho_xi read, rho_xi and r written
    assert bench.kernel_bytes("fwd_rho", N, Nh, 4, D=3) == 5 * Hs + 8 * F
    # state: 2 absorption spectra in, p's spectrum out; c0^2 tau, c0^2 eta, c0^2, r read
    assert bench.kernel_bytes("fwd_p", N, Nh, 4, D=3) == 3 * Hs + 4 * F
    assert bench.kernel_bytes("spec_div", N, Nh, 4, D=3) == 6 * Hs


def test_y_transform_family_at_256_cubed():
    # one forward + adjoint step, 3-D lossy: the y inverse transform follows every spectral
    # operation with its output fields: GRAD 3, DIV 3, ABS 2 (forward); ABS 2, DIVT 3, GRADT 1
    # (adjoint): 14 fields over 6 launches, each field read and written once
    N, Nh, F, Hs = _sizes((256, 256, 256))
    fams = bench.family_totals({}, N, Nh, 4, 3, True)
    assert fams["y_inv"]["launches"] == 6
    assert fams["y_inv"]["bytes"] == 2 * 14 * Hs
    assert fams["y_inv"]["bytes"] / 6 / MB == pytest.approx(315.6, abs=0.1)
    # the forward y transform precedes every operation with its input fields: 1, 3, 2 and 2, 3, 3
    assert fams["y_fwd"]["launches"] == 6
    assert fams["y_fwd"]["bytes"] == 2 * 14 * Hs
    # twelve launches of spectral passes and three row kernels per direction
    sched = bench.step_schedule(3, True)
    for g in ("fwd", "adj"):
        kinds = [p for gg, p, _, _, _ in sched if gg == g]
        assert sum(p.startswith("spec") for p in kinds) == 9 and len(kinds) == 12


def test_family_time_counts_chunks():
    # a 3-D spectral operation split into c chunks of column tiles is c launches of its kernels,
    # each probed at the chunk's time
    N, Nh, F, Hs = _sizes((32, 32, 32))
    k = {"fwd:spec_y_inv": 0.5, "adj:spec_y_inv": 0.25}
    one = bench.family_totals(k, N, Nh, 4, 3, True, chunks=1)["y_inv"]
    four = bench.family_totals(k, N, Nh, 4, 3, True, chunks=4)["y_inv"]
    assert four["launches"] == 4 * one["launches"] and four["bytes"] == one["bytes"]
    assert one["ms"] == pytest.approx(3 * 0.5 + 3 * 0.25)
    assert four["ms"] == pytest.approx(4 * one["ms"])


def test_clock_summary_of_sampled_lines():
    # nvidia-smi --format=csv,noheader,nounits lines: index, clocks.sm, clocks.max.sm, power.draw,
    # active reasons mask, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    lines = [
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.ClockSampler.summarize(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = lines[:1] + ["0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"]
    assert bench.ClockSampler.summarize(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize(["x"]) is None
