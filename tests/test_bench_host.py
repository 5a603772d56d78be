"""Host arithmetic of bench.py (no GPU): the roofline object of the dominant kernel from stage
times given per step, the derived FP32 peak, the HBM fraction on algorithmic bytes, the DRAM
traffic scaled from the per-particle capture, and the algorithmic bytes per particle."""
import math

import bench


def _run(stages, accd):
    return {"stages_ms": stages, "accd": accd}


def test_roofline_of_the_pressure_pass():
    n = 1_200_009
    stages = {"rebuild": 0.1, "interact": 3.4, "control": 0.02, "integrate": 0.64}
    peaks = {"hbm_gbs": 6772.9}
    r = bench.roofline_of(_run(stages, 83_909_599), n, peaks, "measured", dim=3)
    assert r["kernel"] == "interact" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 152 SMs x 128 FP32 lanes x 2 operations x 2,070 MHz
    assert math.isclose(r["peak"], 152 * 128 * 2 * 2070e6 / 1e12, rel_tol=1e-12)
    want = 50.0 * 83_909_599 / 3.4e-3 / 1e12
    assert math.isclose(r["achieved"], want, rel_tol=1e-12)
    assert math.isclose(r["frac"], want / r["peak"], rel_tol=1e-12)
    assert r["avg_launch_ms"] == 3.4
    # traffic: the capture's bytes per particle times the particles of the launch
    assert math.isclose(r["traffic"], bench.DOMINANT_DRAM_BYTES_PER_PARTICLE * n, rel_tol=1e-12)
    # HBM fraction on algorithmic bytes against the measured copy bandwidth
    bpp = bench.algorithmic_bytes("interact", 3)
    assert math.isclose(r["hbm_achieved_gbs"], n * bpp / 3.4e-3 / 1e9, rel_tol=1e-12)
    assert math.isclose(r["hbm_frac"], r["hbm_achieved_gbs"] / 6772.9, rel_tol=1e-12)


def test_roofline_of_a_2d_run_has_no_scaled_traffic():
    r = bench.roofline_of(_run({"interact": 0.08, "integrate": 0.04, "control": 0.01}, 2_000_000), 120_000,
                          {}, "fallback", dim=2)
    assert r["kernel"] == "interact" and r["traffic"] is None
    assert r["hbm_peak_gbs"] == bench.hbm_peak({})


def test_algorithmic_bytes():
    # pressure pass: own record (16 B 2D / 20 B 3D), (v, h) 16, own cell 4 per axis, a_p + V~ 16
    assert bench.algorithmic_bytes("interact", 2) == 16 + 16 + 8 + 16
    assert bench.algorithmic_bytes("interact", 3) == 20 + 16 + 12 + 16
    # update: record, (v, h), a_p, stored cell + offset in; cell, offset, velocity, h, meta, index, key out
    assert bench.algorithmic_bytes("integrate", 3) == 20 + 16 + 16 + 24 + (24 + 12 + 16)
    assert bench.algorithmic_bytes("control", 3) == 0


def test_measured_peak_lookup():
    assert bench.hbm_peak({"hbm_gbs": 7000.0}) == 7000.0
    assert bench.hbm_peak({"other": 1}) == 6800.0


def test_stage_times_are_per_step_not_per_launch():
    # the 3D viscous pass + update stage launches two kernels per step
    times = {"rebuild": (60, 2.0), "interact": (20, 68.0), "integrate": (40, 12.8)}
    st = bench.stages_per_step(times, 20)
    assert st == {"rebuild": 0.1, "interact": 3.4, "integrate": 0.64}
