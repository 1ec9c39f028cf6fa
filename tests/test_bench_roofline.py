"""The benchmark's roofline arithmetic (host logic, no GPU): algorithmic
bytes of the particle phase as the measurement plan counts them -- the
state of each particle alive at step start read once, each survivor written
once (x, mu, nu, w in FP32 plus the 64-bit identity: 24 B in 1D mixed; 40 B
in FP64), plus three FP64 tallies per (cell, group) and per bin -- and the
source iteration's FP64 operations against the FP64 pipe."""
import math

import bench
from paper_2312_16981_gb300 import inputs as I

PEAKS = {"hbm_gbs": 6781.4}


def test_particle_bytes_per_survivor():
    p = I.multigroup_slab()
    n_read, n_out = 1_000_000, 900_000
    tab = 3 * 8 * p.ncell * p.G + 3 * 8 * p.nbins
    assert bench.algorithmic_bytes(p, "particles", n_read, n_out, 3, mixed=True) == 24 * (n_read + n_out) + tab
    assert bench.algorithmic_bytes(p, "particles", n_read, n_out, 3, mixed=False) == 40 * (n_read + n_out) + tab
    q = I.checkerboard_2d()
    tab2 = 3 * 8 * q.ncell * q.G + 3 * 8 * q.nbins
    assert bench.algorithmic_bytes(q, "particles", n_read, n_out, 3, mixed=True) == 32 * (n_read + n_out) + tab2
    assert bench.algorithmic_bytes(p, "source_iteration", n_read, n_out, 3) == 0


def test_particle_roofline_fraction_and_traffic():
    p = I.multigroup_slab()
    n_read, n_out, n_proc, ms = 1_300_000, 1_320_000, 1_330_000, 0.035
    r = bench.roofline(p, "particles", ms, n_proc, n_read, n_out, 3, True, PEAKS, "measured")
    abytes = bench.algorithmic_bytes(p, "particles", n_read, n_out, 3, mixed=True)
    assert r["kernel"] == "k_stream32_fast" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], abytes / (ms * 1e-3) / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / PEAKS["hbm_gbs"])
    assert r["bytes_per_particle"] == 24
    assert math.isclose(r["traffic"], bench.TRAFFIC_PER_PROCESSED["mixed"] * n_proc)
    r64 = bench.roofline(p, "particles", ms, n_proc, n_read, n_out, 3, False, PEAKS, "measured")
    assert r64["kernel"] == "k_stream64" and r64["bytes_per_particle"] == 40
    # no capture of the FP64 kernel's traffic: reported as unknown
    assert r64["traffic"] is None


def test_source_iteration_roofline_against_the_fp64_pipe():
    p = I.multigroup_slab()
    r = bench.roofline(p, "source_iteration", 0.045, 0, 0, 0, 3.0, True, PEAKS, "measured")
    flops = bench.SI_FLOPS_PER_CELL_GROUP[1] * p.ncell * p.G * 3.0
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert math.isclose(r["achieved"], flops / 0.045e-3 / 1e12)
    # 152 SMs x 4 sub-partitions x 0.5 FMA lanes a cycle x 2 flops x 2.07 GHz
    assert math.isclose(r["peak"], 1.25856, rel_tol=1e-9)
    assert 0.0 < r["frac"] < 1.0
