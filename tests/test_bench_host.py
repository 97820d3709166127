"""bench.py's host arithmetic, on CPU.  The roofline line divides
algorithmic bytes and flops per launch by the measured time.  These counts,
taken from a host-only plan of the 115,200-unknown cube (6 levels, 64
columns), must equal the figures written out by hand below (every operand
read once, every result written once, 8 bytes per complex FP32 value; a
translation costs 16 real flops per pair, sample and column: one complex
multiply-add for each of the two tangential components).  The whole-job rate
of N replicas is N x columns x steps over the slowest rank's time.  The
clock sampler reads nvidia-smi's CSV rows into the median SM clock, the
maximum clock and the throttle reasons that were active."""
import bench
import workloads
from paper_1412_1756_gb300 import mlfma as M


def test_algorithmic_counts_of_the_cube_at_64_columns():
    W = workloads.get("cube8m-6lv")
    v, t = W.mesh()
    P = M.MlfmaPlan(v, t, W.k, W.levels, W.digits, host_only=True)
    inf = P.info()
    assert inf["box_count"][4:6] == [1352, 5768] and inf["samples_K"][4:6] == [512, 288]
    assert inf["translations"][5] == 184_896
    field5 = 5768 * 2 * 288 * 64 * 8          # leaf boxes x components x samples x columns x bytes
    field4 = 1352 * 2 * 512 * 64 * 8
    assert field5 == 1_701_052_416
    # translate5: read S_5, write G_5; 16 x pairs x samples x columns flops
    assert bench.algorithmic(inf, 64, "translate5") == (2 * field5, 16 * 184_896 * 288 * 64)
    assert bench.algorithmic(inf, 64, "translate5") == (3_402_104_832, 54_528_049_152)
    # down4: read G_4 and G_5, write G_5; up4: read S_5, write S_4
    assert bench.algorithmic(inf, 64, "down4") == (field4 + 2 * field5, 0) == (4_110_942_208, 0)
    assert bench.algorithmic(inf, 64, "up4") == (field5 + field4, 0)
    # radiate: patterns (N x K x 2 components, complex) + x (real) + S_5
    n, nnz = P.n, inf["near_nnz"]
    assert bench.algorithmic(inf, 64, "radiate")[0] == n * 288 * 2 * 8 + n * 64 * 4 + field5
    # near: CSR values (complex) + x (real) + y (complex); 8 flops per entry and column
    assert bench.algorithmic(inf, 64, "near") == (nnz * 8 + n * 64 * 4 + n * 64 * 8, 8 * nnz * 64)


def test_replica_rate_and_single_process_max():
    assert bench.replica_rate(64, 20, 0.5, 4) == 4 * 64 * 20 / 0.5
    assert bench.reduce_max(3.25, None, "cpu") == 3.25


def test_clock_sampler_summary(tmp_path):
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbled line",
            "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.ClockSampler(0)
    c.proc, c.path = object(), str(path)
    out = c.summary()
    assert out == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    path.write_text("0, 1200, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active\n")
    c.path = str(path)
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
