"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region (median SM clock, maximum, throttle reasons), the algorithmic
bytes per node update and the single-rank aggregation."""
import bench


def _sampler(rows):
    s = bench.ClockSampler(0)
    s.rows = rows
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0,
                            "kill": lambda self: None})()
    return s


def test_clock_record_median_max_and_reasons():
    rows = [["2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
            ["2055", "2070", "950.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
            ["2070", "2070", "1000.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    rec = _sampler(rows).stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]


def test_clock_record_reports_thermal_and_hardware_slowdown():
    rows = [["1500", "2070", "1300", "0x48", "Active", "Active", "Not Active", "Not Active"],
            ["1490", "2070", "1300", "0x20", "Not Active", "Not Active", "Active", "Not Active"]]
    rec = _sampler(rows).stop()
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert rec["sm_mhz"] == 1495.0


def test_clock_record_without_nvidia_smi():
    s = bench.ClockSampler(0)
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_bytes_per_node_update():
    # mixer: 33 densities; exchanger: 26 (FP32 and 16-bit storage)
    assert bench.bytes_per_node(33, 4, "primal") == 269
    assert bench.bytes_per_node(33, 4, "adjoint") == 417
    assert bench.bytes_per_node(26, 4, "primal") == 213
    assert bench.bytes_per_node(26, 4, "adjoint") == 333
    assert bench.bytes_per_node(26, 2, "primal") == 109
    assert bench.bytes_per_node(26, 2, "adjoint") == 281


def test_single_rank_aggregation():
    ms, value = bench.aggregate_ranks(2000.0, 1.0e9, 4, 1, device="cpu")
    assert ms == 2000.0
    assert abs(value - 4.0e9 / 2.0 / 1e6) < 1e-6


def test_fifo_finish_times_of_the_one_at_a_time_baseline():
    from bench import fifo_finish_times
    # idle server: each request starts on arrival
    assert fifo_finish_times([0.0, 5.0, 9.0], [1.0, 2.0, 0.5]) == [1.0, 7.0, 9.5]
    # queueing: a request waits for the previous one to finish
    assert fifo_finish_times([0.0, 0.1, 0.2], [1.0, 1.0, 1.0]) == [1.0, 2.0, 3.0]
    # mixed: the third arrives after the queue drained
    assert fifo_finish_times([0.0, 0.5, 4.0], [2.0, 1.0, 1.0]) == [2.0, 3.0, 5.0]
