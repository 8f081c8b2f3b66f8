"""Host logic of bench.py that needs no GPU: the training-plateau report and
the clock-sample summary's rejection rules."""
import bench


def test_plateau_report_first_crossings():
    hist = [(1000, 1.0, 0.1), (6000, 0.30, 0.6), (11000, 0.12, 1.1), (16000, 0.105, 1.6),
            (20000, 0.10, 2.0)]
    rep = bench.plateau_report([{"history": hist}, {"history": []}])
    assert rep[1] is None
    # within 2x of the final 0.10: first point <= 0.20 is (11000, 0.12)
    assert rep[0]["within_2x"] == {"steps": 11000, "seconds": 1.1}
    # within 10 %: first point <= 0.11 is (16000, 0.105)
    assert rep[0]["within_10pct"] == {"steps": 16000, "seconds": 1.6}


def test_plateau_report_monotone_only_at_the_end():
    # a history that only reaches the band at its last point
    hist = [(1000, 5.0, 0.1), (2000, 4.0, 0.2), (3000, 1.0, 0.3)]
    rep = bench.plateau_report([{"history": hist}])[0]
    assert rep["within_10pct"]["steps"] == 3000 and rep["within_2x"]["steps"] == 3000


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_summary_median_and_reasons():
    """nvidia-smi rows -> median SM clock, max clock, the throttle reasons
    seen Active (a row that is cut short or not numeric is ignored)"""
    cs = bench.ClockSampler()
    cs.proc = _FakeProc()
    row = lambda sm, hw="Not Active", cap="Not Active": [
        "0", sm, "2070", "900.00", "0x0", hw, "Not Active", "Not Active", cap]
    cs.rows = [row("2070"), row("1995", cap="Active"), row("2070"), ["0", "2070"],
               row("[N/A]"), row("2055", hw="Active")]
    out = cs.stop()
    assert out["sm_mhz"] == 2062.5  # median of 2070, 1995, 2070, 2055
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["samples"] == 5


def test_clock_summary_without_nvidia_smi():
    assert bench.ClockSampler().stop()["reasons"] == ["nvidia-smi unavailable"]
