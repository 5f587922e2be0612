"""Host-side pieces of the benchmark, without a GPU: the comment-blind hash
of the stage-kernel sources that keys the recorded DRAM traffic, the clock
sampler's reading of nvidia-smi records (a run that saw a slowdown reason is
rejected, so the parse decides which runs count), and the recorded traffic's
own arithmetic."""
import json

import numpy as np

import bench


def test_kernel_hash_ignores_comments_and_blank_lines_but_not_code(tmp_path, monkeypatch):
    a, b = tmp_path / "a.cuh", tmp_path / "b.cuh"
    code_a = "int f(int x) {\n    return x + 1;\n}\n"
    code_b = "constexpr int N = 8;\n"
    a.write_text(code_a)
    b.write_text(code_b)
    monkeypatch.setattr(bench, "KERNEL_SRC", [str(a), str(b)])
    h0 = bench.kernel_hash()
    assert len(h0) == 16 and int(h0, 16) >= 0
    # comments (line and block), trailing blanks and blank lines do not count
    a.write_text("// leading comment\n/* block\n   comment */\nint f(int x) {   \n\n"
                 "    return x + 1;  // trailing\n}\n\n")
    assert bench.kernel_hash() == h0
    # a changed token in either file does
    a.write_text(code_a.replace("+ 1", "+ 2"))
    assert bench.kernel_hash() != h0
    a.write_text(code_a)
    b.write_text("constexpr int N = 16;\n")
    assert bench.kernel_hash() != h0
    b.write_text(code_b)
    assert bench.kernel_hash() == h0


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s.thread, s.lines = _Proc(), _Thread(), list(lines)
    return s


def test_clock_sampler_takes_the_median_clock_and_every_active_reason():
    quiet = "Not Active, Not Active, Not Active, Not Active"
    c = _sampler([
        f"0, 2070, 2070, 900.1, 0x0000000000000000, {quiet}",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        f"0, 2070, 2070, 1200.0, 0x0000000000000000, {quiet}",
        f"0, [N/A], 2070, 1200.0, 0x0, {quiet}",   # no clock reading: skipped
        "not a record",
    ]).stop()
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    c = _sampler([
        f"0, 1500, 2070, 800.0, 0x0, {quiet}",
        "0, 1400, 2070, 800.0, 0x40, Not Active, Active, Not Active, Not Active",
        "0, 1300, 2070, 800.0, 0x20, Not Active, Not Active, Active, Not Active",
        "0, 1200, 2070, 800.0, 0x8, Active, Not Active, Not Active, Not Active",
    ]).stop()
    assert c["sm_mhz"] == float(np.median([1500, 1400, 1300, 1200]))
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi_says_so():
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


def test_recorded_traffic_is_bytes_over_cells_against_the_algorithmic_words():
    """Per stage, DRAM bytes per cell = (read + write) / cells of the captured
    launch; the algorithmic bytes are the FP32 words a cell moves: stage 1
    reads Q and writes Q' and dQ (21), stage 2 also reads dQ (28), stage 3
    writes no dQ (21)."""
    with open(bench.TRAFFIC_FILE) as f:
        rec = json.load(f)
    assert rec["precision"] == "fp32" and len(rec["kernel_hash"]) == 16
    rd = np.array(rec["dram_read_bytes_by_stage"])
    wr = np.array(rec["dram_write_bytes_by_stage"])
    per = np.array(rec["dram_bytes_per_cell_stage_by_stage"])
    assert np.allclose(per, (rd + wr) / rec["cells"], rtol=1e-12)
    assert rec["algorithmic_bytes_per_cell_stage_by_stage"] == [4.0 * w for w in (21, 28, 21)]
