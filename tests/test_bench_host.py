"""Host-side pieces of the benchmark, checked without a GPU: the clock record
(parsed from nvidia-smi's CSV), the name of the pass kernel a plan runs, and the
DRAM-traffic record (taken only while it names that kernel and its source is
unchanged, scaled from the captured size by the amplitude count)."""
import hashlib
import types

import bench


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_record_median_and_reasons():
    c = bench.Clocks(0)
    c.p = _FakeSmi("2070, 2070, 900.1, Not Active, Not Active, Not Active, Active\n"
                   "2055, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active\n"
                   "[N/A], 2070, 0, Not Active, Not Active, Not Active, Not Active\n"
                   "1980, 2070, 1390.5, Not Active, Not Active, Not Active, Active\n")
    r = c.stop()
    assert r["sm_mhz"] == 2055 and r["sm_max_mhz"] == 2070 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    c.p = _FakeSmi("1500, 2070, 800, Active, Not Active, Not Active, Not Active\n")
    assert bench.Clocks.stop(c)["reasons"] == ["hw_slowdown"]


def test_clock_record_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _info(tb, low, groups):
    return types.SimpleNamespace(tile_bits=tb, low_tile_bits=low, n_groups=groups)


def test_kernel_names_follow_the_plan():
    assert bench.kernel_name(0, _info(13, 12, 3)) == "pass_kernel_ring<12,4,RX>+<13,5,RX>"
    assert bench.kernel_name(5, _info(12, 11, 4)) == "pass_kernel_ring<11,4,RX>+<12,5,RX>"
    assert bench.kernel_name(3, _info(13, 12, 3)) == "pass_kernel_ring<12,4,RX>+<13,4,RX>"
    assert bench.kernel_name(3, _info(11, 11, 2)) == "pass_kernel_ring<11,4,RX>"
    assert bench.kernel_name(4, _info(13, 13, 3)) == "pass_kernel_ring<13,5,RX>"
    assert bench.kernel_name(2, _info(13, 13, 3)) == "pass_kernel_tma<float2,13,RX>"
    assert bench.kernel_name(1, _info(14, 14, 3)) == "pass_kernel_packed<14,4,RX>"
    assert bench.kernel_name(0, _info(14, 14, 2)) == "pass_kernel_packed<14,4,RX>"
    assert bench.kernel_name(0, _info(13, 13, 2)) == "pass_kernel_ring<13,4,RX>+<13,5,RX>"


def test_traffic_record_checks_kernel_and_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    src = tmp_path / "kernel.cuh"
    src.write_bytes(b"// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles" / "pass_kernel_ring_traffic.txt").write_text(
        "# comment\nkernel K<1>\nsource kernel.cuh\n"
        f"qubits 28\nsource_sha256 {sha}\ndram_bytes_per_launch 1000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic(28, "K<1>") == 1000
    assert bench.recorded_traffic(32, "K<1>") == 16000      # scaled by 2^(32 - 28)
    assert bench.recorded_traffic(32, "K<2>") is None       # another kernel
    src.write_bytes(b"// kernel source, edited\n")
    assert bench.recorded_traffic(32, "K<1>") is None       # the source changed since the capture


def test_cpu_baseline_times_the_oracle_on_a_real_state():
    # a workload of at most 30 links is timed on its own lattice (no scaling);
    # at least one Trotter step even with a zero budget
    wl = dict(d=2, L=(3, 2), lam=2.0, T=1.0, M=10)
    cb = bench.cpu_baseline(wl, 1, budget_s=0.0)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert "3x2 lattice (12 qubits" in cb["sample"] and "extrapolated" not in cb["sample"]
    assert cb["cpu"]


def test_l2_note_for_states_near_the_l2_size():
    """Inputs are not flushed between timed steps; the line says whether the
    state dwarfs the 129 MB L2 or is about its size (24 qubits: part of every
    pass is served from L2)."""
    assert ">> L2" in bench.l2_note(8 << 32)
    near = bench.l2_note(8 << 24)
    assert "134 MB" in near and "about the size of L2" in near and ">>" not in near
