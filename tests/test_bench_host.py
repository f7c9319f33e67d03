"""Host logic of bench.py that the GPU runs rely on: the DRAM traffic record
(keyed by precision and steps per launch, valid only for the kernel source it
was taken on) and the clock summary over the sampled window."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_traffic_record_is_keyed_by_steps_per_launch_and_kernel_source(tmp_path, monkeypatch):
    b = _bench()
    csrc = tmp_path / "paper_2102_12163_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("// kernel, first version\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    h = b.source_hash()
    rec = {"batch:fp64:g20": {"dram_bytes_per_update": 25.5, "source_hash": h},
           "batch:fp32:g64": {"dram_bytes_per_update": 4.5, "source_hash": h}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert b.profiled_traffic("batch", "fp64", 20)["dram_bytes_per_update"] == 25.5
    assert b.profiled_traffic("batch", "fp32", 64)["dram_bytes_per_update"] == 4.5
    # another launch length or precision has no record: its DRAM bytes per update differ
    assert b.profiled_traffic("batch", "fp64", 64) is None
    assert b.profiled_traffic("batch", "fp32", 20) is None
    # a changed kernel source invalidates every record
    (csrc / "k.cu").write_text("// kernel, second version\n")
    assert b.source_hash() != h
    assert b.profiled_traffic("batch", "fp64", 20) is None


def test_clock_summary_keeps_the_sampled_window_and_every_throttle_reason():
    b = _bench()
    c = b.ClockSampler(0)
    c.marks = {"load_start": 10.0, "timed_start": 11.5, "timed_end": 12.0}

    def row(mhz, *flags):
        f = ["Not Active"] * 4
        for i in flags:
            f[i] = "Active"
        return ", ".join(["0", str(mhz), "2070", "900.0", "0x0"] + f)

    c.lines = [
        (9.0, row(1000, 0)),      # before the window: ignored, with its hw_slowdown
        (10.5, row(2070)),
        (11.0, row(2055, 3)),     # sw_power_cap during the pre-roll
        (11.7, row(2070)),        # inside the timed region
        (11.9, row(2040)),        # inside the timed region
        (12.5, row(500, 1)),      # after the window: ignored
        (11.8, "garbled line"),
    ]
    s = c.summary()
    assert s["samples"] == 4
    assert s["samples_in_timed_region"] == 2
    assert s["sm_mhz"] == 2062.5
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["window_s"] == 2.0
