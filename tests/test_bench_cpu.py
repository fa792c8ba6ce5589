"""The benchmark's reference arm (the FP64 oracle on the host cores) runs
without a GPU and prints one JSON line with the keys the contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--ref-seconds", "2"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Gpixel/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["h"] == 8192 and d["config"]["w"] == 8192 and d["config"]["channels"] == 3


def test_warmup_below_three_is_refused():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "2"], capture_output=True,
                       text=True, timeout=120, cwd=ROOT)
    assert r.returncode != 0


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp32_peak_from_unit_counts():
    """152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz."""
    assert abs(_bench().fp32_peak_tflops() - 80.5478) < 1e-3


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    """The committed DRAM-traffic figure is used only while the kernel sources
    hash to the value recorded with it; after any edit it reads as null."""
    b = _bench()
    for p in b.KERNEL_SOURCES:
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, p), "rb").read())
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    rec = {"k": {"bytes_per_launch": 123, "source_sha": b.sources_sha()}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert b.traffic_record("k") == 123
    assert b.traffic_record("other") is None
    (tmp_path / b.KERNEL_SOURCES[0]).write_bytes(b"// edited\n" + (tmp_path / b.KERNEL_SOURCES[0]).read_bytes())
    assert b.traffic_record("k") is None                  # sources changed since the capture
    (tmp_path / "profiles" / "traffic.json").write_text("not json")
    assert b.traffic_record("k") is None


def test_clock_samples_are_summarised(tmp_path):
    """nvidia-smi rows: median SM clock under load, the maximum clock, and every
    throttle reason seen active in any sample; malformed rows are skipped."""
    b = _bench()
    c = b.Clocks(0)
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
            "garbage line", "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    path.write_text("\n".join(rows) + "\n")
    c.f = open(path, "r+")
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    path2 = tmp_path / "clocks2.csv"
    path2.write_text("0, 1500, 2070, 700, 0x8, Active, Not Active, Not Active, Not Active\n")
    c.f = open(path2, "r+")
    assert c.summary()["reasons"] == ["hw_slowdown"]
    path3 = tmp_path / "clocks3.csv"
    path3.write_text("")
    c.f = open(path3, "r+")
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
