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


def test_fp32_peak_follows_the_device_counts():
    """The peak uses the SM count and maximum clock the run reads from the device."""
    b = _bench()
    b.set_fp32_peak(160, 2000.0, "test")
    assert abs(b.fp32_peak_tflops() - 160 * 128 * 2 * 2000e6 / 1e12) < 1e-9
    assert abs(b.fp32_peak_tflops(152, 2070.0) - 80.5478) < 1e-3


def test_summary_keys_come_last_in_the_line():
    """The per-pass, Jacobi and precision results close the JSON line, so a
    log cut to its last few kilobytes still holds them."""
    b = _bench()
    extras = {"jacobi_8192x8192_100sweeps": 1, "op2": 2, "passes_f32": 3, "chain": 4, "passes_f16": 5,
              "batched_512": 6, "serving_2000_req_s": 7}
    out = b.ordered_extras(extras, {"worst_err_over_tol": 0.5})
    assert list(out) == ["op2", "chain", "batched_512", "serving_2000_req_s", "passes_f16", "passes_f32",
                         "jacobi_8192x8192_100sweeps", "precision"]
    assert list(b.ordered_extras({"op2": 1}, None)) == ["op2"]


def test_error_ratio_helper():
    import numpy as np
    b = _bench()
    want = np.array([1.0, 2.0, 0.0, 4.0])
    got = np.array([1.0, 2.0 + 2e-6, 0.0, 4.0 - 4e-7], dtype=np.float64)
    assert abs(b._ratio_max(got, want, want) - 1e-6) < 1e-12   # the zero-bound pixel is exact: no 0/0
    pts = b._edge_and_random_points(1, 3, 5, 7, 10)
    assert pts.shape[1] == 3 and pts[:, 0].max() < 3 and pts[:, 1].max() < 5 and pts[:, 2].max() < 7
    assert {(0, 0, 0), (0, 4, 6), (0, 0, 6), (0, 4, 0)} <= {tuple(p) for p in pts}


def test_cpu_leg_states_each_results_error(monkeypatch):
    """The CPU leg on a reduced workload, with CPU tensors standing in for the
    device outputs: results that are the oracle's own values rounded to the
    storage type give error ratios within one rounding, and a planted error
    in one pass shows up in that pass's ratio only."""
    import numpy as np
    import torch

    import oracle
    import synth
    b = _bench()
    monkeypatch.setattr(b, "C", 2)
    monkeypatch.setattr(b, "H", 64)
    monkeypatch.setattr(b, "W", 96)
    img = synth.image_f32(3, 2, 64, 96)
    ks = [synth.filter_f32(4 + K, K, K) for K in b.DIRECT_K]
    g = synth.gaussian_taps_f32(b.GAUSS_R, b.GAUSS_SIGMA)
    outs = [oracle.conv2d(img, k, want_bound=False)[0] for k in ks] + [oracle.conv2d_sep(img, g, g, False)[0]]
    d_out = [torch.from_numpy(o.astype(np.float32)) for o in outs]
    d_out[1][1, 10, 20] += 1e-3                   # a planted error in the 7x7 pass
    x16 = img.astype(np.float16)
    o16 = [torch.from_numpy(oracle.conv2d(x16, k, want_bound=False)[0].astype(np.float16)) for k in ks]
    o16.append(torch.from_numpy(oracle.conv2d_sep(x16, g, g, False)[0].astype(np.float16)))
    small = synth.image_f32(9, 1, 40, 50)
    k5 = synth.filter_f32(10, 5, 5)
    u0 = synth.jacobi_init_f32(11, 40, 48)
    u_ref, r_ref = oracle.jacobi2d(u0, 100, 10)
    keep = {"f16": (torch.from_numpy(x16), o16),
            "plain512": (small, k5, torch.from_numpy(oracle.conv2d(small, k5, False)[0].astype(np.float32))),
            "batch": {"f32": [(0, small, k5, oracle.conv2d(small, k5, False)[0].astype(np.float32))]},
            "jacobi": (u0, torch.from_numpy(u_ref.astype(np.float32)), torch.from_numpy(r_ref))}
    cpu, prec = b.cpu_baseline(torch, img, ks, g, d_out, keep, budget_s=0.01)
    assert cpu["kind"] == "oracle" and cpu["value"] > 0
    f32 = prec["conv_f32_err_over_bound"]
    assert f32["7x7"] > 1e-5                      # the planted error
    assert f32["3x3"] <= 2.0 ** -24 and f32["15x15"] <= 2.0 ** -24 and f32["gauss15-sep"] <= 2.0 ** -24
    assert max(prec["conv_f16_err_over_bound"].values()) <= 2.0 ** -11
    assert prec["plain_512x512_5x5_err_over_bound"] <= 2.0 ** -24
    assert prec["batched_f32_err_over_bound"] <= 2.0 ** -24
    assert prec["jacobi_max_abs_du"] <= 1e-6 and prec["jacobi_residual_rel_err"] <= 1e-6
    assert prec["worst_err_over_tol"] > 10        # the planted error dominates

