"""Host logic of bench.py that decides whether a measurement stands: the clock
summary taken from nvidia-smi rows sampled during the timed region (a run that
saw a hardware or thermal slowdown is rejected; a power cap is kept and noted),
and the measured-peaks file the roofline fractions divide by. CPU only."""
import json
import os

import bench

ROW = "0, {sm}, 2070, {pw}, 0x{mask}, {hw}, {hwt}, {swt}, {pc}"


def row(sm=2070, pw=900.0, hw="Not Active", hwt="Not Active", swt="Not Active", pc="Not Active", mask="0"):
    return ROW.format(sm=sm, pw=pw, hw=hw, hwt=hwt, swt=swt, pc=pc, mask=mask) + "\n"


def test_clean_run_median_and_maxima():
    lines = [row(sm=v, pw=p) for v, p in ((2070, 800.0), (2055, 950.5), (1980, 1010.0), (2070, 700.0), (2040, 990.0))]
    s = bench.summarize_clock_lines(lines)
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == [] and s["samples"] == 5 and s["power_w_max"] == 1010.0


def test_each_throttle_reason_is_reported():
    kinds = {"hw": "hw_slowdown", "hwt": "hw_thermal_slowdown", "swt": "sw_thermal_slowdown", "pc": "sw_power_cap"}
    for key, name in kinds.items():
        lines = [row(), row(**{key: "Active"}), row()]
        assert bench.summarize_clock_lines(lines)["reasons"] == [name], key
    both = [row(hw="Active"), row(pc="Active")]
    assert bench.summarize_clock_lines(both)["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_not_active_is_not_a_reason_and_bad_rows_are_skipped():
    lines = ["index, clocks.current.sm [MHz], ...\n", row(), "0, 2070, 20\n", "0, [N/A], 2070, 900, 0x0, a, b, c, d\n",
             row(sm=2000)]
    s = bench.summarize_clock_lines(lines)
    assert s["samples"] == 2 and s["reasons"] == [] and s["sm_mhz"] == 2035


def test_a_row_without_clocks_still_reports_its_throttle_reason():
    lines = [row(), "0, 1500, [N/A], 900, 0x0, Active, Not Active, Not Active, Not Active\n", row(sm=2000)]
    s = bench.summarize_clock_lines(lines)
    assert s["samples"] == 2 and s["sm_mhz"] == 2035 and s["reasons"] == ["hw_slowdown"]
    only = bench.summarize_clock_lines(["0, [N/A], [N/A], [N/A], 0x0, Not Active, Active, Not Active, Not Active\n"])
    assert only["sm_mhz"] is None and only["reasons"] == ["no samples", "hw_thermal_slowdown"]


def test_no_samples():
    assert bench.summarize_clock_lines([])["reasons"] == ["no samples"]
    assert bench.summarize_clock_lines(["garbage\n"])["sm_mhz"] is None


def test_measured_peaks_file(tmp_path, monkeypatch):
    path = tmp_path / "peaks.json"
    path.write_text(json.dumps({"hbm_gbs": 6753.8, "bf16_tflops": 1923.9}))
    monkeypatch.setattr(bench, "PEAKS_FILE", str(path))
    assert bench.measured_peaks()["hbm_gbs"] == 6753.8
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "absent.json"))
    assert bench.measured_peaks() == {}
    path.write_text("{not json")
    monkeypatch.setattr(bench, "PEAKS_FILE", str(path))
    assert bench.measured_peaks() == {}
    assert os.path.exists(path)


def _run_reference(env_extra):
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        if k not in env_extra:
            env.pop(k, None)
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=300, env=env, cwd=root)
    return res


def test_reference_arm_prints_one_contract_line():
    """The reference arm (the oracle timed on the host cores) prints exactly one JSON
    line with the contract's keys; its ratio inputs are the same metric and unit."""
    res = _run_reference({})
    assert res.returncode == 0, res.stderr[-500:]
    lines = [ln for ln in res.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GDoF/s"
    for key in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"].startswith(bench.WORKLOAD)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "1 thread" in cb["sample"]
    assert d["step_s_extrapolated"] > 0 and d["ms_per_step"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    res = _run_reference({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert res.returncode == 0, res.stderr[-500:]
    assert not [ln for ln in res.stdout.splitlines() if ln.strip().startswith("{")]


def test_precision_forms_are_labelled_and_the_defaults_are_the_fp64_step():
    """Every precision form the benchmark line reports has its label, every solve mode a
    name, and the default options are the FP64 step (fixed-point operator, FP64 basis,
    tensor-core elimination) on the large workload."""
    for name, key in bench.FORMS.items():
        assert key in bench.FORM_DTYPES, name
        assert key[0] in bench.MODE_NAMES
    assert bench.FORM_DTYPES[bench.FORMS["fp64_fixed"]].startswith("f64")
    assert bench.FORM_DTYPES[bench.FORMS["fp64"]].startswith("f64")
    args = bench.parse_args([])
    assert (args.mode, args.basis, args.elim, args.gpus) == (3, 0, "tc", 1)
    assert args.warmup >= 3 and args.config == "n128_m8_p3"
    assert bench.parse_args(["--mode", "0", "--basis", "2"]).basis == 2
