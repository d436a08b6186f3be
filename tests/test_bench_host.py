"""Host-side logic of bench.py, without a GPU: argument handling, the clock
record parsed from nvidia-smi's CSV, the traffic record's source hash, and
the percentile helper."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def parse(monkeypatch, *argv):
    monkeypatch.setattr(sys, "argv", ["bench.py", *argv])
    return bench.parse_args()


def test_defaults_run_every_leg_on_one_gpu(monkeypatch):
    a = parse(monkeypatch)
    assert (a.gpus, a.steps, a.warmup, a.impl, a.evals) == (1, 20, 3, "ours", 100)
    assert a.warmup >= 3
    assert a.leg_set == {"peak", "small", "pme", "backward", "batched", "halo", "million"}
    assert not a.no_tune


def test_leg_selection(monkeypatch):
    assert parse(monkeypatch, "--legs", "backward").leg_set == {"backward"}
    assert parse(monkeypatch, "--legs", " million , halo ").leg_set == {"million", "halo"}
    assert parse(monkeypatch, "--no-extras", "--legs", "backward").leg_set == set()
    with pytest.raises(SystemExit):
        parse(monkeypatch, "--legs", "backward,bogus")


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def sampled(tmp_path, lines):
    s = bench.ClockSampler(0)
    f = open(tmp_path / "clocks.csv", "w+")
    f.write("\n".join(lines) + "\n")
    s.file, s.proc = f, _DoneProc()
    return s.stop()


def test_clock_record(tmp_path):
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c = sampled(tmp_path, rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_names_thermal_and_hw_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1400.0, 0x68, Active, Active, Active, Not Active"]
    c = sampled(tmp_path, rows)
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1500.0


def test_clock_record_without_samples(tmp_path):
    assert sampled(tmp_path, [""]) is None


def test_traffic_record_only_while_the_sources_match(tmp_path, monkeypatch):
    import hashlib
    rec = json.load(open(os.path.join(ROOT, "profiles", "force_kernel_traffic.json")))
    h = hashlib.sha256()
    for f in rec["source_files"]:
        (tmp_path / os.path.dirname(f)).mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), tmp_path / f)
        h.update(open(tmp_path / f, "rb").read())
    rec["source_sha256"] = h.hexdigest()  # a record taken on exactly these sources
    (tmp_path / "profiles").mkdir(exist_ok=True)
    json.dump(rec, open(tmp_path / "profiles" / "force_kernel_traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic() == rec["bytes_per_launch_96k"]
    with open(tmp_path / rec["source_files"][0], "a") as fh:
        fh.write("// edited\n")
    assert bench.load_traffic() is None


def test_percentile():
    ts = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert bench._percentile(ts, 50) == 3.0
    assert bench._percentile(ts, 0) == 1.0
    assert bench._percentile(ts, 100) == 5.0
    assert bench._percentile(ts, 99) == 5.0
