"""Host-side logic of the benchmark (no GPU): workload naming, the measured
peaks, and the DRAM traffic record, which must be dropped as soon as a
source of the kernels it was taken from changes."""
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(root=ROOT):
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(root, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_presets_name_their_workload():
    b = _bench()
    for cfg in (1, 2, 3, 4, 6, 7):
        a = type("A", (), dict(b.PRESETS[cfg]))()
        a.config = cfg
        c = b.config(a, 1)
        hw = f"{a.n}x{getattr(a, 'h', a.n)}"
        assert c["image"] == hw and c["l2_flush"] is True
        assert c["parallelism"] == "single"
        assert hw in c["workload"]
    a = type("A", (), dict(b.PRESETS[7]))()
    assert b.image_hw(a) == (3264, 4896)
    a = type("A", (), dict(b.PRESETS[2]))()
    a.config = 2
    assert b.config(a, 4)["parallelism"] == "replicas4"


def test_measured_peak_is_read_when_present():
    b = _bench()
    peak, kind = b.measured_peaks()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured"
        assert peak == json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    else:
        assert kind == "fallback"


def test_traffic_record_matches_its_capture_and_sources(tmp_path):
    b = _bench()
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for fam, r in rec.items():
        total = sum(k["dram_read_bytes"] + k["dram_write_bytes"] for k in r["kernels"].values())
        launches = sum(k["launches"] for k in r["kernels"].values())
        assert r["dram_bytes_per_launch"] == round(total / launches)
        # the committed record is reported only while its sources are unchanged
        assert b.traffic_record(fam) in (r["dram_bytes_per_launch"], None)
    assert b.traffic_record("no-such-family") is None

    # a copy of the tree whose record names the current sources: reported;
    # then one kernel source changes: that family's record is dropped
    import hashlib
    root = tmp_path / "tree"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "bench.py"), root / "bench.py")
    shutil.copytree(os.path.join(ROOT, "paper_2105_01586_gb300", "csrc"), root / "paper_2105_01586_gb300" / "csrc")
    csrc = root / "paper_2105_01586_gb300" / "csrc"
    for r in rec.values():
        r["sources"] = {n: hashlib.sha256((csrc / n).read_bytes()).hexdigest()[:16] for n in r["sources"]}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    bc = _bench(str(root))
    fam, r = next(iter(rec.items()))
    assert bc.traffic_record(fam) == r["dram_bytes_per_launch"]
    src = root / "paper_2105_01586_gb300" / "csrc" / next(iter(r["sources"]))
    src.write_text(src.read_text() + "\n// changed\n")
    assert bc.traffic_record(fam) is None
