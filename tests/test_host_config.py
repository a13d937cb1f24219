"""Host-side configuration the benchmark and the library read (CPU only): the recorded DRAM
traffic is reported only for the tensor-kernel source and launch count it was captured with,
and the committed tuning table only holds options the library accepts, for every class the
tuner times."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.fixture()
def traffic_file(tmp_path, monkeypatch):
    sha = hashlib.sha256(open(bench.TC_SOURCE, "rb").read()).hexdigest()
    path = tmp_path / "traffic.json"
    rec = {"bytes_per_launch": 1.5e7, "source_sha256": sha, "capture": "test capture", "launches": 80}
    path.write_text(json.dumps({"dense_full:default:factor": rec,
                                "stale:default:factor": dict(rec, source_sha256="0" * 64)}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    return path


def test_traffic_is_reported_for_its_capture(traffic_file):
    assert bench.captured_traffic("dense_full:default:factor", 80.0) == (1.5e7, "test capture")
    assert bench.captured_traffic("dense_full:default:factor") == (1.5e7, "test capture")


def test_traffic_is_withheld_when_stale_or_missing(traffic_file):
    val, why = bench.captured_traffic("dense_full:default:factor", 96.0)
    assert val is None and "launches" in why
    val, why = bench.captured_traffic("stale:default:factor", 80.0)
    assert val is None and "changed" in why
    val, why = bench.captured_traffic("rank_deficient:default:factor", 80.0)
    assert val is None
    val, why = bench.captured_traffic("", 80.0)
    assert val is None


def test_committed_traffic_record_matches_the_kernel_source():
    """The record bench.py reports at the default configuration was taken with this source."""
    data = json.load(open(bench.TRAFFIC_FILE))
    rec = data["dense_full:default:factor"]
    sha = hashlib.sha256(open(bench.TC_SOURCE, "rb").read()).hexdigest()
    assert rec["source_sha256"] == sha
    assert rec["bytes_per_launch"] > 0 and rec["launches"] > 0


def test_tuning_table_holds_accepted_options_for_every_class():
    table = json.load(open(os.path.join(ROOT, "paper_1112_5717_gb300", "tuning.json")))
    classes = set()
    for e in table["entries"]:
        assert 1 <= e["leaf_rows"] <= 64                  # CUP_OPT_LEAF_ROWS range
        assert 1 <= e["window"] <= 128                    # CUP_OPT_WINDOW range
        assert e["tc_min_k"] >= 1
        assert 0 <= e["min_lo"] < e["min_hi"]
        assert e["ms"] <= e["default_ms"] * 1.001         # the pick is never slower than the defaults
        assert min(c[3] for c in e["candidates"]) == pytest.approx(e["ms"])
        classes.add((e["limbs"], e["tall"]))
    assert classes == {(L, t) for L in (1, 2, 3, 4) for t in (0, 1)}
