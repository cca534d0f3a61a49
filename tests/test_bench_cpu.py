"""Host logic of bench.py that needs no GPU: every profiling case names the
kernel whose sources define it, and the DRAM traffic recorded from an ncu
capture is reported only while those sources are the ones it was taken on."""
import json
import os

import bench


def test_every_case_names_a_kernel_with_existing_sources():
    csrc = os.path.join(bench.ROOT, "paper_1705_06661_gb300", "csrc")
    for case in bench.CASES:
        kern = bench.CASE_KERNEL[case]
        for f in bench.KERNEL_SOURCES[kern]:
            assert os.path.isfile(os.path.join(csrc, f)), (case, f)


def test_recorded_traffic_cases_are_known():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for case, c in rec["cases"].items():
        assert case in bench.CASES, case
        assert c["kernel"] == bench.CASE_KERNEL[case], case
        assert c["dram_bytes_per_launch"] == c["read"] + c["write"], case


def test_traffic_is_reported_only_for_unchanged_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    good = bench.kernel_source_hash("k2")
    rec = {"cases": {"paper-3d": {"dram_bytes_per_launch": 123.0, "source_hash": good},
                     "paper-4d": {"dram_bytes_per_launch": 456.0, "source_hash": "0" * 16}}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash is taken over the sources under the new root: recreate them there
    src = tmp_path / "paper_1705_06661_gb300" / "csrc"
    src.mkdir(parents=True)
    real = os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "paper_1705_06661_gb300", "csrc")
    for f in bench.KERNEL_SOURCES["k2"]:
        (src / f).write_bytes(open(os.path.join(real, f), "rb").read())
    assert bench.ncu_traffic("paper-3d") == 123.0
    assert bench.ncu_traffic("paper-4d") is None      # taken on other sources
    assert bench.ncu_traffic("paper-3d-544") is None  # no record
    # an edited source invalidates the record
    with open(src / "ss_k2.cuh", "ab") as fh:
        fh.write(b"\n")
    assert bench.ncu_traffic("paper-3d") is None
