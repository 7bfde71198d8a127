"""The roofline traffic that bench.py reports for the rank-k kernel comes from
the committed ncu record only while the kernel's device code is the code the
counters were taken on: a SHA-256 of k_herk_tc.cu up to its operand
preparation section.  Checked on copies of the record and the source."""
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench_mod():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _copy_tree(tmp_path):
    rec = json.load(open(os.path.join(ROOT, "profiles", "herk_tc_traffic.json")))
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(ROOT, "profiles", "herk_tc_traffic.json"), tmp_path / "profiles")
    dst = tmp_path / rec["source"]
    os.makedirs(dst.parent)
    shutil.copy(os.path.join(ROOT, rec["source"]), dst)
    return rec, dst


def test_traffic_follows_the_recorded_device_code(bench_mod, tmp_path, monkeypatch):
    rec, src = _copy_tree(tmp_path)
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    want = float(rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"])
    # the committed kernel is the captured one
    assert bench_mod.herk_traffic() == want
    text = src.read_text()
    cut = text.index(bench_mod.HERK_DEVICE_END)
    # an edit after the device code (host launch helpers) keeps the record valid
    src.write_text(text + "\n// host-side note\n")
    assert bench_mod.herk_traffic() == want
    # any edit inside the device code, even a comment, voids it
    src.write_text(text[:cut] + "// changed\n" + text[cut:])
    assert bench_mod.herk_traffic() is None
    # so does a missing record or a source without the section marker
    src.write_text(text.replace(bench_mod.HERK_DEVICE_END, "// elsewhere"))
    assert bench_mod.herk_traffic() is None
    os.remove(tmp_path / "profiles" / "herk_tc_traffic.json")
    assert bench_mod.herk_traffic() is None
