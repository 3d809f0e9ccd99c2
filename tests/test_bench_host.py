"""Host-side pieces of the benchmark and of the reference-minimum records (no GPU): the ncu
counter file is used only while the kernel source still has its recorded hash, and a
record is tight only when its last 1000 iterations lowered f by at most 1e-7 relative."""
import hashlib
import os

import bench
from oracle import fstar


def test_counter_file_is_used_only_for_the_recorded_source(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1810_13100_gb300", "csrc", "joseph.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    rel = os.path.relpath(src, bench.ROOT)
    (tmp_path / "counters_w.txt").write_text(
        "# comment line\n"
        "k_gather %s %s 100 200\n"
        "k_fwd %s %s 300 400\n" % (rel, sha, rel, "0" * 64))
    c = bench.load_counters("w", str(tmp_path))
    assert bench.counters_for(c, "joseph_gather") == (100.0, 200.0)
    assert bench.counters_for(c, "joseph_fwd") == (None, None)      # stale: another source
    assert bench.counters_for(c, "fft_rows_fwd") == (None, None)    # never captured
    assert bench.load_counters("absent", str(tmp_path)) == {}


def test_committed_counter_file_parses():
    c = bench.load_counters("ct512")
    assert set(c) >= {"k_gather", "k_fwd_strip", "k_fwd_sum"}
    for v in c.values():
        assert v["traffic"] > 0 and v["warp_instr"] > 0


def test_counters_of_a_class_sum_its_kernels():
    """The strip-form K is two kernels per launch: its class's counters are their sum, and
    a class with any kernel missing or stale has none."""
    cnt = {"k_fwd_strip": {"current": True, "traffic": 4.0, "warp_instr": 90.0},
           "k_fwd_sum": {"current": True, "traffic": 25.0, "warp_instr": 1.0},
           "k_gather": {"current": False, "traffic": 4.0, "warp_instr": 134.0}}
    assert bench.counters_for(cnt, "joseph_fwd") == (29.0, 91.0)
    assert bench.counters_for(cnt, "joseph_gather") == (None, None)
    assert bench.counters_for(cnt, "joseph_fwd", ["k_fwd"]) == (None, None)
    assert bench.counters_for(cnt, "joseph_fwd", "k_fwd_strip") == (4.0, 90.0)


def test_tightness_of_a_record():
    rec = {"f_star": 2.0e6, "iterations": 8000, "decrease_last_1000": 0.1}
    assert fstar.is_tight(rec)                       # 5e-8 relative
    rec["decrease_last_1000"] = 0.3                  # 1.5e-7 relative
    assert not fstar.is_tight(rec)
    assert not fstar.is_tight({"f_star": 1.0, "iterations": 500, "decrease_last_1000": 0.0})


def test_stored_records_carry_their_tightness():
    import glob
    import json
    for path in glob.glob(os.path.join(bench.ROOT, "tests", "golden", "fstar_*.json")):
        rec = json.load(open(path))
        assert rec.get("tight") == fstar.is_tight(rec), path


def test_records_serialise_numpy_values(tmp_path):
    """A record written from numpy scalars (the oracle's history) is plain JSON."""
    import json
    import numpy as np
    hist = [(np.int64(1000), np.float64(10.0)), (np.int64(2000), np.float64(9.999999))]
    P = type("P", (), {"b": np.ones(3)})()
    out = str(tmp_path / "rec.json")
    fstar.write_golden("w", 0, P, {"alpha": 0.003}, np.float64(5.0), hist, out_path=out)
    rec = json.load(open(out))
    assert rec["tight"] is False and rec["iterations"] == 2000
