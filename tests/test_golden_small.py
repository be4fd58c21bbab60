"""Regression pin of the seeded small workload (64 channels, 64 DMs, 8192
samples, one DM-30 pulse): input bytes, the FP32 dmshift table and the oracle
plane must keep the digests that tests/golden/make_golden.py recorded."""
import hashlib
import json
import os

from tests.golden.make_golden import small_case

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "small_workload.json")


def test_small_workload_digests(oracle_lib):
    rec = json.load(open(GOLDEN))
    w, table, dms, S, data = small_case()
    assert S == rec["maxshift"]
    assert hashlib.sha256(data.tobytes()).hexdigest() == rec["input_sha256"]
    assert hashlib.sha256(table.tobytes()).hexdigest() == rec["dmshift_sha256"]
    plane = oracle_lib.dedisperse(data, table, dms, w.nsamp_out)
    assert hashlib.sha256(plane.tobytes()).hexdigest() == rec["plane_sha256"]
    for key, v in rec["plane_samples"].items():
        d, t = map(int, key.split(","))
        assert plane[d, t] == v
