"""bench.py helpers that need no GPU: the ncu traffic record is reported only
for the exact kernel source, workload, dtype and tile shape it was taken on,
and the reference arm's oracle sample is bounded and well formed."""
import os

import numpy as np
import pytest

import bench
import filterbank as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_record_matches_the_current_kernel_source():
    digest = bench._sha256("dd_kernel.cuh", "dd_launch.cpp")
    for rec in bench.PROFILED_TRAFFIC:
        # a record whose kernel or launch code changed must not be reported
        got = bench.profiled_traffic(rec["workload"], rec["dtype"], rec["tiles"])
        assert (got is rec) == (rec["code_sha256"] == digest)
        # another tile shape or dtype never matches
        other = list(rec["tiles"])
        other[1] += 1
        assert bench.profiled_traffic(rec["workload"], rec["dtype"], other) is None
        assert bench.profiled_traffic(rec["workload"], "f32", rec["tiles"]) is None
        assert rec["bytes"] > 0 and os.path.exists(os.path.join(ROOT, rec["source"]))


def test_traffic_digest_covers_kernel_and_launch_code():
    one = bench._sha256("dd_kernel.cuh")
    both = bench._sha256("dd_kernel.cuh", "dd_launch.cpp")
    assert one != both and len(both) == 64


def test_oracle_sample_is_bounded_and_described(oracle_lib):
    prep = bench.prepare_oracle_sample(fb.SMALL, budget_s=0.05)
    res = bench.time_oracle_sample(fb.SMALL, prep)
    assert res["kind"] == "oracle" and res["unit"] == "adds/s" and res["value"] > 0
    assert res["cores"] >= 1 and "channels" in res["sample"]
    assert 1 <= prep["ndm"] <= fb.SMALL.ndm and prep["nsamp"] <= fb.SMALL.nsamp_out
