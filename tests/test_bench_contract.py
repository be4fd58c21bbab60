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
        for dtype in ("u8", "f16", "f32"):
            if dtype != rec["dtype"] and not any(
                    r["workload"] == rec["workload"] and r["dtype"] == dtype
                    and list(r["tiles"]) == list(rec["tiles"]) for r in bench.PROFILED_TRAFFIC):
                assert bench.profiled_traffic(rec["workload"], dtype, rec["tiles"]) is None
        assert rec["bytes"] > 0 and rec["compulsory"] > 0


def test_traffic_digest_covers_kernel_and_launch_code():
    one = bench._sha256("dd_kernel.cuh")
    both = bench._sha256("dd_kernel.cuh", "dd_launch.cpp")
    assert one != both and len(both) == 64


@pytest.mark.parametrize("threads", [True, False])
def test_oracle_sample_is_bounded_and_described(oracle_lib, threads):
    prep = bench.prepare_oracle_sample(fb.SMALL, budget_s=0.05, threads=threads)
    res = bench.time_oracle_sample(fb.SMALL, prep)
    assert res["kind"] == "oracle" and res["unit"] == "adds/s" and res["value"] > 0
    assert res["cores"] >= 1 and "channels" in res["sample"]
    assert (res["cores"] == 1) == (not threads) or os.cpu_count() == 1
    assert ("single-threaded" in res["sample"]) == (not threads)
    assert 1 <= prep["ndm"] <= fb.SMALL.ndm and prep["nsamp"] <= fb.SMALL.nsamp_out


def test_reference_arm_line_reports_its_timed_sample(oracle_lib, capsys):
    """The reference arm prints one line whose ms_per_step is the timed
    sample's own step time (not the full workload extrapolated) and whose
    config names the sample."""
    import json
    import types
    args = types.SimpleNamespace(gpus=1, steps=2, warmup=1)
    os.environ.pop("RANK", None)
    bench.run_reference(args, fb.SMALL)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    smp = line["config"]["timed_sample"]
    assert smp["adds"] == fb.SMALL.nchan * smp["ndm"] * smp["nsamp_out"]
    assert abs(line["ms_per_step"] - smp["adds"] / line["value"] * 1e3) \
        <= 0.5 * line["ms_per_step"]
    assert line["full_workload_ms_extrapolated"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
