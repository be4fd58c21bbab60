"""Boxcar detection (dd_detect) against the oracle.

Integer planes (the planes of uint8 input) must give identical results, bit
for bit: mean, std, S/N and peak times.  FP32 planes are checked within a
tolerance derived from FP32 boxcar rounding, with every reported peak time
checked to be a valid maximiser.  End to end, the search finds the small
workload's injected pulse and the Fig. 3 pulse at their DMs, and on the
full-size L-band beam the rows the oracle recomputes itself agree exactly.
"""
import math

import numpy as np
import pytest

import filterbank as fb
from tests.cases import workload_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _gpu_detect(dd, plane, nlevels, integer, pitch_extra=0):
    ndm, nsamp = plane.shape
    x = torch.zeros((ndm, nsamp + pitch_extra), dtype=torch.float32, device="cuda")
    x[:, :nsamp] = torch.from_numpy(plane.astype(np.float32)).cuda()
    if pitch_extra:
        x[:, nsamp:] = 1e9            # beyond nsamp: must not be read into any result
    res = dd.detect(x, nsamp=nsamp, nlevels=nlevels, integer_valued=integer)
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in res]


@pytest.mark.parametrize("ndm,nsamp,nlevels", [(3, 3000, 9), (2, 200, 9), (4, 9000, 6), (1, 1, 3),
                                               (2, 8192, 9), (1, 17000, 9), (5, 131, 1),
                                               (3, 65537, 9)])
def test_integer_planes_are_bit_identical(dd, oracle_lib, ndm, nsamp, nlevels):
    rng = np.random.default_rng(ndm * 1000 + nsamp)
    plane = rng.integers(0, 1 << 20, size=(ndm, nsamp)).astype(np.float64)
    for d in range(ndm):
        if nsamp > 40:
            t0 = int(rng.integers(0, nsamp - 32))
            plane[d, t0:t0 + (1 << d % 6)] += 400000.0
    want = oracle_lib.detect(plane, nlevels, True)
    got = _gpu_detect(dd, plane, nlevels, True, pitch_extra=13)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_ties_report_the_first_time(dd, oracle_lib):
    plane = np.zeros((2, 5000))
    plane[0, [100, 2100, 4100]] = 50.0         # three equal spikes across warps
    plane[1, :] = 7.0                          # constant: std 0, every boxcar equal
    want = oracle_lib.detect(plane, 9, True)
    got = _gpu_detect(dd, plane, 9, True)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert got[3][0, 0] == 100 and np.all(got[3][1] == 0) and np.all(got[2][1] == 0.0)


def test_non_integer_values_in_integer_mode_give_nan_rows(dd):
    plane = np.full((3, 700), 5.0)
    plane[1, 33] = 2.5
    plane[2, 600] = float(1 << 21)
    mean, std, snr, tpk = _gpu_detect(dd, plane, 4, True)
    assert np.isfinite(mean[0]) and np.all(np.isfinite(snr[0]))
    assert np.all(np.isnan(mean[1:])) and np.all(np.isnan(std[1:])) and np.all(np.isnan(snr[1:]))


@pytest.mark.parametrize("ndm,nsamp", [(3, 5000), (2, 20000)])
def test_float_planes_within_fp32_boxcar_rounding(dd, oracle_lib, ndm, nsamp):
    rng = np.random.default_rng(nsamp)
    plane = (rng.normal(1000.0, 30.0, size=(ndm, nsamp))).astype(np.float32).astype(np.float64)
    plane[0, 1234:1242] += 400.0
    nlev = 9
    mean, std, snr, tpk = _gpu_detect(dd, plane, nlev, False)
    wm, ws, wsnr, wt = oracle_lib.detect(plane, nlev, False)
    assert np.allclose(mean, wm, rtol=1e-9, atol=0) and np.allclose(std, ws, rtol=1e-6, atol=0)
    ci = np.concatenate([np.zeros((ndm, 1)), np.cumsum(plane, axis=1)], axis=1)
    for lev in range(nlev):
        w = 1 << lev
        box = ci[:, w:] - ci[:, :-w]              # FP64 boxcars at every t
        # FP32 tree sum of w terms: each of log2(w) adds rounds once
        tol_b = (lev + 1) * 2.0 ** -23 * np.abs(box).max(axis=1)
        assert np.all(box.max(axis=1) - box[np.arange(ndm), tpk[:, lev]] <= 2 * tol_b)
        tol = 2 * tol_b / (ws * math.sqrt(w)) + 1e-9 * np.abs(wsnr[:, lev])
        assert np.all(np.abs(snr[:, lev] - wsnr[:, lev]) <= tol)
    assert tpk[0, 3] == 1234


def test_search_finds_the_small_workload_pulse(dd, oracle_lib):
    """dd_execute then dd_detect on the small workload (uint8, exact plane):
    identical to oracle.detect on the oracle's own plane, and the best S/N of
    the whole search sits at the injected pulse's DM, width and time."""
    w = fb.SMALL
    table, dms, S, data = workload_input(w)
    nin = w.nsamp_out + S
    want_plane = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, w.nsamp_out)
    want = oracle_lib.detect(want_plane, 6, True)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    x = torch.from_numpy(data).cuda()
    out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device="cuda")
    plan.execute(x, out, nsamp_in=nin)
    got = [r.cpu().numpy() for r in dd.detect(out, nlevels=6, integer_valued=True)]
    plan.sync()
    for g, wv in zip(got, want):
        assert np.array_equal(g, wv)
    p = w.pulses[0]
    d, lev = np.unravel_index(np.argmax(got[2]), got[2].shape)
    assert dms[d] == np.float32(p.dm) and (1 << lev) == p.width and got[3][d, lev] == p.t


def test_lband_full_size_rows_match_the_oracle(dd, oracle_lib):
    """The full L-band beam (1024 ch x 1024 DMs x 131072): the GPU searches its
    own plane; the oracle recomputes 12 rows (including every pulse's DM) from
    the filterbank and searches them; those rows agree bit for bit."""
    w = fb.LBAND
    table, dms, S, data = workload_input(w)
    nin = w.nsamp_out + S
    pulses = fb.all_pulses(w)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    x = torch.from_numpy(data).cuda()
    out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device="cuda")
    plan.execute(x, out, nsamp_in=nin)
    got = [r.cpu().numpy() for r in dd.detect(out, nlevels=9, integer_valued=True)]
    plan.sync()
    rows = sorted(set([0, 1, 511, 1023] + [int(np.argmin(np.abs(dms - p.dm))) for p in pulses]))
    sub = dms[rows]
    want_plane = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, sub,
                                       w.nsamp_out, threads=True)
    want = oracle_lib.detect(want_plane, 9, True)
    for g, wv in zip(got, want):
        assert np.array_equal(g[rows], wv)
    for p in pulses:     # every injected pulse stands out at its DM
        d = int(np.argmin(np.abs(dms - p.dm)))
        assert got[2][d].max() > 8.0
