"""Detection fused into the uint8 de-dispersion kernel (dd_execute_detect)
against the oracle.

The plane must equal the oracle's de-dispersion bit for bit, and the search
results (mean, std, S/N and peak time per DM row and boxcar width) must equal
the oracle's search of that plane bit for bit.  The tiles of the plane are
searched by the CTAs that computed them; the boxcar starts across a tile
boundary by whichever neighbour finishes second, so the cases cover one tile,
ragged last tiles, boundaries every 1024 samples, ragged DM tiles and pulses
placed across tile boundaries.
"""
import numpy as np
import pytest

import filterbank as fb
from tests.cases import lband_input_and_plane, workload_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _fused(dd, plan, data, nin, nsamp_out, nlevels):
    x = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    out = torch.full((plan.ndm, (nsamp_out + 3) // 4 * 4 + 4), -5.0, device="cuda")
    res = plan.execute_detect(x, out, nlevels=nlevels, nsamp_in=nin, nsamp_out=nsamp_out)
    plan.sync()
    got = out.cpu().numpy()
    assert np.all(got[:, nsamp_out:] == -5.0)
    return got[:, :nsamp_out], [r.cpu().numpy() for r in res]


def _check(oracle_lib, plane, want_plane, res, nlevels):
    assert np.array_equal(plane, want_plane)
    want = oracle_lib.detect(want_plane.astype(np.float64), nlevels, True)
    for name, g, w in zip(("mean", "std", "snr", "t"), res, want):
        assert np.array_equal(g, w), name


@pytest.mark.parametrize("nchan,ndm,nsamp_out,nlevels", [
    (64, 48, 1024, 9), (64, 48, 1000, 9), (70, 40, 3000, 9), (33, 100, 4097, 9),
    (130, 96, 9000, 7), (8, 5, 1, 3), (16, 49, 2048, 9), (200, 20, 10240, 9)])
def test_fused_search_equals_the_oracle(dd, oracle_lib, nchan, ndm, nsamp_out, nlevels):
    rng = np.random.default_rng(nchan * 7 + ndm * 3 + nsamp_out)
    band = (1400.0, -1.0, 1e-4)
    table = oracle_lib.dmshift(nchan, *band)
    dms = rng.uniform(0.0, 30.0, size=ndm).astype(np.float32)
    S = oracle_lib.maxshift(table, dms)
    nin = nsamp_out + S
    pitch = (nin + 15) // 16 * 16
    data = np.zeros((nchan, pitch), np.uint8)
    data[:, :nin] = rng.integers(100, 151, size=(nchan, nin), dtype=np.uint8)
    # pulses straddling tile boundaries (1024-sample tiles) in a few DM rows
    for d in range(min(ndm, 4)):
        t_p = max(0, min(nsamp_out - 1, 1024 * (d + 1) - 3 * d - 5))
        w = 1 << (2 * d + 1)
        for c in range(nchan):
            s = oracle_lib.shift(dms[d], table[c])
            data[c, t_p + s:min(t_p + s + w, nin)] += 25     # at most 4 x 25 over 150
    plan = dd.Plan(nchan, *band, dms)
    plane, res = _fused(dd, plan, data, nin, nsamp_out, nlevels)
    want_plane = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, nsamp_out)
    _check(oracle_lib, plane, want_plane, res, nlevels)


def test_fused_search_on_the_small_workload_finds_its_pulse(dd, oracle_lib):
    w = fb.SMALL
    table, dms, S, data = workload_input(w)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    plane, res = _fused(dd, plan, data, w.nsamp_out + S, w.nsamp_out, 9)
    want_plane = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :w.nsamp_out + S]), table,
                                       dms, w.nsamp_out)
    _check(oracle_lib, plane, want_plane, res, 9)
    snr = res[2]
    d, lev = np.unravel_index(int(np.argmax(snr)), snr.shape)
    assert dms[d] == np.float32(30.0) and res[3][d, lev] in range(1990, 2010)


def test_fused_search_on_the_full_lband_beam(dd, oracle_lib):
    """The 1024-channel L-band beam at full size (1024 DMs x 131072 samples,
    128 tiles per row): the plane and every search result equal the oracle's."""
    w = fb.LBAND
    table, dms, S, data, want_plane = lband_input_and_plane(oracle_lib)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    plane, res = _fused(dd, plan, data, w.nsamp_out + S, w.nsamp_out, 9)
    _check(oracle_lib, plane, want_plane, res, 9)


def test_fused_search_equals_the_separate_pass(dd):
    """On the same plane the fused search and dd_detect give identical bits,
    and repeated calls (counters and accumulators cleared each time) too."""
    rng = np.random.default_rng(77)
    nchan, ndm, nsamp_out = 96, 60, 7000
    plan = dd.Plan(nchan, 1400.0, -1.0, 1e-4, rng.uniform(0, 25, ndm).astype(np.float32))
    nin = nsamp_out + plan.maxshift
    x = torch.randint(0, 256, (nchan, (nin + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((ndm, nsamp_out), device="cuda")
    for _ in range(2):
        fused = plan.execute_detect(x, out, nlevels=9, nsamp_in=nin)
        sep = dd.detect(out, nlevels=9, integer_valued=True)
        torch.cuda.synchronize()
        for f, s in zip(fused, sep):
            assert torch.equal(f, s)


def test_fused_search_rejects_what_it_does_not_take(dd):
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, np.arange(8, dtype=np.float32))
    x = torch.zeros((16, 1024), dtype=torch.float16, device="cuda")
    out = torch.empty((8, 512), device="cuda")
    with pytest.raises(dd.DDError):
        plan.execute_detect(x, out)                       # FP16 input: not integer planes
    x8 = torch.zeros((16, 1024), dtype=torch.uint8, device="cuda")
    with pytest.raises(dd.DDError):
        plan.execute_detect(x8, out, nlevels=10)          # widths up to 256 only
