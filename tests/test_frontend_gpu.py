"""Front end (dd_frontend: Stokes I, integration, RFI excision by iterated
sigma clipping, quantisation) against the oracle, bit for bit: codes,
per-channel mean and std.

Covers every integration factor class (1, 2, 4 and the 16-byte load path,
64), one to eight clipping passes, every cluster size of the fused kernel
and the long-row fallback, ragged output lengths and dropped trailing raw samples, the byte-load
path (unaligned rows), channels of constant power (std 0), RFI from the
seeded layout, empty outputs, the full-size L-band block (1024 channels x
147628 output spectra x 16 raw samples, sampled channels recomputed by the
oracle) and the front end feeding dd_execute.
"""
import numpy as np
import pytest

import filterbank as fb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


@pytest.fixture(scope="module")
def vpool():
    return fb.VoltagePool(21, size=1 << 20)


def _gpu(dd, volts, nint, k, niter=1, offset=0, pitch_extra=0):
    """Run dd_frontend on host volts int8 [nchan][nraw][4], rows placed at a
    byte offset inside a wider device buffer; returns (codes, mean, std)."""
    nchan, nraw = volts.shape[0], volts.shape[1]
    pitch = (4 * nraw + 15) // 16 * 16 + pitch_extra
    buf = torch.zeros(nchan * pitch + offset + 16, dtype=torch.int8, device="cuda")
    rows = buf[offset:offset + nchan * pitch].view(nchan, pitch)
    rows[:, :4 * nraw] = torch.from_numpy(volts.reshape(nchan, -1)).cuda()
    v = rows[:, :4 * nraw].unflatten(1, (nraw, 4))
    n = nraw // nint
    opitch = max(16, (n + 16 + 15) // 16 * 16)
    out = torch.full((nchan, opitch), 0xA7, dtype=torch.uint8, device="cuda")
    _, mean, std = dd.frontend(v, nint, k, niter, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:, n:] == 0xA7)        # columns past n untouched
    return got[:, :n], mean.cpu().numpy(), std.cpu().numpy()


def _same(got, want):
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[1], want[1])     # FP64, bit for bit
    assert np.array_equal(got[2], want[2])


@pytest.mark.parametrize("nint", [1, 2, 4, 16, 64])
@pytest.mark.parametrize("nchan,nraw", [(3, 1000), (64, 4099), (17, 70001), (5, 64 * 1031 + 63)])
def test_frontend_matches_oracle(dd, oracle_lib, vpool, nint, nchan, nraw):
    volts = vpool.rows(vpool.layout(nchan, nraw))
    for k, niter in ((4.0, 1), (1e9, 1), (4.0, 3), (2.5, 8)):
        _same(_gpu(dd, volts, nint, k, niter), oracle_lib.frontend(volts, nint, k, niter))


@pytest.mark.parametrize("nint", [4, 16])
def test_byte_path_for_unaligned_rows(dd, oracle_lib, vpool, nint):
    """Rows 4 bytes off a 16-byte boundary, or a pitch of 4 mod 16, take the
    4-byte load path; results are unchanged."""
    volts = vpool.rows(vpool.layout(9, 5003))
    want = oracle_lib.frontend(volts, nint, 3.0, 2)
    _same(_gpu(dd, volts, nint, 3.0, 2, offset=4), want)
    _same(_gpu(dd, volts, nint, 3.0, 2, pitch_extra=4), want)


def test_constant_and_zero_channels(dd, oracle_lib, vpool):
    volts = vpool.rows(vpool.layout(6, 2048, rfi=False))
    volts[1] = (5, -5, 5, -5)        # constant power: std 0 -> every code 128
    volts[4] = 0                     # all-zero channel
    for niter in (1, 4):
        want = oracle_lib.frontend(volts, 8, 4.0, niter)
        assert want[2][1] == 0.0 and np.all(want[0][1] == 128)
        _same(_gpu(dd, volts, 8, 4.0, niter), want)


def test_rfi_is_clipped_to_128(dd, oracle_lib, vpool):
    lay = vpool.layout(128, 64000)
    volts = vpool.rows(lay)
    got = _gpu(dd, volts, 16, 4.0, 3)
    _same(got, oracle_lib.frontend(volts, 16, 4.0, 3))
    # output samples wholly inside an impulse (every channel) or a tone
    for r0, r1 in lay.impulses:
        assert np.all(got[0][:, r0 // 16 + 1:r1 // 16] == 128)
    for c, r0, r1 in lay.tones:
        assert np.all(got[0][c, r0 // 16 + 1:r1 // 16] == 128)


@pytest.mark.parametrize("nraw,nint", [(0, 1), (15, 16), (63, 64)])
def test_no_output_samples(dd, nraw, nint):
    v = torch.zeros((4, max(nraw, 1), 4), dtype=torch.int8, device="cuda")[:, :nraw]
    out = torch.full((4, 16), 0xA7, dtype=torch.uint8, device="cuda")
    _, mean, std = dd.frontend(v, nint, 4.0, 2, out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 0xA7) and torch.all(mean == 0) and torch.all(std == 0)


@pytest.mark.parametrize("n,fused", [(25600, True), (25601, True), (102401, True),
                                     (409600, True), (409601, False), (1 << 19, False)])
def test_cluster_sizes_and_long_row_fallback(dd, oracle_lib, n, fused):
    """Rows up to 409600 output samples run in one fused launch (clusters of
    1, 2, 4 or 8 CTAs with P in shared memory); longer rows take the
    work-array path (niter + 1 launches).  Both agree with the oracle."""
    rng = np.random.default_rng(n)
    volts = rng.normal(0.0, 12.0, size=(2, n, 4)).round().clip(-128, 127).astype(np.int8)
    volts[0, n // 3:n // 3 + 50] = (90, 90, 90, 90)
    n0 = dd.launch_count()
    got = _gpu(dd, volts, 1, 3.5, 3)
    assert dd.launch_count() - n0 == (1 if fused else 4)
    _same(got, oracle_lib.frontend(volts, 1, 3.5, 3))


def test_full_size_lband_block(dd, oracle_lib):
    """1024 channels x 147628 output spectra (the L-band beam's input length)
    from 16 raw samples each: 9.7 GB of voltages built on the device from the
    seeded pools; sampled channels (including every tone) recomputed by the
    oracle from the same layout."""
    nchan, n, nint = 1024, 147628, 16
    pool = fb.VoltagePool(22)
    lay = pool.layout(nchan, n * nint)
    buf, v = pool.rows_torch(lay, "cuda")
    n0 = dd.launch_count()
    out, mean, std = dd.frontend(v, nint, 4.0, 3)
    torch.cuda.synchronize()
    assert dd.launch_count() - n0 == 1        # fused: clusters of 8 CTAs
    rng = np.random.default_rng(8)
    chans = sorted({0, nchan - 1, *(c for c, _, _ in lay.tones),
                    *rng.choice(nchan, size=4, replace=False).tolist()})
    del buf, v
    host = pool.rows(lay, chans)
    want = oracle_lib.frontend(host, nint, 4.0, 3)
    got_codes = out[chans, :n].cpu().numpy()
    assert np.array_equal(got_codes, want[0])
    assert np.array_equal(mean[chans].cpu().numpy(), want[1])
    assert np.array_equal(std[chans].cpu().numpy(), want[2])


def test_frontend_feeds_dedispersion(dd, oracle_lib, vpool):
    """Voltages -> filterbank -> (DM,t) plane on the device, equal to the
    oracle's front end followed by the oracle's de-dispersion."""
    w = fb.SMALL
    dms = fb.dm_grid(w.dm_lo, w.dm_step, w.ndm)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    n = w.nsamp_out + plan.maxshift
    nint = 8
    volts = vpool.rows(vpool.layout(w.nchan, n * nint + 5))
    vt = torch.from_numpy(volts).cuda()
    fbank, _, _ = dd.frontend(vt, nint, 4.0, 3)
    plane = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device="cuda")
    plan.execute(fbank, plane, nsamp_in=n)
    torch.cuda.synchronize()
    codes, _, _ = oracle_lib.frontend(volts, nint, 4.0, 3)
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    want = oracle_lib.dedisperse(codes, table, dms, w.nsamp_out)
    assert np.array_equal(plane.cpu().numpy(), want)
