"""Pins of the oracle's input-side unpacking and its boxcar detection (no GPU).

Unpacking is checked against numpy's own little-endian bit unpacking, hand-made
bytes and the plain transpose of 8-bit spectra.  Detection is checked against
closed forms for a box pulse on a quiet background, numpy's mean and standard
deviation, an independent cumulative-sum search for the peak time, the
degenerate cases, and the Fig. 3 experiment (a square pulse dispersed at
DM 50 is found at DM 50, at its width and time).
"""
import math

import numpy as np
import pytest

import filterbank as fb


# --------------------------------------------------------------------------
# Unpacking: sigproc spectra (time-major, first sample in the low bits)
# --------------------------------------------------------------------------

def test_unpack_hand_made_bytes(oracle_lib):
    # 2-bit: 0xE4 = 0b11_10_01_00 holds channels 0..3 = 0, 1, 2, 3
    assert list(oracle_lib.unpack(np.array([0xE4], np.uint8), 2, 4, 1).ravel()) == [0, 1, 2, 3]
    # 4-bit: 0xA5 holds channel 0 = 5 (low nibble), channel 1 = 10
    assert list(oracle_lib.unpack(np.array([0xA5], np.uint8), 4, 2, 1).ravel()) == [5, 10]
    # 1-bit: 0b0000_0101 holds channels 0 and 2 set
    assert list(oracle_lib.unpack(np.array([0x05], np.uint8), 1, 8, 1).ravel()) == \
        [1, 0, 1, 0, 0, 0, 0, 0]
    # two 4-bit spectra of 2 channels: [t][c] -> out[c][t]
    got = oracle_lib.unpack(np.array([0x21, 0x43], np.uint8), 4, 2, 2)
    assert got.tolist() == [[1, 3], [2, 4]]


@pytest.mark.parametrize("nbits", [1, 2, 4, 8])
def test_unpack_matches_numpy_little_endian_bits(oracle_lib, nbits):
    rng = np.random.default_rng(nbits)
    nchan, nsamp = 48, 37
    raw = rng.integers(0, 256, size=nsamp * nchan * nbits // 8, dtype=np.uint8)
    bits = np.unpackbits(raw, bitorder="little").reshape(nsamp, nchan, nbits)
    want = (bits.astype(np.int64) << np.arange(nbits)).sum(axis=2).T.astype(np.uint8)
    assert np.array_equal(oracle_lib.unpack(raw, nbits, nchan, nsamp), want)


def test_unpack_8bit_is_a_transpose_and_packing_round_trips(oracle_lib):
    rng = np.random.default_rng(8)
    spectra = rng.integers(0, 256, size=(29, 40), dtype=np.uint8)  # [t][c]
    assert np.array_equal(oracle_lib.unpack(spectra.ravel(), 8, 40, 29), spectra.T)
    for nbits in (1, 2, 4):
        vals = rng.integers(0, 1 << nbits, size=(29, 40), dtype=np.uint8)
        bits = ((vals[..., None] >> np.arange(nbits)) & 1).astype(np.uint8)
        raw = np.packbits(bits.ravel(), bitorder="little")
        assert np.array_equal(oracle_lib.unpack(raw, nbits, 40, 29), vals.T)


def test_unpack_rejects_bad_shapes(oracle_lib):
    with pytest.raises(ValueError):
        oracle_lib.unpack(np.zeros(4, np.uint8), 3, 8, 1)
    with pytest.raises(ValueError):
        oracle_lib.unpack(np.zeros(4, np.uint8), 2, 3, 1)   # 6 bits per spectrum
    with pytest.raises(ValueError):
        oracle_lib.unpack(np.zeros(3, np.uint8), 8, 2, 2)   # 4 bytes needed


# --------------------------------------------------------------------------
# Detection: boxcar widths 1, 2, 4, ... with the row's mean and std
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w0,t0,amp,n", [(4, 100, 7.0, 512), (1, 0, 3.0, 64), (16, 40, 2.0, 256),
                                         (8, 250, 5.0, 258)])
@pytest.mark.parametrize("integer", [True, False])
def test_box_pulse_closed_form(oracle_lib, w0, t0, amp, n, integer):
    """A box of height A over w0 samples on a zero background: mean = A w0/n,
    var = A^2 w0/n (1 - w0/n); a window of width w <= w0 inside the box scores
    sqrt(w) (A - mean)/std, a window w > w0 holding the whole box scores
    (A w0 - w mean)/(std sqrt(w)) and first occurs at t = max(0, t0+w0-w).
    The matched width w = w0 scores highest."""
    x = np.zeros((1, n))
    x[0, t0:t0 + w0] = amp
    nlev = 7
    mean, std, snr, tpk = oracle_lib.detect(x, nlev, integer)
    mu = amp * w0 / n
    sd = math.sqrt(amp * amp * w0 / n * (1.0 - w0 / n))
    assert mean[0] == pytest.approx(mu, rel=1e-14)
    assert std[0] == pytest.approx(sd, rel=1e-12)
    for lev in range(nlev):
        w = 1 << lev
        if w <= w0:
            assert tpk[0, lev] == t0
            assert snr[0, lev] == pytest.approx(math.sqrt(w) * (amp - mu) / sd, rel=1e-12)
        else:
            assert tpk[0, lev] == max(0, t0 + w0 - w)
            assert snr[0, lev] == pytest.approx((amp * w0 - w * mu) / (sd * math.sqrt(w)),
                                                rel=1e-12)
    assert int(np.argmax(snr[0])) == int(math.log2(w0))


def test_statistics_match_numpy_and_peaks_match_a_cumsum_search(oracle_lib):
    rng = np.random.default_rng(11)
    x = rng.integers(0, 3000, size=(5, 1000)).astype(np.float64)
    x[2, 400:404] += 5000.0
    mean, std, snr, tpk = oracle_lib.detect(x, 9, True)
    assert np.allclose(mean, x.mean(axis=1), rtol=1e-14, atol=0)
    assert np.allclose(std, x.std(axis=1), rtol=1e-10, atol=0)
    ci = np.concatenate([np.zeros((5, 1), np.int64), np.cumsum(x.astype(np.int64), axis=1)], 1)
    for lev in range(9):
        w = 1 << lev
        box = ci[:, w:] - ci[:, :-w]
        assert np.array_equal(tpk[:, lev], np.argmax(box, axis=1))
        # the reported S/N grows with the boxcar sum at that peak
        assert np.all(np.isfinite(snr[:, lev]))
    assert tpk[2, 2] == 400


def test_integer_and_float_modes_agree_on_integers(oracle_lib):
    rng = np.random.default_rng(12)
    x = rng.integers(0, 1 << 20, size=(3, 700)).astype(np.float64)
    a = oracle_lib.detect(x, 8, True)
    b = oracle_lib.detect(x, 8, False)
    assert np.array_equal(a[3], b[3])
    for u, v in zip(a[:3], b[:3]):
        assert np.allclose(u, v, rtol=1e-12, atol=0)


def test_degenerate_rows(oracle_lib):
    x = np.full((2, 5), 7.0)
    x[1] = 0.0
    mean, std, snr, tpk = oracle_lib.detect(x, 4, True)
    assert list(mean) == [7.0, 0.0] and list(std) == [0.0, 0.0]
    assert np.all(snr[:, :3] == 0.0) and np.all(tpk[:, :3] == 0)   # std 0: S/N 0, first t
    assert np.all(snr[:, 3] == -np.inf) and np.all(tpk[:, 3] == -1)  # width 8 > 5 samples
    with pytest.raises(ValueError):
        oracle_lib.detect(np.array([[0.5, 1.0]]), 1, True)


def test_fig3_pulse_at_dm50_is_found_at_its_dm_width_and_time(oracle_lib):
    """Fig. 3: simulated filterbank data with a square pulse at DM 50; the
    search over trial DMs recovers it.  Here 256 channels at 1.2-1.5 GHz,
    DMs 0..99.5 in steps of 0.5, a 16-sample pulse of +12 counts over N(128,16)
    noise.  The best S/N over every DM and width is at DM 50, width 16, t0."""
    nchan, fch1, foff, tsamp = 256, 1500.0, -300.0 / 256, 64e-6
    table = oracle_lib.dmshift(nchan, fch1, foff, tsamp)
    dms = (np.arange(200) * 0.5).astype(np.float32)
    nsamp_out = 4096
    S = oracle_lib.maxshift(table, dms)
    p = fb.Pulse(50.0, 1500, 16, 12.0)
    delays = np.array([oracle_lib.shift(p.dm, table[c]) for c in range(nchan)])
    data = fb.filterbank(nchan, nsamp_out + S, 31, [p], [delays])
    plane = oracle_lib.dedisperse(data, table, dms, nsamp_out)
    mean, std, snr, tpk = oracle_lib.detect(plane, 6, True)
    d, lev = np.unravel_index(np.argmax(snr), snr.shape)
    assert dms[d] == np.float32(50.0) and lev == 4 and tpk[d, lev] == p.t
    # Expected S/N: the pulse adds h = 256 x 12 counts to 16 samples of the row.
    # The row's variance is the channel noise (256 x 16^2) plus the pulse's own
    # share h^2 w0/n (1 - w0/n); the boxcar holds w0 h above a mean w0 h/n.
    h, w0, n = nchan * p.amp, 16, nsamp_out
    sd = math.sqrt(nchan * 16.0 ** 2 + h * h * w0 / n * (1 - w0 / n))
    expect = w0 * h * (1 - w0 / n) / (sd * math.sqrt(w0))
    assert 0.9 * expect < snr[d, lev] < 1.1 * expect
    assert abs(std[d] - sd) < 0.05 * sd
