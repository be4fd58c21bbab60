"""Pins of the CPU oracle against facts fixed outside it (no GPU).

Each test checks the oracle against something it does not compute itself:
closed forms of the dispersion law, the exact rational value of an FP32
product, a numpy restatement on tiny inputs, invariants of the shifted sum
(DM = 0, impulses, linearity, time-shift equivariance), the injected-pulse
experiment of Sec. 4 / Fig. 3, and numpy's own binary16 decoding.  A dropped
term, a wrong sign or index, a transposed operand or a rounding slip in the
oracle makes at least one of them fail.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import filterbank as fb

BANDS = [
    # (nchan, fch1 MHz, foff MHz, tsamp s) of the three single-beam workloads
    (64, 1500.0, -1.0, 64e-6),
    (1024, 1500.0, -0.29296875, 64e-6),
    (4096, 150.0, -0.00732421875, 327.68e-6),
]


def _freqs(nchan, fch1, foff):
    return np.array([fch1 + c * foff for c in range(nchan)], dtype=np.float64)


# --------------------------------------------------------------------------
# The dispersion law (Sec. 2): delay ~ DM * (f^-2 - f_top^-2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("band", BANDS)
def test_dmshift_matches_textbook_delay_in_ghz_ms(oracle_lib, band):
    """The cold-plasma delay in the usual astronomer's units is
    4.148808 ms * DM * (f_GHz^-2 - f_top,GHz^-2); the oracle's table, times
    tsamp, must give it to FP32 precision for every channel."""
    nchan, fch1, foff, tsamp = band
    table = oracle_lib.dmshift(nchan, fch1, foff, tsamp).astype(np.float64)
    f_ghz = _freqs(nchan, fch1, foff) / 1000.0
    ftop = f_ghz.max()
    delay_ms = 4.148808 * (f_ghz ** -2 - ftop ** -2)
    got_ms = table * tsamp * 1e3
    assert got_ms[np.argmax(f_ghz)] == 0.0
    np.testing.assert_allclose(got_ms, delay_ms, rtol=2e-7, atol=1e-12)


def test_dmshift_reference_delay_dm100_at_1400mhz(oracle_lib):
    """Textbook figure: a DM of 100 pc/cm^3 delays 1.4 GHz by 4.148808e3 * 100 /
    1400^2 s = 0.211674 s relative to infinite frequency.  A two-channel band
    with its top channel far above 1.4 GHz reproduces it to FP32 precision."""
    ftop = 1.0e7  # MHz; f_top^-2 = 1e-14, negligible
    table = oracle_lib.dmshift(2, ftop, 1400.0 - ftop, 1e-3)
    assert table[0] == 0.0
    delay_s = float(table[1]) * 1e-3 * 100.0
    assert abs(delay_s - 0.2116738775510204) < 2e-7 * 0.2117


@pytest.mark.parametrize("band", BANDS)
def test_dmshift_shape_invariants(oracle_lib, band):
    """Zero at the top channel, strictly increasing towards lower frequency, the
    ratio between channels independent of the constant, and exactly inverse in
    tsamp (up to one FP32 rounding)."""
    nchan, fch1, foff, tsamp = band
    t1 = oracle_lib.dmshift(nchan, fch1, foff, tsamp).astype(np.float64)
    t2 = oracle_lib.dmshift(nchan, fch1, foff, tsamp * 4.0).astype(np.float64)
    assert t1[0] == 0.0 and np.all(np.diff(t1) > 0)
    np.testing.assert_allclose(t2 * 4.0, t1, rtol=1.2e-7)
    f = _freqs(nchan, fch1, foff)
    ratio = (f[1:] ** -2 - f[0] ** -2) / (f[-1] ** -2 - f[0] ** -2)
    np.testing.assert_allclose(t1[1:] / t1[-1], ratio, rtol=3e-7)


def test_dmshift_ascending_band_uses_highest_channel(oracle_lib):
    """With foff > 0 channel 0 is the lowest frequency; the delay reference is
    the last channel and the table is the mirror image of the descending band."""
    down = oracle_lib.dmshift(64, 1500.0, -1.0, 64e-6)
    up = oracle_lib.dmshift(64, 1437.0, 1.0, 64e-6)
    assert np.array_equal(up[::-1], down)


def test_invalid_bands_are_rejected(oracle_lib):
    for args in [(0, 1500.0, -1.0, 64e-6), (8, 1500.0, 0.0, 64e-6), (8, 1500.0, -1.0, 0.0),
                 (8, 5.0, -1.0, 64e-6)]:
        with pytest.raises(ValueError):
            oracle_lib.dmshift(*args)


def test_maxshift_of_the_workloads(oracle_lib):
    """The workload statements give maxshift of about 16.6k samples for the
    L-band beam at DM 1023 and about 31.7k for the low-frequency beam at DM 100
    (DM grid up to 99.95), and 162 for the small 64-channel case."""
    for w, approx, tol in [(fb.SMALL, 162, 0), (fb.LBAND, 16600, 100), (fb.LOWFREQ, 31700, 200)]:
        table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
        S = oracle_lib.maxshift(table, w.dm_list())
        assert abs(S - approx) <= tol, (w.name, S)
    # maxshift is attained by the lowest channel at the largest DM
    table = oracle_lib.dmshift(fb.LBAND.nchan, fb.LBAND.fch1, fb.LBAND.foff, fb.LBAND.tsamp)
    assert oracle_lib.maxshift(table, fb.LBAND.dm_list()) == 16556


# --------------------------------------------------------------------------
# The integer shift rule: trunc(fp32(DM * dmshift))
# --------------------------------------------------------------------------

def test_shift_is_floor_of_exact_product_away_from_integers(oracle_lib):
    """For non-negative operands, trunc of the FP32-rounded product equals the
    floor of the exact rational product unless that product lies within one
    FP32 rounding step of an integer (where rounding may carry it across)."""
    w = fb.LBAND
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    rng = np.random.default_rng(11)
    dms = w.dm_list()
    checked = 0
    for _ in range(4000):
        d = int(rng.integers(0, len(dms)))
        c = int(rng.integers(0, len(table)))
        exact = Fraction(float(dms[d])) * Fraction(float(table[c]))
        fl = math.floor(exact)
        frac = exact - fl
        if frac < Fraction(1, 1 << 18) or 1 - frac < Fraction(1, 1 << 18):
            continue
        assert oracle_lib.shift(dms[d], table[c]) == fl
        checked += 1
    assert checked > 3000


def test_shift_rounds_the_product_before_truncating(oracle_lib):
    """0.1f * 10.0f rounds to exactly 1.0f in FP32 (the exact product is
    1.0000000149...), so the shift is 1 -- one FP32 multiply, not an FP64 one
    (which would also give 1) and not a fused form with a different rounding.
    And 3 * 0.99999994 = 2.99999982 truncates to 2, never rounds to 3."""
    assert oracle_lib.shift(np.float32(0.1), np.float32(10.0)) == 1
    assert oracle_lib.shift(np.float32(3.0), np.float32(0.99999994)) == 2
    assert oracle_lib.shift(np.float32(0.0), np.float32(316.42)) == 0
    # a product whose FP32 rounding crosses an integer: float32(0.04) * 25 is
    # 0.99999997765 exactly but rounds to 1.0f, so the shift is 1, not 0
    a = np.float32(0.04)
    assert Fraction(float(a)) * 25 < 1
    assert oracle_lib.shift(a, np.float32(25.0)) == 1
    assert oracle_lib.shift(np.float32(25.0), a) == 1


# --------------------------------------------------------------------------
# The shifted sum (Sec. 2: shift each channel, then integrate over frequency)
# --------------------------------------------------------------------------

def _tiny_case(rng, nchan, ndm, nsamp_out, kind="u8"):
    fch1 = float(rng.uniform(300.0, 1500.0))
    foff = -float(rng.uniform(0.5, 4.0))
    tsamp = float(rng.uniform(1e-4, 1e-3))
    table = None
    import oracle
    table = oracle.dmshift(nchan, fch1, foff, tsamp)
    dms = rng.uniform(0.0, 40.0, size=ndm).astype(np.float32)   # unsorted, non-integer
    dms[0] = 0.0
    S = oracle.maxshift(table, dms)
    data = fb.random_filterbank(rng, nchan, nsamp_out + S + int(rng.integers(0, 5)), kind)
    return data, table, dms


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_numpy_on_tiny_inputs(oracle_lib, seed):
    """A numpy restatement (its own FP32 products, its own loops) on tiny random
    shapes with unsorted, non-integer DM lists."""
    rng = np.random.default_rng(100 + seed)
    nchan, ndm, nsamp = int(rng.integers(1, 9)), int(rng.integers(1, 9)), int(rng.integers(1, 65))
    data, table, dms = _tiny_case(rng, nchan, ndm, nsamp)
    got = oracle_lib.dedisperse(data, table, dms, nsamp)
    prod = (dms[:, None] * table[None, :]).astype(np.float32)       # numpy FP32 multiply
    shifts = np.trunc(prod).astype(np.int64)
    want = np.zeros((ndm, nsamp), dtype=np.int64)
    for d in range(ndm):
        for c in range(nchan):
            want[d] += data[c, shifts[d, c]:shifts[d, c] + nsamp].astype(np.int64)
    assert np.array_equal(got, want.astype(np.float32))


def test_dm_zero_row_is_the_plain_channel_sum(oracle_lib):
    rng = np.random.default_rng(3)
    data, table, dms = _tiny_case(rng, 200, 5, 300)
    got = oracle_lib.dedisperse(data, table, dms, 300)
    assert np.array_equal(got[0], data[:, :300].sum(axis=0, dtype=np.int64).astype(np.float32))


def test_impulse_lands_on_its_dispersion_curve(oracle_lib):
    """An impulse at (c0, t0) contributes 1 exactly to out[d][t0 - s(c0,d)] and
    nowhere else, for every trial DM: the shift moves later samples of lower
    channels back to the top-of-band arrival time."""
    w = fb.SMALL
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms = w.dm_list()
    S = oracle_lib.maxshift(table, dms)
    nsamp = 400
    for c0, t0 in [(63, 300), (0, 10), (40, 200), (63, 162)]:
        data = np.zeros((w.nchan, nsamp + S), dtype=np.uint8)
        data[c0, t0] = 1
        out = oracle_lib.dedisperse(data, table, dms, nsamp)
        for d in range(len(dms)):
            s = oracle_lib.shift(dms[d], table[c0])
            row = np.zeros(nsamp, dtype=np.float32)
            if 0 <= t0 - s < nsamp:
                row[t0 - s] = 1.0
            assert np.array_equal(out[d], row), (c0, t0, d)
    # the lowest channel at the largest DM is delayed by maxshift
    assert oracle_lib.shift(dms[-1], table[-1]) == S


def test_linearity_and_time_shift_equivariance(oracle_lib):
    rng = np.random.default_rng(5)
    data, table, dms = _tiny_case(rng, 48, 12, 256)
    a = (data // 2).astype(np.uint8)
    b = (data - a).astype(np.uint8)
    full = oracle_lib.dedisperse(data, table, dms, 200)
    assert np.array_equal(full, oracle_lib.dedisperse(a, table, dms, 200) +
                          oracle_lib.dedisperse(b, table, dms, 200))
    tau = 37
    shifted = np.ascontiguousarray(data[:, tau:])
    assert np.array_equal(oracle_lib.dedisperse(shifted, table, dms, 200 - tau),
                          full[:, tau:])


def test_injected_pulse_is_recovered_at_its_dm(oracle_lib):
    """The Fig. 3 experiment on the small workload: a square pulse (+40 counts,
    4 samples) dispersed with DM 30 and arriving at t = 2000 at the top of the
    band.  Its boxcar-4 response peaks at the DM-30 row at t = 2000, the pulse
    adds exactly nchan * 40 to each of its 4 samples there, and the S/N gain over
    one channel is about sqrt(nchan)."""
    w = fb.SMALL
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms = w.dm_list()
    S = oracle_lib.maxshift(table, dms)
    nin = w.nsamp_out + S
    p = w.pulses[0]
    delays = np.array([oracle_lib.shift(p.dm, table[c]) for c in range(w.nchan)])
    data = fb.filterbank(w.nchan, nin, w.seed, [p], [delays])
    quiet = fb.filterbank(w.nchan, nin, w.seed)
    out = oracle_lib.dedisperse(data, table, dms, w.nsamp_out)
    base = oracle_lib.dedisperse(quiet, table, dms, w.nsamp_out)
    diff = out - base
    d30 = int(np.where(dms == np.float32(30.0))[0][0])
    assert np.array_equal(diff[d30, p.t:p.t + p.width], np.full(p.width, w.nchan * p.amp))
    box = np.stack([np.convolve(r, np.ones(p.width), mode="valid") for r in out])
    d_best, t_best = np.unravel_index(np.argmax(box), box.shape)
    assert (d_best, t_best) == (d30, p.t)
    noise = base[d30]
    snr = (out[d30, p.t] - noise.mean()) / noise.std()
    single = p.amp / 16.0
    assert 0.8 * single * math.sqrt(w.nchan) < snr < 1.25 * single * math.sqrt(w.nchan)


def test_float_paths_sum_in_fp64_exactly(oracle_lib):
    """FP32 and FP16 inputs are summed in FP64; for these magnitudes every FP64
    partial sum is exact, so each cell equals math.fsum of its curve, and the
    absolute-sum plane equals fsum of |in|."""
    rng = np.random.default_rng(9)
    for kind in ("f32", "f16", "f32-frac", "f16-frac"):
        data, table, dms = _tiny_case(rng, 64, 6, 100, kind)
        out, asum = oracle_lib.dedisperse(data, table, dms, 100, with_abssum=True)
        for d in range(len(dms)):
            s = [oracle_lib.shift(dms[d], table[c]) for c in range(64)]
            for t in (0, 13, 99):
                vals = [float(data[c, t + s[c]]) for c in range(64)]
                assert out[d, t] == math.fsum(vals)
                assert asum[d, t] == math.fsum(abs(v) for v in vals)


def test_half_decoding_matches_numpy_for_every_bit_pattern(oracle_lib):
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle_lib.half_to_double(int(b)) for b in bits])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])


def test_cells_and_checker_build_agree_with_the_plane(oracle_lib):
    rng = np.random.default_rng(21)
    for kind in ("u8", "f32", "f16"):
        data, table, dms = _tiny_case(rng, 37, 9, 123, kind)
        plane = oracle_lib.dedisperse(data, table, dms, 123)
        omp = oracle_lib.dedisperse(data, table, dms, 123, threads=True)
        assert np.array_equal(plane, omp)
        d_idx = rng.integers(0, 9, size=50)
        t_idx = rng.integers(0, 123, size=50)
        vals, _ = oracle_lib.dedisperse_cells(data, table, dms, d_idx, t_idx)
        assert np.array_equal(vals, plane[d_idx, t_idx].astype(np.float64))


def test_short_rows_are_rejected(oracle_lib):
    w = fb.SMALL
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms = w.dm_list()
    S = oracle_lib.maxshift(table, dms)
    with pytest.raises(ValueError):
        oracle_lib.dedisperse(np.zeros((w.nchan, 100 + S - 1), np.uint8), table, dms, 100)
