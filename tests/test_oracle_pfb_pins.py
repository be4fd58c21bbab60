"""Pins of the oracle's polyphase channeliser, without a GPU.

The channeliser is the critically sampled polyphase filter bank (a window of
M*T samples weighted by a prototype filter, then an M-point DFT).  Its
oracle is pinned by what the mathematics fixes: with one tap and a flat
window it is numpy's FFT of each block; an impulse reproduces the prototype
with the DFT phase; a bin-centred tone lands in its channel with gain sum(h);
the output is linear and shifts by one spectrum when the input shifts by M
samples; real input gives conjugate-symmetric bins.  The prototype is
scipy's windowed-sinc design, and the quantiser is checked on hand-worked
values.
"""
import numpy as np
import pytest


def _volts(rng, nsub, nraw, lo=-60, hi=61):
    return rng.integers(lo, hi, size=(nsub, nraw, 4)).astype(np.int8)


def _complex(v, pol):
    return v[..., 2 * pol].astype(np.float64) + 1j * v[..., 2 * pol + 1].astype(np.float64)


@pytest.mark.parametrize("M,T", [(16, 4), (64, 8), (256, 16), (32, 3)])
def test_prototype_is_scipy_windowed_sinc(oracle_lib, M, T):
    signal = pytest.importorskip("scipy.signal")
    h = oracle_lib.pfb_prototype(M, T)
    # firwin's cutoff is relative to Nyquist: 1/M puts the edge at half a channel;
    # without scaling it returns cutoff * sinc(cutoff * m) * window.
    want = M * signal.firwin(M * T, 1.0 / M, window="hamming", scale=False)
    assert np.allclose(h, want, rtol=1e-12, atol=1e-15)
    assert np.allclose(h, h[::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("M", [16, 32, 64, 256])
def test_one_tap_flat_window_is_the_fft_of_each_block(oracle_lib, M):
    rng = np.random.default_rng(M)
    nraw = 5 * M + 7                         # 5 spectra, 7 trailing samples dropped
    v = _volts(rng, 2, nraw)
    y = oracle_lib.pfb(v, M, 1, np.ones(M))
    assert y.shape == (2 * M, 5, 4)
    for s in range(2):
        for pol in range(2):
            x = _complex(v[s], pol)[:5 * M].reshape(5, M)
            want = np.fft.fftshift(np.fft.fft(x, axis=1), axes=1)   # bin M/2 first
            got = y[s * M:(s + 1) * M, :, 2 * pol] + 1j * y[s * M:(s + 1) * M, :, 2 * pol + 1]
            scale = np.abs(x).sum()
            assert np.max(np.abs(got.T - want)) <= 1e-13 * scale


@pytest.mark.parametrize("M,T", [(16, 4), (32, 3), (64, 8)])
def test_impulse_reproduces_the_prototype_with_the_dft_phase(oracle_lib, M, T):
    rng = np.random.default_rng(M + T)
    h = rng.normal(size=M * T)               # any filter: no symmetry to hide an index error
    nraw = (T + 6) * M
    j0 = 3 * M + 5
    v = np.zeros((1, nraw, 4), np.int8)
    v[0, j0] = (3, 0, 0, -2)                 # X = 3, Y = -2i
    y = oracle_lib.pfb(v, M, T, h)
    nspec = nraw // M - T + 1
    assert y.shape == (M, nspec, 4)
    for n in range(nspec):
        m = j0 - n * M
        for k in range(M):
            c = (k + M // 2) % M
            if 0 <= m < M * T:
                ph = np.exp(-2j * np.pi * ((k * m) % M) / M)
                wx, wy = 3 * h[m] * ph, -2j * h[m] * ph
            else:
                wx = wy = 0.0
            got_x = y[c, n, 0] + 1j * y[c, n, 1]
            got_y = y[c, n, 2] + 1j * y[c, n, 3]
            assert abs(got_x - wx) <= 1e-13 and abs(got_y - wy) <= 1e-13, (n, k)


@pytest.mark.parametrize("M,T", [(16, 8), (64, 4)])
def test_bin_centred_tones_land_in_their_channels(oracle_lib, M, T):
    """X carries exp(+i pi j / 2) (bin M/4) and Y exp(-i pi j / 2) (bin 3M/4):
    integer voltages 1, i, -1, -i.  Their bins receive A * sum(h) exactly (up
    to rounding); bins two or more channels away lie in the stopband."""
    h = oracle_lib.pfb_prototype(M, T)
    nraw = (T + 4) * M
    j = np.arange(nraw)
    a = 40
    v = np.zeros((1, nraw, 4), np.int8)
    v[0, :, 0] = np.round(a * np.cos(np.pi * j / 2)).astype(np.int8)
    v[0, :, 1] = np.round(a * np.sin(np.pi * j / 2)).astype(np.int8)
    v[0, :, 2] = v[0, :, 0]
    v[0, :, 3] = -v[0, :, 1]
    y = oracle_lib.pfb(v, M, T, h)
    X = y[:, :, 0] + 1j * y[:, :, 1]
    Y = y[:, :, 2] + 1j * y[:, :, 3]
    cx, cy = (M // 4 + M // 2) % M, (3 * M // 4 + M // 2) % M
    assert np.allclose(X[cx], a * h.sum(), rtol=1e-12, atol=0)
    assert np.allclose(Y[cy], a * h.sum(), rtol=1e-12, atol=0)
    far_x = np.abs(np.arange(M) - cx) >= 2
    far_y = np.abs(np.arange(M) - cy) >= 2
    assert np.max(np.abs(X[far_x])) < 1e-2 * a * h.sum()
    assert np.max(np.abs(Y[far_y])) < 1e-2 * a * h.sum()


def test_linear_and_shift_equivariant(oracle_lib):
    M, T = 32, 4
    rng = np.random.default_rng(11)
    h = oracle_lib.pfb_prototype(M, T)
    v1 = _volts(rng, 2, 12 * M, -30, 31)
    v2 = _volts(rng, 2, 12 * M, -30, 31)
    y1, y2 = oracle_lib.pfb(v1, M, T, h), oracle_lib.pfb(v2, M, T, h)
    y12 = oracle_lib.pfb((2 * v1.astype(np.int16) - v2).astype(np.int8), M, T, h)
    assert np.allclose(y12, 2 * y1 - y2, rtol=0, atol=1e-10)
    # dropping the first M raw samples drops the first spectrum, bit for bit
    ys = oracle_lib.pfb(np.ascontiguousarray(v1[:, M:]), M, T, h)
    assert np.array_equal(ys, y1[:, 1:])
    # the listed-spectra form gives the same bits as the full form
    cells = oracle_lib.pfb(v1, M, T, h, spectra=[(1, 3), (0, 0)])
    assert np.array_equal(cells[0], y1[M:2 * M, 3])
    assert np.array_equal(cells[1], y1[:M, 0])


def test_real_input_gives_conjugate_symmetric_bins(oracle_lib):
    M, T = 64, 4
    rng = np.random.default_rng(5)
    v = _volts(rng, 1, 10 * M)
    v[..., 1] = 0
    v[..., 3] = 0
    y = oracle_lib.pfb(v, M, T, oracle_lib.pfb_prototype(M, T))
    X = y[:, :, 0] + 1j * y[:, :, 1]
    for k in range(1, M):
        c, cm = (k + M // 2) % M, (M - k + M // 2) % M
        assert np.allclose(X[c], np.conj(X[cm]), rtol=0, atol=1e-9)


def test_short_rows_give_no_spectra(oracle_lib):
    M, T = 16, 8
    v = np.zeros((3, M * T - 1, 4), np.int8)
    assert oracle_lib.pfb_nspec(M * T - 1, M, T) == 0
    assert oracle_lib.pfb(v, M, T, np.ones(M * T)).shape == (3 * M, 0, 4)
    assert oracle_lib.pfb_nspec(M * T, M, T) == 1
    assert oracle_lib.pfb_nspec(M * T + M - 1, M, T) == 1


def test_quantiser_hand_values(oracle_lib):
    v = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 126.4, 126.6, 300.0, -300.0, 0.26, -0.74])
    got = oracle_lib.pfb_quantise(v, 1.0)
    assert got.tolist() == [0, 2, 2, 0, -2, 126, 127, 127, -127, 0, -1]
    assert oracle_lib.pfb_quantise(np.array([0.25, 0.75, -3.0]), 2.0).tolist() == [0, 2, -6]


def test_threaded_build_gives_the_same_bits(oracle_lib):
    M, T = 32, 4
    rng = np.random.default_rng(2)
    v = _volts(rng, 3, 20 * M)
    h = oracle_lib.pfb_prototype(M, T)
    assert np.array_equal(oracle_lib.pfb(v, M, T, h), oracle_lib.pfb(v, M, T, h, threads=True))


def test_long_voltage_rows_are_seeded_pool_slices():
    """The channeliser workloads' rows (longer than the pools) are copies of
    seeded pool slices, chunk by chunk: the same seed gives the same bytes,
    every chunk is a contiguous slice of its row's pool, and the noise keeps
    that pool's spread."""
    torch = pytest.importorskip("torch")
    import filterbank as fb
    pool = fb.VoltagePool(5, size=1 << 16)
    a = pool.long_rows_torch(3, 100_003, "cpu", chunk=1 << 14).numpy()
    b = fb.VoltagePool(5, size=1 << 16).long_rows_torch(3, 100_003, "cpu", chunk=1 << 14).numpy()
    assert a.shape == (3, 100_003, 4) and np.array_equal(a, b)
    flat = [p.reshape(-1) for p in pool.pools]
    for r in range(3):
        chunk = a[r, 3 * (1 << 14):4 * (1 << 14)].reshape(-1)
        hits = [i for i, p in enumerate(flat)
                if any(np.array_equal(p[o:o + 64], chunk[:64])
                       for o in range(0, len(p) - chunk.size + 1, 4))]
        assert hits, r
        sd = a[r].astype(np.float64).std()
        assert min(abs(sd - s) for s in fb.VOLT_SIGMAS) < 0.05 * sd
    w = fb.CHANNELISER_LBAND
    assert w.nraw == (w.nspec + w.T - 1) * w.M and w.nsub * w.M == fb.LBAND.nchan
