"""Pins of the oracle's front end (Stokes I, integration, RFI excision by
iterated sigma clipping, quantisation to uint8), without a GPU.

Stokes I and the integration are recomputed with numpy complex arithmetic and
reshapes; the quantiser is checked through closed forms (two-valued channels,
constant channels), its monotonicity in the integrated power, the clipping of
an injected spike, a two-pass clipping case in closed form, and the
N(128, 16) statistics of Gaussian voltages with and without seeded RFI.
"""
import math

import numpy as np
import pytest

import filterbank as fb


def _power(volts, nint):
    """numpy Stokes I: |X|^2 + |Y|^2 from complex voltages, summed over nint."""
    v = volts.astype(np.int64)
    x = v[..., 0] + 1j * v[..., 1]
    y = v[..., 2] + 1j * v[..., 3]
    i = (np.abs(x) ** 2 + np.abs(y) ** 2).round().astype(np.int64)
    n = volts.shape[1] // nint
    return i[:, :n * nint].reshape(volts.shape[0], n, nint).sum(axis=2)


def test_hand_worked_channel(oracle_lib):
    v = np.zeros((1, 4, 4), np.int8)
    v[0, 0] = [3, 4, -1, 2]      # |3+4i|^2 + |-1+2i|^2 = 25 + 5 = 30
    v[0, 1] = [1, 1, 1, 1]       # 4
    v[0, 3] = [2, 0, 0, 0]       # 4
    out, mean, std = oracle_lib.frontend(v, 1, 100.0)
    assert mean[0] == 9.5 and std[0] == pytest.approx(math.sqrt(142.75), rel=1e-15)
    # 128 + 16 (P - 9.5)/11.948: 30 -> 155.45, 4 -> 120.63, 0 -> 115.28
    assert out.tolist() == [[155, 121, 115, 121]]


@pytest.mark.parametrize("nint", [1, 3, 8])
def test_power_and_statistics_match_numpy(oracle_lib, nint):
    rng = np.random.default_rng(nint)
    volts = rng.integers(-128, 128, size=(5, 403, 4), dtype=np.int8)
    out, mean, std = oracle_lib.frontend(volts, nint, 1e9)
    p = _power(volts, nint)
    assert out.shape == p.shape
    assert np.allclose(mean, p.mean(axis=1), rtol=1e-14, atol=0)
    assert np.allclose(std, p.std(axis=1), rtol=1e-10, atol=0)
    for c in range(5):   # codes never decrease as the power grows
        order = np.argsort(p[c], kind="stable")
        assert np.all(np.diff(out[c][order].astype(int)) >= 0)


def test_two_valued_and_constant_channels(oracle_lib):
    # channel 0 alternates P = 4 and P = 16: mean 10, std 6; mean +- std -> 112 / 144
    v = np.zeros((2, 6, 4), np.int8)
    v[0, 0::2] = [2, 0, 0, 0]
    v[0, 1::2] = [4, 0, 0, 0]
    v[1, :] = [5, 5, 5, 5]   # constant: std 0 -> every code 128
    out, mean, std = oracle_lib.frontend(v, 1, 100.0)
    assert (mean[0], std[0]) == (10.0, 6.0)
    assert out[0].tolist() == [112, 144] * 3
    assert std[1] == 0.0 and np.all(out[1] == 128)


def test_spike_above_threshold_is_replaced_by_the_mean(oracle_lib):
    rng = np.random.default_rng(7)
    volts = rng.normal(0.0, 10.0, size=(2, 4000, 4)).round().clip(-128, 127).astype(np.int8)
    volts[0, 1234] = [127, 127, 127, 127]   # 4 x 127^2 = 64516 >> mean + 4 std
    out, mean, std = oracle_lib.frontend(volts, 1, 4.0)
    assert out[0, 1234] == 128
    p = _power(volts, 1)
    kept = p[0] <= math.floor(mean[0] + 4.0 * std[0])
    assert not kept[1234] and kept.sum() > 3990
    # without clipping the spike saturates the code
    out2, _, _ = oracle_lib.frontend(volts, 1, 1e9)
    assert out2[0, 1234] == 255


def test_gaussian_voltages_quantise_to_128_16(oracle_lib):
    """Integrated power of many Gaussian samples is near Gaussian, so the
    codes come out with mean about 128 and standard deviation about 16."""
    rng = np.random.default_rng(11)
    volts = rng.normal(0.0, 20.0, size=(3, 64000, 4)).round().clip(-128, 127).astype(np.int8)
    out, _, _ = oracle_lib.frontend(volts, 16, 1e9)
    codes = out.astype(np.float64)
    assert np.all(np.abs(codes.mean(axis=1) - 128.0) < 0.6)
    assert np.all(np.abs(codes.std(axis=1) - 16.0) < 0.6)


def test_trailing_raw_samples_are_dropped(oracle_lib):
    rng = np.random.default_rng(3)
    volts = rng.integers(-50, 50, size=(2, 103, 4), dtype=np.int8)
    out_a, mean_a, _ = oracle_lib.frontend(volts, 10, 1e9)
    out_b, mean_b, _ = oracle_lib.frontend(volts[:, :100], 10, 1e9)
    assert out_a.shape == (2, 10) and np.array_equal(out_a, out_b)
    assert np.array_equal(mean_a, mean_b)


def test_second_clipping_pass_recovers_the_clean_statistics(oracle_lib):
    """1000 samples alternating P = 4 / 16 and 10 outliers at P = 9800.  Pass
    one: mean 106.93, std 969.3, threshold floor(mean + 4 std) = 3984, so the
    outliers leave the kept set; pass two over the 1000 clean samples gives
    mean 10 and std 6 exactly, codes 112 / 144, and the outliers become 128.
    Further passes change nothing (the kept set is a fixed point)."""
    v = np.zeros((1, 1010, 4), np.int8)
    v[0, 0:1000:2] = [2, 0, 0, 0]
    v[0, 1:1000:2] = [4, 0, 0, 0]
    v[0, 1000:] = [70, 70, 0, 0]
    out1, mean1, std1 = oracle_lib.frontend(v, 1, 4.0, niter=1)
    assert mean1[0] == pytest.approx(108000 / 1010, rel=1e-15)
    p2 = (500 * 16 + 500 * 256 + 10 * 9800 ** 2) / 1010
    assert std1[0] == pytest.approx(math.sqrt(p2 - (108000 / 1010) ** 2), rel=1e-12)
    # one pass: the threshold (3984) already excises the outliers, but the
    # clean samples are scaled by the inflated std: 128 + 16 (P - 106.93) / 969.3
    # is 126.30 for P = 4 and 126.50 (just below) for P = 16
    assert np.all(out1[0, 1000:] == 128) and np.all(out1[0, :1000] == 126)
    for niter in (2, 3, 6):
        out, mean, std = oracle_lib.frontend(v, 1, 4.0, niter=niter)
        assert (mean[0], std[0]) == (10.0, 6.0)
        assert out[0, :1000].tolist() == [112, 144] * 500
        assert np.all(out[0, 1000:] == 128)


def test_iterated_clipping_restores_the_noise_scale(oracle_lib):
    """The seeded RFI layout: broadband impulses inflate one-pass std in every
    channel, so the noise codes lose most of their spread; three passes excise
    every impulse and tone (code 128 wherever they cover a whole output
    sample) and the noise codes come back to a standard deviation near 16."""
    vp = fb.VoltagePool(21, size=1 << 20)
    lay = vp.layout(128, 64000)
    volts = vp.rows(lay)
    mask = np.ones(64000 // 16, bool)
    for r0, r1 in lay.impulses:
        mask[r0 // 16:r1 // 16 + 1] = False
    tone_chans = {c for c, _, _ in lay.tones}
    clean = [c for c in range(128) if c not in tone_chans]
    out1, _, _ = oracle_lib.frontend(volts, 16, 4.0, niter=1)
    assert out1[clean][:, mask].astype(float).std(axis=1).min() < 4.0
    out, _, _ = oracle_lib.frontend(volts, 16, 4.0, niter=3)
    for r0, r1 in lay.impulses:
        assert np.all(out[:, r0 // 16 + 1:r1 // 16] == 128)
    for c, r0, r1 in lay.tones:
        assert np.all(out[c, r0 // 16 + 1:r1 // 16] == 128)
    sd = out[clean][:, mask].astype(float).std(axis=1)
    assert np.all(np.abs(sd - 16.0) < 0.5)
