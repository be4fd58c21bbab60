"""GPU parity of the polyphase channeliser (dd_channelise) against the FP64
oracle.

FP32 output: every element within the stated bound
    |gpu - oracle| <= (T + 6 log2 M + 8) * 2^-23 * sum_m |h[m]| (|re| + |im|)
of the window's magnitudes (the FIR's T roundings, the FFT's log2 M stages
with their twiddle roundings, and margin).
int8 output: the oracle's FP64 value times scale decides the code; where it
lies farther than that bound from a rounding boundary the GPU code must be
equal, elsewhere either neighbouring code is accepted (and such cells must be
rare).
"""
import math

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


def _volts(seed, nsub, nraw, sigma=20.0):
    rng = np.random.default_rng(seed)
    return np.clip(np.rint(rng.normal(0.0, sigma, size=(nsub, nraw, 4))), -128, 127).astype(np.int8)


def _gamma(M, T):
    return (T + 6 * math.log2(M) + 8) * 2.0 ** -23


def _magnitude(v, h, M, T, spectra):
    """sum_m |h[m]| (|re| + |im|) per listed spectrum and polarisation: [n][2]."""
    ah = np.abs(np.asarray(h, np.float64))
    out = np.empty((len(spectra), 2))
    for i, (s, n) in enumerate(spectra):
        w = np.abs(v[s, n * M:n * M + M * T].astype(np.float64))
        out[i, 0] = (ah * (w[:, 0] + w[:, 1])).sum()
        out[i, 1] = (ah * (w[:, 2] + w[:, 3])).sum()
    return out


def _all_spectra(nsub, nspec):
    return [(s, n) for s in range(nsub) for n in range(nspec)]


def _gather(out, M, spectra):
    """GPU output [nsub*M][cols][4] -> [len(spectra)][M][4] in the oracle's order."""
    return np.stack([out[s * M:(s + 1) * M, n] for s, n in spectra])


def _check_cf32(got, want, mag, M, T):
    bound = _gamma(M, T) * mag                               # [n][2]
    b = np.repeat(bound[:, None, :], 2, axis=2)              # [n][1][4] per component
    err = np.abs(got.astype(np.float64) - want)
    assert np.all(err <= b), f"max err/bound {np.max(err / np.maximum(b, 1e-300)):.3g}"
    return float(np.max(err / np.maximum(b, 1e-300)))


def _check_ci8(got, want, mag, M, T, scale, oracle_lib):
    u = want * scale
    b = np.repeat((_gamma(M, T) * mag * scale)[:, None, :], 2, axis=2) + np.abs(u) * 2.0 ** -23
    frac = u - np.floor(u)
    tie = np.abs(frac - 0.5) <= b
    exact = oracle_lib.pfb_quantise(want, scale)
    g = got.astype(np.int64)
    lo = np.clip(np.floor(u), -127, 127)
    hi = np.clip(np.ceil(u), -127, 127)
    ok = np.where(tie, (g == lo) | (g == hi), g == exact)
    assert np.all(ok), f"{np.count_nonzero(~ok)} codes differ"
    # the undecided band is 2b wide per unit interval: its share of the cells
    # stays near 2 * mean(b) (about 1e-3 here), far below 1 %
    assert tie.mean() < 0.01
    return int(tie.sum())


CASES = [  # (M, T, nsub, nraw): several CTAs and rounds, ragged spectra and raw tails
    (16, 8, 3, 16 * 9100 + 5),
    (16, 16, 2, 16 * 5000 + 15),
    (16, 1, 2, 16 * 700),
    (32, 3, 2, 32 * 2200 + 31),
    (64, 4, 3, 64 * 900 + 1),
    (64, 2, 1, 64 * 1300),
    (128, 8, 2, 128 * 600 + 100),
    (256, 8, 2, 256 * 300 + 7),
    (256, 16, 1, 256 * 200),
    (256, 5, 2, 256 * 270),
]


@pytest.mark.parametrize("M,T,nsub,nraw", CASES)
def test_cf32_within_bound_and_ci8_codes(dd, oracle_lib, M, T, nsub, nraw):
    v = _volts(1000 + M + T, nsub, nraw)
    h = oracle_lib.pfb_prototype(M, T).astype(np.float32)
    nspec = oracle_lib.pfb_nspec(nraw, M, T)
    dev = torch.device("cuda:0")
    vt = torch.from_numpy(v).to(dev)
    ht = torch.from_numpy(h).to(dev)
    spectra = _all_spectra(nsub, nspec)
    want = oracle_lib.pfb(v, M, T, h.astype(np.float64), spectra=spectra, threads=True)
    mag = _magnitude(v, h, M, T, spectra)
    out = dd.channelise(vt, M, T, ht, kind="cf32")
    torch.cuda.synchronize()
    _check_cf32(_gather(out.cpu().numpy(), M, spectra), want, mag, M, T)
    # scale: about 12 codes of standard deviation per component
    scale = 12.0 / (20.0 * math.sqrt(float((h.astype(np.float64) ** 2).sum())))
    q = dd.channelise(vt, M, T, ht, kind="ci8", scale=scale)
    torch.cuda.synchronize()
    _check_ci8(_gather(q.cpu().numpy(), M, spectra), want, mag, M, T, scale, oracle_lib)


def test_random_filter_and_extreme_voltages(dd, oracle_lib):
    """A non-symmetric filter and full-scale voltages (every byte value)."""
    M, T, nsub = 64, 4, 2
    rng = np.random.default_rng(9)
    v = rng.integers(-128, 128, size=(nsub, 64 * 400 + 9, 4)).astype(np.int8)
    v[0, :64 * T] = -128
    h = rng.normal(size=M * T).astype(np.float32)
    nspec = oracle_lib.pfb_nspec(v.shape[1], M, T)
    spectra = _all_spectra(nsub, nspec)
    want = oracle_lib.pfb(v, M, T, h.astype(np.float64), spectra=spectra, threads=True)
    mag = _magnitude(v, h, M, T, spectra)
    dev = torch.device("cuda:0")
    out = dd.channelise(torch.from_numpy(v).to(dev), M, T, torch.from_numpy(h).to(dev),
                        kind="cf32")
    torch.cuda.synchronize()
    _check_cf32(_gather(out.cpu().numpy(), M, spectra), want, mag, M, T)


def test_clipped_codes_and_bin_centred_tone(dd, oracle_lib):
    """A bin-centred tone in X saturates its channel's codes at +-127 and
    lands in channel (M/4 + M/2) mod M of its subband only."""
    M, T = 32, 8
    nraw = 32 * 300
    j = np.arange(nraw)
    v = np.zeros((2, nraw, 4), np.int8)
    v[1, :, 0] = np.round(100 * np.cos(np.pi * j / 2)).astype(np.int8)
    v[1, :, 1] = np.round(100 * np.sin(np.pi * j / 2)).astype(np.int8)
    h = oracle_lib.pfb_prototype(M, T).astype(np.float32)
    dev = torch.device("cuda:0")
    q = dd.channelise(torch.from_numpy(v).to(dev), M, T, torch.from_numpy(h).to(dev),
                      kind="ci8", scale=1.0).cpu().numpy()
    nspec = oracle_lib.pfb_nspec(nraw, M, T)
    c = (M // 4 + M // 2) % M
    assert np.all(q[M + c, :nspec, 0] == 127) and np.all(q[M + c, :nspec, 1] == 0)
    others = np.delete(np.arange(2 * M), M + c)
    assert np.max(np.abs(q[others, :nspec].astype(int))) < 127


def test_short_rows_and_untouched_columns(dd, oracle_lib):
    M, T = 16, 8
    dev = torch.device("cuda:0")
    h = torch.from_numpy(oracle_lib.pfb_prototype(M, T).astype(np.float32)).to(dev)
    # fewer than M*T raw samples: no spectra, nothing written
    v = torch.zeros((2, M * T - 1, 4), dtype=torch.int8, device=dev)
    out = torch.full((2 * M, 4, 4), 77, dtype=torch.int8, device=dev)
    dd.channelise(v, M, T, h, kind="ci8", out=out)
    torch.cuda.synchronize()
    assert bool((out == 77).all())
    # exactly one spectrum; columns past it keep their guard value
    vn = _volts(3, 2, M * T)
    out = torch.full((2 * M, 8, 4), -99.0, dtype=torch.float32, device=dev)
    dd.channelise(torch.from_numpy(vn).to(dev), M, T, h, kind="cf32", out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:, 1:] == -99.0)
    want = oracle_lib.pfb(vn, M, T, h.cpu().numpy().astype(np.float64))
    mag = _magnitude(vn, h.cpu().numpy(), M, T, [(0, 0), (1, 0)])
    _check_cf32(np.stack([got[:M, 0], got[M:, 0]]), np.stack([want[:M, 0], want[M:, 0]]),
                mag, M, T)


def test_int8_rows_not_16_byte_aligned(dd, oracle_lib):
    """A row pitch that is a multiple of 4 but not of 16 bytes takes the
    element-by-element store path; codes equal the 16-byte path's and the
    padding column stays untouched."""
    M, T, nsub = 32, 4, 2
    v = _volts(21, nsub, 32 * 1301 + 3)
    nspec = oracle_lib.pfb_nspec(v.shape[1], M, T)
    assert (nspec + 1) * 4 % 16 != 0
    dev = torch.device("cuda:0")
    vt = torch.from_numpy(v).to(dev)
    h = torch.from_numpy(oracle_lib.pfb_prototype(M, T).astype(np.float32)).to(dev)
    ref = dd.channelise(vt, M, T, h, kind="ci8", scale=0.05)
    odd = torch.full((nsub * M, nspec + 1, 4), 55, dtype=torch.int8, device=dev)
    dd.channelise(vt, M, T, h, kind="ci8", scale=0.05, out=odd)
    torch.cuda.synchronize()
    assert torch.equal(odd[:, :nspec], ref[:, :nspec])
    assert bool((odd[:, nspec] == 55).all())


def test_invalid_arguments_are_rejected(dd):
    dev = torch.device("cuda:0")
    v = torch.zeros((1, 1024, 4), dtype=torch.int8, device=dev)
    h = torch.ones(16 * 4, dtype=torch.float32, device=dev)
    for M, T in [(8, 4), (48, 4), (512, 4), (16, 0), (16, 17)]:
        with pytest.raises(dd.DDError):
            dd.channelise(v, M, T, torch.ones(max(1, M * max(T, 1)), device=dev), kind="ci8")
    for scale in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(dd.DDError):
            dd.channelise(v, 16, 4, h, kind="ci8", scale=scale)


def test_full_size_sampled_spectra(dd, oracle_lib):
    """The benchmark workload: 64 subbands x 16 channels, 8 taps, 2,362,048
    spectra per subband (the front end's L-band input); spectra sampled at
    random and at CTA, round and row ends are checked against the oracle."""
    w = fb.CHANNELISER_LBAND
    dev = torch.device("cuda:0")
    pool = fb.VoltagePool(w.seed)
    vt = pool.long_rows_torch(w.nsub, w.nraw, dev)
    h = oracle_lib.pfb_prototype(w.M, w.T).astype(np.float32)
    q = dd.channelise(vt, w.M, w.T, torch.from_numpy(h).to(dev), kind="ci8", scale=w.scale)
    torch.cuda.synchronize()
    nspec = oracle_lib.pfb_nspec(w.nraw, w.M, w.T)
    rng = np.random.default_rng(17)
    picks = [(int(rng.integers(0, w.nsub)), int(rng.integers(0, nspec))) for _ in range(200)]
    per_cta = 16 * 8 * 32
    for s in (0, w.nsub - 1):
        picks += [(s, n) for n in (0, 1, 127, 128, per_cta - 1, per_cta, nspec - 2, nspec - 1)]
    wins = np.stack([vt[s, n * w.M:(n + w.T) * w.M].cpu().numpy() for s, n in picks])
    want = oracle_lib.pfb(wins, w.M, w.T, h.astype(np.float64),
                          spectra=[(i, 0) for i in range(len(picks))], threads=True)
    mag = _magnitude(wins, h, w.M, w.T, [(i, 0) for i in range(len(picks))])
    qh = torch.stack([q[s * w.M:(s + 1) * w.M, n] for s, n in picks]).cpu().numpy()
    _check_ci8(qh, want, mag, w.M, w.T, w.scale, oracle_lib)
