"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

uint8: bit-exact.  FP16/FP32: the same integer-valued noise is exact too (FP32
sums of integers below 2^24); unquantised ("-frac") data must satisfy
|gpu - oracle64| <= 1e-6 * sum_c |in[c][t+s(c,d)]| in every checked cell.
"""
import numpy as np
import pytest

import filterbank as fb
from tests.cases import lband_input_and_plane, sample_cells, workload_input

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative to sum |in| along the curve


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _out(ndm, nsamp_out, pad_rows=0, pad_cols=0, fill=np.nan):
    pitch = (nsamp_out + pad_cols + 3) // 4 * 4
    return torch.full((ndm + pad_rows, pitch), fill, dtype=torch.float32, device="cuda")


def _run(dd, plan, data, nsamp_in, nsamp_out, pad_rows=0, pad_cols=4):
    x = _dev(data)
    if data.dtype == np.float16:
        x = x.view(torch.float16)
    out = _out(plan.ndm, nsamp_out, pad_rows, pad_cols, fill=-7.0)
    plan.execute(x, out[:plan.ndm], nsamp_in=nsamp_in, nsamp_out=nsamp_out)
    plan.sync(torch.cuda.current_stream())
    got = out.cpu().numpy()
    # nothing written outside the plane
    assert np.all(got[:, nsamp_out:] == -7.0)
    assert np.all(got[plan.ndm:] == -7.0)
    return got[:plan.ndm, :nsamp_out]


def _check_float(got, want, asum):
    err = np.abs(got.astype(np.float64) - want)
    bound = TOL * asum
    assert np.all(err <= bound), float(np.max(err / np.maximum(asum, 1e-30)))


def _random_case(rng, nchan, ndm, nsamp_out, kind, dm_hi=80.0, sorted_dms=False):
    fch1 = float(rng.uniform(300.0, 1500.0))
    foff = -float(rng.uniform(0.05, min(2.0, 0.8 * fch1 / nchan)))
    tsamp = float(rng.uniform(6.4e-5, 5e-4))
    import oracle
    table = oracle.dmshift(nchan, fch1, foff, tsamp)
    dms = rng.uniform(0.0, dm_hi, size=ndm).astype(np.float32)
    if sorted_dms:
        dms.sort()
    S = oracle.maxshift(table, dms)
    nin = nsamp_out + S + int(rng.integers(0, 40))
    elem = {"u8": 1, "f16": 2, "f32": 4, "f16-frac": 2, "f32-frac": 4}[kind]
    step = 16 // elem
    pitch = (nin + step - 1) // step * step + step * int(rng.integers(0, 3))
    data = fb.random_filterbank(rng, nchan, nin, kind, pitch=pitch)
    return (fch1, foff, tsamp), table, dms, nin, data


# ---------------------------------------------------------------------------

def test_small_workload_bit_exact(dd, oracle_lib):
    w = fb.SMALL
    table, dms, S, data = workload_input(w)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    got = _run(dd, plan, data, w.nsamp_out + S, w.nsamp_out)
    want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :w.nsamp_out + S]), table, dms,
                                 w.nsamp_out)
    assert np.array_equal(got, want)


TILES_U8 = [(4, 12, 1, 8), (4, 4, 2, 8), (2, 3, 1, 4), (1, 1, 1, 16), (4, 5, 2, 4),
            (4, 10, 2, 8, 4), (2, 12, 2, 8, 4), (1, 24, 1, 4, 4), (2, 8, 1, 32, 4),
            (1, 12, 1, 48, 4), (4, 6, 1, 4), (2, 16, 1, 8), (1, 16, 1, 4), (4, 13, 1, 8)]


def _case_that_fits(dd, rng, nchan, ndm, nsamp_out, kind, tiles, dm_hi=80.0):
    """A random case whose shift spread fits the tile shape's shared memory:
    the DM range is halved until the plan accepts the shape."""
    for _ in range(10):
        band, table, dms, nin, data = _random_case(rng, nchan, ndm, nsamp_out, kind, dm_hi=dm_hi)
        plan = dd.Plan(nchan, *band, dms)
        try:
            plan.set_tiles(kind[:3] if kind != "u8" else "u8", *tiles)
            return plan, table, dms, nin, data
        except dd.DDError:
            dm_hi /= 2.0
    raise AssertionError(f"tile shape {tiles} fits no DM range")


@pytest.mark.parametrize("tiles", TILES_U8)
@pytest.mark.parametrize("seed", [0, 1])
def test_u8_fuzz_bit_exact(dd, oracle_lib, tiles, seed):
    """Ragged nchan/ndm/nsamp (not multiples of any tile), unsorted non-integer
    DMs, padded pitches, several tile shapes: every cell bit-exact."""
    rng = np.random.default_rng(1000 * seed + sum(tiles))
    nchan = int(rng.integers(3, 300))
    ndm = int(rng.integers(1, 150))
    nsamp_out = int(rng.integers(1, 5000))
    plan, table, dms, nin, data = _case_that_fits(dd, rng, nchan, ndm, nsamp_out, "u8", tiles)
    assert plan.get_tiles("u8")[:len(tiles)] == tuple(tiles)
    got = _run(dd, plan, data, nin, nsamp_out)
    want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, nsamp_out)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ndm,nsamp_out,launches", [
    (152, 40960, 2), (3 * 48 + 24, 40960, 2),      # remainder <= 24 DMs, split pays
    (152, 9000, 1),                                 # one round either way: padded launch
    (3 * 48 + 25, 40960, 1), (144, 40960, 1), (40, 40960, 1)])
@pytest.mark.parametrize("kind", ["u8", "f16-frac"])
def test_remainder_dms_launch(dd, oracle_lib, ndm, nsamp_out, launches, kind):
    """With 48 DMs per tile on 152 SMs, a remainder of at most 24 DMs runs as a
    second launch of its own tile shape when that takes fewer tile rounds than
    padding (two launches); a larger remainder, none, fewer DMs than one tile,
    or no round to gain keep one padded launch.  Either way every cell is
    bit-exact (uint8) or within the bound (FP16)."""
    rng = np.random.default_rng(ndm + nsamp_out)
    nchan = 200
    band = (1500.0, -1.5, 64e-6)          # 300 MHz below 1.5 GHz, as the L-band beam
    table = oracle_lib.dmshift(nchan, *band)
    dms = rng.permutation(np.arange(ndm, dtype=np.float32) * np.float32(0.9))
    nin = nsamp_out + oracle_lib.maxshift(table, dms) + 5
    data = fb.random_filterbank(rng, nchan, nin, kind, pitch=(nin + 15) // 16 * 16)
    plan = dd.Plan(nchan, *band, dms)
    plan.set_tiles(kind[:3] if kind != "u8" else "u8", 4, 12, 1, 8)
    n0 = dd.launch_count()
    got = _run(dd, plan, data, nin, nsamp_out)
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        assert dd.launch_count() - n0 == launches
    if kind == "u8":
        want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, nsamp_out,
                                     threads=True)
        assert np.array_equal(got, want)
    else:
        want, asum = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms,
                                           nsamp_out, with_abssum=True, threads=True)
        _check_float(got, want, asum)


@pytest.mark.parametrize("kind", ["f32", "f16", "f32-frac", "f16-frac"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_float_fuzz(dd, oracle_lib, kind, seed):
    rng = np.random.default_rng(77 + seed)
    nchan = int(rng.integers(3, 400))
    ndm = int(rng.integers(1, 80))
    nsamp_out = int(rng.integers(1, 3000))
    band, table, dms, nin, data = _random_case(rng, nchan, ndm, nsamp_out, kind)
    plan = dd.Plan(nchan, *band, dms)
    if seed == 2:
        plan.set_tiles(kind[:3], 1, 3, 2, 4)
    got = _run(dd, plan, data, nin, nsamp_out)
    want, asum = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms,
                                       nsamp_out, with_abssum=True)
    if kind.endswith("frac"):
        _check_float(got, want, asum)
    else:
        assert np.array_equal(got.astype(np.float64), want)


@pytest.mark.parametrize("kind", ["f32-frac", "f16-frac"])
@pytest.mark.parametrize("tiles", [(4, 13, 1, 8), (4, 12, 1, 8), (2, 16, 1, 8),
                                   (4, 12, 1, 12), (4, 10, 1, 24)])
def test_float_fuzz_wide_tiles(dd, oracle_lib, kind, tiles):
    """The widest CTAs of 4 and 2 DMs per thread (16 warps with the producer
    and the phase builders), and the stage sizes with a compile-time
    instantiation (12 channels for FP16, 24 for FP32): ragged sizes, every
    cell within the bound."""
    rng = np.random.default_rng(500 + sum(tiles) + len(kind))
    nchan = int(rng.integers(3, 300))
    ndm = int(rng.integers(60, 150))
    nsamp_out = int(rng.integers(1, 5000))
    plan, table, dms, nin, data = _case_that_fits(dd, rng, nchan, ndm, nsamp_out, kind, tiles)
    got = _run(dd, plan, data, nin, nsamp_out)
    want, asum = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms,
                                       nsamp_out, with_abssum=True)
    _check_float(got, want, asum)


def test_extreme_values_u8_4096_channels(dd, oracle_lib):
    """All-255 input over 4096 channels: the largest sums (1,044,480) are exact,
    including across the 256-channel SWAR widening."""
    nchan, ndm, nsamp_out = 4096, 8, 2048
    dms = np.linspace(0, 5, ndm).astype(np.float32)
    plan = dd.Plan(nchan, 150.0, -0.00732421875, 327.68e-6, dms)
    nin = nsamp_out + plan.maxshift
    data = np.full((nchan, (nin + 15) // 16 * 16), 255, dtype=np.uint8)
    got = _run(dd, plan, data, nin, nsamp_out)
    assert np.all(got == 4096 * 255)


def test_degenerate_shapes(dd, oracle_lib):
    rng = np.random.default_rng(5)
    # one channel, one DM, one output sample; all DMs zero; DM list with repeats
    for nchan, dms, nsamp_out in [(1, [0.0], 1), (1, [7.5], 33), (5, [0.0, 0.0, 0.0], 100),
                                  (7, [3.0, 1.0, 3.0, 1.0, 2.0], 257), (64, [500.0], 64)]:
        dms = np.array(dms, np.float32)
        plan = dd.Plan(nchan, 1400.0, -1.5, 1e-4, dms)
        nin = nsamp_out + plan.maxshift
        data = fb.random_filterbank(rng, nchan, nin, "u8", pitch=(nin + 15) // 16 * 16)
        got = _run(dd, plan, data, nin, nsamp_out)
        table = oracle_lib.dmshift(nchan, 1400.0, -1.5, 1e-4)
        want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, nsamp_out)
        assert np.array_equal(got, want)


def test_zero_samples_is_a_no_op(dd):
    plan = dd.Plan(8, 1400.0, -1.0, 1e-4, [0.0, 1.0])
    out = torch.full((2, 16), 3.0, device="cuda")
    x = torch.zeros((8, 64), dtype=torch.uint8, device="cuda")
    plan.execute(x, out, nsamp_out=0)
    plan.sync()
    assert torch.all(out == 3.0)


def test_execute_host_matches_device_path(dd, oracle_lib):
    """The host-buffer form (blocked, overlap tails copied on the device) gives
    the same plane as the device form, on pinned and pageable buffers."""
    w = fb.SMALL
    rng = np.random.default_rng(8)
    dms = np.arange(0, 300, dtype=np.float32)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    nsamp_out = 150_000  # several 65536-sample blocks and a ragged last block
    nin = nsamp_out + plan.maxshift
    data = fb.random_filterbank(rng, w.nchan, nin, "u8")
    dev = _run(dd, plan, np.pad(data, ((0, 0), (0, (-nin) % 16))), nin, nsamp_out)
    out = np.full((len(dms), nsamp_out), -1.0, np.float32)
    plan.execute_host(data, out)
    assert np.array_equal(out, dev)
    pinned_in = torch.from_numpy(data).pin_memory()
    pinned_out = torch.empty((len(dms), nsamp_out), dtype=torch.float32).pin_memory()
    plan.execute_host(pinned_in, pinned_out)
    assert np.array_equal(pinned_out.numpy(), dev)
    d_idx, t_idx = sample_cells(rng, len(dms), nsamp_out, 500)
    table = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    want, _ = oracle_lib.dedisperse_cells(data, table, dms, d_idx, t_idx)
    assert np.array_equal(out[d_idx, t_idx].astype(np.float64), want)


def test_execute_host_with_tails_longer_than_a_block(dd, oracle_lib):
    """Host-buffer blocks are uneven (short first and last blocks); here maxshift
    (about 32400 samples) exceeds the 12500-sample edge blocks, so every overlap
    tail spans more than one block of input."""
    rng = np.random.default_rng(9)
    nchan = 64
    dms = np.linspace(0.0, 2000.0, 40).astype(np.float32)
    plan = dd.Plan(nchan, 1500.0, -300.0 / nchan, 64e-6, dms)
    assert plan.maxshift > 30000
    nsamp_out = 100_000
    nin = nsamp_out + plan.maxshift
    data = fb.random_filterbank(rng, nchan, nin, "u8")
    dev = _run(dd, plan, np.pad(data, ((0, 0), (0, (-nin) % 16))), nin, nsamp_out)
    out = np.full((len(dms), nsamp_out), -1.0, np.float32)
    plan.execute_host(data, out)
    assert np.array_equal(out, dev)
    table = oracle_lib.dmshift(nchan, 1500.0, -300.0 / nchan, 64e-6)
    d_idx, t_idx = sample_cells(rng, len(dms), nsamp_out, 300)
    want, _ = oracle_lib.dedisperse_cells(data, table, dms, d_idx, t_idx)
    assert np.array_equal(out[d_idx, t_idx].astype(np.float64), want)


def test_lband_full_size_whole_plane(dd, oracle_lib):
    """The 1024-channel L-band beam at full size (1024 DMs x 131072 samples),
    default tiles (the benchmarked launch): every cell of the plane
    bit-exact against the oracle (its OpenMP build, the same sums), the DM-0
    row equal to the plain channel sum, and each injected pulse recovered at
    its DM."""
    w = fb.LBAND
    table, dms, S, data, want = lband_input_and_plane(oracle_lib)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    got = _run(dd, plan, data, w.nsamp_out + S, w.nsamp_out)
    bad = np.argwhere(got != want)
    assert len(bad) == 0, f"{len(bad)} cells differ, first {bad[:4].tolist()}"
    chan_sum = data[:, :w.nsamp_out].sum(axis=0, dtype=np.int64)
    assert np.array_equal(got[0], chan_sum.astype(np.float32))
    for p in fb.all_pulses(w):
        d = int(np.where(dms == np.float32(p.dm))[0][0])
        win = got[d, p.t:p.t + p.width]
        assert win.mean() > got[d].mean() + 0.8 * w.nchan * p.amp


_LOWFREQ_CACHE = {}


def _lowfreq_input(kind):
    if "u8" not in _LOWFREQ_CACHE:
        _LOWFREQ_CACHE.clear()
        _LOWFREQ_CACHE["u8"] = workload_input(fb.LOWFREQ, "u8")
    table, dms, S, data = _LOWFREQ_CACHE["u8"]
    if kind == "u8":
        return table, dms, S, data
    return table, dms, S, data.astype(np.float16 if kind == "f16" else np.float32)


# Every second DM row of the low-frequency beam, compared at full length: half
# the plane (1000 rows x 262144 samples, 1.1e12 oracle adds on the host
# cores), both ends of the DM range included.
LOWFREQ_HALF = np.unique(np.append(np.arange(0, fb.LOWFREQ.ndm, 2), fb.LOWFREQ.ndm - 1))


def _lowfreq_oracle_rows(oracle_lib):
    """The oracle's rows LOWFREQ_HALF of the low-frequency beam's plane
    (uint8 noise), computed once per session."""
    if "plane" not in _LOWFREQ_CACHE:
        w = fb.LOWFREQ
        table, dms, S, data = _lowfreq_input("u8")
        _LOWFREQ_CACHE["plane"] = oracle_lib.dedisperse(
            np.ascontiguousarray(data[:, :w.nsamp_out + S]), table, dms[LOWFREQ_HALF],
            w.nsamp_out, threads=True)
    return _LOWFREQ_CACHE["plane"]


# Tile shapes of the 4096-channel beam: the ones the bench's autotuner picks
# (the benchmarked launch; for uint8 also the plan's default) and, for
# FP16/FP32, the plan's default (None).
LOWFREQ_TILES = {"u8": [(4, 12, 1, 8, 8)],
                 "f16": [(4, 12, 1, 12, 8), None],
                 "f32": [(4, 6, 2, 24, 8), None]}


def _lowfreq_plan(dd, dms, dtype, tiles):
    w = fb.LOWFREQ
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, dms)
    if tiles is not None:
        plan.set_tiles(dtype, *tiles)
    return plan


@pytest.mark.parametrize("kind,tiles", [(k, t) for k, ts in LOWFREQ_TILES.items() for t in ts])
def test_lowfreq_full_size_half_plane(dd, oracle_lib, kind, tiles):
    """The 4096-channel low-frequency beam at full size (2000 DMs x 262144
    samples) in each storage type, in the benchmarked launch (and the default
    tile shape): the same integer-valued noise, so every cell of every second
    DM row must equal the oracle's exactly (for FP16/FP32 input the oracle's
    FP64 sums of integers are the same numbers as its uint8 sums)."""
    w = fb.LOWFREQ
    table, dms, S, data = _lowfreq_input(kind)
    plan = _lowfreq_plan(dd, dms, kind, tiles)
    got = _run(dd, plan, data, w.nsamp_out + S, w.nsamp_out)[LOWFREQ_HALF]
    want = _lowfreq_oracle_rows(oracle_lib)
    bad = np.argwhere(got != want)
    assert len(bad) == 0, f"{len(bad)} cells differ, first {bad[:4].tolist()}"
    for p in fb.all_pulses(w):
        d = int(np.argmin(np.abs(dms[LOWFREQ_HALF] - np.float32(p.dm))))
        assert got[d, p.t:p.t + p.width].mean() > got[d].mean() + 0.8 * w.nchan * p.amp


# DM rows checked at full length for the non-integer variants: 64 rows spread
# over the 2000 DMs, both ends included.
LOWFREQ_ROWS = np.unique(np.linspace(0, fb.LOWFREQ.ndm - 1, 64).round().astype(int))


@pytest.mark.parametrize("kind", ["f16-frac", "f32-frac"])
def test_lowfreq_noninteger_full_length_rows(dd, oracle_lib, kind):
    """Unquantised noise on the 4096-channel band at full size (2000 DMs x
    262144 samples), in the benchmarked launch and the default tile shape: 64
    DM rows spread over the DM range, every sample of each, within 1e-6 of
    sum |in| along its curve against the FP64 oracle."""
    w = fb.LOWFREQ
    table, dms, S, data = workload_input(w, kind)
    sel = dms[LOWFREQ_ROWS]
    Ssel = oracle_lib.maxshift(table, sel)
    want, asum = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :w.nsamp_out + Ssel]),
                                       table, sel, w.nsamp_out, with_abssum=True, threads=True)
    for tiles in LOWFREQ_TILES[kind[:3]]:
        plan = _lowfreq_plan(dd, dms, kind[:3], tiles)
        got = _run(dd, plan, data, w.nsamp_out + S, w.nsamp_out)
        _check_float(got[LOWFREQ_ROWS], want, asum)


def test_launch_count_and_status(dd):
    n0 = dd.launch_count()
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, [0.0, 2.0])
    x = torch.zeros((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((2, 512), device="cuda")
    plan.execute(x, out)
    plan.sync()
    assert dd.launch_count() == n0 + 1  # one de-dispersion kernel per execution


def test_autotuner_picks_a_shape_that_stays_bit_exact(dd, oracle_lib):
    rng = np.random.default_rng(31)
    band, table, dms, nin, data = _random_case(rng, 200, 70, 3000, "u8", sorted_dms=True)
    plan = dd.Plan(200, *band, dms)
    x = _dev(data)
    out = torch.empty((70, 3000), dtype=torch.float32, device="cuda")
    res = plan.autotune(x, out, nsamp_in=nin, reps=1)
    timed = [r for r in res if r[1] >= 0]
    assert len(timed) >= 3
    best = min(timed, key=lambda r: r[1])[0]
    assert plan.get_tiles("u8") == best
    got = _run(dd, plan, data, nin, 3000)
    want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, dms, 3000)
    assert np.array_equal(got, want)


def test_bounded_wait_runs_out_and_reports_without_fault(dd):
    """A wait on an mbarrier nothing arrives on gives up after its limit and
    reports DD_ERR_TIMEOUT; the context stays usable afterwards."""
    import time
    t = time.perf_counter()
    st = dd.lib.dd_selftest_wait_timeout(50_000_000, None)   # 50 ms
    assert st == dd.DD_ERR_TIMEOUT if hasattr(dd, "DD_ERR_TIMEOUT") else st == -5
    assert time.perf_counter() - t < 5.0
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, [0.0, 2.0])
    x = torch.ones((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((2, 512), device="cuda")
    plan.execute(x, out)
    plan.sync()
    assert torch.all(out == 16.0)
