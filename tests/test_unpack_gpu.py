"""Corner turn and bit unpacking (dd_unpack) against the oracle, bit-exact:
every sample width, the 16-byte and byte load paths, ragged channel and time
edges, an unaligned input pointer, and a full-size L-band block."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _run(dd, raw, nbits, nchan, nsamp, offset=0, pitch_extra=16):
    pitch = (nsamp + pitch_extra + 15) // 16 * 16
    buf = torch.zeros(raw.size + offset + 16, dtype=torch.uint8, device="cuda")
    buf[offset:offset + raw.size] = torch.from_numpy(raw).cuda()
    src = buf[offset:offset + raw.size]
    out = torch.full((nchan, pitch), 0xA7, dtype=torch.uint8, device="cuda")
    dd.unpack(src, nbits, nchan, nsamp, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:, nsamp:] == 0xA7)   # columns past nsamp untouched
    return got[:, :nsamp]


@pytest.mark.parametrize("nbits", [1, 2, 4, 8])
@pytest.mark.parametrize("nchan,nsamp", [(128, 1000), (256, 129), (1024, 4096), (136, 333),
                                         (8, 5), (24, 130), (384, 1), (512, 3 * 256 + 17),
                                         (128, 256), (256, 16 * 40 + 9), (1024, 70000)])
def test_unpack_matches_oracle(dd, oracle_lib, nbits, nchan, nsamp):
    if (nchan * nbits) % 8:
        pytest.skip("spectra must be whole bytes")
    rng = np.random.default_rng(nchan * 10 + nbits)
    raw = rng.integers(0, 256, size=nsamp * nchan * nbits // 8, dtype=np.uint8)
    want = oracle_lib.unpack(raw, nbits, nchan, nsamp)
    assert np.array_equal(_run(dd, raw, nbits, nchan, nsamp), want)


@pytest.mark.parametrize("nbits", [2, 8])
def test_unaligned_input_takes_the_byte_path(dd, oracle_lib, nbits):
    rng = np.random.default_rng(77)
    nchan, nsamp = 256, 700
    raw = rng.integers(0, 256, size=nsamp * nchan * nbits // 8, dtype=np.uint8)
    want = oracle_lib.unpack(raw, nbits, nchan, nsamp)
    for off in (1, 3, 8):
        assert np.array_equal(_run(dd, raw, nbits, nchan, nsamp, offset=off), want)


@pytest.mark.parametrize("nbits", [8, 4, 2, 1])
def test_full_size_lband_block(dd, oracle_lib, nbits):
    """1024 channels x 147628 spectra (the L-band beam's input length)."""
    rng = np.random.default_rng(5 + nbits)
    nchan, nsamp = 1024, 147628
    raw = rng.integers(0, 256, size=nsamp * nchan * nbits // 8, dtype=np.uint8)
    want = oracle_lib.unpack(raw, nbits, nchan, nsamp)
    assert np.array_equal(_run(dd, raw, nbits, nchan, nsamp), want)


def test_unpacked_rows_feed_the_dedispersion(dd, oracle_lib):
    """Spectra -> dd_unpack -> dd_execute equals the oracle on the same spectra."""
    rng = np.random.default_rng(3)
    nchan, ndm = 64, 40
    table = oracle_lib.dmshift(nchan, 1500.0, -1.0, 64e-6)
    dms = np.linspace(0.0, 60.0, ndm).astype(np.float32)
    S = oracle_lib.maxshift(table, dms)
    nsamp_out = 3000
    nin = nsamp_out + S
    raw = rng.integers(0, 256, size=nin * nchan // 2, dtype=np.uint8)   # 4-bit spectra
    rows = oracle_lib.unpack(raw, 4, nchan, nin)
    want = oracle_lib.dedisperse(rows, table, dms, nsamp_out)
    pitch = (nin + 15) // 16 * 16
    x = torch.empty((nchan, pitch), dtype=torch.uint8, device="cuda")
    dd.unpack(torch.from_numpy(raw).cuda(), 4, nchan, nin, x)
    plan = dd.Plan(nchan, 1500.0, -1.0, 64e-6, dms)
    out = torch.empty((ndm, (nsamp_out + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    plan.execute(x, out, nsamp_in=nin, nsamp_out=nsamp_out)
    plan.sync()
    assert np.array_equal(out.cpu().numpy()[:, :nsamp_out], want)
