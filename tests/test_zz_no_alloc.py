"""dd_execute_noalloc, the entry point for callers that cannot allocate device
memory (allocator callbacks, real-time threads, hosts that keep device memory
to themselves).  Its planes must equal the CPU oracle's, call after call: its
fixed device array keeps the previous call's contents, so consecutive calls
with plans of different sizes (small then large, and large then small) check
that nothing stale leaks into a result.  The array's status word must read
clear after each good call and report a bounded wait that ran out.

This file is collected last on purpose; it also passes when run alone in a
fresh process.
"""
import numpy as np
import pytest

import filterbank as fb

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # relative to sum |in| along the curve, as for dd_execute


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _plane(plan, x, pitch, nin, nsamp_out, code):
    out = torch.full((plan.ndm, (nsamp_out + 3) // 4 * 4), -3.0, dtype=torch.float32,
                     device="cuda")
    s = torch.cuda.current_stream()
    plan.execute_noalloc_ptr(x.data_ptr(), code, pitch, nin, out.data_ptr(), out.stride(0),
                             nsamp_out, s.cuda_stream)
    plan.sync_noalloc(s.cuda_stream)   # raises on a recorded device failure
    got = out.cpu().numpy()
    assert np.all(got[:, nsamp_out:] == -3.0)
    return got[:, :nsamp_out]


SHAPES = [(96, 48, 5000), (130, 70, 3333), (300, 140, 4000)]


@pytest.mark.parametrize("order", ["growing", "shrinking"])
@pytest.mark.parametrize("kind", ["u8", "f16-frac", "f32-frac"])
def test_noalloc_matches_the_oracle_call_after_call(dd, oracle_lib, kind, order):
    rng = np.random.default_rng(404 if order == "growing" else 405)
    code = {"u8": 0, "f16-frac": 1, "f32-frac": 2}[kind]
    elem = (1, 2, 4)[code]
    shapes = SHAPES if order == "growing" else SHAPES[::-1]
    for call, (nchan, ndm, nsamp_out) in enumerate(shapes):
        band = (1400.0, -1.0, 1e-4)
        dms = rng.uniform(0.0, 60.0, size=ndm).astype(np.float32)
        plan = dd.Plan(nchan, *band, dms)
        nin = nsamp_out + plan.maxshift
        step = 16 // elem
        pitch = (nin + step - 1) // step * step
        data = fb.random_filterbank(rng, nchan, nin, kind, pitch=pitch)
        x = torch.from_numpy(data).cuda()
        got = _plane(plan, x, pitch, nin, nsamp_out, code)
        table = oracle_lib.dmshift(nchan, *band)
        rows = np.ascontiguousarray(data[:, :nin])
        if kind == "u8":
            want = oracle_lib.dedisperse(rows, table, dms, nsamp_out, threads=True)
            assert np.array_equal(got, want), f"call {call}"
        else:
            want, asum = oracle_lib.dedisperse(rows, table, dms, nsamp_out, with_abssum=True,
                                               threads=True)
            err = np.abs(got.astype(np.float64) - want)
            assert np.all(err <= TOL * asum), f"call {call}"


def test_noalloc_takes_large_inputs_and_rejects_tables_beyond_its_array(dd, oracle_lib):
    # The input size is not limited: 1024 channels x 40000 samples of uint8.
    rng = np.random.default_rng(405)
    dms = np.arange(16, dtype=np.float32)
    plan = dd.Plan(1024, 1500.0, -0.29296875, 64e-6, dms)
    nin = 40000
    data = fb.random_filterbank(rng, 1024, nin, "u8", pitch=nin)
    x = torch.from_numpy(data).cuda()
    nsamp_out = nin - plan.maxshift
    got = _plane(plan, x, nin, nin, nsamp_out, 0)
    table = oracle_lib.dmshift(1024, 1500.0, -0.29296875, 64e-6)
    want = oracle_lib.dedisperse(data, table, dms, nsamp_out, threads=True)
    assert np.array_equal(got, want)
    # 140000 DMs: 2 x 4 x 140096 bytes of DM tables exceed the fixed 1 MiB.
    big = dd.Plan(16, 1500.0, -1.0, 64e-6, np.linspace(0.0, 1.0, 140000, dtype=np.float32))
    x = torch.zeros((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((140000, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError) as e:
        big.execute_noalloc_ptr(x.data_ptr(), 0, 1024, 1024, out.data_ptr(), 512, 512)
    assert e.value.status == -1 and "fixed" in str(e.value)


def test_noalloc_status_word_reports_a_wait_that_ran_out(dd):
    """A bounded wait that records into the fixed array's status word (a short
    limit on an mbarrier nothing arrives on; no fault) is reported by
    dd_sync_noalloc as DD_ERR_TIMEOUT, once; the word is clear afterwards and
    the next no-alloc call runs normally."""
    s = torch.cuda.current_stream().cuda_stream
    dd.Plan.sync_noalloc(s)                               # clear to start with
    dd.check(dd.lib.dd_selftest_noalloc_timeout(20_000_000, s))
    with pytest.raises(dd.DDError) as e:
        dd.Plan.sync_noalloc(s)
    assert e.value.status == dd._binding.DD_ERR_TIMEOUT
    dd.Plan.sync_noalloc(s)                               # reported once, then clear
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, [0.0, 2.0])
    x = torch.ones((16, 1024), dtype=torch.uint8, device="cuda")
    got = _plane(plan, x, 1024, 1024, 512, 0)
    assert np.all(got == 16.0)


def test_noalloc_refuses_a_capturing_stream(dd):
    """The table copies come from per-call pageable host memory, so a stream
    under capture is turned away with DD_ERR_INVALID before anything is
    enqueued, and the caller's capture stays valid."""
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, [0.0, 2.0])
    x = torch.ones((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 512), dtype=torch.float32, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g, stream=side):
        try:
            plan.execute_noalloc_ptr(x.data_ptr(), 0, 1024, 1024, out.data_ptr(), 512, 512,
                                     side.cuda_stream)
        except dd.DDError as e:
            refused = e
        out.add_(1.0)                                      # the capture is still usable
    assert refused is not None and refused.status == -1
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(out == 1.0)
