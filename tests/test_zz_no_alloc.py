"""dd_execute_noalloc, the entry point for callers that cannot allocate device
memory (allocator callbacks, real-time threads, hosts that keep device memory
to themselves).  It must give the same planes as dd_execute, call after call:
its fixed device array keeps the previous call's contents, so the second call
checks that nothing stale leaks into a result.

This file is collected last on purpose; it also passes when run alone in a
fresh process.
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


def _plane(plan, fn, x, pitch, nin, nsamp_out, code):
    out = torch.full((plan.ndm, (nsamp_out + 3) // 4 * 4), -3.0, dtype=torch.float32,
                     device="cuda")
    s = torch.cuda.current_stream()
    fn(x.data_ptr(), code, pitch, nin, out.data_ptr(), out.stride(0), nsamp_out, s.cuda_stream)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:, nsamp_out:] == -3.0)
    return got[:, :nsamp_out]


@pytest.mark.parametrize("kind", ["u8", "f16-frac", "f32-frac"])
def test_noalloc_matches_execute_twice(dd, kind):
    rng = np.random.default_rng(404)
    code = {"u8": 0, "f16-frac": 1, "f32-frac": 2}[kind]
    elem = (1, 2, 4)[code]
    for call, (nchan, ndm, nsamp_out) in enumerate([(96, 48, 5000), (130, 70, 3333)]):
        dms = rng.uniform(0.0, 60.0, size=ndm).astype(np.float32)
        plan = dd.Plan(nchan, 1400.0, -1.0, 1e-4, dms)
        nin = nsamp_out + plan.maxshift
        step = 16 // elem
        pitch = (nin + step - 1) // step * step
        data = fb.random_filterbank(rng, nchan, nin, kind, pitch=pitch)
        x = torch.from_numpy(data).cuda()
        want = _plane(plan, plan.execute_ptr, x, pitch, nin, nsamp_out, code)
        got = _plane(plan, plan.execute_noalloc_ptr, x, pitch, nin, nsamp_out, code)
        if kind == "u8":
            assert np.array_equal(got, want), f"call {call}"
        else:
            # both paths run the same kernels; allow the library's FP tolerance anyway
            asum = np.abs(want).astype(np.float64)
            assert np.all(np.abs(got.astype(np.float64) - want) <= 1e-6 * asum), f"call {call}"


def test_noalloc_takes_large_inputs_and_rejects_tables_beyond_its_array(dd, oracle_lib):
    # The input size is not limited: 1024 channels x 40000 samples of uint8.
    rng = np.random.default_rng(405)
    dms = np.arange(16, dtype=np.float32)
    plan = dd.Plan(1024, 1500.0, -0.29296875, 64e-6, dms)
    nin = 40000
    data = fb.random_filterbank(rng, 1024, nin, "u8", pitch=nin)
    x = torch.from_numpy(data).cuda()
    nsamp_out = nin - plan.maxshift
    got = _plane(plan, plan.execute_noalloc_ptr, x, nin, nin, nsamp_out, 0)
    table = oracle_lib.dmshift(1024, 1500.0, -0.29296875, 64e-6)
    d = rng.integers(0, 16, size=64)
    t = rng.integers(0, nsamp_out, size=64)
    want, _ = oracle_lib.dedisperse_cells(data, table, dms, d, t)
    assert np.array_equal(got[d, t].astype(np.float64), want)
    # 140000 DMs: 2 x 4 x 140096 bytes of DM tables exceed the fixed 1 MiB.
    big = dd.Plan(16, 1500.0, -1.0, 64e-6, np.linspace(0.0, 1.0, 140000, dtype=np.float32))
    x = torch.zeros((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((140000, 512), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError) as e:
        big.execute_noalloc_ptr(x.data_ptr(), 0, 1024, 1024, out.data_ptr(), 512, 512)
    assert e.value.status == -1 and "fixed" in str(e.value)
