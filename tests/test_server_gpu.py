"""Serving runtime: streaming blocks of many beams with continuous batching.

Each block's outputs must equal the oracle's plane of the concatenated stream
at the block's stream samples (bit-exact for uint8), and a beam's results must
be the same served alone and served in a mix of other beams.
"""
import time

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


class Stream:
    """One beam's seeded input stream, served block by block."""

    def __init__(self, oracle_lib, seed, nchan, ndm, bw, B, nblocks):
        rng = np.random.default_rng(seed)
        self.nchan, self.B, self.nblocks = nchan, B, nblocks
        self.fch1, self.foff, self.tsamp = 1500.0, -bw / nchan, 64e-6
        self.dms = rng.uniform(0.0, float(rng.integers(20, 120)), size=ndm).astype(np.float32)
        self.table = oracle_lib.dmshift(nchan, self.fch1, self.foff, self.tsamp)
        self.S = oracle_lib.maxshift(self.table, self.dms)
        self.data = fb.NoisePool(seed, 1 << 22).rows(nchan, B * nblocks)
        self.outs = [np.full((ndm, B), -9.0, np.float32) for _ in range(nblocks)]
        self.got = {}

    def plan(self, dd):
        return dd.Plan(self.nchan, self.fch1, self.foff, self.tsamp, self.dms)

    def block(self, k):
        return np.ascontiguousarray(self.data[:, k * self.B:(k + 1) * self.B])

    def check(self, oracle_lib, cells=None, threads=False):
        total = self.B * self.nblocks - self.S
        if cells is None:
            want = oracle_lib.dedisperse(self.data, self.table, self.dms, total, threads=threads)
        for k in range(self.nblocks):
            first_t, n = self.got[k]
            assert first_t == (0 if k == 0 else k * self.B - self.S)
            assert n == (self.B - self.S if k == 0 else self.B)
            plane = self.outs[k][:, :n]
            assert np.all(self.outs[k][:, n:] == -9.0)
            if cells is None:
                assert np.array_equal(plane, want[:, first_t:first_t + n]), f"block {k}"
            else:
                rng = np.random.default_rng(k)
                d = rng.integers(0, len(self.dms), size=cells)
                t = rng.integers(0, n, size=cells)
                w, _ = oracle_lib.dedisperse_cells(self.data, self.table, self.dms, d, first_t + t)
                assert np.array_equal(plane[d, t].astype(np.float64), w), f"block {k}"


def _serve(dd, streams, budget=8 << 30, inflight=8, interleave=True, window_us=0):
    srv = dd.Server(budget, inflight, "u8")
    if window_us is not None:
        srv.set_batch_window(window_us)
    ids = [srv.add_beam(s.plan(dd), s.B) for s in streams]
    pending = {}
    order = [(i, k) for k in range(max(s.nblocks for s in streams)) for i in range(len(streams))
             if k < streams[i].nblocks] if interleave else \
        [(i, k) for i in range(len(streams)) for k in range(streams[i].nblocks)]
    busy = 0
    for i, k in order:
        while True:
            t = srv.submit(ids[i], streams[i].block(k), streams[i].outs[k])
            if t is not None:
                pending[t] = (i, k)
                break
            busy += 1
            time.sleep(0.001)
            for tt in list(pending):
                r = srv.poll(tt)
                if r is not None:
                    ii, kk = pending.pop(tt)
                    streams[ii].got[kk] = r
    srv.drain()
    for tt in list(pending):
        r = srv.poll(tt)
        assert r is not None
        ii, kk = pending.pop(tt)
        streams[ii].got[kk] = r
    stats = srv.stats()
    srv.close()
    return stats, busy


def test_streams_match_the_oracle_on_the_concatenated_stream(dd, oracle_lib):
    streams = [Stream(oracle_lib, 10 + i, nchan, ndm, bw, B, 5) for i, (nchan, ndm, bw, B) in
               enumerate([(64, 40, 64.0, 2048), (130, 72, 300.0, 3000), (256, 17, 64.0, 4096)])]
    stats, _ = _serve(dd, streams)
    for s in streams:
        s.check(oracle_lib)
    assert stats["completed"] == stats["submitted"] == 15
    assert stats["p50_ms"] > 0 and stats["p99_ms"] >= stats["p50_ms"]


def test_a_beam_served_alone_and_in_a_mix_gives_the_same_bytes(dd, oracle_lib):
    alone = Stream(oracle_lib, 99, 128, 64, 300.0, 3000, 4)
    _serve(dd, [alone])
    mixed = Stream(oracle_lib, 99, 128, 64, 300.0, 3000, 4)
    others = [Stream(oracle_lib, 200 + i, 96, 50, 64.0, 2500, 4) for i in range(5)]
    stats, _ = _serve(dd, [others[0], others[1], mixed, others[2], others[3], others[4]],
                      window_us=200_000)
    assert stats["mean_batch"] > 1.0   # blocks of different beams shared launches
    for k in range(4):
        assert alone.got[k] == mixed.got[k]
        assert np.array_equal(alone.outs[k], mixed.outs[k])
    alone.check(oracle_lib)


def test_full_queue_returns_busy_and_all_accepted_blocks_complete(dd, oracle_lib):
    streams = [Stream(oracle_lib, 30 + i, 64, 32, 64.0, 2048, 6) for i in range(4)]
    # one slot: two staging buffers, so a tight submit loop must see DD_ERR_BUSY
    stats, busy = _serve(dd, streams, budget=64 << 20, inflight=1, interleave=True)
    assert busy > 0 and stats["rejected_busy"] == busy
    assert stats["slots"] == 1
    for s in streams:
        s.check(oracle_lib)


def test_default_batch_window_and_copy_statistics(dd, oracle_lib):
    """Without an explicit window the server waits up to 1/64 of the shortest
    block duration for more ready blocks; its statistics count every block's
    staging, host-to-device and device-to-host bytes with positive times, and
    the results stay bit-exact."""
    streams = [Stream(oracle_lib, 40 + i, 64, 32, 64.0, 4096, 3) for i in range(3)]
    stats, _ = _serve(dd, streams, window_us=None)
    assert stats["batch_window_us"] == int(4096 * 64e-6 * 1e6 / 64)
    n = stats["completed"]
    assert n == 9 and stats["staging_bytes"] == n * 64 * 4096
    assert stats["h2d_bytes"] == stats["staging_bytes"]
    assert stats["d2h_bytes"] == sum(4 * 32 * (4096 - s.S if k == 0 else 4096)
                                     for s in streams for k in range(3))
    assert stats["staging_ms"] > 0 and stats["h2d_ms"] > 0 and stats["d2h_ms"] > 0
    for s in streams:
        s.check(oracle_lib)


def test_budget_below_one_slot_is_refused(dd):
    srv = dd.Server(1024, 4, "u8")
    plan = dd.Plan(64, 1500.0, -1.0, 64e-6, np.arange(16, dtype=np.float32))
    bid = srv.add_beam(plan, 1024)
    with pytest.raises(dd.DDError) as e:
        srv.submit(bid, np.zeros((64, 1024), np.uint8), np.zeros((16, 1024), np.float32))
    assert e.value.status == -3   # DD_ERR_NOMEM
    with pytest.raises(dd.DDError):
        srv.add_beam(plan, 8)      # block shorter than maxshift
    srv.close()


def test_lband_blocks_full_size_whole_planes(dd, oracle_lib):
    """Blocks of 65536 samples of 1024-channel, 1024-DM beams (DMs 0..1023, the
    serving workload's beam shape), 8 beams x 3 blocks served with continuous
    batching: every cell of every block's plane bit-exact against the oracle's
    plane of the beam's concatenated stream."""
    streams = []
    for i in range(8):
        s = Stream.__new__(Stream)
        s.nchan, s.B, s.nblocks = 1024, 65536, 3
        s.fch1, s.foff, s.tsamp = 1500.0, -0.29296875, 64e-6
        s.dms = fb.dm_grid(0.0, 1.0, 1024)
        s.table = oracle_lib.dmshift(1024, s.fch1, s.foff, s.tsamp)
        s.S = oracle_lib.maxshift(s.table, s.dms)
        s.data = fb.NoisePool(500 + i).rows(1024, 3 * 65536)
        s.outs = [np.full((1024, 65536), -9.0, np.float32) for _ in range(3)]
        s.got = {}
        streams.append(s)
    stats, _ = _serve(dd, streams, budget=24 << 30, inflight=12)
    assert stats["completed"] == 24
    for s in streams:
        s.check(oracle_lib, threads=True)
