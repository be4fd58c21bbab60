"""Batched uneven beams in one persistent launch (CUDA-graph replay) against
the CPU oracle and against each beam's own single-beam execution."""
import numpy as np
import pytest

import filterbank as fb
from tests.cases import pulse_delays, sample_cells

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dd(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return request.getfixturevalue("built_lib")


def _beam_input(spec, table, pool, kind="u8"):
    import oracle
    S = oracle.maxshift(table, spec.dm_list())
    nin = spec.nsamp_out + S
    elem = {"u8": 1, "f16": 2, "f32": 4}[kind]
    step = 16 // elem
    pitch = (nin + step - 1) // step * step
    data = pool.rows(spec.nchan, nin, pitch)
    for p, dl in zip(spec.pulses, pulse_delays(table, spec.pulses)):
        fb.add_pulse_u8(data, dl, p, nin)
    if kind != "u8":
        data = data.astype(np.float16 if kind == "f16" else np.float32)
    return data, nin


def _run_batch(dd, specs, kind, oracle_lib, tiles=None, autotune=False):
    pool = fb.NoisePool(123)
    plans, ins, outs, datas, tables = [], [], [], [], []
    for sp in specs:
        table = oracle_lib.dmshift(sp.nchan, sp.fch1, sp.foff, sp.tsamp)
        plan = dd.Plan(sp.nchan, sp.fch1, sp.foff, sp.tsamp, sp.dm_list())
        data, nin = _beam_input(sp, table, pool, kind)
        assert nin == sp.nsamp_out + plan.maxshift
        plans.append(plan)
        datas.append((data, nin))
        tables.append(table)
        ins.append(torch.from_numpy(data).cuda())
        outs.append(torch.full((sp.ndm, (sp.nsamp_out + 3) // 4 * 4), -5.0, device="cuda"))
    batch = dd.Batch(plans, kind)
    for i, sp in enumerate(specs):
        batch.set_io(i, ins[i], outs[i], nsamp_in=datas[i][1], nsamp_out=sp.nsamp_out)
    if tiles:
        batch.set_tiles(*tiles)
    if autotune:
        res = batch.autotune(reps=1)
        assert any(ms >= 0 for _, ms in res)
    return batch, plans, ins, outs, datas, tables


def _check_beam(dd, oracle_lib, sp, plan, inp, out, data, nin, table, full=True):
    got = out.cpu().numpy()
    assert np.all(got[:, sp.nsamp_out:] == -5.0)
    got = got[:, :sp.nsamp_out]
    # equal to the beam's own single-beam launch
    solo = torch.empty((sp.ndm, (sp.nsamp_out + 3) // 4 * 4), device="cuda")
    plan.execute(inp, solo, nsamp_in=nin, nsamp_out=sp.nsamp_out)
    plan.sync()
    assert np.array_equal(got, solo.cpu().numpy()[:, :sp.nsamp_out])
    if full:
        want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nin]), table, sp.dm_list(),
                                     sp.nsamp_out)
        if data.dtype == np.uint8:
            assert np.array_equal(got, want)
        else:
            assert np.array_equal(got.astype(np.float64), want)   # integer-valued data
    else:
        rng = np.random.default_rng(sp.index)
        d_idx, t_idx = sample_cells(rng, sp.ndm, sp.nsamp_out, 48)
        want, _ = oracle_lib.dedisperse_cells(data, table, sp.dm_list(), d_idx, t_idx)
        assert np.array_equal(got[d_idx, t_idx].astype(np.float64), want)


def _small_specs(seed, n, kind="u8"):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nchan = int(rng.choice([24, 64, 130, 256]))
        bw = float(rng.choice([64.0, 300.0]))
        nsamp = int(rng.integers(500, 9000))
        ndm = int(rng.integers(5, 150))
        pulses = (fb.Pulse(float(rng.integers(0, ndm)), int(rng.integers(0, nsamp - 16)), 3),)
        out.append(fb.BeamSpec(i, nchan, 1500.0, -bw / nchan, 64e-6, nsamp, ndm, pulses))
    return out


@pytest.mark.parametrize("kind", ["u8", "f16", "f32"])
def test_small_uneven_batch_is_exact_and_equal_to_solo(dd, oracle_lib, kind):
    specs = _small_specs(7, 6)
    batch, plans, ins, outs, datas, tables = _run_batch(dd, specs, kind, oracle_lib)
    batch.execute()          # eager run + graph capture
    batch.sync()
    for i, sp in enumerate(specs):
        _check_beam(dd, oracle_lib, sp, plans[i], ins[i], outs[i], *datas[i], tables[i])
    # graph replay after the inputs change in place
    for i in range(len(specs)):
        outs[i][:, :specs[i].nsamp_out].fill_(-1.0)
        ins[i].copy_(torch.flip(ins[i], dims=[0]))
        datas[i] = (np.ascontiguousarray(datas[i][0][::-1]), datas[i][1])
    batch.execute()
    batch.sync()
    for i, sp in enumerate(specs):
        _check_beam(dd, oracle_lib, sp, plans[i], ins[i], outs[i], *datas[i], tables[i])


def test_batch_tile_shapes_and_autotuner(dd, oracle_lib):
    specs = _small_specs(11, 5)
    for tiles in [(2, 6, 1, 8, 8), (4, 8, 1, 12, 4), (1, 12, 1, 4, 8)]:
        batch, plans, ins, outs, datas, tables = _run_batch(dd, specs, "u8", oracle_lib, tiles)
        assert batch.get_tiles() == tiles
        batch.execute()
        batch.execute()
        batch.sync()
        for i, sp in enumerate(specs):
            _check_beam(dd, oracle_lib, sp, plans[i], ins[i], outs[i], *datas[i], tables[i])
    batch, plans, ins, outs, datas, tables = _run_batch(dd, specs, "u8", oracle_lib,
                                                        autotune=True)
    batch.execute()
    batch.sync()
    for i, sp in enumerate(specs):
        _check_beam(dd, oracle_lib, sp, plans[i], ins[i], outs[i], *datas[i], tables[i])


def test_batch_rejects_unbound_beams(dd):
    plan = dd.Plan(16, 1400.0, -1.0, 1e-4, [0.0, 3.0])
    batch = dd.Batch([plan, plan], "u8")
    x = torch.zeros((16, 1024), dtype=torch.uint8, device="cuda")
    out = torch.empty((2, 512), device="cuda")
    batch.set_io(0, x, out)
    with pytest.raises(dd.DDError):
        batch.execute()
    with pytest.raises(dd.DDError):
        batch.set_io(1, x, out, nsamp_in=10, nsamp_out=512)   # rows too short


def test_uneven_beams_full_size(dd, oracle_lib):
    """The 64-beam batch at full size (about 10^13 adds), one persistent launch
    replayed from a CUDA graph: every beam equals its own single-beam launch;
    16 DM rows of every beam, spread over its DM range, match the oracle at
    full length; and the whole planes of the eight beams with the fewest adds
    match the oracle cell by cell."""
    specs = fb.uneven_beams()
    batch, plans, ins, outs, datas, tables = _run_batch(dd, specs, "u8", oracle_lib)
    batch.execute()
    batch.execute()          # graph replay
    batch.sync()
    whole = set(int(i) for i in np.argsort([sp.adds() for sp in specs])[:8])
    for i, sp in enumerate(specs):
        data, nin = datas[i]
        got = outs[i].cpu().numpy()
        assert np.all(got[:, sp.nsamp_out:] == -5.0)
        got = got[:, :sp.nsamp_out]
        solo = torch.empty((sp.ndm, (sp.nsamp_out + 3) // 4 * 4), device="cuda")
        plans[i].execute(ins[i], solo, nsamp_in=nin, nsamp_out=sp.nsamp_out)
        plans[i].sync()
        assert np.array_equal(got, solo.cpu().numpy()[:, :sp.nsamp_out]), f"beam {i}"
        del solo
        dms = sp.dm_list()
        rows = np.arange(sp.ndm) if i in whole else \
            np.unique(np.linspace(0, sp.ndm - 1, 16).round().astype(int))
        sel = dms[rows]
        nneed = sp.nsamp_out + oracle_lib.maxshift(tables[i], sel)
        want = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :nneed]), tables[i], sel,
                                     sp.nsamp_out, threads=True)
        bad = np.argwhere(got[rows] != want)
        assert len(bad) == 0, f"beam {i}: {len(bad)} cells differ, first {bad[:4].tolist()}"
