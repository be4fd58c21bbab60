"""C-ABI library: loads, exports every declared symbol, and the host plan and
argument validation behave -- all without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import filterbank as fb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dd(request):
    return request.getfixturevalue("built_lib")


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(dd_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(dd):
    declared = _declared()
    assert "dd_execute" in declared and "dd_plan" in declared
    lib = ctypes.CDLL(dd._binding.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(dd._binding.EXPORTS) == sorted(n for n in declared if n in dd._binding.EXPORTS)


def test_plan_table_is_bit_identical_to_the_oracle(dd, oracle_lib):
    for w in (fb.SMALL, fb.LBAND, fb.LOWFREQ):
        p = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
        want = oracle_lib.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
        assert np.array_equal(p.dmshift().view(np.uint32), want.view(np.uint32))
        assert p.maxshift == oracle_lib.maxshift(want, w.dm_list())
        assert (p.nchan, p.ndm) == (w.nchan, w.ndm)


def test_plan_on_random_bands_and_unsorted_dms(dd, oracle_lib):
    rng = np.random.default_rng(4)
    for _ in range(30):
        nchan = int(rng.integers(1, 3000))
        fch1 = float(rng.uniform(50, 3000))
        foff = float(rng.choice([-1, 1]) * rng.uniform(1e-4, 0.9 * fch1 / max(nchan, 2)))
        tsamp = float(rng.uniform(1e-6, 1e-2))
        dms = rng.uniform(0, 3000, size=int(rng.integers(1, 50))).astype(np.float32)
        p = dd.Plan(nchan, fch1, foff, tsamp, dms)
        want = oracle_lib.dmshift(nchan, fch1, foff, tsamp)
        assert np.array_equal(p.dmshift().view(np.uint32), want.view(np.uint32))
        assert p.maxshift == oracle_lib.maxshift(want, dms)


@pytest.mark.parametrize("args", [
    (0, 1500.0, -1.0, 64e-6, [0.0]),
    (8, 1500.0, 0.0, 64e-6, [0.0]),
    (8, 1500.0, -1.0, 0.0, [0.0]),
    (8, 1500.0, -1.0, -1e-3, [0.0]),
    (8, 5.0, -1.0, 64e-6, [0.0]),          # channel centres below zero
    (8, 1500.0, -1.0, 64e-6, []),
    (8, 1500.0, -1.0, 64e-6, [1.0, -2.0]),
    (8, 1500.0, -1.0, 64e-6, [float("nan")]),
    (8, 1500.0, -1.0, 64e-6, [float("inf")]),
])
def test_invalid_plans_are_rejected(dd, args):
    with pytest.raises(dd.DDError) as e:
        dd.Plan(*args)
    assert e.value.status == -1


def test_tile_validation(dd):
    w = fb.LBAND
    p = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    assert p.get_tiles("u8") == (4, 12, 1, 8, 8)
    p.set_tiles("u8", 2, 6, 2, 4, 4)
    assert p.get_tiles("u8") == (2, 6, 2, 4, 4)
    for bad in [(3, 8, 1, 8), (4, 16, 1, 8), (4, 8, 1, 7), (4, 8, 1, 6), (4, 8, 1, 0), (1, 1, 1, 96),
                (4, 12, 1, 64),    # needs more shared memory than a CTA has
                (4, 20, 1, 8, 4)]:  # 80 DMs per CTA (limit 64)
        with pytest.raises(dd.DDError):
            p.set_tiles("u8", *bad)
    with pytest.raises(dd.DDError):
        p.set_tiles("f32", 2, 8, 1, 128)


def test_execute_validates_before_touching_a_gpu(dd):
    """Every layout error is reported as DD_ERR_INVALID by host checks alone."""
    w = fb.SMALL
    p = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    S = p.maxshift
    good = dict(in_ptr=4096, dtype=0, in_pitch=8512, nsamp_in=8192 + S, out_ptr=8192,
                out_pitch=8192, nsamp_out=8192)
    bad = [
        dict(nsamp_in=8192 + S - 1),       # rows too short for maxshift
        dict(in_pitch=8500),               # pitch not a multiple of 16 bytes
        dict(out_pitch=8190),              # output pitch not a multiple of 4 floats
        dict(in_pitch=8000),               # pitch shorter than the row
        dict(in_ptr=4097),                 # misaligned pointer
        dict(out_ptr=0),                   # NULL output
        dict(dtype=7),                     # unknown dtype
        dict(nsamp_out=-1),
    ]
    for b in bad:
        args = {**good, **b}
        with pytest.raises(dd.DDError) as e:
            p.execute_ptr(args["in_ptr"], args["dtype"], args["in_pitch"], args["nsamp_in"],
                          args["out_ptr"], args["out_pitch"], args["nsamp_out"])
        assert e.value.status == -1, b
    # nsamp_out == 0 is a no-op and needs no device
    p.execute_ptr(0, 0, 16, 0, 0, 0, 0)
    # the no-alloc entry point runs the same host checks first
    for b in bad:
        args = {**good, **b}
        with pytest.raises(dd.DDError) as e:
            p.execute_noalloc_ptr(args["in_ptr"], args["dtype"], args["in_pitch"],
                                  args["nsamp_in"], args["out_ptr"], args["out_pitch"],
                                  args["nsamp_out"])
        assert e.value.status == -1, b
    p.execute_noalloc_ptr(0, 0, 16, 0, 0, 0, 0)


def test_unpack_validates_before_touching_a_gpu(dd):
    """dd_unpack argument errors are DD_ERR_INVALID from host checks alone."""
    good = dict(inp=4096, nbits=2, nchan=64, nsamp=100, out=8192, pitch=112)
    bad = [
        dict(nbits=3), dict(nbits=0), dict(nbits=16),
        dict(nchan=3),                   # 3 x 2 bits is not whole bytes
        dict(nchan=0),
        dict(pitch=96),                  # shorter than nsamp
        dict(pitch=104),                 # not a multiple of 16
        dict(nsamp=-1),
        dict(inp=0), dict(out=0),
        dict(out=8200),                  # output not 16-byte aligned
    ]
    for b in bad:
        a = {**good, **b}
        st = dd.lib.dd_unpack(ctypes.c_void_p(a["inp"]), a["nbits"], a["nchan"], a["nsamp"],
                              ctypes.c_void_p(a["out"]), a["pitch"], None)
        assert st == -1, b
    # nsamp == 0 is a no-op and needs no device
    assert dd.lib.dd_unpack(None, 8, 16, 0, None, 0, None) == 0


def test_detect_validates_before_touching_a_gpu(dd):
    """dd_detect argument errors are DD_ERR_INVALID from host checks alone."""
    P = 4096
    good = dict(plane=P, pitch=1000, ndm=4, nsamp=1000, nlev=9, integer=1, mean=P, std=P,
                snr=P, t=P)
    bad = [
        dict(nlev=0), dict(nlev=10),       # widths 1..256 only
        dict(nsamp=0), dict(pitch=999),    # empty rows, pitch shorter than a row
        dict(nsamp=(1 << 21) + 1, pitch=(1 << 21) + 1),   # integer planes: nsamp <= 2^21
        dict(ndm=-1),
        dict(plane=0), dict(mean=0), dict(snr=0), dict(t=0),
        dict(plane=P + 2), dict(std=P + 4), # misaligned
    ]
    for b in bad:
        a = {**good, **b}
        st = dd.lib.dd_detect(ctypes.c_void_p(a["plane"]), a["pitch"], a["ndm"], a["nsamp"],
                              a["nlev"], a["integer"], ctypes.c_void_p(a["mean"]),
                              ctypes.c_void_p(a["std"]), ctypes.c_void_p(a["snr"]),
                              ctypes.c_void_p(a["t"]), None)
        assert st == -1, b
    # no rows: a no-op that needs no device
    assert dd.lib.dd_detect(None, 10, 0, 10, 3, 1, None, None, None, None, None) == 0


def test_frontend_validates_before_touching_a_gpu(dd):
    """dd_frontend argument errors are DD_ERR_INVALID from host checks alone."""
    P = 4096
    need = dd.frontend_work_bytes(8, 1000, 4, 3)
    assert need == 4 * 8 * 252 + 24 * 3 * 8          # P rows of 250 -> 252, 3 sum sets
    good = dict(volts=P, vpitch=4000, nchan=8, nraw=1000, nint=4, k=4.0, niter=3, out=P,
                opitch=256, work=P, wbytes=need, mean=P, std=P)
    bad = [
        dict(nint=3), dict(nint=0), dict(nint=128),     # powers of two up to 64
        dict(niter=0), dict(niter=9),
        dict(nchan=0), dict(nchan=65536),
        dict(nraw=-1),
        dict(nraw=(1 << 19) * 4 + 4, vpitch=16 * (1 << 21)),   # more than 2^19 outputs
        dict(vpitch=3996),               # shorter than 4*nsamp_raw
        dict(vpitch=4002),               # not a multiple of 4
        dict(opitch=240),                # shorter than nsamp_raw / nint
        dict(opitch=264),                # not a multiple of 16
        dict(k=0.0), dict(k=-1.0), dict(k=2e9), dict(k=float("nan")),
        dict(wbytes=need - 1),
        dict(volts=0), dict(out=0), dict(work=0), dict(mean=0), dict(std=0),
        dict(volts=P + 2), dict(out=P + 4), dict(work=P + 4), dict(mean=P + 4),
    ]
    for b in bad:
        a = {**good, **b}
        st = dd.lib.dd_frontend(ctypes.c_void_p(a["volts"]), a["vpitch"], a["nchan"], a["nraw"],
                                a["nint"], a["k"], a["niter"], ctypes.c_void_p(a["out"]),
                                a["opitch"], ctypes.c_void_p(a["work"]), a["wbytes"],
                                ctypes.c_void_p(a["mean"]), ctypes.c_void_p(a["std"]), None)
        assert st == -1, b
    for shape in [(0, 1000, 4, 1), (8, 1000, 3, 1), (8, 1000, 4, 0), (8, 1 << 22, 4, 1)]:
        assert dd.lib.dd_frontend_work_bytes(*shape) == -1, shape
    with pytest.raises(dd.DDError):
        dd.frontend_work_bytes(8, 1000, 4, 9)


def test_status_codes_and_messages(dd):
    with pytest.raises(dd.DDError) as e:
        dd.Plan(8, 1500.0, -1.0, 0.0, [0.0])
    assert "tsamp" in str(e.value)
    assert dd.lib.dd_plan_maxshift(None) == -1


def test_channeliser_host_routines_match_the_oracle(dd, oracle_lib):
    """The library's prototype is the oracle's FP64 prototype rounded once to
    FP32, and both count the same spectra."""
    for M, T in [(16, 8), (32, 3), (64, 1), (128, 16), (256, 8)]:
        got = dd.pfb_prototype(M, T)
        want = oracle_lib.pfb_prototype(M, T).astype(np.float32)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), (M, T)
    rng = np.random.default_rng(3)
    for _ in range(200):
        M = int(rng.choice([16, 32, 64, 128, 256]))
        T = int(rng.integers(1, 17))
        nraw = int(rng.integers(0, 40 * M))
        assert dd.channelise_nspec(nraw, M, T) == oracle_lib.pfb_nspec(nraw, M, T)
    for bad in [(100, 8, 4), (100, 48, 4), (100, 512, 4), (100, 16, 0), (100, 16, 17),
                (-1, 16, 4)]:
        assert dd.lib.dd_channelise_nspec(*bad) == -1, bad
    with pytest.raises(dd.DDError):
        dd.pfb_prototype(1, 1)


def test_channelise_validates_before_touching_a_gpu(dd):
    """dd_channelise argument errors are DD_ERR_INVALID from host checks alone."""
    P = 4096
    good = dict(volts=P, vpitch=4096, nsub=2, nraw=1024, M=16, T=4, h=P, kind=1, scale=0.5,
                out=P, opitch=256)
    bad = [
        dict(M=8), dict(M=48), dict(M=512), dict(T=0), dict(T=17),
        dict(nsub=0), dict(nsub=65536), dict(nraw=-1),
        dict(kind=2), dict(kind=-1),
        dict(scale=0.0), dict(scale=-1.0), dict(scale=float("nan")), dict(scale=float("inf")),
        dict(vpitch=4092),                    # shorter than 4*nraw
        dict(vpitch=4098),                    # not a multiple of 4
        dict(opitch=240),                     # shorter than 4 bytes x 61 spectra
        dict(opitch=246),                     # not a multiple of the 4-byte element
        dict(kind=0, opitch=512),             # FP32 elements: 16 x 61 bytes needed
        dict(kind=0, opitch=984),             # not a multiple of 16
        dict(volts=0), dict(h=0), dict(out=0),
        dict(volts=P + 2), dict(h=P + 2), dict(out=P + 2),
        dict(kind=0, opitch=1024, out=P + 4),  # FP32 output must be 16-byte aligned
    ]
    for b in bad:
        a = {**good, **b}
        st = dd.lib.dd_channelise(ctypes.c_void_p(a["volts"]), a["vpitch"], a["nsub"],
                                  a["nraw"], a["M"], a["T"], ctypes.c_void_p(a["h"]), a["kind"],
                                  a["scale"], ctypes.c_void_p(a["out"]), a["opitch"], None)
        assert st == -1, b
    # fewer than M*T raw samples: no spectra, a no-op that needs no device
    assert dd.lib.dd_channelise(None, 252, 2, 63, 16, 4, None, 1, 0.5, None, 0, None) == 0



def test_execute_detect_validates_before_touching_a_gpu(dd):
    """dd_execute_detect takes uint8 input, nlevels 1..9 and aligned outputs;
    anything else is DD_ERR_INVALID from host checks alone."""
    import ctypes
    w = fb.SMALL
    p = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    S = p.maxshift
    lib = dd.lib
    good = dict(inp=4096, dtype=0, pitch=8512, nin=8192 + S, out=8192, opitch=8192,
                nout=8192, nlev=9, mean=1024, std=2048, snr=4096, tpk=8192)
    bad = [dict(dtype=1), dict(dtype=2), dict(nlev=0), dict(nlev=10), dict(nin=8192 + S - 1),
           dict(inp=4097), dict(mean=1028), dict(tpk=0), dict(nout=0), dict(nout=(1 << 21) + 1)]
    for b in bad:
        a = {**good, **b}
        st = lib.dd_execute_detect(p.handle, ctypes.c_void_p(a["inp"]), a["dtype"], a["pitch"],
                                   a["nin"], ctypes.c_void_p(a["out"]), a["opitch"], a["nout"],
                                   a["nlev"], ctypes.c_void_p(a["mean"]),
                                   ctypes.c_void_p(a["std"]), ctypes.c_void_p(a["snr"]),
                                   ctypes.c_void_p(a["tpk"]), None)
        assert st == -1, b
