"""CPU oracle for brute-force incoherent de-dispersion (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py`` may import it.  The GPU library
(``paper_1111_6399_gb300``) never imports, links or runs anything here, and this
package imports nothing from the library.

The arithmetic lives in ``dedisp_oracle.c`` (plain single-threaded C, built with
``-ffp-contract=off``); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  Two builds are made from the same source:

* ``liboracle.so``      -- single-threaded, the oracle proper;
* ``liboracle_omp.so``  -- the same loops with the DM loop under OpenMP (the
  "checker" build), used for large parity cases; each (d,t) cell is summed in
  the same order, so both give identical results.

Definitions follow Sec. 2 of the paper (shift each channel by its dispersion
delay, then sum over frequency, for every trial DM); the integer shift rule is
spelled out in the C file's header.  The same file states, beside each
function, the stages around the search that the paper names without formulas
(Sec. 1, Sec. 4, Sec. 5): the polyphase channeliser and its prototype filter,
the front end (Stokes I, integration, RFI clipping, quantisation), sigproc
unpacking and the boxcar detection search.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dedisp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[bool, ctypes.CDLL] = {}

_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (seconds)."""
    os.makedirs(_BUILD, exist_ok=True)
    for omp in (False, True):
        out = _lib_path(omp)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = ["gcc", *_CFLAGS, _SRC, "-o", out + ".tmp", "-lm"]
        if omp:
            cmd.insert(1, "-fopenmp")
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


def _lib_path(omp: bool) -> str:
    return os.path.join(_BUILD, "liboracle_omp.so" if omp else "liboracle.so")


def _lib(omp: bool = False) -> ctypes.CDLL:
    with _LOCK:
        if omp not in _LIBS:
            build()
            lib = ctypes.CDLL(_lib_path(omp))
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_dmshift.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, p]
            lib.oracle_dmshift.restype = ctypes.c_int
            lib.oracle_shift.argtypes = [ctypes.c_float, ctypes.c_float]
            lib.oracle_shift.restype = ctypes.c_int
            lib.oracle_maxshift.argtypes = [ctypes.c_int, p, ctypes.c_int, p]
            lib.oracle_maxshift.restype = i64
            lib.oracle_dedisperse_u8.argtypes = [p, ctypes.c_int, i64, p, p, ctypes.c_int,
                                                 i64, p, i64]
            lib.oracle_dedisperse_u8.restype = None
            lib.oracle_half_to_double.argtypes = [ctypes.c_uint16]
            lib.oracle_half_to_double.restype = ctypes.c_double
            lib.oracle_dedisperse_float.argtypes = [p, ctypes.c_int, ctypes.c_int, i64, p, p,
                                                    ctypes.c_int, i64, p, p, i64]
            lib.oracle_dedisperse_float.restype = None
            lib.oracle_dedisperse_cells.argtypes = [p, ctypes.c_int, ctypes.c_int, i64, p, p,
                                                    i64, p, p, p, p]
            lib.oracle_dedisperse_cells.restype = None
            lib.oracle_unpack.argtypes = [p, ctypes.c_int, ctypes.c_int, i64, p, i64]
            lib.oracle_unpack.restype = None
            lib.oracle_detect.argtypes = [p, ctypes.c_int, i64, i64, ctypes.c_int, ctypes.c_int,
                                          p, p, p, p]
            lib.oracle_detect.restype = None
            lib.oracle_frontend.argtypes = [p, i64, ctypes.c_int, i64, ctypes.c_int,
                                            ctypes.c_double, ctypes.c_int, p, i64, p, p]
            lib.oracle_frontend.restype = None
            lib.oracle_pfb.argtypes = [p, i64, i64, ctypes.c_int, ctypes.c_int, p, ctypes.c_int,
                                       p, p, p]
            lib.oracle_pfb.restype = None
            lib.oracle_pfb_quantise.argtypes = [p, i64, ctypes.c_double, p]
            lib.oracle_pfb_quantise.restype = None
            lib.oracle_pfb_prototype.argtypes = [ctypes.c_int, ctypes.c_int, p]
            lib.oracle_pfb_prototype.restype = ctypes.c_int
            _LIBS[omp] = lib
        return _LIBS[omp]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def dmshift(nchan: int, fch1: float, foff: float, tsamp: float) -> np.ndarray:
    """FP32 per-channel delay per unit DM, in samples (FP64 evaluation, one rounding)."""
    out = np.empty(nchan, dtype=np.float32)
    if _lib().oracle_dmshift(nchan, fch1, foff, tsamp, _ptr(out)) != 0:
        raise ValueError("invalid band description")
    return out


def shift(dm: float, dmshift_c: float) -> int:
    """s(c,d) = trunc(float32(dm) * float32(dmshift[c])) with one FP32 multiply."""
    return int(_lib().oracle_shift(float(np.float32(dm)), float(np.float32(dmshift_c))))


def shift_table(dms: np.ndarray, table: np.ndarray) -> np.ndarray:
    """int32 [ndm][nchan] of s(c,d), one oracle_shift call per cell (small inputs)."""
    lib = _lib()
    out = np.empty((len(dms), len(table)), dtype=np.int32)
    for d, dm in enumerate(np.asarray(dms, dtype=np.float32)):
        for c, ds in enumerate(np.asarray(table, dtype=np.float32)):
            out[d, c] = lib.oracle_shift(float(dm), float(ds))
    return out


def maxshift(table: np.ndarray, dms: np.ndarray) -> int:
    table = np.ascontiguousarray(table, dtype=np.float32)
    dms = np.ascontiguousarray(dms, dtype=np.float32)
    return int(_lib().oracle_maxshift(len(table), _ptr(table), len(dms), _ptr(dms)))


def half_to_double(bits: int) -> float:
    return float(_lib().oracle_half_to_double(bits))


def dedisperse(data: np.ndarray, table: np.ndarray, dms: np.ndarray, nsamp_out: int,
               with_abssum: bool = False, threads: bool = False):
    """Full (DM,t) plane.

    data: [nchan][nsamp_in] uint8, float16 or float32 (C-contiguous rows).
    uint8 -> float32 plane (exact); float16/float32 -> float64 plane
    (and, if with_abssum, the float64 plane of sum |in| along each curve).
    """
    data = np.ascontiguousarray(data)
    table = np.ascontiguousarray(table, dtype=np.float32)
    dms = np.ascontiguousarray(dms, dtype=np.float32)
    nchan, nsamp_in = data.shape
    if len(table) != nchan:
        raise ValueError("dmshift length does not match nchan")
    if nsamp_in < nsamp_out + maxshift(table, dms):
        raise ValueError("rows are shorter than nsamp_out + maxshift")
    lib = _lib(threads)
    ndm = len(dms)
    if data.dtype == np.uint8:
        out = np.empty((ndm, nsamp_out), dtype=np.float32)
        lib.oracle_dedisperse_u8(_ptr(data), nchan, nsamp_in, _ptr(table), _ptr(dms), ndm,
                                 nsamp_out, _ptr(out), nsamp_out)
        return (out, out.astype(np.float64)) if with_abssum else out
    if data.dtype == np.float16:
        elem, raw = 2, data.view(np.uint16)
    elif data.dtype == np.float32:
        elem, raw = 4, data
    else:
        raise TypeError(f"unsupported dtype {data.dtype}")
    out = np.empty((ndm, nsamp_out), dtype=np.float64)
    asum = np.empty((ndm, nsamp_out), dtype=np.float64) if with_abssum else None
    lib.oracle_dedisperse_float(_ptr(raw), elem, nchan, nsamp_in, _ptr(table), _ptr(dms), ndm,
                                nsamp_out, _ptr(out), _ptr(asum) if asum is not None else None,
                                nsamp_out)
    return (out, asum) if with_abssum else out


def dedisperse_cells(data: np.ndarray, table: np.ndarray, dms: np.ndarray,
                     d_idx: np.ndarray, t_idx: np.ndarray, threads: bool = True):
    """Selected cells (d_idx[i], t_idx[i]) of the plane, for full-size inputs.

    Returns (values, abssum) as float64 arrays; for uint8 the value is the
    exact FP32 sum widened to float64.
    """
    data = np.ascontiguousarray(data)
    table = np.ascontiguousarray(table, dtype=np.float32)
    dms = np.ascontiguousarray(dms, dtype=np.float32)
    d_idx = np.ascontiguousarray(d_idx, dtype=np.int32)
    t_idx = np.ascontiguousarray(t_idx, dtype=np.int64)
    nchan, nsamp_in = data.shape
    if data.dtype == np.uint8:
        elem, raw = 1, data
    elif data.dtype == np.float16:
        elem, raw = 2, data.view(np.uint16)
    elif data.dtype == np.float32:
        elem, raw = 4, data
    else:
        raise TypeError(f"unsupported dtype {data.dtype}")
    if len(d_idx) != len(t_idx):
        raise ValueError("index arrays differ in length")
    if len(d_idx):
        need = int(t_idx.max()) + maxshift(table, dms[np.unique(d_idx)])
        if need >= nsamp_in or d_idx.min() < 0 or d_idx.max() >= len(dms) or t_idx.min() < 0:
            raise ValueError("cell outside the plane")
    out = np.empty(len(d_idx), dtype=np.float64)
    asum = np.empty(len(d_idx), dtype=np.float64)
    _lib(threads).oracle_dedisperse_cells(_ptr(raw), elem, nchan, nsamp_in, _ptr(table),
                                          _ptr(dms), len(d_idx), _ptr(d_idx), _ptr(t_idx),
                                          _ptr(out), _ptr(asum))
    return out, asum


def unpack(raw: np.ndarray, nbits: int, nchan: int, nsamp: int) -> np.ndarray:
    """Corner turn of nsamp sigproc-order spectra of nchan nbits-bit samples
    (first sample in the lowest bits of a byte) into uint8 [nchan][nsamp]."""
    raw = np.ascontiguousarray(raw, dtype=np.uint8)
    if nbits not in (1, 2, 4, 8) or (nchan * nbits) % 8:
        raise ValueError("nbits must be 1, 2, 4 or 8 and nchan*nbits a multiple of 8")
    if raw.size < nsamp * nchan * nbits // 8:
        raise ValueError("input shorter than nsamp spectra")
    out = np.empty((nchan, nsamp), dtype=np.uint8)
    _lib().oracle_unpack(_ptr(raw), nbits, nchan, nsamp, _ptr(out), nsamp)
    return out


def detect(plane: np.ndarray, nlevels: int, integer_valued: bool):
    """Boxcar search of every DM row of a (DM,t) plane over widths 1, 2, ...,
    2^(nlevels-1) (the rules are in the C file).  Returns (mean[ndm], std[ndm],
    snr[ndm][nlevels], t[ndm][nlevels])."""
    x = np.ascontiguousarray(plane, dtype=np.float64)
    ndm, nsamp = x.shape
    if integer_valued and (np.any(x != np.floor(x)) or np.any(x < 0) or np.any(x >= 2 ** 21)
                           or nsamp > 2 ** 21):
        raise ValueError("integer mode needs integers in [0, 2^21) and nsamp <= 2^21")
    mean = np.empty(ndm, dtype=np.float64)
    std = np.empty(ndm, dtype=np.float64)
    snr = np.empty((ndm, nlevels), dtype=np.float64)
    tpk = np.empty((ndm, nlevels), dtype=np.int64)
    _lib().oracle_detect(_ptr(x), ndm, nsamp, nsamp, nlevels, int(bool(integer_valued)),
                         _ptr(mean), _ptr(std), _ptr(snr), _ptr(tpk))
    return mean, std, snr, tpk


def frontend(volts: np.ndarray, nint: int, k_clip: float, niter: int = 1):
    """Stokes I, integration over nint raw samples, RFI excision by niter
    passes of sigma clipping at mean + k_clip*std, and quantisation to uint8
    (rules in the C file).  volts: int8 [nchan][nsamp_raw][4] (Xre, Xim, Yre,
    Yim).  Returns (out uint8 [nchan][nsamp_raw // nint], mean[nchan],
    std[nchan]), mean and std those of the last pass."""
    v = np.ascontiguousarray(volts, dtype=np.int8)
    if v.ndim != 3 or v.shape[2] != 4 or nint < 1 or niter < 1:
        raise ValueError("volts must be int8 [nchan][nsamp_raw][4], nint >= 1, niter >= 1")
    nchan, nraw = v.shape[0], v.shape[1]
    n = nraw // nint
    out = np.empty((nchan, n), dtype=np.uint8)
    mean = np.empty(nchan, dtype=np.float64)
    std = np.empty(nchan, dtype=np.float64)
    _lib().oracle_frontend(_ptr(v), 4 * nraw, nchan, nraw, nint, float(k_clip), int(niter),
                           _ptr(out), n, _ptr(mean), _ptr(std))
    return out, mean, std


def pfb_nspec(nraw: int, M: int, T: int) -> int:
    """Spectra of the channeliser: floor(nraw/M) - T + 1, or 0."""
    return max(0, nraw // M - T + 1)


def pfb(volts: np.ndarray, M: int, T: int, h: np.ndarray, spectra=None, threads: bool = False):
    """Polyphase channeliser (definition in the C file), FP64.

    volts: int8 [nsub][nraw][4] (Xre, Xim, Yre, Yim) subband voltages;
    h: prototype filter, M*T values (taken as FP64).
    spectra: None for every spectrum -> float64 [nsub*M][nspec][4] (row
    s*M + c, channel c in increasing frequency); or a list of (s, n) ->
    float64 [len][M][4].
    """
    v = np.ascontiguousarray(volts, dtype=np.int8)
    if v.ndim != 3 or v.shape[2] != 4:
        raise ValueError("volts must be int8 [nsub][nraw][4]")
    h = np.ascontiguousarray(h, dtype=np.float64)
    if M < 1 or T < 1 or h.size != M * T:
        raise ValueError("h must hold M*T values")
    nsub, nraw = v.shape[0], v.shape[1]
    nspec = pfb_nspec(nraw, M, T)
    full = spectra is None
    if full:
        sub = np.repeat(np.arange(nsub, dtype=np.int32), nspec)
        spec = np.tile(np.arange(nspec, dtype=np.int64), nsub)
    else:
        sel = np.asarray(spectra, dtype=np.int64).reshape(-1, 2)
        sub = np.ascontiguousarray(sel[:, 0], dtype=np.int32)
        spec = np.ascontiguousarray(sel[:, 1], dtype=np.int64)
        if len(sel) and (sub.min() < 0 or sub.max() >= nsub or spec.min() < 0
                         or spec.max() >= nspec):
            raise ValueError("spectrum outside the output")
    out = np.empty((len(sub), M, 4), dtype=np.float64)
    if len(sub):
        _lib(threads).oracle_pfb(_ptr(v), 4 * nraw, nraw, M, T, _ptr(h), len(sub), _ptr(sub),
                                 _ptr(spec), _ptr(out))
    if full:
        return out.reshape(nsub, nspec, M, 4).transpose(0, 2, 1, 3).reshape(nsub * M, nspec, 4)
    return out


def pfb_quantise(v: np.ndarray, scale: float) -> np.ndarray:
    """int8 clamp(rint(v * scale), -127, 127) in FP64 (same shape as v)."""
    x = np.ascontiguousarray(v, dtype=np.float64)
    q = np.empty(x.shape, dtype=np.int8)
    _lib().oracle_pfb_quantise(_ptr(x), x.size, float(scale), _ptr(q))
    return q


def pfb_prototype(M: int, T: int) -> np.ndarray:
    """Hamming-windowed sinc prototype of M*T taps (FP64)."""
    h = np.empty(M * T, dtype=np.float64)
    if _lib().oracle_pfb_prototype(M, T, _ptr(h)) != 0:
        raise ValueError("need M >= 1, T >= 1 and M*T >= 2")
    return h
