"""ctypes binding of libdd.so (argument marshalling only).

Every step of the de-dispersion path runs in the CUDA library; this module
converts Python/numpy/torch arguments to plain pointers and sizes and raises
on a non-OK status.  It never falls back to another implementation: if the
library is missing or fails to load, importing the package raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdd.so")

DD_U8, DD_F16, DD_F32 = 0, 1, 2
STATUS = {0: "DD_OK", 1: "DD_PENDING", -1: "DD_ERR_INVALID", -2: "DD_ERR_CUDA",
          -3: "DD_ERR_NOMEM", -4: "DD_ERR_BUSY", -5: "DD_ERR_TIMEOUT", -6: "DD_ERR_DEVICE"}
DD_OK, DD_PENDING, DD_ERR_INVALID, DD_ERR_CUDA = 0, 1, -1, -2
DD_ERR_NOMEM, DD_ERR_BUSY, DD_ERR_TIMEOUT, DD_ERR_DEVICE = -3, -4, -5, -6

# Every symbol include/dd.h declares (checked by the tests).
EXPORTS = [
    "dd_plan", "dd_plan_destroy", "dd_plan_maxshift", "dd_plan_nchan", "dd_plan_ndm",
    "dd_plan_dmshift", "dd_plan_get_tiles", "dd_plan_set_tiles", "dd_execute",
    "dd_execute_host", "dd_sync", "dd_profile_events", "dd_launch_count", "dd_last_error",
    "dd_autotune", "dd_execute_noalloc", "dd_batch_create", "dd_batch_destroy",
    "dd_batch_set_io", "dd_batch_execute", "dd_batch_get_tiles", "dd_batch_set_tiles",
    "dd_batch_autotune", "dd_batch_sync", "dd_server_create", "dd_server_add_beam",
    "dd_submit", "dd_poll", "dd_server_drain", "dd_server_get_stats", "dd_server_destroy",
    "dd_selftest_wait_timeout", "dd_server_set_batch_window", "dd_unpack", "dd_detect",
    "dd_frontend", "dd_frontend_work_bytes", "dd_channelise", "dd_channelise_nspec",
    "dd_pfb_prototype", "dd_sync_noalloc", "dd_selftest_noalloc_timeout", "dd_add_peak",
    "dd_execute_detect",
]


class DDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Tiles(ctypes.Structure):
    _fields_ = [("dm_per_thread", ctypes.c_int), ("dm_warps", ctypes.c_int),
                ("time_warps", ctypes.c_int), ("chan_per_stage", ctypes.c_int),
                ("words_per_thread", ctypes.c_int)]

    def as_tuple(self):
        return (self.dm_per_thread, self.dm_warps, self.time_warps, self.chan_per_stage,
                self.words_per_thread)


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected_busy", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_batch", ctypes.c_double),
                ("slots", ctypes.c_int), ("device_bytes", ctypes.c_int64),
                ("staging_bytes", ctypes.c_int64), ("staging_ms", ctypes.c_double),
                ("h2d_bytes", ctypes.c_int64), ("h2d_ms", ctypes.c_double),
                ("d2h_bytes", ctypes.c_int64), ("d2h_ms", ctypes.c_double),
                ("batch_window_us", ctypes.c_int64), ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class TuneResult(ctypes.Structure):
    _fields_ = [("tiles", Tiles), ("ms", ctypes.c_float)]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdd.so not built ({LIB_PATH}); run "
                          "python __graft_entry__.py")
    lib = ctypes.CDLL(LIB_PATH)
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sig = {
        "dd_plan": (i32, [i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, p, i32,
                          ctypes.POINTER(p)]),
        "dd_plan_destroy": (None, [p]),
        "dd_plan_maxshift": (i64, [p]),
        "dd_plan_nchan": (i32, [p]),
        "dd_plan_ndm": (i32, [p]),
        "dd_plan_dmshift": (i32, [p, p]),
        "dd_plan_get_tiles": (i32, [p, i32, ctypes.POINTER(Tiles)]),
        "dd_plan_set_tiles": (i32, [p, i32, ctypes.POINTER(Tiles)]),
        "dd_execute": (i32, [p, p, i32, i64, i64, p, i64, i64, p]),
        "dd_execute_host": (i32, [p, p, i32, i64, i64, p, i64, i64]),
        "dd_execute_noalloc": (i32, [p, p, i32, i64, i64, p, i64, i64, p]),
        "dd_sync": (i32, [p, p]),
        "dd_sync_noalloc": (i32, [p]),
        "dd_execute_detect": (i32, [p, p, i32, i64, i64, p, i64, i64, i32, p, p, p, p, p]),
        "dd_add_peak": (i32, [i32, i32, p, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)]),
        "dd_selftest_noalloc_timeout": (i32, [i64, p]),
        "dd_unpack": (i32, [p, i32, i32, i64, p, i64, p]),
        "dd_detect": (i32, [p, i64, i32, i64, i32, i32, p, p, p, p, p]),
        "dd_frontend": (i32, [p, i64, i32, i64, i32, ctypes.c_double, i32, p, i64, p, i64, p,
                              p, p]),
        "dd_frontend_work_bytes": (i64, [i32, i64, i32, i32]),
        "dd_channelise": (i32, [p, i64, i32, i64, i32, i32, p, i32, ctypes.c_float, p, i64, p]),
        "dd_channelise_nspec": (i64, [i64, i32, i32]),
        "dd_pfb_prototype": (i32, [i32, i32, p]),
        "dd_profile_events": (None, [p, p]),
        "dd_autotune": (i32, [p, p, i32, i64, i64, p, i64, i64, p, i32,
                              ctypes.POINTER(TuneResult), i32, ctypes.POINTER(i32)]),
        "dd_batch_create": (i32, [ctypes.POINTER(p), i32, i32, ctypes.POINTER(p)]),
        "dd_batch_destroy": (None, [p]),
        "dd_batch_set_io": (i32, [p, i32, p, i64, i64, p, i64, i64]),
        "dd_batch_execute": (i32, [p, p]),
        "dd_batch_get_tiles": (i32, [p, ctypes.POINTER(Tiles)]),
        "dd_batch_set_tiles": (i32, [p, ctypes.POINTER(Tiles)]),
        "dd_batch_autotune": (i32, [p, p, i32, ctypes.POINTER(TuneResult), i32,
                                    ctypes.POINTER(i32)]),
        "dd_batch_sync": (i32, [p, p]),
        "dd_server_create": (i32, [ctypes.c_size_t, i32, i32, ctypes.POINTER(p)]),
        "dd_server_add_beam": (i32, [p, p, i64, ctypes.POINTER(i32)]),
        "dd_submit": (i32, [p, i32, p, i64, p, i64, ctypes.POINTER(ctypes.c_uint64)]),
        "dd_poll": (i32, [p, ctypes.c_uint64, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "dd_server_drain": (i32, [p, i64]),
        "dd_server_set_batch_window": (i32, [p, i64]),
        "dd_server_get_stats": (i32, [p, ctypes.POINTER(ServerStats)]),
        "dd_server_destroy": (i32, [p]),
        "dd_selftest_wait_timeout": (i32, [i64, p]),
        "dd_launch_count": (i64, []),
        "dd_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def check(status: int) -> int:
    if status < 0:
        raise DDError(status, lib.dd_last_error().decode(errors="replace"))
    return status


def dtype_code(dtype) -> int:
    """numpy / torch dtype (or 'u8'/'f16'/'f32') -> dd_dtype."""
    name = str(dtype).replace("torch.", "")
    table = {"uint8": DD_U8, "u8": DD_U8, "float16": DD_F16, "f16": DD_F16,
             "float32": DD_F32, "f32": DD_F32}
    if name not in table:
        raise TypeError(f"unsupported input dtype {dtype}")
    return table[name]


def elem_size(code: int) -> int:
    return (1, 2, 4)[code]


def warp_span(code: int, words: int = 8) -> int:
    return 32 * words * (4 // (1, 2, 4)[code])


ADD_KINDS = {"fadd": 0, "iadd": 1, "fadd2": 2}


def add_peak(kind: str = "fadd", ctas_per_sm: int = 4, stream=None) -> tuple[float, float]:
    """dd_add_peak: (adds per second, kernel ms) of the add-throughput
    microbenchmark on the current device ("fadd", "iadd" or "fadd2")."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    rate, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib.dd_add_peak(ADD_KINDS[kind], int(ctas_per_sm), ctypes.c_void_p(s.cuda_stream),
                          ctypes.byref(rate), ctypes.byref(ms)))
    return float(rate.value), float(ms.value)


def launch_count() -> int:
    return int(lib.dd_launch_count())


def unpack(raw, nbits: int, nchan: int, nsamp: int, out, stream=None) -> None:
    """dd_unpack on torch CUDA tensors: raw holds nsamp sigproc-order spectra of
    nchan nbits-bit samples (any dtype, contiguous bytes); out is a uint8
    [nchan][pitch] tensor with contiguous rows.  Asynchronous on stream."""
    import torch
    if not (raw.is_cuda and out.is_cuda):
        raise ValueError("dd_unpack takes CUDA tensors")
    if out.dtype != torch.uint8 or out.dim() != 2 or out.stride(1) != 1 or not raw.is_contiguous():
        raise ValueError("out must be a 2-D uint8 tensor with contiguous rows; raw contiguous")
    s = torch.cuda.current_stream(out.device) if stream is None else stream
    check(lib.dd_unpack(ctypes.c_void_p(raw.data_ptr()), int(nbits), int(nchan), int(nsamp),
                        ctypes.c_void_p(out.data_ptr()), out.stride(0),
                        ctypes.c_void_p(s.cuda_stream)))


def detect(plane, nsamp: int | None = None, nlevels: int = 9, integer_valued: bool = True,
           stream=None):
    """dd_detect on a float32 CUDA plane [ndm][pitch]: returns CUDA tensors
    (mean[ndm], std[ndm], snr[ndm][nlevels], t[ndm][nlevels]).  Asynchronous."""
    import torch
    if not plane.is_cuda or plane.dtype != torch.float32 or plane.dim() != 2 \
            or plane.stride(1) != 1:
        raise ValueError("plane must be a 2-D float32 CUDA tensor with contiguous rows")
    ndm = plane.shape[0]
    nsamp = plane.shape[1] if nsamp is None else nsamp
    dev = plane.device
    mean = torch.empty(ndm, dtype=torch.float64, device=dev)
    std = torch.empty(ndm, dtype=torch.float64, device=dev)
    snr = torch.empty((ndm, nlevels), dtype=torch.float64, device=dev)
    tpk = torch.empty((ndm, nlevels), dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    check(lib.dd_detect(ctypes.c_void_p(plane.data_ptr()), plane.stride(0), ndm, int(nsamp),
                        int(nlevels), int(bool(integer_valued)), ctypes.c_void_p(mean.data_ptr()),
                        ctypes.c_void_p(std.data_ptr()), ctypes.c_void_p(snr.data_ptr()),
                        ctypes.c_void_p(tpk.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
    return mean, std, snr, tpk


def frontend(volts, nint: int, k_clip: float, niter: int = 1, out=None, work=None,
             stream=None):
    """dd_frontend on an int8 CUDA tensor volts [nchan][nsamp_raw][4] (rows
    contiguous): returns (out uint8 [nchan][pitch], mean[nchan], std[nchan]),
    out's first nsamp_raw // nint columns the filterbank.  out may be given
    (uint8, 2-D, contiguous rows, 16-byte aligned pitch); work may be given
    (a CUDA uint8 tensor of at least frontend_work_bytes).  Asynchronous."""
    import torch
    if not volts.is_cuda or volts.dtype != torch.int8 or volts.dim() != 3 \
            or volts.shape[2] != 4 or volts.stride(2) != 1 or volts.stride(1) != 4:
        raise ValueError("volts must be an int8 CUDA tensor [nchan][nsamp_raw][4] with "
                         "contiguous rows")
    nchan, nraw = volts.shape[0], volts.shape[1]
    n = nraw // int(nint) if int(nint) > 0 else 0
    dev = volts.device
    if out is None:
        out = torch.empty((nchan, max(16, (n + 15) // 16 * 16)), dtype=torch.uint8, device=dev)
    elif out.dtype != torch.uint8 or out.dim() != 2 or out.stride(1) != 1 or not out.is_cuda \
            or out.shape[0] < nchan or out.shape[1] < n:
        raise ValueError("out must be a 2-D uint8 CUDA tensor [>= nchan][>= n] with contiguous "
                         "rows")
    need = frontend_work_bytes(nchan, nraw, nint, niter)
    if work is None:
        work = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)
    mean = torch.empty(nchan, dtype=torch.float64, device=dev)
    std = torch.empty(nchan, dtype=torch.float64, device=dev)
    s = torch.cuda.current_stream(dev) if stream is None else stream
    check(lib.dd_frontend(ctypes.c_void_p(volts.data_ptr()), volts.stride(0), nchan, nraw,
                          int(nint), float(k_clip), int(niter), ctypes.c_void_p(out.data_ptr()),
                          out.stride(0), ctypes.c_void_p(work.data_ptr()),
                          work.numel() * work.element_size(), ctypes.c_void_p(mean.data_ptr()),
                          ctypes.c_void_p(std.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
    return out, mean, std


DD_PFB_CF32, DD_PFB_CI8 = 0, 1


def channelise_nspec(nraw: int, nchan_sub: int, ntaps: int) -> int:
    """dd_channelise_nspec; raises DDError for an invalid M, T or nraw."""
    n = int(lib.dd_channelise_nspec(int(nraw), int(nchan_sub), int(ntaps)))
    if n < 0:
        raise DDError(-1, "invalid channeliser shape (nraw, nchan_sub, ntaps)")
    return n


def pfb_prototype(nchan_sub: int, ntaps: int):
    """dd_pfb_prototype: the windowed-sinc prototype as a float32 numpy array."""
    import numpy as np
    h = np.empty(int(nchan_sub) * int(ntaps), dtype=np.float32)
    check(lib.dd_pfb_prototype(int(nchan_sub), int(ntaps), ctypes.c_void_p(h.ctypes.data)))
    return h


def channelise(volts, nchan_sub: int, ntaps: int, coeffs, kind: str = "ci8",
               scale: float = 1.0, out=None, stream=None):
    """dd_channelise on an int8 CUDA tensor volts [nsub][nraw][4] (rows
    contiguous) with float32 CUDA coeffs [nchan_sub*ntaps].  kind "ci8"
    returns int8 [nsub*M][pitch][4] (the front end's element, pitch a
    multiple of 4 spectra), "cf32" float32 [nsub*M][nspec][4]; the first
    nspec columns hold the spectra.  out may be given with that layout.
    Asynchronous."""
    import torch
    if not volts.is_cuda or volts.dtype != torch.int8 or volts.dim() != 3 \
            or volts.shape[2] != 4 or volts.stride(2) != 1 or volts.stride(1) != 4:
        raise ValueError("volts must be an int8 CUDA tensor [nsub][nraw][4] with contiguous "
                         "rows")
    if not coeffs.is_cuda or coeffs.dtype != torch.float32 or not coeffs.is_contiguous():
        raise ValueError("coeffs must be a contiguous float32 CUDA tensor")
    nsub, nraw = volts.shape[0], volts.shape[1]
    M = int(nchan_sub)
    nspec = channelise_nspec(nraw, M, ntaps)
    code = {"ci8": DD_PFB_CI8, "cf32": DD_PFB_CF32}[kind]
    dt = torch.int8 if code == DD_PFB_CI8 else torch.float32
    dev = volts.device
    if out is None:
        cols = max(4, (nspec + 3) // 4 * 4) if code == DD_PFB_CI8 else max(1, nspec)
        out = torch.empty((nsub * M, cols, 4), dtype=dt, device=dev)
    elif out.dtype != dt or out.dim() != 3 or out.shape[2] != 4 or out.stride(2) != 1 \
            or out.stride(1) != 4 or out.shape[0] < nsub * M or out.shape[1] < nspec:
        raise ValueError("out must be a CUDA tensor [>= nsub*M][>= nspec][4] of the kind's "
                         "dtype with contiguous rows")
    s = torch.cuda.current_stream(dev) if stream is None else stream
    check(lib.dd_channelise(ctypes.c_void_p(volts.data_ptr()), volts.stride(0), nsub, nraw, M,
                            int(ntaps), ctypes.c_void_p(coeffs.data_ptr()), code, float(scale),
                            ctypes.c_void_p(out.data_ptr()), out.stride(0) * out.element_size(),
                            ctypes.c_void_p(s.cuda_stream)))
    return out


def frontend_work_bytes(nchan: int, nsamp_raw: int, nint: int, niter: int = 1) -> int:
    """dd_frontend_work_bytes; raises DDError for an invalid shape."""
    b = int(lib.dd_frontend_work_bytes(int(nchan), int(nsamp_raw), int(nint), int(niter)))
    if b < 0:
        raise DDError(-1, "invalid front-end shape (nchan, nsamp_raw, nint, niter)")
    return b


def profile_events(start=None, stop=None) -> None:
    """dd_profile_events with torch.cuda.Event objects (None clears)."""
    h = (lambda e: ctypes.c_void_p(e.cuda_event) if e is not None else None)
    lib.dd_profile_events(h(start), h(stop))


class Plan:
    """dd_plan: the host plan (FP64 delay table rounded to FP32, DM list, maxshift)."""

    def __init__(self, nchan: int, fch1: float, foff: float, tsamp: float, dm_list):
        dms = np.ascontiguousarray(dm_list, dtype=np.float32)
        h = ctypes.c_void_p()
        check(lib.dd_plan(int(nchan), float(fch1), float(foff), float(tsamp),
                          dms.ctypes.data, len(dms), ctypes.byref(h)))
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib.dd_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def maxshift(self) -> int:
        return int(lib.dd_plan_maxshift(self.handle))

    @property
    def nchan(self) -> int:
        return int(lib.dd_plan_nchan(self.handle))

    @property
    def ndm(self) -> int:
        return int(lib.dd_plan_ndm(self.handle))

    def dmshift(self) -> np.ndarray:
        out = np.empty(self.nchan, dtype=np.float32)
        check(lib.dd_plan_dmshift(self.handle, out.ctypes.data))
        return out

    def get_tiles(self, dtype) -> tuple:
        t = Tiles()
        check(lib.dd_plan_get_tiles(self.handle, dtype_code(dtype), ctypes.byref(t)))
        return t.as_tuple()

    def set_tiles(self, dtype, dm_per_thread, dm_warps, time_warps, chan_per_stage,
                  words_per_thread=8):
        t = Tiles(dm_per_thread, dm_warps, time_warps, chan_per_stage, words_per_thread)
        check(lib.dd_plan_set_tiles(self.handle, dtype_code(dtype), ctypes.byref(t)))

    # -- execution --------------------------------------------------------
    def execute_ptr(self, in_ptr: int, dtype: int, in_pitch: int, nsamp_in: int,
                    out_ptr: int, out_pitch: int, nsamp_out: int, stream: int = 0):
        """dd_execute on raw device pointers (asynchronous on stream)."""
        check(lib.dd_execute(self.handle, ctypes.c_void_p(in_ptr), dtype, in_pitch, nsamp_in,
                             ctypes.c_void_p(out_ptr), out_pitch, nsamp_out,
                             ctypes.c_void_p(stream)))

    def execute(self, inp, out, nsamp_in: int | None = None, nsamp_out: int | None = None,
                stream=None):
        """dd_execute on torch CUDA tensors: inp [nchan][pitch] (uint8/float16/float32),
        out [ndm][pitch] float32.  Asynchronous on stream (default: torch's current)."""
        import torch
        if not (inp.is_cuda and out.is_cuda):
            raise ValueError("dd_execute takes CUDA tensors; use execute_host for host arrays")
        if inp.dim() != 2 or out.dim() != 2 or inp.stride(1) != 1 or out.stride(1) != 1:
            raise ValueError("inp and out must be 2-D with contiguous rows")
        if out.dtype != torch.float32:
            raise TypeError("out must be float32")
        nsamp_in = inp.shape[1] if nsamp_in is None else nsamp_in
        nsamp_out = out.shape[1] if nsamp_out is None else nsamp_out
        s = torch.cuda.current_stream(inp.device) if stream is None else stream
        self.execute_ptr(inp.data_ptr(), dtype_code(inp.dtype), inp.stride(0), nsamp_in,
                         out.data_ptr(), out.stride(0), nsamp_out, s.cuda_stream)

    def execute_noalloc_ptr(self, in_ptr: int, dtype: int, in_pitch: int, nsamp_in: int,
                            out_ptr: int, out_pitch: int, nsamp_out: int, stream: int = 0):
        """dd_execute_noalloc on raw device pointers: for callers that cannot
        allocate device memory; uses the library's fixed 1 MiB device array."""
        check(lib.dd_execute_noalloc(self.handle, ctypes.c_void_p(in_ptr), dtype, in_pitch,
                                     nsamp_in, ctypes.c_void_p(out_ptr), out_pitch, nsamp_out,
                                     ctypes.c_void_p(stream)))

    def execute_detect(self, inp, out, nlevels: int = 9, nsamp_in: int | None = None,
                       nsamp_out: int | None = None, stream=None):
        """dd_execute_detect on torch CUDA tensors: inp uint8 [nchan][pitch], out
        float32 [ndm][pitch] (the plane, written as by execute).  Returns CUDA
        tensors (mean[ndm], std[ndm], snr[ndm][nlevels], t[ndm][nlevels]) of the
        fused boxcar search.  Asynchronous on stream."""
        import torch
        if not (inp.is_cuda and out.is_cuda) or inp.dim() != 2 or out.dim() != 2 \
                or inp.stride(1) != 1 or out.stride(1) != 1 or out.dtype != torch.float32:
            raise ValueError("inp/out must be 2-D CUDA tensors with contiguous rows; out float32")
        nsamp_in = inp.shape[1] if nsamp_in is None else nsamp_in
        nsamp_out = out.shape[1] if nsamp_out is None else nsamp_out
        dev = out.device
        ndm = self.ndm
        mean = torch.empty(ndm, dtype=torch.float64, device=dev)
        std = torch.empty(ndm, dtype=torch.float64, device=dev)
        snr = torch.empty((ndm, nlevels), dtype=torch.float64, device=dev)
        tpk = torch.empty((ndm, nlevels), dtype=torch.int64, device=dev)
        s = torch.cuda.current_stream(dev) if stream is None else stream
        check(lib.dd_execute_detect(self.handle, ctypes.c_void_p(inp.data_ptr()),
                                    dtype_code(inp.dtype), inp.stride(0), nsamp_in,
                                    ctypes.c_void_p(out.data_ptr()), out.stride(0), nsamp_out,
                                    int(nlevels), ctypes.c_void_p(mean.data_ptr()),
                                    ctypes.c_void_p(std.data_ptr()),
                                    ctypes.c_void_p(snr.data_ptr()),
                                    ctypes.c_void_p(tpk.data_ptr()),
                                    ctypes.c_void_p(s.cuda_stream)))
        return mean, std, snr, tpk

    @staticmethod
    def sync_noalloc(stream: int = 0) -> None:
        """dd_sync_noalloc: wait for stream and raise if a dd_execute_noalloc
        kernel recorded a failure in the fixed array's status word."""
        check(lib.dd_sync_noalloc(ctypes.c_void_p(stream)))

    def execute_host(self, inp: np.ndarray, out: np.ndarray, nsamp_in: int | None = None,
                     nsamp_out: int | None = None):
        """dd_execute_host on host arrays (numpy or CPU torch tensors, pinned or not)."""
        inp_np = inp.numpy() if hasattr(inp, "numpy") and not isinstance(inp, np.ndarray) else inp
        out_np = out.numpy() if hasattr(out, "numpy") and not isinstance(out, np.ndarray) else out
        if inp_np.ndim != 2 or out_np.ndim != 2 or inp_np.strides[1] != inp_np.itemsize \
                or out_np.strides[1] != 4 or out_np.dtype != np.float32:
            raise ValueError("inp/out must be 2-D with contiguous rows; out float32")
        code = dtype_code(inp_np.dtype)
        nsamp_in = inp_np.shape[1] if nsamp_in is None else nsamp_in
        nsamp_out = out_np.shape[1] if nsamp_out is None else nsamp_out
        check(lib.dd_execute_host(self.handle, inp_np.ctypes.data, code,
                                  inp_np.strides[0] // inp_np.itemsize, nsamp_in,
                                  out_np.ctypes.data, out_np.strides[0] // 4, nsamp_out))

    def autotune(self, inp, out, nsamp_in: int | None = None, nsamp_out: int | None = None,
                 stream=None, reps: int = 2) -> list:
        """dd_autotune on torch CUDA tensors; returns [(tiles, ms), ...] for every
        candidate (ms < 0: rejected) and leaves the fastest shape set on the plan."""
        import torch
        nsamp_in = inp.shape[1] if nsamp_in is None else nsamp_in
        nsamp_out = out.shape[1] if nsamp_out is None else nsamp_out
        s = torch.cuda.current_stream(inp.device) if stream is None else stream
        res = (TuneResult * 512)()
        n = ctypes.c_int(0)
        check(lib.dd_autotune(self.handle, ctypes.c_void_p(inp.data_ptr()), dtype_code(inp.dtype),
                              inp.stride(0), nsamp_in, ctypes.c_void_p(out.data_ptr()),
                              out.stride(0), nsamp_out, ctypes.c_void_p(s.cuda_stream), reps,
                              res, 512, ctypes.byref(n)))
        return [(res[i].tiles.as_tuple(), float(res[i].ms)) for i in range(min(n.value, 512))]

    def sync(self, stream=None) -> None:
        """dd_sync: synchronize the stream and raise if a kernel recorded a failure."""
        h = 0
        if stream is not None:
            h = stream if isinstance(stream, int) else stream.cuda_stream
        check(lib.dd_sync(self.handle, ctypes.c_void_p(h)))


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


class Batch:
    """dd_batch: many beams (own plans and buffers) in one persistent launch,
    replayed from a CUDA graph.  Keeps references to its plans and tensors."""

    def __init__(self, plans, dtype):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[pl.handle.value for pl in self.plans])
        h = ctypes.c_void_p()
        check(lib.dd_batch_create(arr, len(self.plans), dtype_code(dtype), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib.dd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_io(self, beam: int, inp, out, nsamp_in: int | None = None,
               nsamp_out: int | None = None):
        """Bind torch CUDA tensors inp [nchan][pitch] and out [ndm][pitch] to a beam."""
        nsamp_in = inp.shape[1] if nsamp_in is None else nsamp_in
        nsamp_out = out.shape[1] if nsamp_out is None else nsamp_out
        check(lib.dd_batch_set_io(self.handle, beam, ctypes.c_void_p(inp.data_ptr()),
                                  inp.stride(0), nsamp_in, ctypes.c_void_p(out.data_ptr()),
                                  out.stride(0), nsamp_out))
        self._keep[beam] = (inp, out)

    def execute(self, stream=None):
        check(lib.dd_batch_execute(self.handle, ctypes.c_void_p(_stream_handle(stream))))

    def sync(self, stream=None):
        check(lib.dd_batch_sync(self.handle, ctypes.c_void_p(_stream_handle(stream))))

    def get_tiles(self) -> tuple:
        t = Tiles()
        check(lib.dd_batch_get_tiles(self.handle, ctypes.byref(t)))
        return t.as_tuple()

    def set_tiles(self, dm_per_thread, dm_warps, time_warps, chan_per_stage, words_per_thread=8):
        t = Tiles(dm_per_thread, dm_warps, time_warps, chan_per_stage, words_per_thread)
        check(lib.dd_batch_set_tiles(self.handle, ctypes.byref(t)))

    def autotune(self, stream=None, reps: int = 1) -> list:
        res = (TuneResult * 256)()
        n = ctypes.c_int(0)
        check(lib.dd_batch_autotune(self.handle, ctypes.c_void_p(_stream_handle(stream)), reps,
                                    res, 256, ctypes.byref(n)))
        return [(res[i].tiles.as_tuple(), float(res[i].ms)) for i in range(min(n.value, 256))]


class Server:
    """dd_server: streaming blocks of many beams, continuous batching.
    Host buffers are numpy arrays (or CPU torch tensors); the server keeps a
    reference to every out buffer until its ticket is collected."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int, dtype="u8"):
        h = ctypes.c_void_p()
        check(lib.dd_server_create(int(hbm_budget_bytes), int(max_inflight), dtype_code(dtype),
                                   ctypes.byref(h)))
        self._h = h
        self._plans = []
        self._outs = {}

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server destroyed")
        return self._h

    def add_beam(self, plan, block_nsamp: int) -> int:
        bid = ctypes.c_int(-1)
        check(lib.dd_server_add_beam(self.handle, plan.handle, int(block_nsamp),
                                     ctypes.byref(bid)))
        self._plans.append(plan)
        return bid.value

    def submit(self, beam: int, block, out):
        """Queue a block ([nchan][>=B] host array); returns a ticket, or None if busy."""
        b = block.numpy() if hasattr(block, "numpy") and not isinstance(block, np.ndarray) else block
        o = out.numpy() if hasattr(out, "numpy") and not isinstance(out, np.ndarray) else out
        if o.dtype != np.float32 or o.strides[1] != 4 or b.strides[1] != b.itemsize:
            raise ValueError("block rows must be contiguous; out must be float32 rows")
        t = ctypes.c_uint64(0)
        st = lib.dd_submit(self.handle, beam, b.ctypes.data, b.strides[0] // b.itemsize,
                           o.ctypes.data, o.strides[0] // 4, ctypes.byref(t))
        if st == DD_ERR_BUSY:
            return None
        check(st)
        self._outs[t.value] = out
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (first_t, nsamp)."""
        f, n = ctypes.c_int64(0), ctypes.c_int64(0)
        st = lib.dd_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(f), ctypes.byref(n))
        if st == DD_PENDING:
            return None
        self._outs.pop(ticket, None)
        check(st)
        return f.value, n.value

    def set_batch_window(self, microseconds: int):
        check(lib.dd_server_set_batch_window(self.handle, int(microseconds)))

    def drain(self, timeout_ms: int = 60000):
        check(lib.dd_server_drain(self.handle, int(timeout_ms)))

    def stats(self) -> dict:
        s = ServerStats()
        check(lib.dd_server_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None:
            st = lib.dd_server_destroy(self._h)
            self._h = None
            check(st)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
