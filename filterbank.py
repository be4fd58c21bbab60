"""Seeded synthetic filterbank inputs (shared by the tests, the oracle checks
and the benchmark).

This module draws inputs only.  It holds none of the de-dispersion
arithmetic: the per-channel arrival delays of an injected pulse are passed in
by the caller (the tests take them from the oracle, the benchmark from the
library's own plan), so neither side's shift rule lives here.

The paper's test data are sigproc simulations of a dispersed pulse in noise
(Sec. 2, Fig. 1); those files are not available, so every workload below is a
seeded stand-in with the same structure: Gaussian total-intensity noise per
(f,t) cell plus broadband square pulses that follow a dispersion curve.

Recipe (all workloads):
  * noise: FP64 N(128, 16) from numpy's PCG64(seed), drawn row by row
    (channel-major), so chunked generation gives the same values;
  * pulses: +amp counts added in FP64 to in[c][t_p + delay[c] + k], k < width;
  * uint8: round half to even, clip to [0, 255];
  * float16/float32 "same noise" variants: the uint8 values converted exactly;
  * "non-integer" variants: the FP64 values clipped to [0, 255] and rounded
    to float16/float32 (stress cases for the floating-point error bound).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Pulse:
    dm: float          # trial DM the pulse is dispersed with (pc cm^-3)
    t: int             # arrival sample at the top of the band
    width: int         # samples
    amp: float = 40.0  # counts added per sample


@dataclass(frozen=True)
class Workload:
    name: str
    nchan: int
    fch1: float        # MHz, centre of channel 0
    foff: float        # MHz, channel step (negative: descending)
    tsamp: float       # seconds
    nsamp_out: int     # output samples per DM
    ndm: int
    dm_lo: float
    dm_step: float
    seed: int
    pulses: tuple = field(default_factory=tuple)
    random_pulses: int = 0   # extra pulses drawn from the seed (grid DMs)

    def dm_list(self) -> np.ndarray:
        """Trial DMs, built in FP64 and handed over as FP32."""
        return dm_grid(self.dm_lo, self.dm_step, self.ndm)

    def duration_s(self) -> float:
        return self.nsamp_out * self.tsamp

    def adds(self) -> int:
        return self.nchan * self.ndm * self.nsamp_out


def dm_grid(dm_lo: float, dm_step: float, ndm: int) -> np.ndarray:
    return (float(dm_lo) + np.arange(ndm, dtype=np.float64) * float(dm_step)).astype(np.float32)


# The workloads, by what they are.
SMALL = Workload("small-64ch-64dm-8k", nchan=64, fch1=1500.0, foff=-1.0, tsamp=64e-6,
                 nsamp_out=8192, ndm=64, dm_lo=0.0, dm_step=1.0, seed=1,
                 pulses=(Pulse(30.0, 2000, 4, 40.0),))
LBAND = Workload("lband-1024ch-1024dm-131072", nchan=1024, fch1=1500.0, foff=-0.29296875,
                 tsamp=64e-6, nsamp_out=131072, ndm=1024, dm_lo=0.0, dm_step=1.0, seed=2,
                 random_pulses=8)
LOWFREQ = Workload("lowfreq-4096ch-2000dm-262144", nchan=4096, fch1=150.0,
                   foff=-0.00732421875, tsamp=327.68e-6, nsamp_out=262144, ndm=2000,
                   dm_lo=0.0, dm_step=0.05, seed=3,
                   pulses=(Pulse(12.3, 262144 // 3, 4, 40.0),
                           Pulse(57.8, 2 * 262144 // 3, 4, 40.0)))

WORKLOADS = {w.name: w for w in (SMALL, LBAND, LOWFREQ)}


def random_pulses(w: Workload) -> list[Pulse]:
    """Pulses drawn from the seed: grid DMs, t in [0, nsamp_out - 16), widths 1..16."""
    rng = np.random.Generator(np.random.PCG64(w.seed + 7919))
    out = []
    dms = w.dm_list()
    for _ in range(w.random_pulses):
        d = int(rng.integers(0, w.ndm))
        t = int(rng.integers(0, w.nsamp_out - 16))
        width = int(rng.integers(1, 17))
        out.append(Pulse(float(dms[d]), t, width, 40.0))
    return out


def all_pulses(w: Workload) -> list[Pulse]:
    return list(w.pulses) + random_pulses(w)


def noise_rows(seed: int, nchan: int, nsamp: int, chunk_rows: int = 64):
    """Yield (c0, block) with block = FP64 N(128,16) rows c0..c0+len(block)-1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for c0 in range(0, nchan, chunk_rows):
        n = min(chunk_rows, nchan - c0)
        yield c0, rng.normal(128.0, 16.0, size=(n, nsamp))


def add_pulse(block: np.ndarray, c0: int, delays: np.ndarray, pulse: Pulse) -> None:
    """Add a square pulse to rows c0.. of block; delays[c] is its arrival offset
    (samples) in channel c relative to the top of the band."""
    n, nsamp = block.shape
    for r in range(n):
        start = pulse.t + int(delays[c0 + r])
        lo, hi = max(start, 0), min(start + pulse.width, nsamp)
        if lo < hi:
            block[r, lo:hi] += pulse.amp


def to_u8(block: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(block), 0.0, 255.0).astype(np.uint8)


def filterbank(nchan: int, nsamp_in: int, seed: int, pulses=(), delays=(),
               kind: str = "u8", pitch: int | None = None) -> np.ndarray:
    """Seeded (f,t) power array, channel-major [nchan][pitch] (pitch >= nsamp_in;
    padding samples are zero).

    pulses[i] is dispersed with delays[i] (int array [nchan]).
    kind: "u8"; "f16"/"f32" (the uint8 values, exactly); "f16-frac"/"f32-frac"
    (unquantised clipped noise rounded to the storage type).
    """
    pitch = nsamp_in if pitch is None else pitch
    if pitch < nsamp_in:
        raise ValueError("pitch shorter than the row")
    dtype = {"u8": np.uint8, "f16": np.float16, "f32": np.float32,
             "f16-frac": np.float16, "f32-frac": np.float32}[kind]
    out = np.zeros((nchan, pitch), dtype=dtype)
    for c0, block in noise_rows(seed, nchan, nsamp_in):
        for p, dl in zip(pulses, delays):
            add_pulse(block, c0, dl, p)
        if kind.endswith("-frac"):
            out[c0:c0 + len(block), :nsamp_in] = np.clip(block, 0.0, 255.0).astype(dtype)
        else:
            out[c0:c0 + len(block), :nsamp_in] = to_u8(block).astype(dtype)
    return out


def random_filterbank(rng: np.random.Generator, nchan: int, nsamp: int, kind: str = "u8",
                      pitch: int | None = None) -> np.ndarray:
    """Unstructured random rows for fuzz cases: the full uint8 range ("u8", and
    the same integers stored as "f16"/"f32"), or non-integer uniform values in
    [0, 255) rounded to the storage type ("f16-frac"/"f32-frac")."""
    pitch = nsamp if pitch is None else pitch
    dt = {"u8": np.uint8, "f16": np.float16, "f32": np.float32,
          "f16-frac": np.float16, "f32-frac": np.float32}[kind]
    out = np.zeros((nchan, pitch), dtype=dt)
    if kind.endswith("-frac"):
        out[:, :nsamp] = rng.uniform(0.0, 255.0, size=(nchan, nsamp)).astype(dt)
    else:
        out[:, :nsamp] = rng.integers(0, 256, size=(nchan, nsamp), dtype=np.uint8).astype(dt)
    return out


# ---------------------------------------------------------------------------
# Uneven beams for one batched launch (64 beams, seed 4).  Each beam draws its
# channel count from {256, 512, 1024, 4096}, its output length 2^k with k in
# 14..18, its DM count from 128..2048 (DMs 0..ndm-1, step 1), and a band like
# the small or the L-band workload: top channel 1500 MHz, 64 or 300 MHz wide
# (foff = -bandwidth/nchan), tsamp 64 us; 1-3 pulses per beam.
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class BeamSpec:
    index: int
    nchan: int
    fch1: float
    foff: float
    tsamp: float
    nsamp_out: int
    ndm: int
    pulses: tuple

    def dm_list(self) -> np.ndarray:
        return dm_grid(0.0, 1.0, self.ndm)

    def adds(self) -> int:
        return self.nchan * self.ndm * self.nsamp_out


def uneven_beams(seed: int = 4, nbeams: int = 64, scale_nsamp: int = 1) -> list[BeamSpec]:
    """The batched-beams workload; scale_nsamp > 1 divides every output length
    (a smaller case with the same mix, for quick tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(nbeams):
        nchan = int(rng.choice([256, 512, 1024, 4096]))
        nsamp = int(2 ** int(rng.integers(14, 19))) // scale_nsamp
        ndm = int(rng.integers(128, 2049))
        bw = float(rng.choice([64.0, 300.0]))
        npulse = int(rng.integers(1, 4))
        pulses = tuple(Pulse(float(rng.integers(0, ndm)), int(rng.integers(0, max(1, nsamp - 16))),
                             int(rng.integers(1, 17)), 40.0) for _ in range(npulse))
        out.append(BeamSpec(i, nchan, 1500.0, -bw / nchan, 64e-6, nsamp, ndm, pulses))
    return out


class NoisePool:
    """Seeded pool of uint8 N(128, 16) noise (round half to even, clipped);
    beam rows are slices of it at seeded offsets -- Gaussian values per sample
    at memory-copy speed for multi-GB batches."""

    def __init__(self, seed: int, size: int = 1 << 26):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.pool = to_u8(rng.normal(128.0, 16.0, size=size))
        self.rng = np.random.Generator(np.random.PCG64(seed + 1))

    def rows(self, nchan: int, nsamp: int, pitch: int | None = None) -> np.ndarray:
        pitch = nsamp if pitch is None else pitch
        if nsamp > len(self.pool):
            raise ValueError("row longer than the noise pool")
        out = np.zeros((nchan, pitch), dtype=np.uint8)
        offs = self.rng.integers(0, len(self.pool) - nsamp + 1, size=nchan)
        for c, o in enumerate(offs):
            out[c, :nsamp] = self.pool[o:o + nsamp]
        return out


def add_pulse_u8(data: np.ndarray, delays: np.ndarray, pulse: Pulse, nsamp: int) -> None:
    """Add a square pulse to uint8 rows in place, saturating at 255."""
    for c in range(data.shape[0]):
        start = pulse.t + int(delays[c])
        lo, hi = max(start, 0), min(start + pulse.width, nsamp)
        if lo < hi:
            seg = data[c, lo:hi].astype(np.int32) + int(pulse.amp)
            data[c, lo:hi] = np.minimum(seg, 255).astype(np.uint8)


# ---------------------------------------------------------------------------
# Dual-polarisation voltages for the front end (Stokes I, integration, RFI
# clipping, quantisation).  Each raw sample is four int8 values (Xre, Xim,
# Yre, Yim).  Recipe:
#   * four seeded pools (PCG64(seed)) of N(0, sigma) components, sigma in
#     (8, 12, 18, 27), rounded half to even and clipped to [-128, 127]; channel
#     c takes pool which[c] (a stand-in for the bandpass) from raw-sample
#     offset offs[c] (both drawn from PCG64(seed + 1));
#   * RFI: narrowband tones -- about one channel in 64 holds (100, 0, 100, 0)
#     over a seeded range of 0.5..4 % of its samples -- and two broadband
#     impulses, every channel (50, 50, 50, 50) over a seeded range of 0.1 % of
#     the samples.
# The paper names the steps of its front end but not its signal levels; these
# put the RFI far above mean + 4 std of the integrated power.
# ---------------------------------------------------------------------------

VOLT_SIGMAS = (8.0, 12.0, 18.0, 27.0)


@dataclass(frozen=True)
class VoltageLayout:
    nchan: int
    nraw: int
    which: np.ndarray      # pool index per channel
    offs: np.ndarray       # raw-sample offset into the pool per channel
    tones: tuple           # (channel, r0, r1)
    impulses: tuple        # (r0, r1), all channels


class VoltagePool:
    def __init__(self, seed: int, size: int = 1 << 22):
        rng = np.random.Generator(np.random.PCG64(seed))
        self.seed = seed
        self.size = size
        self.pools = np.stack([
            np.clip(np.rint(rng.normal(0.0, s, size=(size, 4))), -128, 127).astype(np.int8)
            for s in VOLT_SIGMAS])

    def layout(self, nchan: int, nraw: int, rfi: bool = True) -> VoltageLayout:
        if nraw > self.size:
            raise ValueError("rows longer than the voltage pool")
        rng = np.random.Generator(np.random.PCG64(self.seed + 1))
        which = rng.integers(0, len(VOLT_SIGMAS), size=nchan)
        offs = rng.integers(0, self.size - nraw + 1, size=nchan)
        tones, impulses = [], []
        if rfi and nraw > 0:
            for c in rng.choice(nchan, size=max(1, nchan // 64), replace=False):
                ln = max(1, int(nraw * rng.uniform(0.005, 0.04)))
                r0 = int(rng.integers(0, nraw - ln + 1))
                tones.append((int(c), r0, r0 + ln))
            for _ in range(2):
                ln = max(1, nraw // 1000)
                r0 = int(rng.integers(0, nraw - ln + 1))
                impulses.append((r0, r0 + ln))
        return VoltageLayout(nchan, nraw, which, offs, tuple(tones), tuple(impulses))

    def rows(self, lay: VoltageLayout, chans=None) -> np.ndarray:
        """int8 [len(chans)][nraw][4] on the host (all channels by default)."""
        chans = range(lay.nchan) if chans is None else chans
        out = np.empty((len(chans), lay.nraw, 4), dtype=np.int8)
        for i, c in enumerate(chans):
            o = int(lay.offs[c])
            out[i] = self.pools[lay.which[c], o:o + lay.nraw]
            for tc, r0, r1 in lay.tones:
                if tc == c:
                    out[i, r0:r1] = (100, 0, 100, 0)
            for r0, r1 in lay.impulses:
                out[i, r0:r1] = (50, 50, 50, 50)
        return out

    def rows_torch(self, lay: VoltageLayout, device, pitch_bytes: int | None = None):
        """The same rows built on a torch device (copies and fills only):
        an int8 tensor [nchan][pitch_bytes] whose first 4*nraw bytes of row c
        are rows(lay)[c]; returned with the [nchan][nraw][4] view."""
        import torch
        pitch = 4 * lay.nraw if pitch_bytes is None else pitch_bytes
        buf = torch.zeros((lay.nchan, pitch), dtype=torch.int8, device=device)
        pools = torch.from_numpy(self.pools.reshape(len(VOLT_SIGMAS), -1)).to(device)
        for c in range(lay.nchan):
            o = 4 * int(lay.offs[c])
            buf[c, :4 * lay.nraw] = pools[int(lay.which[c]), o:o + 4 * lay.nraw]
        view = buf[:, :4 * lay.nraw].unflatten(1, (lay.nraw, 4))
        tone = torch.tensor([100, 0, 100, 0], dtype=torch.int8, device=device)
        for c, r0, r1 in lay.tones:
            view[c, r0:r1] = tone
        for r0, r1 in lay.impulses:
            view[:, r0:r1] = 50
        return buf, view

    def long_rows_torch(self, nrows: int, nraw: int, device, chunk: int = 1 << 21):
        """int8 [nrows][nraw][4] on a torch device for rows longer than the
        pool (copies only): row r takes pool which[r] and is filled chunk by
        chunk from seeded pool offsets (PCG64(seed + 2)).  No RFI."""
        import torch
        rng = np.random.Generator(np.random.PCG64(self.seed + 2))
        which = rng.integers(0, len(VOLT_SIGMAS), size=nrows)
        chunk = min(chunk, self.size)
        nchunk = (nraw + chunk - 1) // chunk
        offs = rng.integers(0, self.size - chunk + 1, size=(nrows, max(nchunk, 1)))
        pools = torch.from_numpy(self.pools).to(device)        # [4][size][4]
        out = torch.empty((nrows, nraw, 4), dtype=torch.int8, device=device)
        for r in range(nrows):
            for k in range(nchunk):
                a, b = k * chunk, min(nraw, (k + 1) * chunk)
                o = int(offs[r, k])
                out[r, a:b] = pools[int(which[r]), o:o + (b - a)]
        return out


# ---------------------------------------------------------------------------
# Channeliser workloads (subband voltages for the polyphase filter bank).
# Each subband row is int8 (Xre, Xim, Yre, Yim) noise from the voltage pools
# above, filled chunk by chunk (VoltagePool.long_rows_torch).  The scale
# brings a pool of sigma 18 to about 16 codes per component after the
# prototype's gain (sqrt(sum h^2) is 3.8 for 16 x 8 taps, 15.2 for 256 x 8).
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class ChanneliserWorkload:
    name: str
    nsub: int      # subbands (rows of raw samples)
    M: int         # channels per subband
    T: int         # taps per branch
    nspec: int     # output spectra per subband
    seed: int
    scale: float   # int8 output: codes = rint(value * scale)

    @property
    def nraw(self) -> int:
        return (self.nspec + self.T - 1) * self.M

    def raw_bytes(self) -> int:
        return 4 * self.nsub * self.nraw


# 64 subbands x 16 channels = the 1024 channels of the L-band front-end block
# (147628 output samples x 16 raw samples each per channel).
CHANNELISER_LBAND = ChanneliserWorkload("pfb-64sub-16ch-8tap", nsub=64, M=16, T=8,
                                        nspec=147628 * 16, seed=6, scale=0.25)
# The same 1024 channels from 4 wide subbands of 256 channels.
CHANNELISER_WIDE = ChanneliserWorkload("pfb-4sub-256ch-8tap", nsub=4, M=256, T=8,
                                       nspec=147628 * 16, seed=7, scale=0.0625)
