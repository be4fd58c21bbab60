"""Seeded test inputs: the workloads with pulses dispersed by the oracle's own
shift rule (so the expected planes never depend on the library)."""
from __future__ import annotations

import numpy as np

import filterbank as fb
import oracle


def pulse_delays(table: np.ndarray, pulses) -> list[np.ndarray]:
    return [np.array([oracle.shift(p.dm, table[c]) for c in range(len(table))]) for p in pulses]


def workload_input(w: fb.Workload, kind: str = "u8", pitch_align: int = 16,
                   nsamp_out: int | None = None):
    """(table, dms, S, data[nchan][pitch]) for a workload; rows hold exactly
    nsamp_out + S valid samples, the pitch is padded to pitch_align bytes."""
    nsamp_out = w.nsamp_out if nsamp_out is None else nsamp_out
    table = oracle.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms = w.dm_list()
    S = oracle.maxshift(table, dms)
    nin = nsamp_out + S
    elem = {"u8": 1, "f16": 2, "f32": 4, "f16-frac": 2, "f32-frac": 4}[kind]
    step = max(1, pitch_align // elem)
    pitch = (nin + step - 1) // step * step
    pulses = fb.all_pulses(w)
    data = fb.filterbank(w.nchan, nin, w.seed, pulses, pulse_delays(table, pulses), kind,
                         pitch=pitch)
    return table, dms, S, data


def sample_cells(rng, ndm: int, nsamp_out: int, n: int):
    """Random cells plus the corners and the ragged end of the plane."""
    d = list(rng.integers(0, ndm, size=n))
    t = list(rng.integers(0, nsamp_out, size=n))
    for dd in (0, ndm - 1):
        for tt in (0, 1, nsamp_out - 1, nsamp_out - 2):
            if 0 <= tt < nsamp_out:
                d.append(dd)
                t.append(tt)
    return np.array(d, dtype=np.int32), np.array(t, dtype=np.int64)


_CACHE: dict = {}


def lband_input_and_plane(oracle_lib):
    """The full-size L-band beam (table, dms, S, data) and the oracle's whole
    plane of it (OpenMP build), computed once per test session."""
    if "lband" not in _CACHE:
        w = fb.LBAND
        table, dms, S, data = workload_input(w)
        plane = oracle_lib.dedisperse(np.ascontiguousarray(data[:, :w.nsamp_out + S]), table,
                                      dms, w.nsamp_out, threads=True)
        _CACHE["lband"] = (table, dms, S, data, plane)
    return _CACHE["lband"]
