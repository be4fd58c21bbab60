"""Benchmark: brute-force incoherent de-dispersion on GB300.

One step = one de-dispersion of the 4096-channel low-frequency beam (120-150
MHz, tsamp 327.68 us, 2000 trial DMs 0..99.95 step 0.05, 262144 output
samples plus maxshift, uint8 seeded noise with pulses at DM 12.3 and 57.8)
through the C ABI, with the input resident in HBM.  The line reports
channel*DM*sample adds/s, the roofline of the dominant kernel against a
measured add peak (an in-library microbenchmark), the real-time factor, an
end-to-end number through the host-buffer entry point, and the CPU oracle's
throughput on bounded samples (single-threaded and OpenMP).  Sections on the
same line: the same beam stored as FP16 and FP32 (precision), the L-band
beam, detection, the 64-beam batch, serving, unpacking, the front end, the
channeliser and a compact form of the Fig. 4 sweeps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload lowfreq|lband|small] [--dtype u8|f16|f32]

Under torchrun (N > 1) every rank de-disperses its own independent beam (no
data-path collective; weak scaling); timing is the max over ranks.
`--impl reference` times the CPU oracle (the only reference this path has) on
a bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import filterbank as fb  # noqa: E402

METRIC = ("channel·DM·sample adds/s and % roofline on 1 GB300; real-time factor; "
          "p50/p99 block latency")
UNIT = "adds/s"
WORKLOADS = {"small": fb.SMALL, "lband": fb.LBAND, "lowfreq": fb.LOWFREQ}
ADD_LANES_PER_SM = 128  # FP32/INT32 lanes per SM per clock (nominal figure beside the measured one)
# Output samples the autotuner times each candidate on (a prefix of the
# beam's output; the full beam when it is shorter).
TUNE_NSAMP = 65536


# DRAM traffic of one de-dispersion step from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of its launches), valid only
# for the kernel and launch code it was taken on (sha256 of csrc/dd_kernel.cuh
# and csrc/dd_launch.cpp) and the same workload, dtype and tile shape; any
# other run reports traffic null.
TRAFFIC_SOURCE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum "
                  "--clock-control none, one step's de-dispersion launches")
PROFILED_TRAFFIC: list[dict] = [
    # one step, 4096-channel beam, tiles (4,12,1,8,8): a single launch of 42 x 256 tiles
    {"workload": "lowfreq-4096ch-2000dm-262144", "dtype": "u8", "tiles": [4, 12, 1, 8, 8],
     "code_sha256": "81b799d99197287efbc40fdfa738662c596bf5a398684d03d44737ff4d1d8816",
     "bytes": 4790403072 + 2875413504, "compulsory": 1203281920 + 2097152000},
    # one step, the same beam stored as FP16, tiles (4,12,1,12,8): a single launch
    {"workload": "lowfreq-4096ch-2000dm-262144", "dtype": "f16", "tiles": [4, 12, 1, 12, 8],
     "code_sha256": "81b799d99197287efbc40fdfa738662c596bf5a398684d03d44737ff4d1d8816",
     "bytes": 20705216768 + 2230952960, "compulsory": 2406563840 + 2097152000},
    # one step, the same beam stored as FP32, tiles (4,6,2,24,8): main launch (1992 DMs) +
    # remainder (8 DMs)
    {"workload": "lowfreq-4096ch-2000dm-262144", "dtype": "f32", "tiles": [4, 6, 2, 24, 8],
     "code_sha256": "81b799d99197287efbc40fdfa738662c596bf5a398684d03d44737ff4d1d8816",
     "bytes": (86389575424 + 2099985408) + (4307168768 + 7886080),
     "compulsory": 4813127680 + 2097152000},
    # one step, L-band beam, tiles (4,12,1,8,8): main launch (1008 DMs) + remainder (16 DMs)
    {"workload": "lband-1024ch-1024dm-131072", "dtype": "u8", "tiles": [4, 12, 1, 8, 8],
     "code_sha256": "81b799d99197287efbc40fdfa738662c596bf5a398684d03d44737ff4d1d8816",
     "bytes": (153392640 + 506828544) + (135646464 + 358912),
     "compulsory": 151171072 + 536870912},
]


def _sha256(*parts) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in parts:
        with open(os.path.join(ROOT, "paper_1111_6399_gb300", "csrc", rel), "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    return h.hexdigest()


def profiled_traffic(workload: str, dtype: str, tiles) -> dict | None:
    digest = _sha256("dd_kernel.cuh", "dd_launch.cpp")
    for rec in PROFILED_TRAFFIC:
        if (rec["code_sha256"] == digest and rec["workload"] == workload
                and rec["dtype"] == dtype and list(rec["tiles"]) == list(tiles)):
            return rec
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def nominal_add_peak(sms: int, sm_mhz: float) -> float:
    """Nominal plain-ALU add peak: SMs x 128 lanes x clock (adds/s)."""
    return sms * ADD_LANES_PER_SM * sm_mhz * 1e6


def measured_add_peak(dd, torch, dev) -> dict:
    """The add-throughput microbenchmark (dd_add_peak) for each add kind, with
    the SM clock sampled while it runs; the roofline denominator is the
    largest measured rate."""
    res = {}
    with ClockSampler(dev.index or 0) as clk:
        for _ in range(3):  # a few seconds of load so the clock sampler sees it
            for kind in ("fadd", "iadd", "fadd2"):
                rate, ms = dd.add_peak(kind, 4)
                if kind not in res or rate > res[kind]["adds_per_s"]:
                    res[kind] = {"adds_per_s": rate, "ms": ms}
    best = max(res, key=lambda k: res[k]["adds_per_s"])
    return {"kinds": res, "best": best, "adds_per_s": res[best]["adds_per_s"],
            "clocks": clk.summary()}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_input(w: fb.Workload, dmshift: np.ndarray, maxshift: int):
    """Seeded uint8 beam; pulses dispersed with the plan's own shifts."""
    nin = w.nsamp_out + maxshift
    pitch = (nin + 15) // 16 * 16
    pulses = fb.all_pulses(w)
    delays = [np.trunc((np.float32(p.dm) * dmshift).astype(np.float32)).astype(np.int64)
              for p in pulses]
    return fb.filterbank(w.nchan, nin, w.seed, pulses, delays, pitch=pitch), nin


def prepare_oracle_sample(w: fb.Workload, budget_s: float = 12.0, threads: bool = True) -> dict:
    """A bounded sample of the workload for the oracle -- its OpenMP build (DM
    loop over all host cores) or, with threads=False, the single-threaded
    oracle proper: all channels, a spread of the DMs, a slice of time, sized
    from a short calibration run to take about budget_s."""
    import oracle
    table = oracle.dmshift(w.nchan, w.fch1, w.foff, w.tsamp)
    dms_all = w.dm_list()
    S = oracle.maxshift(table, dms_all)
    rng = np.random.default_rng(w.seed)
    cores = (os.cpu_count() or 1) if threads else 1
    nsamp = min(w.nsamp_out, 4096 if threads else 1024)
    ndm = max(1, min(w.ndm, 2 * cores))
    data = rng.integers(0, 256, size=(w.nchan, nsamp + S), dtype=np.uint8)
    t = time.perf_counter()
    oracle.dedisperse(data, table, dms_all[np.linspace(0, w.ndm - 1, ndm).astype(int)], nsamp,
                      threads=threads)
    rate = w.nchan * ndm * nsamp / max(time.perf_counter() - t, 1e-4)
    target = rate * budget_s
    ndm = int(max(1, min(w.ndm, target / (w.nchan * nsamp))))
    nsamp = int(max(1024, min(w.nsamp_out, target / (w.nchan * ndm))))
    return {"data": rng.integers(0, 256, size=(w.nchan, nsamp + S), dtype=np.uint8),
            "table": table, "sel": dms_all[np.linspace(0, w.ndm - 1, ndm).astype(int)],
            "nsamp": nsamp, "ndm": ndm, "cores": cores, "threads": threads}


def time_oracle_sample(w: fb.Workload, prep: dict) -> dict:
    """One timed oracle run over a prepared sample."""
    import oracle
    t = time.perf_counter()
    oracle.dedisperse(prep["data"], prep["table"], prep["sel"], prep["nsamp"],
                      threads=prep["threads"])
    dt = time.perf_counter() - t
    adds = w.nchan * prep["ndm"] * prep["nsamp"]
    how = "OpenMP over DMs" if prep["threads"] else "single-threaded"
    return {"value": adds / dt, "unit": UNIT, "cores": prep["cores"], "kind": "oracle",
            "sample": f"{w.nchan} channels x {prep['ndm']} of {w.ndm} DMs x {prep['nsamp']} "
                      f"samples ({adds:.3g} adds, {dt:.2f} s, {how})",
            "seconds": dt, "sample_adds": adds}


def cpu_oracle_sample(w: fb.Workload) -> dict:
    """The oracle's OpenMP build on a ~10 s sample (the line's value, all host
    cores) and the single-threaded oracle on a ~6 s sample."""
    omp = time_oracle_sample(w, prepare_oracle_sample(w, 10.0, threads=True))
    one = time_oracle_sample(w, prepare_oracle_sample(w, 6.0, threads=False))
    for r in (omp, one):
        r.pop("seconds")
        r.pop("sample_adds")
    return {**omp, "single_thread": one}


def _plan_delays(table: np.ndarray, pulses):
    return [np.trunc((np.float32(p.dm) * table).astype(np.float32)).astype(np.int64)
            for p in pulses]


def batch_section(dd, torch, dev, steps: int, tiles=None):
    """64 uneven beams: one persistent launch replayed from a CUDA graph versus
    one plain single-beam launch per beam, on the same device buffers."""
    specs = fb.uneven_beams()
    pool = fb.NoisePool(4)
    plans, ins, outs_b, outs_p, nins = [], [], [], [], []
    for sp in specs:
        plan = dd.Plan(sp.nchan, sp.fch1, sp.foff, sp.tsamp, sp.dm_list())
        nin = sp.nsamp_out + plan.maxshift
        data = pool.rows(sp.nchan, nin, (nin + 15) // 16 * 16)
        for p, dl in zip(sp.pulses, _plan_delays(plan.dmshift(), sp.pulses)):
            fb.add_pulse_u8(data, dl, p, nin)
        plans.append(plan)
        nins.append(nin)
        ins.append(torch.from_numpy(data).to(dev))
        outs_b.append(torch.empty((sp.ndm, (sp.nsamp_out + 3) // 4 * 4), device=dev))
        outs_p.append(torch.empty_like(outs_b[-1]))
    batch = dd.Batch(plans, "u8")
    for i, sp in enumerate(specs):
        batch.set_io(i, ins[i], outs_b[i], nsamp_in=nins[i], nsamp_out=sp.nsamp_out)
    if tiles is not None:  # the headline's tuned shape, for the batch and every single beam
        try:
            batch.set_tiles(*tiles)
            for pl in plans:
                pl.set_tiles("u8", *tiles)
        except dd.DDError:
            pass
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        batch.execute(stream)           # eager run + capture, then replays
        for i, sp in enumerate(specs):
            plans[i].execute(ins[i], outs_p[i], nsamp_in=nins[i], nsamp_out=sp.nsamp_out,
                             stream=stream)
    batch.sync(stream)
    reps = max(2, min(steps, 5))
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    for _ in range(reps):
        batch.execute(stream)
    e[1].record(stream)
    for _ in range(reps):
        for i, sp in enumerate(specs):
            plans[i].execute(ins[i], outs_p[i], nsamp_in=nins[i], nsamp_out=sp.nsamp_out,
                             stream=stream)
    e[2].record(stream)
    torch.cuda.synchronize(dev)
    t_batch = e[0].elapsed_time(e[1]) / reps / 1e3
    t_plain = e[1].elapsed_time(e[2]) / reps / 1e3
    same = all(torch.equal(outs_b[i][:, :sp.nsamp_out], outs_p[i][:, :sp.nsamp_out])
               for i, sp in enumerate(specs))
    adds = sum(sp.adds() for sp in specs)
    res = {"workload": "64 uneven beams (nchan 256-4096, nsamp 2^14-2^18, ndm 128-2048)",
           "adds": adds, "batched_adds_per_s": adds / t_batch,
           "per_beam_adds_per_s": adds / t_plain, "speedup": t_plain / t_batch,
           "batched_ms": t_batch * 1e3, "per_beam_ms": t_plain * 1e3,
           "identical_outputs": bool(same), "tiles": batch.get_tiles(),
           "launch": "one persistent kernel, CUDA graph replay"}
    del ins, outs_b, outs_p
    batch.close()
    torch.cuda.empty_cache()
    return res


def unpack_section(dd, torch, dev, w: fb.Workload, nin: int, hbm_gbs: float, reps: int = 20):
    """dd_unpack on one beam's worth of sigproc spectra (nin spectra of
    w.nchan channels) at 8, 4, 2 and 1 bits: HBM-bound, bytes read + written
    per launch over CUDA-event time, against the measured copy bandwidth.
    Each launch moves more than L2 holds except at 1-2 bits, where the timed
    launches alternate between two input/output pairs."""
    res = {"workload": f"{nin} spectra x {w.nchan} channels -> uint8 [{w.nchan}][{nin}]",
           "bound": "hbm", "peak_gbs": hbm_gbs}
    pitch = (nin + 15) // 16 * 16
    g = torch.Generator(device=dev)
    g.manual_seed(6)
    outs = [torch.empty((w.nchan, pitch), dtype=torch.uint8, device=dev) for _ in range(2)]
    for nbits in (8, 4, 2, 1):
        nbytes = nin * w.nchan * nbits // 8
        raws = [torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=dev, generator=g)
                for _ in range(2)]
        for i in range(3):
            dd.unpack(raws[i % 2], nbits, w.nchan, nin, outs[i % 2])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for i in range(reps):
            dd.unpack(raws[i % 2], nbits, w.nchan, nin, outs[i % 2])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        moved = nbytes + w.nchan * nin
        res[f"{nbits}bit"] = {"ms": ms, "gbs": moved / ms / 1e6,
                              "frac": moved / ms / 1e6 / hbm_gbs, "bytes": moved}
        del raws
    return res


def frontend_section(dd, torch, dev, w: fb.Workload, nin: int, hbm_gbs: float, nint: int = 16,
                     niter: int = 3, k_clip: float = 4.0, reps: int = 10, nchan: int = 0):
    """dd_frontend producing the beam's uint8 input block (w.nchan channels x
    nin spectra) from nint raw dual-polarisation samples per spectrum, with
    niter clipping passes: HBM-bound.  'compulsory' bytes are the voltages
    read and the codes written; 'moved' adds the integrated powers written
    once and read niter times.  Voltages (several GB) exceed L2.  nchan > 0
    takes only the first nchan channels (a smaller case for profiling)."""
    nchan = w.nchan if nchan <= 0 else min(nchan, w.nchan)
    pool = fb.VoltagePool(23)
    lay = pool.layout(nchan, nin * nint)
    buf, v = pool.rows_torch(lay, dev)
    pitch = (nin + 15) // 16 * 16
    out = torch.empty((nchan, pitch), dtype=torch.uint8, device=dev)
    work = torch.empty(dd.frontend_work_bytes(nchan, nin * nint, nint, niter),
                       dtype=torch.uint8, device=dev)
    for _ in range(3):
        dd.frontend(v, nint, k_clip, niter, out=out, work=work)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    n0 = dd.launch_count()
    e0.record()
    for _ in range(reps):
        _, mean, std = dd.frontend(v, nint, k_clip, niter, out=out, work=work)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    launches = (dd.launch_count() - n0) // reps
    volts_b = nchan * nin * nint * 4
    codes_b = nchan * nin
    compulsory = volts_b + codes_b
    moved = compulsory + nchan * nin * 4 * (1 + niter)
    std_h = std.cpu().numpy()
    res = {"workload": f"{nchan} channels x {nin} spectra x {nint} raw samples "
                       f"(int8 Xre,Xim,Yre,Yim), {niter} clipping passes at {k_clip} sigma",
           "bound": "hbm", "ms": ms, "peak_gbs": hbm_gbs, "launches": launches,
           "compulsory_bytes": compulsory, "moved_bytes": moved,
           "gbs": compulsory / ms / 1e6, "frac": compulsory / ms / 1e6 / hbm_gbs,
           "moved_gbs": moved / ms / 1e6, "moved_frac": moved / ms / 1e6 / hbm_gbs,
           "spectra_per_s": nin / (ms / 1e3),
           "real_time_factor": (nin * w.tsamp) / (ms / 1e3),
           "std_range": [float(std_h.min()), float(std_h.max())]}
    del buf, v, out, work
    torch.cuda.empty_cache()
    return res


def channeliser_section(dd, torch, dev, hbm_gbs: float, sm_mhz: float, sms: int,
                        nsub: int = 0, reps: int = 10, which: str = "both") -> dict:
    """dd_channelise (int8 output, the front end's element) on the two
    channeliser workloads: 64 subbands x 16 channels and 4 subbands x 256
    channels, 8 taps, the 1024 channels of the L-band front-end block.
    Algorithmic bytes: the raw words read and the codes written; algorithmic
    flops per spectrum and polarisation: 4*M*T for the FIR (a real tap times
    a complex sample as two fused multiply-adds) and 5*M*log2(M) for the FFT.
    The FP32 peak is the SM count x 128 lanes x 2 flops x the measured
    maximum SM clock.  Inputs (9.7 GB) exceed L2.  nsub > 0 keeps the first nsub
    subbands of each workload (a smaller case for profiling); which picks one
    workload ("16ch", "256ch") or both."""
    res = {"fp32_peak_tflops": sms * ADD_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12,
           "peak_gbs": hbm_gbs}
    for w in (fb.CHANNELISER_LBAND, fb.CHANNELISER_WIDE):
        if which != "both" and which != f"{w.M}ch":
            continue
        ns = w.nsub if nsub <= 0 else min(nsub, w.nsub)
        pool = fb.VoltagePool(w.seed)
        v = pool.long_rows_torch(ns, w.nraw, dev)
        h = torch.from_numpy(dd.pfb_prototype(w.M, w.T)).to(dev)
        nspec = dd.channelise_nspec(w.nraw, w.M, w.T)
        out = torch.empty((ns * w.M, (nspec + 3) // 4 * 4, 4), dtype=torch.int8, device=dev)
        for _ in range(3):
            dd.channelise(v, w.M, w.T, h, kind="ci8", scale=w.scale, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        n0 = dd.launch_count()
        e0.record()
        for _ in range(reps):
            dd.channelise(v, w.M, w.T, h, kind="ci8", scale=w.scale, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        launches = (dd.launch_count() - n0) // reps
        nbytes = 4 * ns * w.nraw + 4 * ns * w.M * nspec
        flops = ns * nspec * 2 * (4 * w.M * w.T + 5 * w.M * math.log2(w.M))
        gbs = nbytes / ms / 1e6
        tflops = flops / ms / 1e9
        t_hbm = nbytes / (hbm_gbs * 1e9)
        t_fp = flops / (res["fp32_peak_tflops"] * 1e12)
        res[w.name] = {
            "workload": f"{ns} subbands x {w.M} channels x {w.T} taps, {nspec} spectra per "
                        f"subband, int8 (Xre,Xim,Yre,Yim) in and out",
            "ms": ms, "launches": launches, "bytes": nbytes, "gbs": gbs,
            "hbm_frac": gbs / hbm_gbs, "flops": flops, "tflops": tflops,
            "fp32_frac": tflops / res["fp32_peak_tflops"],
            "bound": "hbm" if t_hbm >= t_fp else "fp32",
            "roofline_frac": max(t_hbm, t_fp) / (ms / 1e3),
            "raw_samples_per_s": ns * w.nraw / (ms / 1e3)}
        del v, out
        torch.cuda.empty_cache()
    return res


def detect_section(dd, torch, out, w: fb.Workload, hbm_gbs: float, dms, reps: int = 20):
    """dd_detect (boxcar widths 1..256) on the beam's own (DM,t) plane: the
    plane (FP32, larger than L2) is read once per launch; bytes over
    CUDA-event time against the measured copy bandwidth.  Also reports the
    strongest detection."""
    for _ in range(3):
        res = dd.detect(out, nlevels=9, integer_valued=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        res = dd.detect(out, nlevels=9, integer_valued=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = w.ndm * w.nsamp_out * 4
    snr = res[2].cpu().numpy()
    tpk = res[3].cpu().numpy()
    d, lev = np.unravel_index(int(np.argmax(snr)), snr.shape)
    return {"workload": f"(DM,t) plane {w.ndm} x {w.nsamp_out} FP32, widths 1..256",
            "bound": "hbm", "ms": ms, "gbs": nbytes / ms / 1e6, "peak_gbs": hbm_gbs,
            "frac": nbytes / ms / 1e6 / hbm_gbs, "bytes": nbytes,
            "launches": 2, "best": {"dm": float(dms[d]), "width": 1 << int(lev),
                                    "t": int(tpk[d, lev]), "snr": float(snr[d, lev])}}


def fused_detect_section(dd, torch, dev, w: fb.Workload, reps: int = 10) -> dict:
    """dd_execute_detect (the boxcar search fused into the de-dispersion
    kernel) against dd_execute followed by dd_detect on the same beam and
    plane, both timed with CUDA events over `reps` steps (inputs larger than
    L2); the two give identical search results, which is checked."""
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    host, nin = beam_input(w, plan, "u8")
    x = torch.from_numpy(host).to(dev)
    out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def fused():
        return plan.execute_detect(x, out, nlevels=9, nsamp_in=nin, stream=stream)

    def separate():
        plan.execute(x, out, nsamp_in=nin, stream=stream)
        return dd.detect(out, nlevels=9, integer_valued=True, stream=stream)

    res = {}
    for name, fn in (("fused", fused), ("separate", separate)):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = dd.launch_count()
        e0.record(stream)
        for _ in range(reps):
            r = fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        res[name] = {"ms": e0.elapsed_time(e1) / reps,
                     "launches": (dd.launch_count() - n0) // reps,
                     "result": [t.clone() for t in r]}
    same = all(torch.equal(a, b) for a, b in zip(res["fused"]["result"],
                                                 res["separate"]["result"]))
    snr = res["fused"]["result"][2].cpu().numpy()
    tpk = res["fused"]["result"][3].cpu().numpy()
    d, lev = np.unravel_index(int(np.argmax(snr)), snr.shape)
    out_d = {"workload": w.name, "tiles": plan.get_tiles("u8"),
             "fused_ms": res["fused"]["ms"], "separate_ms": res["separate"]["ms"],
             "fused_launches": res["fused"]["launches"],
             "separate_launches": res["separate"]["launches"],
             "saved_ms": res["separate"]["ms"] - res["fused"]["ms"],
             "identical_results": bool(same),
             "best": {"dm": float(w.dm_list()[d]), "width": 1 << int(lev), "t": int(tpk[d, lev]),
                      "snr": float(snr[d, lev])}}
    del x, out
    torch.cuda.empty_cache()
    return out_d


def serving_section(dd, torch, dev, seconds: float = 8.0, speed: float = 1.25):
    """128 streaming L-band beams (1024 channels, 1024 DMs, blocks of 65536
    samples = 4.194 s) served with continuous batching (the server's default
    batching window, 1/64 of a block's duration): Poisson arrivals at
    `speed` x the aggregate real-time rate for `seconds`, then a saturating
    phase (blocks submitted as fast as the server accepts them)."""
    w = fb.LBAND
    B, nbeams = 65536, 128
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    block_s = B * w.tsamp
    rng = np.random.default_rng(5)
    pool = fb.NoisePool(5)
    blocks = [pool.rows(w.nchan, B) for _ in range(4)]
    slots = 8
    srv = dd.Server(24 << 30, slots, "u8")
    ids = [srv.add_beam(plan, B) for _ in range(nbeams)]
    outs = [torch.empty((w.ndm, B), dtype=torch.float32).pin_memory() for _ in range(2 * slots)]
    free = list(range(len(outs)))
    pending = {}

    def reap():
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                free.append(pending.pop(t))

    def submit(beam, k):
        while not free:
            reap()
            time.sleep(0.0002)
        o = free.pop()
        t = srv.submit(ids[beam], blocks[k % 4], outs[o])
        if t is None:
            free.append(o)
            return False
        pending[t] = o
        return True

    # real-time phase: aggregate Poisson arrivals, beams in turn
    rate = speed * nbeams / block_s
    t0 = time.perf_counter()
    t_next, n, late = 0.0, 0, 0
    kblock = [0] * nbeams
    while True:
        now = time.perf_counter() - t0
        if now >= seconds:
            break
        if now >= t_next:
            b = n % nbeams
            if submit(b, kblock[b]):
                kblock[b] += 1
                n += 1
            else:
                late += 1
            t_next += rng.exponential(1.0 / rate)
        else:
            reap()
            time.sleep(min(0.0005, t_next - now))
    srv.drain()
    reap()
    st_rt = srv.stats()
    wall_rt = time.perf_counter() - t0
    # saturating phase
    done0 = st_rt["completed"]
    t1 = time.perf_counter()
    m = 0
    while m < 96:
        b = (n + m) % nbeams
        if submit(b, kblock[b]):
            kblock[b] += 1
            m += 1
        else:
            reap()
            time.sleep(0.0002)
    srv.drain()
    reap()
    wall_sat = time.perf_counter() - t1
    st = srv.stats()
    srv.close()
    sat_blocks = st["completed"] - done0
    adds_block = w.nchan * w.ndm * B

    def gbs(nbytes, ms):
        return nbytes / ms / 1e6 if ms > 0 else None
    return {"workload": "128 streaming beams x (1024 ch, 1024 DMs, 65536-sample blocks)",
            "arrivals": f"Poisson at {speed}x aggregate real time for {seconds:.0f} s",
            "blocks_real_time": st_rt["completed"], "busy_rejections": st_rt["rejected_busy"],
            "late_arrivals": late,
            "p50_ms": st_rt["p50_ms"], "p99_ms": st_rt["p99_ms"], "max_ms": st_rt["max_ms"],
            "block_duration_ms": block_s * 1e3,
            "p99_below_block_duration": st_rt["p99_ms"] < block_s * 1e3,
            "mean_batch": st_rt["mean_batch"], "slots": st_rt["slots"],
            "device_bytes": st_rt["device_bytes"],
            "saturated_blocks_per_s": sat_blocks / wall_sat,
            "saturated_mean_batch": sat_blocks / max(1, st["batches"] - st_rt["batches"]),
            "saturated_adds_per_s": sat_blocks * adds_block / wall_sat,
            "real_time_beams_sustained": sat_blocks / wall_sat * block_s,
            "batch_window_ms": st_rt["batch_window_us"] / 1e3,
            "copies": {"host_staging_gbs": gbs(st["staging_bytes"], st["staging_ms"]),
                       "h2d_gbs": gbs(st["h2d_bytes"], st["h2d_ms"]),
                       "d2h_gbs": gbs(st["d2h_bytes"], st["d2h_ms"]),
                       "kernel_ms_per_block": st["kernel_ms"] / max(1, st["completed"]),
                       "per_block_bytes": {"staging": w.nchan * B, "h2d": w.nchan * B,
                                           "d2h": w.ndm * B * 4},
                       "note": "host staging: dd_submit's copy into pinned memory (host "
                               "threads, wall clock); h2d/d2h: device time of the batches' "
                               "input and result copy phases"},
            "wall_s": wall_rt + wall_sat}


def max_over_ranks(value: float, dist, device) -> float:
    """Max of a per-rank timing over all ranks (a timing reduction only: the
    ranks de-disperse independent beams and exchange no data)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    # each step: one oracle run (OpenMP build, all host cores) over the same
    # bounded sample of the workload, sized so the whole run takes about a
    # minute and a half; ms_per_step is the sample's own time
    prep = prepare_oracle_sample(w, budget_s=max(0.25, 90.0 / (args.warmup + args.steps)))
    vals, secs = [], []
    last = None
    for i in range(args.warmup + args.steps):
        res = time_oracle_sample(w, prep)
        if i >= args.warmup:
            vals.append(res["value"])
            secs.append(res["seconds"])
        last = res
    v = statistics.mean(vals)
    sample = {"ndm": prep["ndm"], "nsamp_out": prep["nsamp"], "adds": last["sample_adds"]}
    base = {k: last[k] for k in ("unit", "cores", "kind", "sample")}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "nchan": w.nchan, "ndm": w.ndm,
                       "nsamp_out": w.nsamp_out, "l2": "inputs larger than L2",
                       "timed_sample": sample,
                       "step": "one oracle run over the timed sample (all channels, a spread "
                               "of the DMs, a slice of time); value = its adds per second"},
            "full_workload_ms_extrapolated": w.adds() / v * 1e3,
            "cpu_baseline": {**base, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def beam_input(w: fb.Workload, plan, dtype: str):
    """The workload's seeded uint8 beam (pulses dispersed with the plan's own
    shifts), stored as dtype (the same integers for FP16/FP32)."""
    host, nin = make_input(w, plan.dmshift(), plan.maxshift)
    if dtype != "u8":
        host = host.astype(np.float16 if dtype == "f16" else np.float32)
    return host, nin


def tune_beam(plan, x, out, nin: int, nsamp_out: int, stream, tiles: str, no_tune: bool,
              dtype: str, log: bool):
    """Tile shape for a beam: fixed (tiles "a,b,c,d[,e]"), the plan's default,
    or the autotuner timing every candidate on the first TUNE_NSAMP output
    samples."""
    if tiles:
        plan.set_tiles(dtype, *[int(v) for v in tiles.split(",")])
        return "fixed"
    if no_tune:
        return "default"
    nt = min(nsamp_out, TUNE_NSAMP)
    S = plan.maxshift
    res = plan.autotune(x, out[:, :nt], nsamp_in=nt + S, nsamp_out=nt, stream=stream, reps=1)
    if log:
        for tl, ms in sorted(res, key=lambda r: (r[1] < 0, r[1])):
            print(f"# tune {dtype} {tl} {ms:.3f} ms" if ms >= 0 else f"# tune {dtype} {tl} "
                  "rejected", file=sys.stderr)
    return f"autotuner ({nt} output samples)"


def time_steps(dd, torch, plan, x, out, nin: int, stream, steps: int, warmup: int, barrier):
    """warmup untimed steps, then `steps` timed ones, each bracketed by CUDA
    events on the launching stream, with the de-dispersion kernel itself
    bracketed by a second pair (dd_profile_events).  Returns per-step ms,
    mean kernel ms, the library's launches in the timed region and wall s."""
    def step():
        plan.execute(x, out, nsamp_in=nin, stream=stream)

    for _ in range(warmup):
        step()
    plan.sync(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for a, b in kev:  # torch only times events it has seen recorded; the library re-records
        a.record(stream)
        b.record(stream)
    n0 = dd.launch_count()
    barrier()
    t0 = time.perf_counter()
    for i in range(steps):
        dd.profile_events(*kev[i])   # around the de-dispersion kernel itself
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    barrier()
    wall = time.perf_counter() - t0
    dd.profile_events(None, None)
    launches = dd.launch_count() - n0
    plan.sync(stream)
    per_step = [a.elapsed_time(b) for a, b in ev]
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)
    return per_step, kernel_ms, launches, wall


def e2e_rate(plan, host, nin: int, w: fb.Workload, torch, reps: int, barrier) -> float:
    """Seconds per step through dd_execute_host from pinned host buffers
    (host-to-device copies of the step's input and device-to-host copies of
    its plane inside the timed region)."""
    h_in = torch.from_numpy(host).pin_memory()
    h_out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32).pin_memory()
    plan.execute_host(h_in, h_out, nsamp_in=nin)
    barrier()
    t = time.perf_counter()
    for _ in range(reps):
        plan.execute_host(h_in, h_out, nsamp_in=nin)
    dt = (time.perf_counter() - t) / reps
    del h_in, h_out
    return dt


def roofline_of(adds: float, kernel_ms: float, peak: dict, nominal: float, w: fb.Workload,
                dtype: str, tiles, traffic_ok: bool = True) -> dict:
    achieved = adds / (kernel_ms / 1e3)
    prof = profiled_traffic(w.name, dtype, tiles) if traffic_ok else None
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak["adds_per_s"] / 1e12,
            "traffic_over_compulsory": prof["bytes"] / prof["compulsory"] if prof else None,
            "unit": "Tadd/s", "frac": achieved / peak["adds_per_s"],
            "peak_source": f"measured: dd_add_peak microbenchmark ({peak['best']}), "
                           "best of 3 launches",
            "peak_nominal": nominal / 1e12, "frac_of_nominal": achieved / nominal,
            "traffic": prof["bytes"] if prof else None,
            "traffic_unit": "bytes per step (ncu dram read + write of its launches)",
            "traffic_source": TRAFFIC_SOURCE if prof else None,
            "kernel": "dedisperse_kernel<%d,%d,%d>" % ({"u8": 1, "f16": 2, "f32": 4}[dtype],
                                                       tiles[0], tiles[4]),
            "kernel_ms": kernel_ms}


def beam_section(dd, torch, dev, w: fb.Workload, dtype: str, steps: int, warmup: int, peak,
                 nominal, args, e2e_reps: int = 2) -> dict:
    """One beam in one storage type, single GPU: tuned tile shape, timed
    steps, kernel roofline, real-time factor and end-to-end rate."""
    stream = torch.cuda.current_stream(dev)
    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    host, nin = beam_input(w, plan, dtype)
    x = torch.from_numpy(host).to(dev)
    out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device=dev)
    tiles_from = tune_beam(plan, x, out, nin, w.nsamp_out, stream, "", args.no_tune, dtype,
                           False)

    def barrier():
        torch.cuda.synchronize(dev)

    per_step, kernel_ms, launches, _ = time_steps(dd, torch, plan, x, out, nin, stream, steps,
                                                  warmup, barrier)
    step_ms = sum(per_step) / len(per_step)
    tiles = plan.get_tiles(dtype)
    rl = roofline_of(w.adds(), kernel_ms, peak, nominal, w, dtype, tiles)
    rl["compulsory_bytes"] = int(w.nchan * nin * host.itemsize + w.ndm * w.nsamp_out * 4)
    del x, out
    torch.cuda.empty_cache()
    e2e_s = e2e_rate(plan, host, nin, w, torch, e2e_reps, barrier)
    return {"workload": w.name, "dtype": dtype, "tiles": tiles, "tiles_from": tiles_from,
            "steps": steps, "ms_per_step": step_ms, "adds_per_s": w.adds() / (step_ms / 1e3),
            "roofline": rl, "real_time_factor": w.duration_s() / (step_ms / 1e3),
            "gpu_launches": launches,
            "e2e": {"value": w.adds() / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(w.nchan * nin * host.itemsize),
                    "d2h_bytes_per_step": int(w.ndm * w.nsamp_out * 4)}}


def run_ours(args, w):
    import torch
    import paper_1111_6399_gb300 as dd

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    pk, pk_kind = peaks()
    peak = measured_add_peak(dd, torch, dev)
    nominal = nominal_add_peak(sms, pk.get("sm_max_mhz", 2070.0))

    plan = dd.Plan(w.nchan, w.fch1, w.foff, w.tsamp, w.dm_list())
    S = plan.maxshift
    dt = args.dtype
    host, nin = beam_input(w, plan, dt)
    x = torch.from_numpy(host).to(dev)
    out = torch.empty((w.ndm, w.nsamp_out), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tiles_from = tune_beam(plan, x, out, nin, w.nsamp_out, stream, args.tiles, args.no_tune, dt,
                           rank == 0)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    with ClockSampler(local) as clk:
        per_step_ms, kernel_ms, launches, wall = time_steps(dd, torch, plan, x, out, nin, stream,
                                                            args.steps, args.warmup, barrier)
    step_ms = sum(per_step_ms) / len(per_step_ms)
    total_ms = max_over_ranks(sum(per_step_ms), dist, dev)
    adds = w.adds()
    value = adds * world * args.steps / (total_ms / 1e3)
    tiles = plan.get_tiles(dt)

    # end-to-end: host buffers through dd_execute_host, copies inside the timed region
    detect = None
    if not args.no_detect and dt == "u8" and rank == 0:
        detect = detect_section(dd, torch, out, w, pk.get("hbm_gbs", 6800.0), w.dm_list())
    del x, out
    torch.cuda.empty_cache()
    e2e_s = max_over_ranks(e2e_rate(plan, host, nin, w, torch, max(1, min(args.steps, 3)),
                                    barrier), dist, dev)

    if rank != 0:
        dist.destroy_process_group()
        return
    clocks = clk.summary()
    rl = roofline_of(adds, kernel_ms, peak, nominal, w, dt, tiles)
    rl["compulsory_bytes"] = int(w.nchan * nin * host.itemsize + w.ndm * w.nsamp_out * 4)
    rl["step_ms"] = step_ms
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dt, "data": "synthetic",
        "config": {"workload": w.name, "nchan": w.nchan, "ndm": w.ndm,
                   "nsamp_out": w.nsamp_out, "maxshift": S, "tiles": tiles,
                   "tiles_from": tiles_from,
                   "l2": "inputs larger than L2 (%.0f MB in + %.0f MB out per step, L2 126 MB)"
                         % (w.nchan * nin * host.itemsize / 1e6, w.ndm * w.nsamp_out * 4 / 1e6),
                   "parallelism": f"replicas{world}" if world > 1 else "single-gpu"},
        "roofline": rl,
        "add_peak": {"kinds": {k: v["adds_per_s"] / 1e12 for k, v in peak["kinds"].items()},
                     "unit": "Tadd/s", "best": peak["best"], "clocks": peak["clocks"],
                     "nominal": nominal / 1e12, "sms": sms,
                     "nominal_source": f"{sms} SMs x {ADD_LANES_PER_SM} lanes x "
                                       f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz ({pk_kind} "
                                       "max clock)"},
        "real_time_factor": w.duration_s() / (step_ms / 1e3),
        "e2e": {"value": adds * world / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(w.nchan * nin * host.itemsize),
                "d2h_bytes_per_step": int(w.ndm * w.nsamp_out * 4)},
        "gpu_launches": launches,
        "wall_s_timed": wall,
    }
    if clocks:
        line["clocks"] = clocks
    if detect:
        line["detect"] = detect
    del host
    if world == 1 and not args.no_precision and w is fb.LOWFREQ and dt == "u8":
        line["precision"] = {
            "data": "the same integer noise stored as FP16 and FP32, summed in FP32",
            **{d: beam_section(dd, torch, dev, w, d, max(3, min(args.steps, 10)), 3, peak,
                               nominal, args) for d in ("f16", "f32")}}
    if world == 1 and not args.no_lband and w is not fb.LBAND:
        line["lband"] = beam_section(dd, torch, dev, fb.LBAND, "u8", max(3, min(args.steps, 100)),
                                     3, peak, nominal, args)
    if not args.no_detect and world == 1:
        line["fused_detect"] = {wl.name: fused_detect_section(dd, torch, dev, wl)
                                for wl in (w, fb.LBAND) if wl.nsamp_out <= (1 << 21)}
    lb = fb.LBAND
    lb_nin = lb.nsamp_out + dd.Plan(lb.nchan, lb.fch1, lb.foff, lb.tsamp, lb.dm_list()).maxshift
    if not args.no_batch and world == 1:
        line["batch"] = batch_section(dd, torch, dev, args.steps)
    if not args.no_serve and world == 1:
        line["serving"] = serving_section(dd, torch, dev)
    if not args.no_unpack and world == 1:
        line["unpack"] = unpack_section(dd, torch, dev, lb, lb_nin, pk.get("hbm_gbs", 6800.0))
    if not args.no_frontend and world == 1:
        line["frontend"] = frontend_section(dd, torch, dev, lb, lb_nin, pk.get("hbm_gbs", 6800.0),
                                            nchan=args.frontend_chans)
    if not args.no_pfb and world == 1:
        line["channeliser"] = channeliser_section(dd, torch, dev, pk.get("hbm_gbs", 6800.0),
                                                  pk.get("sm_max_mhz", 2070.0), sms,
                                                  nsub=args.pfb_subs, which=args.pfb_workload)
    if not args.no_sweep and world == 1:
        line["fig4_sweep"] = sweep(dd, torch, dev, compact=True)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(w)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sweep(dd, torch, dev, compact: bool = False) -> dict:
    """The Fig. 4 experiments as a second workload: execution time as a
    percentage of real time (i) over the channel count with the maximum DM at
    200 and as many trial DMs as channels, (ii) over the maximum DM with 2000
    channels and 2000 trial DMs.  DMs are equally spaced from 0.  The band and
    sampling the paper does not state are the L-band beam's: 1500 MHz down by
    300 MHz, 64 us, 2^17 output samples (8.39 s of data).  Full form: six
    points per axis, each autotuned; compact form: three points per axis with
    the plan's default tile shape.  Each point is the median of 7 launches
    (inputs larger than L2 except at the smallest points)."""
    pool = fb.NoisePool(7)
    fch1, bw, tsamp, nsamp_out = 1500.0, 300.0, 64e-6, 1 << 17
    duration = nsamp_out * tsamp

    def point(nchan, ndm, maxdm):
        dms = np.linspace(0.0, maxdm, ndm).astype(np.float32)
        plan = dd.Plan(nchan, fch1, -bw / nchan, tsamp, dms)
        nin = nsamp_out + plan.maxshift
        pitch = (nin + 15) // 16 * 16
        x = torch.from_numpy(pool.rows(nchan, nin, pitch)).to(dev)
        out = torch.empty((ndm, nsamp_out), dtype=torch.float32, device=dev)
        if not compact:
            plan.autotune(x, out, nsamp_in=nin, reps=1)
        ts = []
        for i in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.execute(x, out, nsamp_in=nin)
            e1.record()
            torch.cuda.synchronize()
            if i >= 3:
                ts.append(e0.elapsed_time(e1))
        plan.sync()
        ms = statistics.median(ts)
        adds = nchan * ndm * nsamp_out
        return {"nchan": nchan, "ndm": ndm, "max_dm": maxdm, "maxshift": plan.maxshift,
                "ms": ms, "pct_real_time": 100.0 * ms / 1e3 / duration,
                "adds_per_s": adds / ms * 1e3, "tiles": plan.get_tiles("u8")}

    nchans = (512, 2048, 4096) if compact else (128, 256, 512, 1024, 2048, 4096)
    maxdms = (100.0, 400.0, 1600.0) if compact else (50.0, 100.0, 200.0, 400.0, 800.0, 1600.0)
    return {"metric": "execution time as % of real time (Fig. 4)", "data": "synthetic",
            "form": "compact, default tiles" if compact else "full, autotuned",
            "band": "1500 MHz down 300 MHz, tsamp 64 us, 131072 samples (8.39 s)",
            "nchan_sweep": [point(n, n, 200.0) for n in nchans],
            "maxdm_sweep": [point(2000, 2000, m) for m in maxdms]}


def run_sweep(args):
    import torch
    import paper_1111_6399_gb300 as dd
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    with ClockSampler(0) as clk:
        res = sweep(dd, torch, dev, compact=False)
    res["clocks"] = clk.summary()
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lowfreq", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tune", action="store_true", help="use the plan's default tile shape")
    ap.add_argument("--dtype", default="u8", choices=["u8", "f16", "f32"],
                    help="storage type of the beam (the same integer noise)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-beam batch section")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the FP16/FP32 section of the low-frequency beam")
    ap.add_argument("--no-lband", action="store_true", help="skip the L-band beam section")
    ap.add_argument("--no-sweep", action="store_true", help="skip the compact Fig. 4 sweep")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving section")
    ap.add_argument("--no-unpack", action="store_true", help="skip the input unpacking section")
    ap.add_argument("--no-detect", action="store_true", help="skip the detection section")
    ap.add_argument("--no-frontend", action="store_true",
                    help="skip the voltage front-end section")
    ap.add_argument("--frontend-chans", type=int, default=0,
                    help="front-end section on the first N channels only (0: all)")
    ap.add_argument("--no-pfb", action="store_true", help="skip the channeliser section")
    ap.add_argument("--pfb-subs", type=int, default=0,
                    help="channeliser section on the first N subbands only (0: all)")
    ap.add_argument("--pfb-workload", default="both", choices=["both", "16ch", "256ch"],
                    help="channeliser workloads to run")
    ap.add_argument("--sweep", action="store_true",
                    help="run the Fig. 4 sweeps instead (one JSON line)")
    ap.add_argument("--tiles", default="",
                    help="fixed tile shape dthr,dm_warps,time_warps,cstage[,words]")
    ap.add_argument("--nsamp-out", type=int, default=0,
                    help="a shorter output (samples) of the same beam: the smaller case ncu "
                         "captures run on (0: the workload's own)")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.nsamp_out > 0 and args.nsamp_out != w.nsamp_out:
        import dataclasses
        w = dataclasses.replace(w, nsamp_out=args.nsamp_out,
                                name=f"{w.name}-first{args.nsamp_out}")
    if args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
