"""Benchmark: GPS L1 C/A FFT parallel code-phase acquisition on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one step = one whole acquisition request through the hot path:
unpack + wipe-off + fold + FFT, conj-multiply + IFFT + |.|^2 + non-coherent
sum, peak search): the weak-signal cloud request of 100 ms at 4.096 MHz,
2-bit packed I/Q (204,800 bytes), 32 PRNs x 81 Doppler bins (+-10 kHz,
250 Hz) x 4096 code phases, 10 ms coherent x 10 blocks with half-bit sets;
8 synthetic satellites at 28-45 dB-Hz.  Metric: acquisition cells per
second, cells = PRN x Doppler bin x code phase x ms processed.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the launching stream; L2 (126 MB) is flushed between steps by writing a
256 MB buffer outside the events.  'value' has the recording resident in
HBM; 'e2e' goes through gnss_acquire with pinned host buffers, so the
host->device copy of the recording and the device->host copy of the
detections are inside the timed region.  Under torchrun each rank runs an
independent replica on its own GPU (no data-path collective); the step
time is the max over ranks and 'value' sums the cells of all ranks.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample per step, see cpu_sample_doppler_bins) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import siggen  # noqa: E402

METRIC = "acq cells/s (PRN x Doppler x phase x ms)"
UNIT = "cells/s"
WORKLOAD = "weak_100ms: fs 4.096 MHz, 100 ms 2-bit I/Q, 32 PRN x 81 Doppler (250 Hz) x 4096 phases, 10 ms coh x 10 half-bit"
L2_FLUSH_BYTES = 256 << 20
# Doppler bins of the oracle's bounded sample: every third bin (27 of 81)
CPU_SAMPLE_EVERY = 3


def _cells(P, D, N, B, coh):
    return P * D * N * B * coh


def _flops_xcorr(P, D, B, N):
    """Algorithmic FLOPs of one correlate launch (radix-2 convention):
    per (PRN, Doppler, block) conj-multiply 6N + IFFT 5N log2 N + |.|^2 3N +
    accumulate N."""
    return P * D * B * (6 * N + 5 * N * int(np.log2(N)) + 3 * N + N)


def _flops_total(P, D, B, N, coh):
    return D * B * (8 * coh * N + 5 * N * int(np.log2(N))) + _flops_xcorr(P, D, B, N)


class _Nvml:
    """Read-only NVML queries through the driver's libnvidia-ml (ctypes)."""

    def __init__(self):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        rc = self.lib.nvmlInit_v2()
        if rc != 0:
            raise RuntimeError("nvmlInit_v2 returned %d" % rc)

    def handle(self, idx):
        h = self.C.c_void_p()
        rc = self.lib.nvmlDeviceGetHandleByIndex_v2(self.C.c_uint(idx), self.C.byref(h))
        if rc != 0:
            raise RuntimeError("nvmlDeviceGetHandleByIndex_v2 returned %d" % rc)
        return h

    def _clock(self, fn, h):
        v = self.C.c_uint()
        rc = fn(h, self.C.c_int(1), self.C.byref(v))  # NVML_CLOCK_SM = 1
        if rc != 0:
            raise RuntimeError("NVML clock query returned %d" % rc)
        return v.value

    def sm_clock(self, h):
        return self._clock(self.lib.nvmlDeviceGetClockInfo, h)

    def max_sm_clock(self, h):
        return self._clock(self.lib.nvmlDeviceGetMaxClockInfo, h)

    def event_reasons(self, h):
        v = self.C.c_ulonglong()
        rc = self.lib.nvmlDeviceGetCurrentClocksEventReasons(h, self.C.byref(v))
        if rc != 0:
            raise RuntimeError("nvmlDeviceGetCurrentClocksEventReasons returned %d" % rc)
        return v.value


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled every 5 ms through
    NVML in a background thread while the timed region runs (read-only)."""

    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, gpu_index: int, period_s: float = 0.005):
        self.gpu = gpu_index
        self.period = period_s
        self.sm = []
        self.reasons = set()
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self.error = None

    def start(self):
        try:
            self._nv = _Nvml()
            vis = os.environ.get("CUDA_VISIBLE_DEVICES")
            idx = self.gpu
            if vis:
                try:
                    idx = int(vis.split(",")[self.gpu])
                except ValueError:
                    idx = self.gpu
            self._h = self._nv.handle(idx)
            self.max_mhz = float(self._nv.max_sm_clock(self._h))
        except Exception as e:  # no NVML: report no samples
            self.error = repr(e)
            return
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()

    def _run(self):
        nv = self._nv
        while not self._stop.is_set():
            try:
                self.sm.append(float(nv.sm_clock(self._h)))
                r = nv.event_reasons(self._h)
                for name, bit in self.REASONS.items():
                    if r & bit:
                        self.reasons.add(name)
            except Exception as e:
                self.error = repr(e)
                return
            time.sleep(self.period)

    def stop(self):
        self._stop.set()
        if self._thread is not None:
            self._thread.join(timeout=2)
        out = {"sm_mhz": statistics.median(self.sm) if self.sm else None, "sm_max_mhz": self.max_mhz,
               "reasons": sorted(self.reasons), "samples": len(self.sm), "source": "nvml (libnvidia-ml)"}
        if self.error:
            out["error"] = self.error
        return out


def make_workloads(args):
    """All synthetic inputs, generated before any CUDA call (the process pool
    uses spawn; a pool forked after CUDA initialisation can hang)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    rec = siggen.weak_100ms()
    long_rec = None if args.no_code_doppler else siggen.long_400ms()
    ref_rec = None if args.no_refine else siggen.refine_12ms()
    trk_rec = None if args.no_track else siggen.track_1s()
    batch, serve = [], []
    if not args.no_batch or not args.no_serve:
        n = os.cpu_count() or 1
        ctx = mp.get_context("spawn")
        with cf.ProcessPoolExecutor(max_workers=min(n, 32), mp_context=ctx) as ex:
            if not args.no_batch:
                chunks = [list(range(i, args.batch_requests, 8)) for i in range(8)]
                parts = list(ex.map(siggen.batch_requests_subset, [(args.batch_requests, c) for c in chunks]))
                by_idx = {}
                for c, part in zip(chunks, parts):
                    for i, r in zip(c, part):
                        by_idx[i] = r
                batch = [by_idx[i] for i in range(args.batch_requests)]
            if not args.no_serve:
                chunks = [list(range(i, args.serve_pool, 16)) for i in range(min(16, args.serve_pool))]
                parts = list(ex.map(siggen.serving_requests_subset, [(args.serve_pool, c) for c in chunks]))
                by_idx = {}
                for c, part in zip(chunks, parts):
                    for i, r in zip(c, part):
                        by_idx[i] = r
                serve = [by_idx[i] for i in range(args.serve_pool)]
    return rec, batch, serve, long_rec, ref_rec, trk_rec


def run_batch(g, torch, batch, stream, flush, steps, peak_tflops):
    """256 uneven recordings: one gnss_acquire_batch per step, one replay of
    the same batch captured into a CUDA graph (gnss_batch_graph_*), and one
    gnss_acquire_device per recording; recordings resident on the device.
    fp32_frac: the batch's algorithmic FLOPs (wipe + fold + forward FFT per
    Doppler bin and block, correlate per PRN as well) over the time, against
    the derived FP32 peak."""
    plans = {}
    items = []
    for r in batch:
        key = (r.fs, r.coh_ms, r.dopp_min_hz, r.dopp_step_hz, r.n_dopp, r.fmt, r.half_bit)
        if key not in plans:
            plans[key] = g.Plan.for_recording(r)
        plan = plans[key]
        raw = torch.from_numpy(np.ascontiguousarray(r.raw)).cuda()
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        items.append((plan, raw, r.n_samples, out, None))
    cells = sum(_cells(p.n_prn, p.n_dopp, p.N, p.n_blocks(n), p.desc.coh_ms) for p, _, n, _, _ in items)
    flops = sum(_flops_total(p.n_prn, p.n_dopp, p.n_blocks(n), p.N, p.desc.coh_ms) for p, _, n, _, _ in items)

    def batched():
        g.acquire_batch(items, stream=stream)

    def per_request():
        for plan, raw, n, out, _ in items:
            plan.acquire_device(raw, n, out, stream=stream)

    graph = g.BatchGraph(items)  # captured once, outside the timed region

    def graph_replay():
        graph.launch(stream=stream)

    res = {}
    for name, fn in (("batched", batched), ("graph", graph_replay), ("one_request_per_launch", per_request)):
        with torch.cuda.stream(stream):
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                fn()
                e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        t = statistics.median(ms)
        res[name] = {"ms_per_batch": t, "cells_per_s": cells / (t * 1e-3), "requests_per_s": len(items) / (t * 1e-3),
                     "fp32_frac": flops / (t * 1e-3) / 1e12 / peak_tflops}
    graph.close()
    res["speedup"] = res["one_request_per_launch"]["ms_per_batch"] / res["batched"]["ms_per_batch"]
    res["graph_speedup"] = res["one_request_per_launch"]["ms_per_batch"] / res["graph"]["ms_per_batch"]
    res["requests"] = len(items)
    res["cells_per_batch"] = cells
    res["gflop_per_batch"] = flops / 1e9
    res["workload"] = ("uneven recordings 20-200 ms, fs {2.048, 4.096, 8.192} MHz, 2-bit, 32 PRN, "
                       "+-10 kHz at 250/500 Hz, coherent 500/step ms, all blocks")
    return res


def run_code_doppler(g, torch, rec, stream, flush, steps):
    """The 400 ms weak-signal request with and without code-Doppler
    compensation (GNSS_CODE_DOPPLER): device time per request and the
    satellites detected."""
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    res = {"workload": "long_400ms: fs 4.096 MHz, 400 ms 2-bit I/Q, 32 PRN x 81 Doppler (250 Hz) x 4096 phases, "
                       "10 ms coh x 40 half-bit, 8 satellites at 27-36 dB-Hz",
           "injected_prns": sorted(s.prn for s in rec.sats)}
    for name, cd in (("plain", False), ("compensated", True)):
        plan = g.Plan.for_recording(rec, code_doppler=cd)
        B = plan.n_blocks(rec.n_samples)
        cells = _cells(plan.n_prn, plan.n_dopp, plan.N, B, rec.coh_ms)
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            plan.acquire_device(raw, rec.n_samples, out, stream=stream)
        torch.cuda.synchronize()
        ms = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                plan.acquire_device(raw, rec.n_samples, out, stream=stream)
                e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        det = g.detections_from_bytes(out.cpu().numpy())
        t = statistics.median(ms)
        res[name] = {"ms_per_request": t, "cells_per_s": cells / (t * 1e-3),
                     "detected_prns": sorted(int(d["prn"]) for d in det if d["detected"])}
    return res


def run_refine(g, torch, rec, stream, steps, peak_tflops):
    """Fine acquisition of the 12 ms recording: the detections of a plain
    acquisition (true candidates) plus 1000 seeded random candidates, refined
    over 10 ms on the device (Doppler pre-search +-250 Hz, then gradient
    ascent); time per call and the refined error of the true candidates
    against the injected truth (delay at the middle of the window)."""
    coh = 10
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    det = plan.acquire(raw, rec.n_samples)
    true = [(int(d["prn"]), float(d["dopp_hz"]), int(d["code_phase"]) * 1023.0 / plan.N) for d in det if d["detected"]]
    rprn, rf, rtau = siggen.refine_candidates(rec)
    prn = [t[0] for t in true] + list(rprn)
    cands = g.candidates(prn, [t[1] for t in true] + list(rf), [t[2] for t in true] + list(rtau))
    cands_dev = torch.from_numpy(cands.view(np.uint8)).cuda()
    out_dev = torch.zeros(len(cands) * g.REFINED_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

    def call():
        plan.refine_device(raw, rec.n_samples, cands_dev, len(cands), coh, 100, out_dev, search_hz=250.0,
                           stream=stream)

    with torch.cuda.stream(stream):
        call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            call()
            e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    out = np.frombuffer(out_dev.cpu().numpy().tobytes(), g.REFINED_DTYPE)
    # algorithmic FP32 work of the ascent actually run: per sample of the
    # L = coh * N window, 20 flops for P alone (carrier rotation 6, wipe-off
    # 6, interpolated chip 4, z += w c 4) and 10 more for the gradient sums
    # ((n - L/2) w c 6, -w slope 4); evaluations counted by the kernel
    L = coh * plan.N
    flops = float(L * (20.0 * out["n_eval"].astype(np.float64).sum() + 30.0 * out["n_eval_grad"].astype(np.float64).sum()))
    T = coh * plan.N / rec.fs
    truth = {s.prn: s for s in rec.sats}
    df, dt = [], []
    for k, (p, _, _) in enumerate(true):
        s = truth.get(p)
        if s is None:
            continue
        df.append(out[k]["f_hz"] - s.dopp_hz)
        mid = s.code_phase_chips - s.dopp_hz * T / (2 * 1540.0)
        dt.append((out[k]["tau_chips"] - mid + 511.5) % 1023 - 511.5)
    t = statistics.median(ms)
    achieved = flops / (t * 1e-3) / 1e12
    return {"workload": "refine_12ms: 2.048 MHz int8, %d true + %d random candidates, 10 ms window, "
                        "pre-search +-250 Hz, <= 100 iterations" % (len(true), len(rprn)),
            "ms_per_call": t, "candidates_per_s": len(cands) / (t * 1e-3),
            "true_candidates": len(df),
            "rms_doppler_error_hz": float(np.sqrt(np.mean(np.square(df)))) if df else None,
            "rms_delay_error_chips": float(np.sqrt(np.mean(np.square(dt)))) if dt else None,
            "status_counts": {int(k): int(v) for k, v in zip(*np.unique(out["status"], return_counts=True))},
            "evaluations_per_call": {"p": int(out["n_eval"].sum()), "p_and_gradient": int(out["n_eval_grad"].sum())},
            "roofline": {"bound": "alu", "kernel": "k_refine", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops, "flops_per_call": flops,
                         "flop_count": "per window sample: 20 for P alone, 30 with the gradient (of derived peak)"}}


def run_track(g, torch, rec, stream, steps, peak_tops, n_chan=1280):
    """Tracking channels over the 1 s recording: the 8 injected satellites
    from perturbed truth plus seeded channels on every PRN at random (f, tau)
    up to n_chan, 1000 intervals of 1 ms each, one launch; channel-ms per
    second and the lock of the true channels."""
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    prn, f, tau = siggen.track_starts(rec)
    rng = np.random.default_rng(1309005207)
    extra = n_chan - len(prn)
    prn = np.concatenate([prn, 1 + np.arange(extra) % 32])
    f = np.concatenate([f, rng.uniform(-5000.0, 5000.0, extra)])
    tau = np.concatenate([tau, rng.uniform(0.0, 1023.0, extra)])
    cands = g.candidates(prn, f, tau)
    cdev = torch.from_numpy(cands.view(np.uint8)).cuda()
    n_int = rec.n_samples // plan.N
    out = torch.zeros(len(cands) * n_int * g.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

    def call():
        plan.track(raw, rec.n_samples, cdev, len(cands), out, n_int, 1, 1.0, 15.0, 2.0, stream=stream)

    with torch.cuda.stream(stream):
        call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            call()
            e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    recs = g.track_records(out[: len(rec.sats) * n_int * g.TRACK_DTYPE.itemsize].cpu().numpy())
    recs = recs.reshape(len(rec.sats), n_int)[:, -200:]
    lock = [float(np.mean(r["zp"][:, 1] ** 2) / max(np.mean(r["zp"][:, 0] ** 2), 1e-30)) for r in recs]
    t = statistics.median(ms)
    # algorithmic operations per channel-sample (32): wipe-off x e^{-j theta}
    # (complex product, 6 flops) and the carrier's advance (rotation, 6),
    # the 64-bit code NCO advance (2 integer ops), the early / prompt / late
    # replica chips (index and bit, 2 integer ops each: 6) and their sign-
    # applied accumulation (3 x (2 sign flips + 2 adds): 12); against the
    # issue roof of one operation per lane of each SM sub-partition per cycle
    cs = len(cands) * rec.n_samples
    ops = 32.0 * cs
    achieved = ops / (t * 1e-3) / 1e12
    return {"roofline": {"bound": "issue", "kernel": "k_track", "achieved": achieved, "peak": peak_tops,
                         "unit": "Tops/s", "frac": achieved / peak_tops, "ops_per_channel_sample": 32,
                         "peak_basis": "148 SMs x 4 sub-partitions x 32 lanes x max SM clock (of derived)"},
            "workload": "track_1s: 4.096 MHz 2-bit, 1 s, %d channels (8 injected satellites + seeded channels "
                        "on every PRN), 1000 intervals of 1 ms, E/P/L spacing 1 chip, PLL 15 Hz, DLL 2 Hz" % n_chan,
            "ms_per_launch": t, "channel_ms_per_s": len(cands) * n_int / (t * 1e-3),
            "sample_correlations_per_s": 3 * len(cands) * rec.n_samples / (t * 1e-3),
            "true_channels_q2_over_i2_last_200ms": lock}


def run_zoom(g, torch, rec, stream, steps):
    """Second-stage fine Doppler search (grid step / 5 over +-1 step) around
    the detections of the 100 ms request: time per call (host clock, records
    copied in and the stream synchronised) and the Doppler error of the
    coarse and the zoomed estimates against the injected truth."""
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    det = plan.acquire(raw, rec.n_samples)
    det = det[det["detected"] == 1]
    fine = plan.zoom(raw, rec.n_samples, det, 5, 1, stream=stream)
    ms = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fine = plan.zoom(raw, rec.n_samples, det, 5, 1, stream=stream)
        ms.append((time.perf_counter() - t0) * 1e3)
    truth = {s.prn: s.dopp_hz + 0.5 * s.dopp_rate * (rec.n_samples / rec.fs) for s in rec.sats}
    # algorithmic FP32 work of one call: per detection, the fine bins' fold and
    # forward FFTs and one PRN's correlations over every block (the counts of
    # the acquisition itself, on 11 bins)
    D, B, N = 11, plan.n_blocks(rec.n_samples), plan.N
    flops = float(len(det)) * (_flops_total(1, D, B, N, rec.coh_ms))
    peak = 148 * 128 * 2 * 2032e6 / 1e12
    zoom_tflops = flops / (statistics.median(ms) * 1e-3) / 1e12
    ec = [int(d["dopp_hz"]) - truth[int(d["prn"])] for d in det if int(d["prn"]) in truth]
    ez = [int(d["dopp_hz"]) - truth[int(d["prn"])] for d in fine if int(d["prn"]) in truth]
    return {"workload": "weak_100ms detections, fine grid 50 Hz over +-250 Hz (11 bins) per detection",
            "detections": len(det), "ms_per_call": statistics.median(ms),
            "rms_doppler_error_hz": {"coarse": float(np.sqrt(np.mean(np.square(ec)))) if ec else None,
                                     "zoom": float(np.sqrt(np.mean(np.square(ez)))) if ez else None},
            "ratio_mean": {"coarse": float(det["ratio"].mean()) if len(det) else None,
                           "zoom": float(fine["ratio"].mean()) if len(fine) else None},
            "roofline": {"bound": "alu", "kernel": "zoom call (k_fold, k_carrier_fft, correlate; host time)",
                         "achieved": zoom_tflops, "peak": peak, "unit": "TFLOP/s", "frac": zoom_tflops / peak,
                         "flops_per_call": flops,
                         "note": "host-timed call of a few small launches: launch- and latency-bound, not ALU-bound"}}


def _chip_err(a, b):
    """Circular code-delay difference in chips, in [-511.5, 511.5)."""
    return (a - b + 511.5) % 1023.0 - 511.5


def zoom_vs_refine(g, torch, rec, zoom, stream=None, steps=5):
    """The two fine searches on the same coarse detections of one recording:
    gnss_acquire_zoom (grid step / zoom over +-1 step; coherent blocks of the
    plan, integrated over the whole recording) and gnss_refine (gradient
    ascent over a 10 ms window from the recording start, pre-search +-half a
    coarse step).  Errors against the injected truth at the middle of the
    samples each method integrates; times per call (host clock, stream
    synchronised, records back on the host)."""
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    det = plan.acquire(raw, rec.n_samples)
    truth = {s.prn: s for s in rec.sats}
    det = det[(det["detected"] == 1) & np.isin(det["prn"], list(truth))]
    cands = g.candidates(det["prn"], det["dopp_hz"].astype(float), det["code_phase"] * 1023.0 / rec.N)
    win_ms = 10
    search = rec.dopp_step_hz / 2.0

    def do_zoom():
        return plan.zoom(raw, rec.n_samples, det, zoom, 1, stream=stream)

    def do_refine():
        return plan.refine(raw, rec.n_samples, cands, win_ms, 100, search_hz=search, stream=stream)

    fine, ref = do_zoom(), do_refine()
    tz, tr = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        do_zoom()
        t1 = time.perf_counter()
        do_refine()
        t2 = time.perf_counter()
        tz.append((t1 - t0) * 1e3)
        tr.append((t2 - t1) * 1e3)
    t_all = 0.5 * rec.n_samples / rec.fs  # coarse and zoom: the whole recording
    t_win = 0.5 * win_ms * 1e-3           # refine: its window
    rows = []
    for d, z, r in zip(det, fine, ref):
        s = truth[int(d["prn"])]
        f_all, c_all = rec.truth_at(s, t_all)
        f_win, c_win = rec.truth_at(s, t_win)
        rows.append({"prn": int(d["prn"]), "cn0_dbhz": s.cn0_dbhz, "bit_edge_in_window": s.bit_edge_ms < win_ms,
                     "doppler_error_hz": {"coarse": float(d["dopp_hz"] - f_all), "zoom": float(z["dopp_hz"] - f_all),
                                          "refine": float(r["f_hz"] - f_win)},
                     "code_error_chips": {"coarse": float(_chip_err(d["code_phase"] * 1023.0 / rec.N, c_all)),
                                          "zoom": float(_chip_err(z["code_phase"] * 1023.0 / rec.N, c_all)),
                                          "refine": float(_chip_err(r["tau_chips"], c_win))}})

    def rms(key, method, subset=None):
        v = [row[key][method] for row in rows if subset is None or subset(row)]
        return float(np.sqrt(np.mean(np.square(v)))) if v else None

    clean = lambda row: not row["bit_edge_in_window"]
    return {"detections": len(rows), "zoom": zoom, "zoom_step_hz": rec.dopp_step_hz / zoom,
            "refine_window_ms": win_ms, "ms_per_call": {"zoom": statistics.median(tz), "refine": statistics.median(tr)},
            "rms_doppler_error_hz": {m: rms("doppler_error_hz", m) for m in ("coarse", "zoom", "refine")},
            "rms_code_error_chips": {m: rms("code_error_chips", m) for m in ("coarse", "zoom", "refine")},
            "rms_doppler_error_hz_edge_free_window": {m: rms("doppler_error_hz", m, clean)
                                                      for m in ("coarse", "zoom", "refine")},
            "per_detection": rows}


def run_zoom_vs_refine(g, torch, stream):
    """zoom_vs_refine on the 12 ms recording (2.048 MHz, 1 ms blocks, 500 Hz
    grid, no bit edge in the first 10 ms) and on the 100 ms one (4.096 MHz,
    10 ms blocks with half-bit sets, 250 Hz grid)."""
    import siggen
    return {"refine_12ms": zoom_vs_refine(g, torch, siggen.refine_12ms(), 10, stream),
            "weak_100ms": zoom_vs_refine(g, torch, siggen.weak_100ms(), 10, stream)}


def run_fft_sizes(g, torch, stream, flush, steps, peak_tflops, sizes=(2048, 4096, 8192, 16384)):
    """The correlate kernel at each FFT size on a 100 ms 2-bit recording at
    fs = N kHz (one satellite at 45 dB-Hz), 32 PRNs x 81 Doppler bins of 250 Hz,
    1 ms coherent blocks, in the default launch shape of that size: launch time
    from the traced entry point's events (L2 flushed before each step) and the
    fraction of the derived FP32 peak under the 5 N log2 N convention."""
    import siggen
    res = {}
    for N in sizes:
        fs, n = N * 1000, 100 * N
        rng = np.random.default_rng(1309005210 + N)
        sats = [siggen.Sat(prn=9, cn0_dbhz=45.0, dopp_hz=-1750.0, code_phase_chips=100.7, carrier_phase=0.3,
                           bit_edge_ms=3.0)]
        x = siggen.synthesize(rng, fs, n, sats)
        li, lq = siggen.quantize_2bit(x, sats, fs)
        raw = torch.from_numpy(np.ascontiguousarray(siggen.pack(li, lq, siggen.FMT_2BIT_IQ))).cuda()
        plan = g.Plan(fs, 1, -10000, 250, 81, prns=range(1, 33), fmt=siggen.FMT_2BIT_IQ)
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(3):
                plan.acquire_device(raw, n, out, stream=stream)
        torch.cuda.synchronize()
        tev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(float(k))
                plan.acquire_device_traced(raw, n, out, tev[k], stream=stream)
        torch.cuda.synchronize()
        ms = statistics.mean(e[2].elapsed_time(e[3]) for e in tev)
        B = plan.n_blocks(n)
        fl = _flops_xcorr(plan.n_prn, plan.n_dopp, B, N)
        res[str(N)] = {"kernel": xcorr_kernel_name(plan.xcorr_variant(), N, half=False),
                       "correlate_ms": ms, "tflops": fl / (ms * 1e-3) / 1e12,
                       "frac": fl / (ms * 1e-3) / 1e12 / peak_tflops}
        plan.close()
    return {"workload": "100 ms at fs = N kHz, 2-bit, 32 PRN x 81 Doppler (250 Hz), 1 ms coherent x 100",
            "sizes": res}


def run_variants(g, torch, rec, stream, flush, steps=20):
    """Every correlate variant the library accepts on this GPU, forced in turn
    and timed like the roofline leg (traced correlate launch, L2 flushed,
    mean of 'steps'): the 100 ms request, and 100 ms at fs = N kHz with 1 ms
    blocks for N = 2048 ... 16384.  Variant codes as gnss_autotune takes them;
    the default of each size is restored afterwards."""
    import siggen
    TM, CL, ST, OCC = 0x400, 0x200, 0x100, 0x800
    K2, M2 = 1 << 12, 1 << 14
    cand = [16, 32, 8, 16 | ST, 16 | CL, 32 | CL, 16 | TM, 16 | TM | K2, 16 | TM | M2, 16 | TM | K2 | M2,
            16 | TM | OCC, 32 | TM, 32 | TM | M2]

    def time_plan(plan, raw, n):
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        default = plan.xcorr_variant()
        res = {}
        for code in cand:
            try:
                plan.autotune(code)
            except g.GnssError:
                continue
            with torch.cuda.stream(stream):
                for _ in range(3):
                    plan.acquire_device(raw, n, out, stream=stream)
            torch.cuda.synchronize()
            tev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
            with torch.cuda.stream(stream):
                for k in range(steps):
                    flush.fill_(float(k))
                    plan.acquire_device_traced(raw, n, out, tev[k], stream=stream)
            torch.cuda.synchronize()
            res[hex(code)] = statistics.mean(e[2].elapsed_time(e[3]) for e in tev)
        plan.autotune(default)
        return {"default": hex(default), "correlate_ms": res}

    out = {"weak_100ms": time_plan(g.Plan.for_recording(rec),
                                   torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda(), rec.n_samples)}
    for N in (2048, 4096, 8192, 16384):
        fs, n = N * 1000, 100 * N
        rng = np.random.default_rng(1309005210 + N)
        sats = [siggen.Sat(prn=9, cn0_dbhz=45.0, dopp_hz=-1750.0, code_phase_chips=100.7, carrier_phase=0.3,
                           bit_edge_ms=3.0)]
        li, lq = siggen.quantize_2bit(siggen.synthesize(rng, fs, n, sats), sats, fs)
        raw = torch.from_numpy(np.ascontiguousarray(siggen.pack(li, lq, siggen.FMT_2BIT_IQ))).cuda()
        plan = g.Plan(fs, 1, -10000, 250, 81, prns=range(1, 33), fmt=siggen.FMT_2BIT_IQ)
        out[str(N)] = time_plan(plan, raw, n)
        plan.close()
    return out


def _serve_points(spec, seconds):
    """'rate[:seconds],...' -> [(rate, seconds)]; a point without its own
    duration runs for 'seconds'."""
    out = []
    for item in spec.split(","):
        item = item.strip()
        if item:
            r, _, sec = item.partition(":")
            out.append((float(r), float(sec) if sec else float(seconds)))
    return out


def run_serving_curve(g, serve, rates, seconds, bound_ms, seed=1309005205):
    """Latency against offered load through gnss_submit / gnss_poll: one
    server (plans and code spectra made resident once, before timing) takes
    Poisson arrivals over the pooled recordings at each rate for 'seconds';
    latency = submit -> result seen by the polling thread (host clock).  With
    bound_ms the server refuses submissions whose projected wait exceeds it
    (GNSS_EBUSY, counted as refused), which bounds latency past saturation."""
    import threading
    srv = g.Server(max_batch=64, streams=2, max_queue_wait_ms=bound_ms)
    descs = [g.Server.desc_for(r) for r in serve]
    for d, r in zip(descs, serve):
        srv.wait(srv.submit(d, r.raw, r.n_samples), 600000)
    req_cells = [_cells(32, r.n_dopp, r.N, r.n_blocks, r.coh_ms) for r in serve]
    rng = np.random.default_rng(seed)
    points = []
    for rate, seconds in rates:
        pending, done, done_cells, queued = {}, [], [0], []
        refused = 0
        lock = threading.Lock()
        stop = threading.Event()

        def poller():
            while not stop.is_set() or pending:
                with lock:
                    items = list(pending.items())
                for t, (t0, kk) in items:
                    try:
                        r = srv.poll(t)
                    except g.GnssError:
                        r = "err"
                    if r is not None:
                        with lock:
                            pending.pop(t, None)
                        done.append(time.perf_counter() - t0)
                        done_cells[0] += req_cells[kk % len(serve)]
                time.sleep(0.0002)

        def sampler():
            while not stop.is_set():
                queued.append(srv.stats()["queued"])
                time.sleep(0.05)

        th, ts = threading.Thread(target=poller, daemon=True), threading.Thread(target=sampler, daemon=True)
        refused0 = srv.stats()["refused"]
        th.start()
        ts.start()
        t_start = time.perf_counter()
        t_next, k = t_start, 0
        while t_next - t_start < seconds:
            now = time.perf_counter()
            if now < t_next:
                time.sleep(t_next - now)
            r = serve[k % len(serve)]
            try:
                tk = srv.submit(descs[k % len(serve)], r.raw, r.n_samples)
                with lock:
                    pending[tk] = (time.perf_counter(), k)
            except g.GnssError:
                refused += 1
            k += 1
            t_next += rng.exponential(1.0 / rate)
        stop.set()
        th.join(timeout=600)
        ts.join(timeout=10)
        t_total = time.perf_counter() - t_start
        lat = np.array(done) * 1e3
        pct = lambda q: float(np.percentile(lat, q)) if len(lat) else None
        points.append({"offered_req_per_s": rate, "seconds": seconds, "submitted": k, "refused": refused,
                       "refused_by_bound": srv.stats()["refused"] - refused0, "completed": len(done),
                       "requests_per_s": len(done) / t_total, "cells_per_s": done_cells[0] / t_total,
                       "p50_ms": pct(50), "p99_ms": pct(99), "p999_ms": pct(99.9),
                       "queued_mean": float(np.mean(queued)) if queued else 0.0,
                       "queued_max": int(max(queued)) if queued else 0})
    srv.close()
    return {"workload": "Poisson arrivals over %d pooled recordings 10-500 ms, fs up to 16.384 MHz, 2-bit, "
                        "32 PRN, +-10 kHz at 250/500 Hz" % len(serve),
            "admission_bound_ms": bound_ms, "device_budget_gib": 16, "points": points}


def run_cufft_comparator(g, torch, plan, raw_dev, n_samples, stream, flush, steps, ours_ms):
    """Library comparison on the same GPU: this library's forward stage gives
    the Doppler-bin spectra Y, then the correlate stage runs as a cuFFT
    pipeline (torch.fft): Y x conj(C_p) for all PRNs at once, one batched
    IFFT, |.|^2, the per-set block sums and the per-PRN surface maxima.
    Timed with CUDA events like the native correlate launch it is set
    against; also reports how far its surfaces are from the native ones."""
    B = plan.n_blocks(n_samples)
    P, D, N, S = plan.n_prn, plan.n_dopp, plan.N, plan.n_sets
    Y = torch.empty((D, B, N, 2), dtype=torch.float32, device="cuda")
    Cs = torch.empty((P, N, 2), dtype=torch.float32, device="cuda")
    ours = torch.zeros((S, P, D, N), dtype=torch.float32, device="cuda")
    out = torch.zeros(P * 28, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        plan.stage_wipe_fft(raw_dev, n_samples, B, Y, stream=stream)
        plan.code_spectra(Cs, stream=stream)
        plan.stage_correlate(Y, B, out, surface=ours, stream=stream)
    torch.cuda.synchronize()
    Yc = torch.view_as_complex(Y)
    Cc = torch.view_as_complex(Cs).conj()

    def correlate():
        Z = Yc.unsqueeze(0) * Cc[:, None, None, :]          # [P, D, B, N]
        R = torch.fft.ifft(Z, dim=-1)                        # cuFFT, 1/N scaled
        pw = R.real.square() + R.imag.square()
        surf = torch.stack([pw[:, :, s::S].sum(dim=2) for s in range(S)])  # [S, P, D, N]
        peak = surf.flatten(2).max(dim=2)
        return surf, peak

    with torch.cuda.stream(stream):
        surf, _ = correlate()
    torch.cuda.synchronize()
    err = float(((surf - ours).abs().amax(dim=(2, 3)) / ours.amax(dim=(2, 3))).max())
    ms = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            correlate()
            e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    return {"kind": "cuFFT pipeline (torch.fft batched IFFT + torch elementwise/reductions) for the correlate "
                    "stage, on this library's Doppler-bin spectra",
            "correlate_ms": t, "native_correlate_ms": ours_ms, "native_speedup": t / ours_ms,
            "cells_per_s_correlate_only": _cells(P, D, N, B, plan.desc.coh_ms) / (t * 1e-3),
            "max_rel_surface_diff_vs_native": err}


def reduce_max_over_ranks(value: float, device) -> float:
    """Largest value over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(cells_per_step_per_rank: float, steps: int, n_ranks: int, max_total_ms: float) -> float:
    """Whole-job throughput: the cells every rank processed over the slowest
    rank's time (replicas: each rank runs its own recording stream)."""
    return n_ranks * cells_per_step_per_rank * steps / (max_total_ms * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_ours(args):
    rec, batch, serve, long_rec, ref_rec, trk_rec = make_workloads(args)
    import torch
    import paper_1309_0052_b300 as g

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    plan = g.Plan.for_recording(rec, prns=range(1, 33))
    B = plan.n_blocks(rec.n_samples)
    P, D, N, coh = plan.n_prn, plan.n_dopp, plan.N, rec.coh_ms
    cells = _cells(P, D, N, B, coh)
    stream = torch.cuda.Stream()
    raw_dev = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    out_dev = torch.zeros(P * 28, dtype=torch.uint8, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def step():
        plan.acquire_device(raw_dev, rec.n_samples, out_dev, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if ws > 1:
        torch.distributed.barrier()
    ck = clocks.stop()
    total_ms = reduce_max_over_ranks(sum(step_ms), torch.device("cuda"))

    # roofline of the dominant kernel (correlate: conj-mult + IFFT + |.|^2 +
    # accumulate + detection), timed live inside the same acquisition step:
    # the traced entry point records CUDA events on the launching stream at
    # the stage boundaries (before fold, before carrier FFT, around correlate)
    tev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))
            plan.acquire_device_traced(raw_dev, rec.n_samples, out_dev, tev[k], stream=stream)
    torch.cuda.synchronize()
    x_ms = statistics.mean(ev[2].elapsed_time(ev[3]) for ev in tev)
    stage_ms = {"fold": statistics.mean(ev[0].elapsed_time(ev[1]) for ev in tev),
                "carrier_fft": statistics.mean(ev[1].elapsed_time(ev[2]) for ev in tev),
                "correlate": x_ms}
    x_flops = _flops_xcorr(P, D, B, N)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clock_for_peak = ck["sm_max_mhz"] or 2032.0
    peak_tflops = sms * 128 * 2 * clock_for_peak * 1e6 / 1e12
    achieved = x_flops / (x_ms * 1e-3) / 1e12
    traffic = _load_traffic()

    # e2e through the public C ABI with pinned host buffers
    raw_pin = torch.from_numpy(np.ascontiguousarray(rec.raw)).pin_memory()
    # page-locked record buffer: the device-to-host copy of the results is asynchronous
    out_pin = torch.zeros(P * g.DETECTION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    out_host = out_pin.numpy().view(g.DETECTION_DTYPE)
    e2e_ms = []
    for k in range(max(args.warmup, 1) + args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        det = plan.acquire(raw_pin.numpy(), rec.n_samples, stream=stream, out=out_host)
        t1 = time.perf_counter()
        if k >= max(args.warmup, 1):
            e2e_ms.append((t1 - t0) * 1e3)
    h2d = g.recording_bytes(rec.fmt, B * coh * N)
    ffma_tflops, _ = g.probe_ffma(2048)

    value = job_value(cells, args.steps, ws, total_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded siggen)",
        "config": {"workload": WORKLOAD, "requests_per_step_per_gpu": 1, "cells_per_request": cells,
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if ws > 1 else "single"},
        "requests_per_s": ws * args.steps / (total_ms * 1e-3),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "kind": "device step time, recording resident"},
        "e2e": {"value": cells / (statistics.mean(e2e_ms) * 1e-3) * ws, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": P * 28,
                "p50_ms": float(np.percentile(e2e_ms, 50)), "p99_ms": float(np.percentile(e2e_ms, 99))},
        "gpu_launches": 3 * args.steps,
        "stage_ms": stage_ms,
        "roofline": {"bound": "alu", "kernel": xcorr_kernel_name(plan.xcorr_variant(), N, half=rec.half_bit),
                     "variant_code": plan.xcorr_variant(), "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": traffic, "flops_per_launch": x_flops, "launch_ms": x_ms,
                     "peak_basis": "148 SMs x 128 FP32 lanes x 2 x max SM clock (of derived)",
                     "ffma_probe_tflops": ffma_tflops,
                     "flop_convention": "5 N log2 N per complex FFT"},
        "clocks": ck,
        "total_gflop_per_request": _flops_total(P, D, B, N, coh) / 1e9,
    }
    det_ok = int(det["detected"].sum())
    line["detected_prns"] = det_ok
    if not args.no_cufft:
        line["cufft_comparator"] = run_cufft_comparator(g, torch, plan, raw_dev, rec.n_samples, stream, flush,
                                                        steps=10, ours_ms=x_ms)
    if long_rec is not None:
        line["code_doppler"] = run_code_doppler(g, torch, long_rec, stream, flush, steps=10)
    if not args.no_zoom:
        line["zoom"] = run_zoom(g, torch, rec, stream, steps=10)
        line["zoom_vs_refine"] = run_zoom_vs_refine(g, torch, stream)
    if not args.no_sizes:
        line["fft_sizes"] = run_fft_sizes(g, torch, stream, flush, steps=5, peak_tflops=peak_tflops)
    if args.variants:
        line["variants"] = run_variants(g, torch, rec, stream, flush)
    if ref_rec is not None:
        line["refine"] = run_refine(g, torch, ref_rec, stream, steps=10, peak_tflops=peak_tflops)
    if trk_rec is not None:
        line["track"] = run_track(g, torch, trk_rec, stream, steps=3, peak_tops=sms * 4 * 32 * clock_for_peak * 1e6 / 1e12)
    if batch:
        line["batch"] = run_batch(g, torch, batch, stream, flush, steps=3, peak_tflops=peak_tflops)
    if serve:
        line["serving"] = run_serving_curve(g, serve, _serve_points(args.serve_rates, args.serve_seconds),
                                            args.serve_seconds, args.serve_bound_ms)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(rec, args)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def xcorr_kernel_name(code, N, half):
    """Name of the correlate kernel a variant code launches at FFT size N."""
    e, sets = code & 0xFF, "half-bit" if half else "one set"
    if code & 0x400:
        k, m = ((code >> 12) & 3) + 1, ((code >> 14) & 3) + 1
        occ = {2048: "6 CTAs/SM", 4096: "4 CTAs/SM, one buffer", 8192: "2 CTAs/SM, one buffer",
               16384: "1 CTA/SM of 1024, one buffer"}.get(N, "")
        form = occ if code & 0x800 else ("%d PRN%s, %d bin%s" % (k, "s" * (k > 1), m, "s" * (m > 1)))
        return "k_xcorr_tm<%d,%d,%s,%s>" % (N, e, sets, form)
    if code & 0x200:
        return ("k_xcorr_split<%s>" % sets) if N == 16384 else "k_xcorr<%d,%d,%s,class-local>" % (N, e, sets)
    return "k_xcorr<%d,%d,%s%s>" % (N, e, sets, ",staged" if code & 0x100 else "")


def _kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("fft.cuh", "xcorr.cuh", "acq.cu", "xcorr_tm.cu"):
        with open(os.path.join(ROOT, "paper_1309_0052_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _load_traffic():
    """DRAM bytes per correlate launch from the committed ncu summary; None when
    there is none or when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic_k_xcorr_weak_100ms.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != _kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def _oracle_sample(rec, threads, every=CPU_SAMPLE_EVERY):
    """One bounded oracle step: every 'every'-th Doppler bin of the workload,
    all 32 PRNs, all blocks, both half-bit sets.  Returns cells."""
    import oracle
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    dopp = rec.dopp_hz[::every]
    S = oracle.surfaces(x, rec.fs, rec.coh_ms, rec.n_blocks, rec.half_bit, np.arange(1, 33), dopp, threads)
    oracle.detect(S, np.arange(1, 33))
    return _cells(32, len(dopp), rec.N, rec.n_blocks, rec.coh_ms)


def cpu_fft_acquire(rec, threads, every=CPU_SAMPLE_EVERY):
    """Optimised CPU acquisition beside the plain oracle, with the paper's CPU
    lessons (Section 4: persistent worker threads, dynamic scheduling,
    vectorised FFT library): a pool of 'threads' workers takes Doppler bins
    as they free up; per bin, the coherent fold uses the per-millisecond
    carrier constant (so only N samples per block take a carrier), then a
    complex64 FFT of every block, the conj-multiply with all 32 code spectra,
    a batched IFFT (scipy.fft / pocketfft), |.|^2, the half-bit set sums and
    the per-PRN peak.  FP32 like the GPU path.  Runs every 'every'-th
    Doppler bin; returns (cells, per-set per-PRN peaks)."""
    import concurrent.futures as cf
    import scipy.fft as sf
    N, coh, B, fs = rec.N, rec.coh_ms, rec.n_blocks, rec.fs
    L = coh * N
    raw = np.frombuffer(np.asarray(rec.raw).tobytes(), np.uint8)[: (B * L + 1) // 2]
    lv = np.array([-3, -1, 1, 3], np.float32)
    x = np.empty(2 * len(raw), np.complex64)
    x[0::2] = lv[raw & 3] + 1j * lv[(raw >> 2) & 3]
    x[1::2] = lv[(raw >> 4) & 3] + 1j * lv[(raw >> 6) & 3]
    X3 = x[: B * L].reshape(B, coh, N)
    table = siggen.chip_table()
    m = np.arange(N)
    conjC = np.conj(sf.fft(table[:, (m * 1023) // N].astype(np.complex64), axis=-1)).astype(np.complex64)
    sets = 2 if rec.half_bit else 1
    bm = (np.arange(B, dtype=np.int64)[:, None] * L + m[None, :])  # sample index of (b, m)

    def one_bin(f):
        f = int(f)
        w = np.exp(-2j * np.pi * ((f * np.arange(coh)) % 1000) / 1000.0).astype(np.complex64)
        car = np.exp(-2j * np.pi * ((f * bm) % fs) / fs).astype(np.complex64)
        y = np.einsum("i,bim->bm", w, X3) * car
        Y = sf.fft(y, axis=-1)
        R = sf.ifft(Y[None] * conjC[:, None, :], axis=-1)           # [P, B, N]
        pw = R.real * R.real + R.imag * R.imag
        return np.stack([pw[:, s::sets].sum(axis=1).max(axis=1) for s in range(sets)])

    dopp = rec.dopp_hz[::every]
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        peaks = list(ex.map(one_bin, dopp))
    best = np.max(np.stack(peaks), axis=0)
    return _cells(32, len(dopp), N, B, coh), best


def cpu_baseline(rec, args):
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    cells = 0
    reps = 0
    while reps < 1 or (time.perf_counter() - t0 < 3.0 and reps < 3):
        cells += _oracle_sample(rec, threads)
        reps += 1
    dt = time.perf_counter() - t0
    # one thread on a smaller sample (3 of 81 Doppler bins)
    t1 = time.perf_counter()
    cells1 = _oracle_sample(rec, 1, every=27)
    dt1 = time.perf_counter() - t1
    # optimised CPU pipeline (scipy.fft on all cores, complex64) on the same sample
    cpu_fft_acquire(rec, threads, every=27)  # warm the FFT plans
    t2 = time.perf_counter()
    cells2, reps2 = 0, 0
    while reps2 < 1 or (time.perf_counter() - t2 < 2.0 and reps2 < 50):
        cells2 += cpu_fft_acquire(rec, threads)[0]
        reps2 += 1
    dt2 = time.perf_counter() - t2
    return {"value": cells / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d x (27 of 81 Doppler bins, all 32 PRNs, 10 blocks, both sets), FP64 C oracle, "
                      "%d threads over Doppler rows, %.1f s wall" % (reps, threads, dt),
            "single_thread": {"value": cells1 / dt1, "unit": UNIT, "cores": 1,
                              "sample": "3 of 81 Doppler bins, all 32 PRNs, 10 blocks, both sets, %.1f s" % dt1},
            "optimised_cpu": {"value": cells2 / dt2, "unit": UNIT, "cores": threads,
                              "kind": "numpy + scipy.fft (pocketfft) complex64 pipeline, %d persistent workers "
                                      "taking Doppler bins as they free up" % threads,
                              "sample": "%d x (27 of 81 Doppler bins, all 32 PRNs, 10 blocks, both sets), %.1f s"
                                        % (reps2, dt2)}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    rec = siggen.weak_100ms()
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        _oracle_sample(rec, threads)
    times = []
    cells = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cells += _oracle_sample(rec, threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = cells / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded siggen)",
        "config": {"workload": WORKLOAD, "sample": "every 3rd Doppler bin (27 of 81) per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "27 of 81 Doppler bins x 32 PRNs x 10 blocks per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cufft", action="store_true")
    ap.add_argument("--no-code-doppler", action="store_true")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--no-track", action="store_true")
    ap.add_argument("--no-zoom", action="store_true")
    ap.add_argument("--no-sizes", action="store_true", help="skip the correlate at N = 2048 ... 16384")
    ap.add_argument("--variants", action="store_true",
                    help="also time every correlate variant the GPU accepts (100 ms request, N = 2048 ... 16384)")
    ap.add_argument("--batch-requests", type=int, default=256)
    ap.add_argument("--serve-rates", default="50,100,150,175,200,250,500:5,1000:5,2000:5",
                    help="offered request rates of the serving curve (requests/s), each 'rate' or "
                         "'rate:seconds' (overload points run shorter)")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="seconds of Poisson arrivals per rate")
    ap.add_argument("--serve-pool", type=int, default=64, help="distinct recordings in the serving pool")
    ap.add_argument("--serve-bound-ms", type=int, default=250,
                    help="server admission bound on the projected wait (ms, 0 = none)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
