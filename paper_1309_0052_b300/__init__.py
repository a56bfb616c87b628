"""Python binding of the B300 GPS L1 C/A acquisition library (libgnss.so).

Argument marshalling only: every step of the acquisition runs in the CUDA
kernels behind the C ABI declared in include/gnss.h.  Device buffers are
torch CUDA tensors (their data_ptr() is passed through); host buffers are
numpy arrays.  There is no CPU fallback: importing this package fails
loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgnss.so")

OK, EINVAL, ENOMEM, ECUDA, EBUSY, EAGAIN, ETIMEOUT, ECANCELLED = range(8)
STATUS_NAMES = ["GNSS_OK", "GNSS_EINVAL", "GNSS_ENOMEM", "GNSS_ECUDA", "GNSS_EBUSY", "GNSS_EAGAIN",
                "GNSS_ETIMEOUT", "GNSS_ECANCELLED"]
FMT_I8_IQ = 0
FMT_2BIT_IQ = 1
HALF_BIT = 0x1
SECOND_WHOLE = 0x2
CODE_DOPPLER = 0x4


class PlanDesc(C.Structure):
    _fields_ = [("fs_hz", C.c_uint32), ("coh_ms", C.c_uint32), ("noncoh", C.c_uint32),
                ("dopp_min_hz", C.c_int32), ("dopp_step_hz", C.c_uint32), ("n_dopp", C.c_uint32),
                ("prn_mask", C.c_uint64), ("threshold", C.c_float), ("flags", C.c_uint32),
                ("format", C.c_uint32), ("reserved", C.c_uint32)]


class Request(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("samples_dev", C.c_void_p), ("n_samples", C.c_size_t),
                ("out_dev", C.c_void_p), ("surface_dev", C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [("device_mem_budget", C.c_size_t), ("host_staging_bytes", C.c_size_t), ("max_batch", C.c_uint32),
                ("streams", C.c_uint32), ("queue_timeout_ms", C.c_uint32), ("max_queue_wait_ms", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("queued", C.c_uint64), ("batches_in_flight", C.c_uint32),
                ("refused", C.c_uint32), ("device_bytes_reserved", C.c_size_t)]


class TuneResult(C.Structure):
    _fields_ = [("N", C.c_uint32), ("n_variants", C.c_uint32), ("elems", C.c_uint32 * 16), ("ms", C.c_float * 16),
                ("chosen", C.c_uint32), ("prns_per_cta", C.c_uint32), ("bins_per_cta", C.c_uint32),
                ("reserved", C.c_uint32)]


class PlanInfo(C.Structure):
    _fields_ = [("N", C.c_uint32), ("n_prn", C.c_uint32), ("n_dopp", C.c_uint32), ("n_sets", C.c_uint32),
                ("excl", C.c_uint32), ("block_len", C.c_uint32), ("xcorr_variant", C.c_uint32)]


CANDIDATE_DTYPE = np.dtype([("prn", "u1"), ("reserved", "u1", (7,)), ("f_hz", "<f8"), ("tau_chips", "<f8")])
REFINED_DTYPE = np.dtype([("f_hz", "<f8"), ("tau_chips", "<f8"), ("power", "<f4"), ("iters", "<u4"),
                          ("status", "<i4"), ("n_eval", "<u2"), ("n_eval_grad", "<u2")])
assert CANDIDATE_DTYPE.itemsize == 24 and REFINED_DTYPE.itemsize == 32

TRACK_DTYPE = np.dtype([("f_hz", "<f8"), ("tau_chips", "<f8"), ("ze", "<f4", (2,)), ("zp", "<f4", (2,)),
                        ("zl", "<f4", (2,)), ("e_phi", "<f4"), ("e_tau", "<f4"), ("status", "<i4"),
                        ("reserved", "<u4")])
assert TRACK_DTYPE.itemsize == 56


class TrackConfig(C.Structure):
    _fields_ = [("coh_ms", C.c_uint32), ("n_int", C.c_uint32), ("spacing_chips", C.c_float),
                ("pll_bw_hz", C.c_float), ("dll_bw_hz", C.c_float), ("reserved", C.c_uint32)]


DETECTION_DTYPE = np.dtype([("prn", "u1"), ("detected", "u1"), ("set", "u1"), ("flags", "u1"),
                            ("dopp_bin", "<i4"), ("dopp_hz", "<i4"), ("code_phase", "<u4"),
                            ("peak", "<f4"), ("second", "<f4"), ("ratio", "<f4")])
assert DETECTION_DTYPE.itemsize == 28

_P = C.c_void_p
_st = C.c_int
_SIGS = {
    "gnss_plan_create": ([C.POINTER(PlanDesc), C.POINTER(_P)], _st),
    "gnss_plan_destroy": ([_P], _st),
    "gnss_plan_get_info": ([_P, C.POINTER(PlanInfo)], _st),
    "gnss_plan_codes": ([_P, _P, C.c_size_t], _st),
    "gnss_plan_code_spectra": ([_P, _P, C.c_size_t, _P], _st),
    "gnss_recording_bytes": ([C.c_uint32, C.c_size_t], C.c_size_t),
    "gnss_acquire": ([_P, _P, C.c_size_t, C.c_int, _P, _P, _P], _st),
    "gnss_acquire_device": ([_P, _P, C.c_size_t, _P, _P, _P], _st),
    "gnss_acquire_device_traced": ([_P, _P, C.c_size_t, _P, _P, _P, C.POINTER(_P)], _st),
    "gnss_acquire_noalloc": ([_P, _P, C.c_size_t, _P, _P, _P], _st),
    "gnss_stage_wipe_fft": ([_P, _P, C.c_size_t, C.c_uint32, _P, _P], _st),
    "gnss_stage_correlate": ([_P, _P, C.c_uint32, _P, _P, _P], _st),
    "gnss_refine_eval": ([_P, _P, C.c_size_t, C.c_uint32, _P, _P, _P, C.c_size_t, _P, _P, _P, _P], _st),
    "gnss_refine": ([_P, _P, C.c_size_t, C.c_int, _P, C.c_size_t, C.c_uint32, C.c_uint32, C.c_double, _P, _P],
                    _st),
    "gnss_refine_device": ([_P, _P, C.c_size_t, _P, C.c_size_t, C.c_uint32, C.c_uint32, C.c_double, _P, _P], _st),
    "gnss_acquire_batch": ([_P, C.c_size_t, C.c_size_t, _P], _st),
    "gnss_batch_graph_create": ([_P, C.c_size_t, C.c_size_t, C.POINTER(_P)], _st),
    "gnss_batch_graph_launch": ([_P, _P], _st),
    "gnss_batch_graph_destroy": ([_P], _st),
    "gnss_acquire_zoom": ([_P, _P, C.c_size_t, _P, C.c_size_t, C.c_uint32, C.c_uint32, _P, _P, _P], _st),
    "gnss_track": ([_P, _P, C.c_size_t, _P, C.c_size_t, C.POINTER(TrackConfig), _P, _P], _st),
    "gnss_server_create": ([_P, C.POINTER(_P)], _st),
    "gnss_server_destroy": ([_P], _st),
    "gnss_submit": ([_P, C.POINTER(PlanDesc), _P, C.c_size_t, C.POINTER(C.c_uint64)], _st),
    "gnss_poll": ([_P, C.c_uint64, _P, C.c_size_t, C.POINTER(C.c_size_t)], _st),
    "gnss_wait": ([_P, C.c_uint64, C.c_uint32, _P, C.c_size_t, C.POINTER(C.c_size_t)], _st),
    "gnss_cancel": ([_P, C.c_uint64], _st),
    "gnss_server_get_stats": ([_P, _P], _st),
    "gnss_server_inject_alloc_failure": ([_P, C.c_int], _st),
    "gnss_autotune": ([_P, C.c_uint32, _P], _st),
    "gnss_probe_ffma": ([C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), _P], _st),
    "gnss_testing_set_stage_wait_limit": ([C.c_uint32, _P], _st),
    "gnss_testing_set_buf_wait_limit": ([C.c_uint32, _P], _st),
    "gnss_last_error": ([], C.c_char_p),
}
_lib = None


def load():
    """Load libgnss.so (once).  Raises ImportError when it has not been built:
    there is no CPU fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libgnss.so is not built: run `python -m paper_1309_0052_b300.build` "
                              "(or __graft_entry__.build()) first; there is no CPU fallback")
        handle = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def __getattr__(name):
    if name == "lib":
        return load()
    raise AttributeError(name)


class GnssError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().gnss_last_error().decode(errors="replace")
        super().__init__("%s failed: %s: %s" % (where, STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


def check(status: int, where: str) -> None:
    if status != OK:
        raise GnssError(status, where)


def _ptr(obj) -> int | None:
    """Address of a torch tensor (device or host), numpy array or bytes; None for None."""
    if obj is None:
        return None
    if hasattr(obj, "data_ptr"):
        return obj.data_ptr()
    if isinstance(obj, np.ndarray):
        return obj.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


def recording_bytes(fmt: int, n_samples: int) -> int:
    return load().gnss_recording_bytes(fmt, n_samples)


def prn_mask(prns) -> int:
    m = 0
    for p in prns:
        m |= 1 << (int(p) - 1)
    return m


class Plan:
    """An acquisition plan (gnss_plan_create): Gold codes and code spectra of
    the searched PRNs resident on the current device."""

    def __init__(self, fs_hz: int, coh_ms: int, dopp_min_hz: int, dopp_step_hz: int, n_dopp: int,
                 prns=range(1, 33), noncoh: int = 0, threshold: float = 2.0, half_bit: bool = False,
                 second_whole: bool = False, fmt: int = FMT_2BIT_IQ, code_doppler: bool = False):
        self.desc = PlanDesc(fs_hz=fs_hz, coh_ms=coh_ms, noncoh=noncoh, dopp_min_hz=dopp_min_hz,
                             dopp_step_hz=dopp_step_hz, n_dopp=n_dopp, prn_mask=prn_mask(prns),
                             threshold=threshold,
                             flags=((HALF_BIT if half_bit else 0) | (SECOND_WHOLE if second_whole else 0)
                                    | (CODE_DOPPLER if code_doppler else 0)),
                             format=fmt)
        h = _P()
        check(load().gnss_plan_create(C.byref(self.desc), C.byref(h)), "gnss_plan_create")
        self._h = h
        info = PlanInfo()
        check(load().gnss_plan_get_info(h, C.byref(info)), "gnss_plan_get_info")
        self.N, self.n_prn, self.n_dopp, self.n_sets = info.N, info.n_prn, info.n_dopp, info.n_sets
        self.excl, self.block_len = info.excl, info.block_len
        self.fmt = fmt

    @classmethod
    def for_recording(cls, rec, prns=range(1, 33), **kw):
        """Plan matching a siggen.Recording's workload parameters."""
        return cls(rec.fs, rec.coh_ms, rec.dopp_min_hz, rec.dopp_step_hz, rec.n_dopp, prns=prns,
                   noncoh=rec.noncoh, half_bit=rec.half_bit, fmt=rec.fmt, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().gnss_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_blocks(self, n_samples: int) -> int:
        B = n_samples // self.block_len
        return min(B, self.desc.noncoh) if self.desc.noncoh else B

    def codes(self) -> np.ndarray:
        out = np.zeros((self.n_prn, 1023), np.int8)
        check(load().gnss_plan_codes(self._h, out.ctypes.data, out.nbytes), "gnss_plan_codes")
        return out

    def code_spectra(self, out, stream=None):
        """Copy C_p into a float32 CUDA tensor [n_prn, N, 2]."""
        check(load().gnss_plan_code_spectra(self._h, _ptr(out), out.numel() * 4, _stream_ptr(stream)),
              "gnss_plan_code_spectra")
        return out

    def autotune(self, force_elems: int = 0) -> dict:
        """gnss_autotune: time (or force) the correlate kernel's elements per
        thread for this plan's FFT size on the current device."""
        r = TuneResult()
        check(load().gnss_autotune(self._h, force_elems, C.byref(r)), "gnss_autotune")
        return {"N": r.N, "chosen": r.chosen, "prns_per_cta": r.prns_per_cta, "bins_per_cta": r.bins_per_cta,
                "timed": {int(r.elems[k]): float(r.ms[k]) for k in range(r.n_variants)}}

    def xcorr_variant(self) -> int:
        """Correlate-kernel variant code used for this plan's N on the current
        device now (gnss_plan_get_info)."""
        info = PlanInfo()
        check(load().gnss_plan_get_info(self._h, C.byref(info)), "gnss_plan_get_info")
        return int(info.xcorr_variant)

    def surface_shape(self):
        return (self.n_sets, self.n_prn, self.n_dopp, self.N)

    def acquire(self, samples, n_samples: int, surface=None, stream=None, out=None) -> np.ndarray:
        """gnss_acquire.  samples: numpy (host) or CUDA tensor (device).  out:
        optional host array of n_prn DETECTION_DTYPE records to fill (page-locked
        memory lets the records come back by an asynchronous copy).  Returns the
        detection records; synchronises the stream."""
        if out is None:
            out = np.zeros(self.n_prn, DETECTION_DTYPE)
        elif out.dtype != DETECTION_DTYPE or out.shape != (self.n_prn,) or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous array of n_prn DETECTION_DTYPE records")
        on_dev = int(hasattr(samples, "is_cuda") and samples.is_cuda)
        if not on_dev:
            samples = np.ascontiguousarray(samples)
        check(load().gnss_acquire(self._h, _ptr(samples), n_samples, on_dev, out.ctypes.data, _ptr(surface),
                               _stream_ptr(stream)), "gnss_acquire")
        if stream is not None:
            stream.synchronize()
        return out

    def acquire_device(self, samples_dev, n_samples: int, out_dev, surface=None, stream=None) -> None:
        """gnss_acquire_device: out_dev is a CUDA uint8 tensor of n_prn * 28 bytes."""
        check(load().gnss_acquire_device(self._h, _ptr(samples_dev), n_samples, _ptr(out_dev), _ptr(surface),
                                      _stream_ptr(stream)), "gnss_acquire_device")

    def acquire_noalloc(self, samples_dev, n_samples: int, out_dev, surface=None, stream=None) -> None:
        """gnss_acquire_noalloc: acquire_device with the library's fixed scratch
        (no allocation).  Asynchronous."""
        check(load().gnss_acquire_noalloc(self._h, _ptr(samples_dev), n_samples, _ptr(out_dev), _ptr(surface),
                                          _stream_ptr(stream)), "gnss_acquire_noalloc")

    def acquire_device_traced(self, samples_dev, n_samples: int, out_dev, events, surface=None,
                              stream=None) -> None:
        """gnss_acquire_device_traced: events are four torch.cuda.Event
        (enable_timing=True) recorded at the stage boundaries (before the fold,
        before the carrier FFT, before and after the correlate launch)."""
        import torch
        handles = (_P * 4)()
        for k, ev in enumerate(events):
            if ev is not None and not ev.cuda_event:  # torch creates the event on its first record
                ev.record(stream if stream is not None else torch.cuda.current_stream())
            handles[k] = ev.cuda_event if ev is not None else None
        check(load().gnss_acquire_device_traced(self._h, _ptr(samples_dev), n_samples, _ptr(out_dev),
                                             _ptr(surface), _stream_ptr(stream), handles),
              "gnss_acquire_device_traced")

    def stage_wipe_fft(self, samples_dev, n_samples: int, n_blocks: int, spectra_dev, stream=None) -> None:
        check(load().gnss_stage_wipe_fft(self._h, _ptr(samples_dev), n_samples, n_blocks, _ptr(spectra_dev),
                                      _stream_ptr(stream)), "gnss_stage_wipe_fft")

    def refine(self, samples, n_samples: int, cands: np.ndarray, coh_ms: int, max_iter: int = 100,
               search_hz: float = 0.0, stream=None) -> np.ndarray:
        """gnss_refine: Doppler pre-search over +-search_hz, then gradient
        ascent from each candidate (records from candidates()).  samples:
        numpy (host) or CUDA tensor.  Synchronises."""
        cands = np.ascontiguousarray(cands, CANDIDATE_DTYPE)
        out = np.zeros(len(cands), REFINED_DTYPE)
        on_dev = int(hasattr(samples, "is_cuda") and samples.is_cuda)
        if not on_dev:
            samples = np.ascontiguousarray(samples)
        check(load().gnss_refine(self._h, _ptr(samples), n_samples, on_dev, cands.ctypes.data, len(cands), coh_ms,
                                 max_iter, search_hz, out.ctypes.data, _stream_ptr(stream)), "gnss_refine")
        if stream is not None:
            stream.synchronize()
        return out

    def refine_device(self, samples_dev, n_samples: int, cands_dev, n_cand: int, coh_ms: int, max_iter: int,
                      out_dev, search_hz: float = 0.0, stream=None) -> None:
        check(load().gnss_refine_device(self._h, _ptr(samples_dev), n_samples, _ptr(cands_dev), n_cand, coh_ms,
                                        max_iter, search_hz, _ptr(out_dev), _stream_ptr(stream)),
              "gnss_refine_device")

    def refine_eval(self, samples_dev, n_samples: int, coh_ms: int, prn_dev, f_dev, tau_dev, P_dev,
                    dPdf_dev=None, dPdtau_dev=None, stream=None) -> None:
        """gnss_refine_eval on CUDA tensors: prn int32, f/tau float64, outputs float32."""
        check(load().gnss_refine_eval(self._h, _ptr(samples_dev), n_samples, coh_ms, _ptr(prn_dev), _ptr(f_dev),
                                      _ptr(tau_dev), prn_dev.numel(), _ptr(P_dev), _ptr(dPdf_dev),
                                      _ptr(dPdtau_dev), _stream_ptr(stream)), "gnss_refine_eval")

    def zoom(self, samples_dev, n_samples: int, detections, zoom: int = 5, span: int = 1, surface=None,
             stream=None) -> np.ndarray:
        """gnss_acquire_zoom: fine Doppler search (grid step / zoom over +-span
        steps) around each record of 'detections' (numpy DETECTION_DTYPE).
        Returns the fine records; synchronises the stream."""
        det = np.ascontiguousarray(detections, DETECTION_DTYPE)
        import torch  # device memory for the records
        out = torch.zeros(max(len(det), 1) * DETECTION_DTYPE.itemsize, dtype=torch.uint8,
                          device=samples_dev.device)
        check(load().gnss_acquire_zoom(self._h, _ptr(samples_dev), n_samples, det.ctypes.data, len(det), zoom,
                                       span, _ptr(out), _ptr(surface), _stream_ptr(stream)), "gnss_acquire_zoom")
        if stream is not None:
            stream.synchronize()
        else:
            torch.cuda.synchronize()
        return detections_from_bytes(out.cpu().numpy())[: len(det)]

    def track(self, samples_dev, n_samples: int, chans_dev, n_chan: int, out_dev, n_int: int, coh_ms: int = 1,
              spacing: float = 1.0, pll_bw_hz: float = 15.0, dll_bw_hz: float = 1.0, stream=None) -> None:
        """gnss_track on CUDA tensors: chans_dev holds n_chan candidate
        records (candidates()), out_dev n_chan * n_int track records."""
        cfg = TrackConfig(coh_ms, n_int, spacing, pll_bw_hz, dll_bw_hz, 0)
        check(load().gnss_track(self._h, _ptr(samples_dev), n_samples, _ptr(chans_dev), n_chan, C.byref(cfg),
                                _ptr(out_dev), _stream_ptr(stream)), "gnss_track")

    def stage_correlate(self, spectra_dev, n_blocks: int, out_dev, surface=None, stream=None) -> None:
        check(load().gnss_stage_correlate(self._h, _ptr(spectra_dev), n_blocks, _ptr(surface), _ptr(out_dev),
                                       _stream_ptr(stream)), "gnss_stage_correlate")


def acquire_batch(requests, scratch_budget: int = 0, stream=None) -> None:
    """gnss_acquire_batch.  requests: iterable of (plan, samples_dev, n_samples,
    out_dev, surface_dev or None) with CUDA tensors.  Asynchronous."""
    reqs = list(requests)
    arr = (Request * len(reqs))()
    for k, (plan, smp, n, out, surf) in enumerate(reqs):
        arr[k] = Request(plan.handle.value if hasattr(plan.handle, "value") else plan.handle, _ptr(smp), n,
                         _ptr(out), _ptr(surf))
    check(load().gnss_acquire_batch(arr, len(reqs), scratch_budget, _stream_ptr(stream)), "gnss_acquire_batch")


class BatchGraph:
    """gnss_batch_graph_*: a batch of requests (as for acquire_batch) captured
    once into a CUDA graph; launch() replays it.  The tensors of the requests
    are kept referenced for the graph's life (their addresses are baked in)."""

    def __init__(self, requests, scratch_budget: int = 0):
        self._reqs = list(requests)
        arr = (Request * len(self._reqs))()
        for k, (plan, smp, n, out, surf) in enumerate(self._reqs):
            arr[k] = Request(plan.handle.value if hasattr(plan.handle, "value") else plan.handle, _ptr(smp), n,
                             _ptr(out), _ptr(surf))
        self._h = C.c_void_p()
        check(load().gnss_batch_graph_create(arr, len(self._reqs), scratch_budget, C.byref(self._h)),
              "gnss_batch_graph_create")

    def launch(self, stream=None) -> None:
        check(load().gnss_batch_graph_launch(self._h, _stream_ptr(stream)), "gnss_batch_graph_launch")

    def close(self) -> None:
        if self._h:
            load().gnss_batch_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server with continuous batching (gnss_server_*)."""

    def __init__(self, device_mem_budget: int = 0, host_staging_bytes: int = 0, max_batch: int = 0,
                 streams: int = 0, queue_timeout_ms: int = 0, max_queue_wait_ms: int = 0):
        cfg = ServerConfig(device_mem_budget, host_staging_bytes, max_batch, streams, queue_timeout_ms,
                           max_queue_wait_ms)
        h = _P()
        check(load().gnss_server_create(C.byref(cfg), C.byref(h)), "gnss_server_create")
        self._h = h

    @staticmethod
    def desc_for(rec, prns=range(1, 33), threshold: float = 2.0) -> PlanDesc:
        return PlanDesc(fs_hz=rec.fs, coh_ms=rec.coh_ms, noncoh=rec.noncoh, dopp_min_hz=rec.dopp_min_hz,
                        dopp_step_hz=rec.dopp_step_hz, n_dopp=rec.n_dopp, prn_mask=prn_mask(prns),
                        threshold=threshold, flags=HALF_BIT if rec.half_bit else 0, format=rec.fmt)

    def submit(self, desc: PlanDesc, samples: np.ndarray, n_samples: int) -> int:
        t = C.c_uint64()
        samples = np.ascontiguousarray(samples)
        check(load().gnss_submit(self._h, C.byref(desc), samples.ctypes.data, n_samples, C.byref(t)), "gnss_submit")
        return t.value

    def poll(self, ticket: int, cap: int = 32):
        """Records (numpy) when done, None while pending; raises GnssError on failure."""
        out = np.zeros(cap, DETECTION_DTYPE)
        n = C.c_size_t()
        st = load().gnss_poll(self._h, ticket, out.ctypes.data, cap, C.byref(n))
        if st == EAGAIN:
            return None
        check(st, "gnss_poll")
        return out[: min(n.value, cap)]

    def wait(self, ticket: int, timeout_ms: int = 60000, cap: int = 32):
        out = np.zeros(cap, DETECTION_DTYPE)
        n = C.c_size_t()
        check(load().gnss_wait(self._h, ticket, timeout_ms, out.ctypes.data, cap, C.byref(n)), "gnss_wait")
        return out[: min(n.value, cap)]

    def cancel(self, ticket: int) -> None:
        check(load().gnss_cancel(self._h, ticket), "gnss_cancel")

    def stats(self) -> dict:
        s = ServerStats()
        check(load().gnss_server_get_stats(self._h, C.byref(s)), "gnss_server_get_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def inject_alloc_failure(self, k: int) -> None:
        check(load().gnss_server_inject_alloc_failure(self._h, k), "gnss_server_inject_alloc_failure")

    def close(self):
        if getattr(self, "_h", None):
            load().gnss_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def candidates(prn, f_hz, tau_chips) -> np.ndarray:
    """Pack candidate arrays into gnss_candidate records."""
    prn = np.atleast_1d(np.asarray(prn))
    out = np.zeros(len(prn), CANDIDATE_DTYPE)
    out["prn"] = prn
    out["f_hz"] = f_hz
    out["tau_chips"] = tau_chips
    return out


def probe_ffma(iters: int = 4096, stream=None):
    """Measured FP32 FMA throughput (TFLOP/s) and kernel time (ms)."""
    tf, ms = C.c_double(), C.c_double()
    check(load().gnss_probe_ffma(iters, C.byref(tf), C.byref(ms), _stream_ptr(stream)), "gnss_probe_ffma")
    return tf.value, ms.value


def set_stage_wait_limit(iters: int, stream=None) -> None:
    """gnss_testing_set_stage_wait_limit (a testing hook): polls of each
    staged-correlate wait before it gives up (0: every wait gives up at once;
    the default is 4194304)."""
    check(load().gnss_testing_set_stage_wait_limit(iters, _stream_ptr(stream)), "gnss_testing_set_stage_wait_limit")


def set_buf_wait_limit(iters: int, stream=None) -> None:
    """gnss_testing_set_buf_wait_limit (a testing hook): polls of each wait of
    the class-local occupancy forms (4096, 8192, 16384) for their exchange
    buffer's release (0: every wait gives up at once and the call's records
    are flagged WAIT_TIMEOUT; the default is 4194304)."""
    check(load().gnss_testing_set_buf_wait_limit(iters, _stream_ptr(stream)), "gnss_testing_set_buf_wait_limit")


STAGE_TIMEOUT = 0x01  # GNSS_DET_STAGE_TIMEOUT: a record's flags bit
WAIT_TIMEOUT = 0x02  # GNSS_DET_WAIT_TIMEOUT: a record's flags bit (records not valid)
STAGE_WAIT_DEFAULT = 1 << 22


def detections_from_bytes(buf) -> np.ndarray:
    """View a device-side detection buffer copied to host (uint8) as records."""
    return np.frombuffer(np.asarray(buf, np.uint8).tobytes(), DETECTION_DTYPE)


def track_records(buf) -> np.ndarray:
    """Track records from the raw bytes of a device output buffer."""
    return np.frombuffer(np.asarray(buf).tobytes(), TRACK_DTYPE)
