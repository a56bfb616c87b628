"""FP64 CPU oracle for GPS L1 C/A FFT parallel code-phase acquisition.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA library is checked against; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code
with the CUDA path: the arithmetic lives in ``oracle/oracle.c`` (plain C,
double precision, no SIMD, no FFT library) and this module only marshals
numpy arrays through ctypes.

The method follows the acquisition channel of Section 3 (Fig. 2): code NCO
-> replica, carrier NCO -> first mixing (wipe-off), FFT of the mixed signal
and of the replica, frequency-domain mixing with the conjugate code
spectrum, IFFT, then signal detection.  Fine acquisition (the hand-off to
tracking of Fig. 1) is the gradient ascent in ``refine``.

Parity unpinned (conventions, not results of the paper): the half-bit set
choice, the detection threshold, the second-peak exclusion region and the
refinement step rule.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CHIPS = 1023
CHIP_RATE = 1.023e6


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (gcc, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        d, i, i64 = C.c_double, C.c_int, C.c_int64
        P = C.c_void_p
        _lib.orc_ca_code.argtypes = [i, P]
        _lib.orc_replica.argtypes = [P, i, P]
        _lib.orc_unpack.argtypes = [P, i64, i, P, P]
        _lib.orc_wipe_fold.argtypes = [P, P, i64, i, i, i64, i, P, P]
        _lib.orc_fft.argtypes = [P, P, i, i]
        _lib.orc_dft.argtypes = [P, P, i, i, P, P]
        _lib.orc_corr_direct.argtypes = [P, P, i64, i, i, i64, i, P, P, P]
        _lib.orc_corr_fft.argtypes = [P, P, i64, i, i, i64, i, P, P, P]
        _lib.orc_surfaces.argtypes = [P, P, i64, i64, i, i, i, P, i, P, i, i, i, P]
        _lib.orc_detect.argtypes = [P, i, i, i, i, i, i, d, P, P]
        _lib.orc_refine_eval.argtypes = [P, P, i64, d, P, d, d, P, P]
        _lib.orc_refine.argtypes = [P, P, i64, d, P, d, d, i, d, i, P]
        _lib.orc_track.argtypes = [P, P, i64, i64, i, i, P, d, d, d, d, d, P]
        _lib.orc_track.restype = i
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _split(x):
    x = np.asarray(x, dtype=np.complex128)
    return np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)


class _Peak(C.Structure):
    _fields_ = [("prn", C.c_int), ("detected", C.c_int), ("set", C.c_int),
                ("dopp_bin", C.c_int), ("code_phase", C.c_int), ("peak", C.c_double),
                ("second", C.c_double), ("ratio", C.c_double)]


class _Refined(C.Structure):
    _fields_ = [("f", C.c_double), ("tau", C.c_double), ("P", C.c_double),
                ("iters", C.c_int), ("status", C.c_int)]


def ca_code(prn: int) -> np.ndarray:
    """C/A code of PRN 1..32 as +-1 int8 chips (G2-delay formulation)."""
    out = np.zeros(CHIPS, np.int8)
    if _L().orc_ca_code(int(prn), _p(out)) != 0:
        raise ValueError("PRN must be 1..32")
    return out


def replica(chips: np.ndarray, N: int) -> np.ndarray:
    """c_s[m] = c[floor(m*1023/N)], m < N."""
    chips = np.ascontiguousarray(chips, np.int8)
    out = np.zeros(N, np.float64)
    _L().orc_replica(_p(chips), int(N), _p(out))
    return out


def unpack(raw: np.ndarray, n: int, fmt: int) -> np.ndarray:
    """Raw recording bytes -> complex128 samples (fmt 0 int8 I/Q, 1 2-bit I/Q)."""
    raw = np.ascontiguousarray(np.frombuffer(np.asarray(raw).tobytes(), np.uint8))
    re = np.zeros(n, np.float64)
    im = np.zeros(n, np.float64)
    if _L().orc_unpack(_p(raw), int(n), int(fmt), _p(re), _p(im)) != 0:
        raise ValueError("bad format")
    return re + 1j * im


def wipe_fold(x, fs: int, coh: int, f: int, b: int) -> np.ndarray:
    xr, xi = _split(x)
    N = fs // 1000
    yr = np.zeros(N)
    yi = np.zeros(N)
    _L().orc_wipe_fold(_p(xr), _p(xi), int(fs), N, int(coh), int(f), int(b), _p(yr), _p(yi))
    return yr + 1j * yi


def fft(x, inverse: bool = False) -> np.ndarray:
    """Textbook radix-2 FFT (forward unscaled, inverse scaled 1/N)."""
    xr, xi = _split(x)
    xr = xr.copy()
    xi = xi.copy()
    if _L().orc_fft(_p(xr), _p(xi), len(xr), int(inverse)) != 0:
        raise ValueError("N must be a power of two")
    return xr + 1j * xi


def dft(x, inverse: bool = False) -> np.ndarray:
    """Direct O(N^2) DFT with the same conventions as fft()."""
    xr, xi = _split(x)
    n = len(xr)
    outr = np.zeros(n)
    outi = np.zeros(n)
    _L().orc_dft(_p(xr), _p(xi), n, int(inverse), _p(outr), _p(outi))
    return outr + 1j * outi


def corr_direct(x, fs: int, coh: int, f: int, b: int, chips) -> np.ndarray:
    """Brute-force coherent correlation R[tau] of block b (time-domain sum)."""
    xr, xi = _split(x)
    N = fs // 1000
    chips = np.ascontiguousarray(chips, np.int8)
    rr = np.zeros(N)
    ri = np.zeros(N)
    _L().orc_corr_direct(_p(xr), _p(xi), int(fs), N, int(coh), int(f), int(b), _p(chips),
                         _p(rr), _p(ri))
    return rr + 1j * ri


def corr_fft(x, fs: int, coh: int, f: int, b: int, chips) -> np.ndarray:
    """FFT form of corr_direct: IFFT(FFT(fold(wipe(x))) * conj(FFT(replica)))."""
    xr, xi = _split(x)
    N = fs // 1000
    chips = np.ascontiguousarray(chips, np.int8)
    rr = np.zeros(N)
    ri = np.zeros(N)
    _L().orc_corr_fft(_p(xr), _p(xi), int(fs), N, int(coh), int(f), int(b), _p(chips),
                      _p(rr), _p(ri))
    return rr + 1j * ri


def code_doppler_shift(f: int, b: int, L: int) -> int:
    """Code-Doppler shift of block b at Doppler f, in samples: the nearest
    integer to f b L / f_L1 (halves up), f_L1 = 1540 x 1.023 MHz.  Computed
    with Python integers (exact)."""
    f_l1 = 1540 * 1023000
    return (2 * int(f) * int(b) * int(L) + f_l1) // (2 * f_l1)


def surfaces(x, fs: int, coh: int, nblocks: int, half_bit: bool, prns, dopp_hz,
             nthreads: int = 1, code_doppler: bool = False) -> np.ndarray:
    """Non-coherent power surfaces, float64 [sets][P][D][N]; with code_doppler
    block b enters as |R_b[(tau - sigma_b) mod N]|^2."""
    xr, xi = _split(x)
    N = fs // 1000
    prns = np.ascontiguousarray(prns, np.int32)
    dopp = np.ascontiguousarray(dopp_hz, np.int64)
    sets = 2 if half_bit else 1
    surf = np.zeros((sets, len(prns), len(dopp), N), np.float64)
    rc = _L().orc_surfaces(_p(xr), _p(xi), len(xr), int(fs), int(coh), int(nblocks),
                           int(bool(half_bit)), _p(prns), len(prns), _p(dopp), len(dopp),
                           int(nthreads), int(bool(code_doppler)), _p(surf))
    if rc != 0:
        raise ValueError("bad surface arguments")
    return surf


def exclusion(N: int) -> int:
    """Second-peak exclusion half-width in samples: ceil(N / 1023) (one chip)."""
    return -(-N // CHIPS)


def detect(surf: np.ndarray, prns, threshold: float = 2.0, excl: int | None = None,
           whole_surface: bool = False) -> list[dict]:
    """Peak / second-peak detection per PRN from surfaces [sets][P][D][N]."""
    surf = np.ascontiguousarray(surf, np.float64)
    sets, P, D, N = surf.shape
    if excl is None:
        excl = exclusion(N)
    prns = np.ascontiguousarray(prns, np.int32)
    out = (_Peak * P)()
    _L().orc_detect(_p(surf), sets, P, D, N, int(excl), int(bool(whole_surface)),
                    float(threshold), _p(prns), out)
    return [dict(prn=o.prn, detected=bool(o.detected), set=o.set, dopp_bin=o.dopp_bin,
                 code_phase=o.code_phase, peak=o.peak, second=o.second, ratio=o.ratio)
            for o in out]


def acquire(raw, n_samples: int, fmt: int, fs: int, coh: int, dopp_hz, prns,
            half_bit: bool = False, noncoh: int = 0, threshold: float = 2.0,
            nthreads: int = 1, whole_surface: bool = False, code_doppler: bool = False):
    """Whole acquisition: unpack, surfaces over all whole blocks (or the first
    noncoh), detection.  Returns (detections, surfaces)."""
    x = unpack(raw, n_samples, fmt)
    N = fs // 1000
    B = n_samples // (coh * N)
    if noncoh:
        B = min(B, noncoh)
    surf = surfaces(x, fs, coh, B, half_bit, prns, dopp_hz, nthreads, code_doppler)
    det = detect(surf, prns, threshold, whole_surface=whole_surface)
    for d in det:
        d["dopp_hz"] = int(np.asarray(dopp_hz)[d["dopp_bin"]])
    return det, surf


def refine_eval(x, L: int, fs: float, chips, f: float, tau: float):
    """Coherent power P(f, tau) over the first L samples and (dP/df, dP/dtau)."""
    xr, xi = _split(x)
    chips = np.ascontiguousarray(chips, np.float64)
    P = C.c_double()
    g = np.zeros(2)
    _L().orc_refine_eval(_p(xr), _p(xi), int(L), float(fs), _p(chips), float(f), float(tau),
                         C.byref(P), _p(g))
    return P.value, g


def refine(x, L: int, fs: float, chips, f0: float, tau0: float, max_iter: int = 100,
           search_hz: float = 0.0, flat_accept: bool = True) -> dict:
    """Gradient-ascent fine acquisition from (f0 Hz, tau0 chips), after a
    Doppler pre-search over +-search_hz at half-lobe spacing fs / (2 L).
    flat_accept: also take a Doppler trial that lowers |dP/df| at a loss of
    at most 1e-5 of P (the FP32 kernel's rule); off, Armijo alone."""
    xr, xi = _split(x)
    chips = np.ascontiguousarray(chips, np.float64)
    r = _Refined()
    _L().orc_refine(_p(xr), _p(xi), int(L), float(fs), _p(chips), float(f0), float(tau0),
                    int(max_iter), float(search_hz), int(bool(flat_accept)), C.byref(r))
    return dict(f=r.f, tau=r.tau, P=r.P, iters=r.iters, status=r.status)


TRACK_DTYPE = np.dtype([("f_hz", "<f8"), ("tau_chips", "<f8"), ("ze", "<f8", (2,)), ("zp", "<f8", (2,)),
                        ("zl", "<f8", (2,)), ("e_phi", "<f8"), ("e_tau", "<f8")])


def track(x, fs: int, coh_ms: int, n_int: int, chips, f0: float, tau0: float, spacing: float = 1.0,
          b_pll: float = 15.0, b_dll: float = 1.0) -> np.ndarray:
    """Tracking channel over n_int intervals of coh_ms ms from the recording
    start: per interval the NCO frequency, the replica delay at its start,
    the early / prompt / late correlators and both discriminators."""
    xr, xi = _split(x)
    chips = np.ascontiguousarray(chips, np.int8)
    out = np.zeros(n_int, TRACK_DTYPE)
    rc = _L().orc_track(_p(xr), _p(xi), len(xr), int(fs), int(coh_ms), int(n_int), _p(chips), float(f0),
                        float(tau0), float(spacing), float(b_pll), float(b_dll), _p(out))
    if rc != 0:
        raise ValueError("bad tracking arguments (%d)" % rc)
    return out
