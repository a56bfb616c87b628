"""Seeded synthetic GPS L1 C/A recordings shared by the tests and the benchmark.

The paper's input (a proprietary 12-channel client recording) is not
available, so every input is synthesised here with the shape of the paper's
workload: complex baseband at IF 0, a handful of visible satellites with
random code phase, Doppler, carrier phase and +-1 navigation bits every
20 ms, complex AWGN of unit power, and a 2-bit ADC (Section 4.2 notes the
limited resolution of the front-end samples).

This module holds none of the acquisition arithmetic: it only synthesises the
transmitted signal from a stored chip table (``ca_chips.txt``, written by
``write_ca_chips.py`` from the oracle) and packs the samples in the two
recording formats.  Every random number comes from
``numpy.random.Generator(PCG64(seed))`` drawn in a fixed order (satellites,
then noise).

Signal model (per satellite, t = n / fs):
    s(t) = A d(t) c[floor(pos(t)) mod 1023] exp(j (2 pi (f_d t + rate t^2 / 2) + phi0))
    pos(t) = R_c t - tau0 + (f_d t + rate t^2 / 2) / 1540      (code Doppler)
    A = sqrt(10^(CN0/10) / fs)                                 (noise power 1)
The truth code phase in samples at t = 0 is tau0 * N / 1023 (mod N).
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

CHIP_RATE = 1.023e6
CHIPS = 1023
L1_PER_CHIP = 1540  # carrier cycles per chip (f_L1 / R_c)
SEED_BASE = 1309005200

FMT_I8_IQ = 0
FMT_2BIT_IQ = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_TABLE = None


def chip_table() -> np.ndarray:
    """int8 [32][1023] of +-1 chips from ca_chips.txt (row p-1 = PRN p)."""
    global _TABLE
    if _TABLE is None:
        rows = []
        with open(os.path.join(_HERE, "ca_chips.txt")) as fh:
            for line in fh:
                prn, bits = line.split()
                rows.append((int(prn), np.array([1 - 2 * int(ch) for ch in bits], np.int8)))
        rows.sort()
        _TABLE = np.stack([r[1] for r in rows])
    return _TABLE


@dataclass
class Sat:
    prn: int
    cn0_dbhz: float
    dopp_hz: float
    code_phase_chips: float
    carrier_phase: float
    bit_edge_ms: float
    dopp_rate: float = 0.0
    bits: np.ndarray = field(default_factory=lambda: np.ones(1, np.int8))


@dataclass
class Recording:
    raw: np.ndarray          # uint8 bytes in the recording format
    fmt: int
    fs: int
    n_samples: int
    sats: list
    # acquisition parameters of the workload this recording stands for
    coh_ms: int = 1
    dopp_min_hz: int = 0
    dopp_step_hz: int = 500
    n_dopp: int = 1
    half_bit: bool = False
    noncoh: int = 0

    @property
    def N(self) -> int:
        return self.fs // 1000

    @property
    def dopp_hz(self) -> np.ndarray:
        return self.dopp_min_hz + self.dopp_step_hz * np.arange(self.n_dopp, dtype=np.int64)

    @property
    def n_blocks(self) -> int:
        B = self.n_samples // (self.coh_ms * self.N)
        return min(B, self.noncoh) if self.noncoh else B

    def truth_code_phase(self, sat: Sat) -> float:
        """Injected code phase in samples at t = 0, in [0, N)."""
        return (sat.code_phase_chips * self.N / CHIPS) % self.N

    def truth_at(self, sat: Sat, t: float):
        """Injected Doppler (Hz) and code delay (chips, in [0, 1023)) of a
        satellite at time t (s) from the recording start: the Doppler moves
        at its rate, and the delay falls by the carrier cycles over 1540
        (code Doppler), as synthesize builds them."""
        cycles = sat.dopp_hz * t + 0.5 * sat.dopp_rate * t * t
        return sat.dopp_hz + sat.dopp_rate * t, (sat.code_phase_chips - cycles / L1_PER_CHIP) % CHIPS


def draw_sats(rng, n_sats, cn0, dopp, rec_ms, rate=0.0, edge_range=(0.0, 20.0), prns=None):
    """Draw n_sats distinct satellites: PRN, C/N0 ~ U(cn0), Doppler ~ U(dopp),
    code phase ~ U[0, 1023) chips, carrier phase ~ U[0, 2 pi), first bit edge
    ~ U(edge_range) ms and one +-1 bit per 20 ms period."""
    if prns is None:
        prns = rng.choice(np.arange(1, 33), size=n_sats, replace=False)
    sats = []
    nbits = int(np.ceil(rec_ms / 20.0)) + 2
    for prn in prns:
        s = Sat(prn=int(prn),
                cn0_dbhz=float(rng.uniform(*cn0)),
                dopp_hz=float(rng.uniform(*dopp)),
                code_phase_chips=float(rng.uniform(0.0, CHIPS)),
                carrier_phase=float(rng.uniform(0.0, 2 * np.pi)),
                bit_edge_ms=float(rng.uniform(*edge_range)),
                dopp_rate=float(rate))
        s.bits = rng.choice(np.array([-1, 1], np.int8), size=nbits)
        sats.append(s)
    return sats


def synthesize(rng, fs: int, n: int, sats, noise: bool = True, nav_bits: bool = True,
               code_doppler: bool = True, amplitude: float | None = None) -> np.ndarray:
    """Complex baseband samples (complex128) of the satellites plus AWGN."""
    table = chip_table()
    t = np.arange(n, dtype=np.float64) / fs
    x = np.zeros(n, np.complex128)
    for s in sats:
        A = amplitude if amplitude is not None else np.sqrt(10.0 ** (s.cn0_dbhz / 10.0) / fs)
        dph = s.dopp_hz * t + 0.5 * s.dopp_rate * t * t
        pos = CHIP_RATE * t - s.code_phase_chips
        if code_doppler:
            pos = pos + dph / L1_PER_CHIP
        chip = table[s.prn - 1][np.floor(pos).astype(np.int64) % CHIPS].astype(np.float64)
        sig = chip * np.exp(1j * (2 * np.pi * dph + s.carrier_phase))
        if nav_bits:
            k = np.floor((t * 1000.0 - s.bit_edge_ms) / 20.0).astype(np.int64) + 1
            sig = sig * s.bits[np.clip(k, 0, len(s.bits) - 1)]
        x += A * sig
    if noise:
        x += (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.sqrt(0.5)
    return x


def quantize_2bit(x: np.ndarray, sats, fs: int, noise: bool = True):
    """2-bit ADC per component: thresholds {-t, 0, +t}, t = per-component total
    standard deviation, levels {-3, -1, +1, +3}.  Returns int8 (I, Q) levels."""
    p = (0.5 if noise else 0.0) + sum(10.0 ** (s.cn0_dbhz / 10.0) / fs for s in sats) / 2.0
    thr = np.sqrt(p) if p > 0 else 1.0

    def q(v):
        return np.where(v < -thr, -3, np.where(v < 0, -1, np.where(v < thr, 1, 3))).astype(np.int8)

    return q(x.real), q(x.imag)


def pack(li: np.ndarray, lq: np.ndarray, fmt: int) -> np.ndarray:
    """Levels -> recording bytes.  fmt 0: int8 I,Q interleaved.  fmt 1: two
    complex samples per byte, byte = I0 | Q0<<2 | I1<<4 | Q1<<6 with code
    c = (level + 3) / 2."""
    if fmt == FMT_I8_IQ:
        out = np.empty(2 * len(li), np.int8)
        out[0::2] = li
        out[1::2] = lq
        return out.view(np.uint8)
    if fmt == FMT_2BIT_IQ:
        n = len(li)
        ci = ((li.astype(np.int16) + 3) // 2).astype(np.uint8)
        cq = ((lq.astype(np.int16) + 3) // 2).astype(np.uint8)
        if n % 2:
            ci = np.append(ci, np.uint8(1))
            cq = np.append(cq, np.uint8(1))
        return (ci[0::2] | (cq[0::2] << 2) | (ci[1::2] << 4) | (cq[1::2] << 6)).astype(np.uint8)
    raise ValueError("unknown format")


def recording_bytes(n_samples: int, fmt: int) -> int:
    return 2 * n_samples if fmt == FMT_I8_IQ else (n_samples + 1) // 2


def make_recording(seed: int, fs: int, n_samples: int, fmt: int, n_sats: int, cn0, dopp,
                   rate=0.0, edge_range=(0.0, 20.0), **acq) -> Recording:
    rng = np.random.Generator(np.random.PCG64(seed))
    rec_ms = 1000.0 * n_samples / fs
    sats = draw_sats(rng, n_sats, cn0, dopp, rec_ms, rate=rate, edge_range=edge_range)
    x = synthesize(rng, fs, n_samples, sats)
    li, lq = quantize_2bit(x, sats, fs)
    return Recording(raw=pack(li, lq, fmt), fmt=fmt, fs=fs, n_samples=n_samples, sats=sats, **acq)


# --------------------------------------------------------------------------
# The five workloads (seed = 1309005200 + workload number)
# --------------------------------------------------------------------------

def plain_4ms(seed: int = SEED_BASE + 1) -> Recording:
    """Plain acquisition: fs 2.048 MHz, 4 ms (8192 samples), int8 I/Q from a
    2-bit ADC, 21 Doppler bins of 500 Hz over +-5 kHz, 1 ms coherent x 4
    non-coherent, 4 satellites at C/N0 42-48 dB-Hz, Doppler in +-4.5 kHz."""
    return make_recording(seed, 2_048_000, 8192, FMT_I8_IQ, 4, (42.0, 48.0), (-4500.0, 4500.0),
                          coh_ms=1, dopp_min_hz=-5000, dopp_step_hz=500, n_dopp=21)


def weak_100ms(seed: int = SEED_BASE + 2) -> Recording:
    """Single cloud request, weak signals: fs 4.096 MHz, 100 ms, 2-bit packed
    I/Q (204,800 bytes), 81 Doppler bins of 250 Hz over +-10 kHz, 10 ms
    coherent x 10 blocks with half-bit sets, 8 satellites at C/N0 28-45 dB-Hz,
    Doppler in +-9.5 kHz, Doppler rate 0.5 Hz/s."""
    return make_recording(seed, 4_096_000, 409_600, FMT_2BIT_IQ, 8, (28.0, 45.0),
                          (-9500.0, 9500.0), rate=0.5,
                          coh_ms=10, dopp_min_hz=-10000, dopp_step_hz=250, n_dopp=81,
                          half_bit=True)


def _batch_params(n_req, seed, fs_choices, ms_range, sats_range):
    """Per-request (fs, ms, step, n_sats, sub-seed), drawn in request order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    params = []
    for _ in range(n_req):
        fs = int(rng.choice(fs_choices))
        ms = int(rng.integers(ms_range[0], ms_range[1] + 1))
        step = int(rng.choice([250, 500]))
        nsat = int(rng.integers(sats_range[0], sats_range[1] + 1))
        sub = int(rng.integers(0, 2**31))
        params.append((fs, ms, step, nsat, sub))
    return params


def _batch_recording(p, cn0) -> Recording:
    fs, ms, step, nsat, sub = p
    coh = 500 // step
    return make_recording(sub, fs, fs // 1000 * ms, FMT_2BIT_IQ, nsat, cn0, (-9500.0, 9500.0),
                          coh_ms=coh, dopp_min_hz=-10000, dopp_step_hz=step, n_dopp=20000 // step + 1)


def batch_requests(n_req: int = 256, seed: int = SEED_BASE + 3, fs_choices=(2_048_000, 4_096_000, 8_192_000),
                   ms_range=(20, 200), sats_range=(4, 10), cn0=(30.0, 48.0)) -> list:
    """Batched workload: uneven recordings, 2-bit packed, each with its own
    fs, length (integer ms), Doppler step in {250, 500} Hz over +-10 kHz and
    coherent length 500 / step ms."""
    return [_batch_recording(p, cn0) for p in _batch_params(n_req, seed, fs_choices, ms_range, sats_range)]


def batch_requests_subset(arg) -> list:
    """Requests idx of batch_requests(n) with its default parameters, for
    generation in parallel worker processes: arg = (n, idx)."""
    n, idx = arg
    params = _batch_params(n, SEED_BASE + 3, (2_048_000, 4_096_000, 8_192_000), (20, 200), (4, 10))
    return [_batch_recording(params[i], (30.0, 48.0)) for i in idx]


def refine_12ms(seed: int = SEED_BASE + 4) -> Recording:
    """Fine-acquisition recording: plain-acquisition parameters (2.048 MHz,
    int8 I/Q, 21 bins of 500 Hz, 1 ms coherent) with 8 satellites over 12 ms
    and the navigation-bit edges placed after the first 10 ms."""
    return make_recording(seed, 2_048_000, 24_576, FMT_I8_IQ, 8, (42.0, 48.0),
                          (-4500.0, 4500.0), edge_range=(10.0, 20.0),
                          coh_ms=1, dopp_min_hz=-5000, dopp_step_hz=500, n_dopp=21)


def refine_candidates(rec: Recording, n_random: int = 1000, seed: int = SEED_BASE + 4):
    """1000 seeded random off-peak candidates (prn, f Hz, tau chips); drawn
    from a second stream of the same seed."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    prn = rng.integers(1, 33, size=n_random)
    f = rng.uniform(-5000.0, 5000.0, size=n_random)
    tau = rng.uniform(0.0, CHIPS, size=n_random)
    return prn, f, tau


def long_400ms(seed: int = SEED_BASE + 6) -> Recording:
    """Long weak-signal request where code Doppler matters: fs 4.096 MHz,
    400 ms 2-bit packed I/Q (819,200 bytes), 81 Doppler bins of 250 Hz over
    +-10 kHz, 10 ms coherent x 40 blocks with half-bit sets, 8 satellites at
    C/N0 27-36 dB-Hz, Doppler in +-9.5 kHz (up to 2.5 chips of code walk over
    the recording), Doppler rate 0.5 Hz/s."""
    return make_recording(seed, 4_096_000, 1_638_400, FMT_2BIT_IQ, 8, (27.0, 36.0),
                          (-9500.0, 9500.0), rate=0.5,
                          coh_ms=10, dopp_min_hz=-10000, dopp_step_hz=250, n_dopp=81,
                          half_bit=True)


def track_1s(seed: int = SEED_BASE + 7) -> Recording:
    """Tracking recording: fs 4.096 MHz, 1 s 2-bit packed I/Q (2,048,000
    bytes), 8 satellites at C/N0 38-48 dB-Hz, Doppler in +-4.5 kHz, Doppler
    rate 0.5 Hz/s, data bits every 20 ms."""
    return make_recording(seed, 4_096_000, 4_096_000, FMT_2BIT_IQ, 8, (38.0, 48.0), (-4500.0, 4500.0),
                          rate=0.5, coh_ms=1, dopp_min_hz=-5000, dopp_step_hz=500, n_dopp=21)


def track_starts(rec: Recording, seed: int = SEED_BASE + 7):
    """Tracking start points of the injected satellites, as a refined
    acquisition would hand them over: truth Doppler + U(-5, 5) Hz, truth code
    phase + U(-0.1, 0.1) chip.  Returns (prn, f Hz, tau chips) arrays."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    prn = np.array([s.prn for s in rec.sats])
    f = np.array([s.dopp_hz for s in rec.sats]) + rng.uniform(-5.0, 5.0, len(prn))
    tau = (np.array([s.code_phase_chips for s in rec.sats]) + rng.uniform(-0.1, 0.1, len(prn))) % CHIPS
    return prn, f, tau


def serving_requests(n_req: int, seed: int = SEED_BASE + 5, ms_range=(10, 500),
                     fs_choices=(2_048_000, 4_096_000, 8_192_000, 16_384_000)) -> list:
    """Serving workload: recordings 10-500 ms, fs in {2.048 .. 16.384} MHz,
    2-12 satellites at 28-48 dB-Hz, Doppler +-10 kHz with step 250 or 500 Hz
    and coherent length 500 / step ms."""
    return batch_requests(n_req, seed=seed, fs_choices=fs_choices, ms_range=ms_range,
                          sats_range=(2, 12), cn0=(28.0, 48.0))


def serving_requests_subset(arg) -> list:
    """Requests idx of serving_requests(n) with its default parameters, for
    generation in parallel worker processes: arg = (n, idx)."""
    n, idx = arg
    params = _batch_params(n, SEED_BASE + 5, (2_048_000, 4_096_000, 8_192_000, 16_384_000), (10, 500), (2, 12))
    return [_batch_recording(params[i], (28.0, 48.0)) for i in idx]
