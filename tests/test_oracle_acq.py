"""Pins of the oracle's acquisition chain (Section 3, Fig. 2): unpack, carrier
wipe-off + fold, FFT-form correlation, surfaces and detection.

Pins: format round trip against the generator's packer, closed forms for an
on-grid tone and for a noise-free replica, brute-force time-domain
correlation, and the injected satellites of the seeded 4 ms workload.
"""
import numpy as np
import pytest

import oracle
import siggen

rng = np.random.default_rng(11)


@pytest.mark.parametrize("fmt", [siggen.FMT_I8_IQ, siggen.FMT_2BIT_IQ])
@pytest.mark.parametrize("n", [1, 2, 7, 4096])
def test_unpack_inverts_pack(fmt, n):
    levels = np.array([-3, -1, 1, 3], np.int8)
    li = rng.choice(levels, n)
    lq = rng.choice(levels, n)
    raw = siggen.pack(li, lq, fmt)
    assert len(raw) == siggen.recording_bytes(n, fmt)
    x = oracle.unpack(raw, n, fmt)
    np.testing.assert_array_equal(x.real, li)
    np.testing.assert_array_equal(x.imag, lq)


def test_2bit_byte_layout():
    # byte = I0 | Q0<<2 | I1<<4 | Q1<<6, code c -> level 2c - 3
    raw = np.array([0b11_10_01_00], np.uint8)
    x = oracle.unpack(raw, 2, siggen.FMT_2BIT_IQ)
    np.testing.assert_array_equal(x, [-3 - 1j, 1 + 3j])


@pytest.mark.parametrize("coh", [1, 3])
def test_wipe_fold_tone_closed_form(coh):
    fs, N = 256_000, 256
    n = np.arange(coh * N * 2)
    f0 = 3250
    x = np.exp(2j * np.pi * f0 * n / fs)
    # on the bin: the carrier cancels exactly, every folded sample equals coh
    y = oracle.wipe_fold(x, fs, coh, f0, 1)
    np.testing.assert_allclose(y, coh * np.ones(N), atol=1e-11)
    # off the bin: geometric sum over the coherent milliseconds
    f = 1000
    y = oracle.wipe_fold(x, fs, coh, f, 1)
    m = np.arange(N)
    w = np.exp(2j * np.pi * (f0 - f) / fs)
    expect = sum(w ** (coh * N + i * N + m) for i in range(coh))
    np.testing.assert_allclose(y, expect, atol=1e-9)


def test_negative_doppler_phase_is_exact():
    fs, N = 256_000, 256
    n = np.arange(2 * N)
    x = np.exp(-2j * np.pi * 4750 * n / fs)
    np.testing.assert_allclose(oracle.wipe_fold(x, fs, 2, -4750, 0), 2 * np.ones(N), atol=1e-11)


@pytest.mark.parametrize("coh", [1, 2])
def test_fft_correlation_equals_brute_force(coh):
    """The FFT form is an exact rewrite of the time-domain correlation sum."""
    fs, N = 2_048_000, 2048
    n = (coh * 2) * N
    x = (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    for prn in (5, 27):
        chips = oracle.ca_code(prn)
        for f in (-3000, 0, 1500):
            a = oracle.corr_direct(x, fs, coh, f, 1, chips)
            b = oracle.corr_fft(x, fs, coh, f, 1, chips)
            assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_correlation_of_replica_is_its_autocorrelation():
    """Noise-free shifted replica: R[tau] = A * coh * periodic autocorrelation
    of the sampled replica at lag tau - tau_s (integer sums)."""
    fs, N, coh, tau_s, A = 1_024_000, 1024, 2, 300, 0.75
    chips = siggen.chip_table()[13].astype(np.int64)
    cs = chips[(np.arange(N) * 1023) // N]
    n = np.arange(coh * N)
    x = A * cs[(n - tau_s) % N]
    R = oracle.corr_fft(x.astype(complex), fs, coh, 0, 0, chips.astype(np.int8))
    auto = np.array([int(np.dot(cs, np.roll(cs, k))) for k in range(N)])
    expect = A * coh * auto[(np.arange(N) - tau_s) % N]
    np.testing.assert_allclose(R.real, expect, atol=1e-9)
    np.testing.assert_allclose(R.imag, 0, atol=1e-9)


def test_surface_closed_form_noise_free():
    """On-grid Doppler, integer-sample code phase, no noise: the cell at truth is
    A^2 L^2 per block of its set and is the maximum of the surface."""
    fs, N, coh, B = 2_048_000, 2048, 2, 4
    A, tau_s, f0, phi = 0.3, 1234, -1500, 0.4
    chips = siggen.chip_table()[6].astype(np.int64)  # PRN 7
    cs = chips[(np.arange(N) * 1023) // N]
    n = np.arange(coh * N * B)
    x = A * cs[(n - tau_s) % N] * np.exp(1j * (2 * np.pi * f0 * n / fs + phi))
    dopp = np.array([-2000, -1500, -1000], np.int64)
    for half in (False, True):
        S = oracle.surfaces(x, fs, coh, B, half, [7, 8], dopp)
        L = coh * N
        per_set = B // 2 if half else B
        for s in range(S.shape[0]):
            assert abs(S[s, 0, 1, tau_s] - per_set * A * A * L * L) <= 1e-9 * per_set * (A * L) ** 2
            assert np.unravel_index(np.argmax(S[s, 0]), S[s, 0].shape) == (1, tau_s)
        det = oracle.detect(S, [7, 8])
        assert det[0]["detected"] and det[0]["dopp_bin"] == 1 and det[0]["code_phase"] == tau_s
        assert not det[1]["detected"]


def test_detects_injected_satellites_plain_4ms():
    rec = siggen.plain_4ms()
    det, S = oracle.acquire(rec.raw, rec.n_samples, rec.fmt, rec.fs, rec.coh_ms, rec.dopp_hz,
                            np.arange(1, 33), nthreads=4)
    truth = {s.prn: s for s in rec.sats}
    found = {d["prn"] for d in det if d["detected"]}
    assert found == set(truth)
    for d in det:
        if d["prn"] in truth:
            s = truth[d["prn"]]
            tau = rec.truth_code_phase(s)
            drift = abs(s.dopp_hz) / 1540 * rec.n_samples / rec.fs * rec.N  # samples over the record
            dist = abs(d["code_phase"] - tau)
            assert min(dist, rec.N - dist) <= 1 + drift
            assert abs(d["dopp_hz"] - s.dopp_hz) <= rec.dopp_step_hz  # half a bin + scalloping


def test_peak_conventions_on_planted_surfaces():
    """Ties go to the smallest linear index; the second peak skips a circular
    band of ceil(N/1023) samples around the peak in the peak's row; the
    half-bit set with the larger ratio wins, ties to set 0.  (Conventions of
    this library; the paper gives no detection statistic.)"""
    N, D = 2048, 3
    S = np.full((2, 1, D, N), 1.0)
    S[0, 0, 1, 5] = S[0, 0, 2, 3] = 10.0        # tie: row 1 wins (smaller index)
    S[0, 0, 1, N - 1] = 9.0                     # circular distance 6 > 3: counts
    S[0, 0, 1, 7] = 9.5                         # distance 2 <= 3: excluded
    S[1] = S[0]                                 # identical set B: tie -> set 0
    d = oracle.detect(S, [1])[0]
    assert (d["set"], d["dopp_bin"], d["code_phase"]) == (0, 1, 5)
    assert d["second"] == 9.0
    S[1, 0, 0, 100] = 50.0                      # set B now has the larger ratio
    d = oracle.detect(S, [1])[0]
    assert d["set"] == 1 and d["ratio"] == 50.0
    assert oracle.exclusion(2048) == 3 and oracle.exclusion(4096) == 5
    assert oracle.exclusion(8192) == 9 and oracle.exclusion(16384) == 17
