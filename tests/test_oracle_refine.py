"""Pins of the oracle's fine-acquisition objective, gradient and ascent.

P(f, tau) = |sum_n x[n] exp(-j 2 pi f n / fs) ctilde(t_n)|^2 with a linearly
interpolated replica.  Pins: the Dirichlet closed form with the code removed
(and its derivative), a chip-run closed form at fs = 2.046 MHz, central
finite differences, and convergence to the injected (f, tau).
"""
import numpy as np
import pytest

import oracle
import siggen

FS = 2_048_000
L = 20_480


def _dirichlet(df, L, fs):
    a = np.pi * df / fs
    return (np.sin(a * L) / np.sin(a)) ** 2


def _dirichlet_deriv(df, L, fs):
    # d/d(df) of sin^2(aL)/sin^2(a), a = pi df / fs; P depends on f via df = f0 - f
    a = np.pi * df / fs
    s, sl = np.sin(a), np.sin(a * L)
    dP_da = 2 * sl * np.cos(a * L) * L / s ** 2 - 2 * sl ** 2 * np.cos(a) / s ** 3
    return dP_da * np.pi / fs


@pytest.mark.parametrize("df", [0.37, 13.0, -41.5, 77.7])
def test_pure_tone_dirichlet(df):
    f0 = 1500.0
    n = np.arange(L)
    x = np.exp(2j * np.pi * f0 * n / FS)
    ones = np.ones(1023)
    f = f0 - df
    P, g = oracle.refine_eval(x, L, FS, ones, f, 123.4)
    ref = _dirichlet(df, L, FS)
    assert abs(P - ref) <= 1e-9 * L * L
    # dP/df = dP/d(df) * d(df)/df = -dP/d(df)
    assert abs(g[0] + _dirichlet_deriv(df, L, FS)) <= 1e-7 * L * L / (FS / L)
    assert g[1] == 0.0  # a constant code has no slope


def test_chip_run_closed_form():
    """fs = 2.046 MHz gives exactly two samples per chip.  For the rectangular
    chip signal at delay 0 and tau = 0, even samples meet the midpoint of two
    interpolated chips and odd samples meet a chip centre, so over one period
    z = 1023 + (1023 + A1) / 2 with A1 the lag-1 periodic autocorrelation."""
    fs = 2_046_000.0
    chips = siggen.chip_table()[9].astype(np.int64)  # PRN 10
    n = np.arange(2046)
    x = chips[(n // 2) % 1023].astype(complex)
    A1 = int(np.dot(chips, np.roll(chips, -1)))
    assert A1 in (-1, 63, -65)
    P, _ = oracle.refine_eval(x, 2046, fs, chips.astype(float), 0.0, 0.0)
    z = 1023 + (1023 + A1) / 2
    assert abs(P - z * z) <= 1e-9 * z * z


def _signal(prn=7, f=1234.5, tau=300.3, noise=False, seed=3):
    rng = np.random.default_rng(seed)
    s = siggen.Sat(prn=prn, cn0_dbhz=45.0, dopp_hz=f, code_phase_chips=tau, carrier_phase=0.7,
                   bit_edge_ms=15.0)
    return siggen.synthesize(rng, FS, L, [s], noise=noise, nav_bits=False, code_doppler=False,
                             amplitude=None if noise else 1.0)


def test_gradient_matches_central_differences_noise_free():
    """Central differences with 1e-3 Hz / 1e-3 chip steps.  P is smooth in f,
    so dP/df is compared directly (tolerance 1e-3 of P_peak T).  In tau, P is
    piecewise quadratic with a kink about every 1/2048 chip, so the 1e-3 chip
    central difference equals the MEAN of the analytic right derivative over
    the window; that mean (201 points) is compared (1e-4 of P_peak)."""
    x = _signal()
    chips = oracle.ca_code(7).astype(float)
    Ppk, _ = oracle.refine_eval(x, L, FS, chips, 1234.5, 300.3)
    T = L / FS
    for f, tau in [(1230.0, 300.1), (1250.0, 300.7), (1200.0, 299.8), (1234.5, 300.45)]:
        P, g = oracle.refine_eval(x, L, FS, chips, f, tau)
        hf, ht = 1e-3, 1e-3
        fd_f = (oracle.refine_eval(x, L, FS, chips, f + hf, tau)[0]
                - oracle.refine_eval(x, L, FS, chips, f - hf, tau)[0]) / (2 * hf)
        fd_t = (oracle.refine_eval(x, L, FS, chips, f, tau + ht)[0]
                - oracle.refine_eval(x, L, FS, chips, f, tau - ht)[0]) / (2 * ht)
        assert abs(g[0] - fd_f) <= 1e-3 * Ppk * T
        grid = tau - ht + (np.arange(201) + 0.5) * (2 * ht / 201)
        mean_g = np.mean([oracle.refine_eval(x, L, FS, chips, f, t)[1][1] for t in grid])
        assert abs(mean_g - fd_t) <= 1e-4 * Ppk


def test_tau_gradient_is_the_segment_slope_with_noise():
    """With noise every interpolation kink (about every 1/2048 chip) changes the
    slope by O(|z| |x[n]|), so the analytic dP/dtau is checked as the right
    derivative: a difference with a step far below the kink spacing.
    dP/df is smooth and keeps the 1e-3 Hz central difference."""
    x = _signal(noise=True)
    chips = oracle.ca_code(7).astype(float)
    Ppk, _ = oracle.refine_eval(x, L, FS, chips, 1234.5, 300.3)
    T = L / FS
    for f, tau in [(1230.0, 300.1), (1250.0, 300.7), (1100.0, 299.2)]:
        P, g = oracle.refine_eval(x, L, FS, chips, f, tau)
        fd_f = (oracle.refine_eval(x, L, FS, chips, f + 1e-3, tau)[0]
                - oracle.refine_eval(x, L, FS, chips, f - 1e-3, tau)[0]) / 2e-3
        assert abs(g[0] - fd_f) <= 1e-3 * Ppk * T
        ht = 1e-8  # far inside one linear segment of the replica
        fd_t = (oracle.refine_eval(x, L, FS, chips, f, tau + ht)[0]
                - oracle.refine_eval(x, L, FS, chips, f, tau - ht)[0]) / (2 * ht)
        assert abs(g[1] - fd_t) <= 1e-4 * Ppk


def test_doppler_gradient_vanishes_at_truth_noise_free():
    x = _signal()
    chips = oracle.ca_code(7).astype(float)
    P, g = oracle.refine_eval(x, L, FS, chips, 1234.5, 300.3)
    T = L / FS
    assert abs(g[0]) <= 1e-9 * P * T


def test_ascent_converges_to_truth_noise_free():
    x = _signal()
    chips = oracle.ca_code(7).astype(float)
    r = oracle.refine(x, L, FS, chips, 1234.5 + 180.0, 300.3 + 0.3, search_hz=250.0)
    assert abs(r["f"] - 1234.5) < 1e-2
    assert abs(r["tau"] - 300.3) < 1e-3
    P0, _ = oracle.refine_eval(x, L, FS, chips, 1234.5 + 180.0, 300.3 + 0.3)
    assert r["P"] > P0


def _refine_12ms_starts():
    """The 12 ms workload's satellites, started where the plain acquisition
    would hand them over: the nearest 500 Hz bin and the nearest sample."""
    rec = siggen.refine_12ms()
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    starts = []
    for s in rec.sats:
        f0 = 500.0 * round(s.dopp_hz / 500.0)
        tau0 = round(s.code_phase_chips * rec.N / 1023.0) * 1023.0 / rec.N
        starts.append((s.prn, f0, tau0))
    return rec, x, starts


def test_ascent_endpoint_is_the_local_maximum_noisy():
    """The ascent's result, not only its rule: for every satellite of the
    noisy 12 ms workload (coarse start, 250 Hz pre-search, 10 ms window), a
    brute-force search of P(f, tau) with plain loops around the oracle's
    endpoint -- a line of +-0.5 Hz at 1e-2 Hz, a line of +-0.01 chip at 1e-4
    chip, and a +-0.5 Hz x +-0.01 chip grid at 0.05 Hz x 1e-3 chip -- finds no
    cell above the endpoint's power beyond the ascent's stopping tolerance
    (tau step < 1e-5 chip: P within 2e-5 of the peak's on the correlation
    triangle, whose slope is about 2 P per chip)."""
    rec, x, starts = _refine_12ms_starts()
    Lw = 10 * rec.N
    for prn, f0, tau0 in starts:
        chips = oracle.ca_code(prn).astype(float)
        r = oracle.refine(x, Lw, rec.fs, chips, f0, tau0, max_iter=100, search_hz=250.0)
        fs_, ts_, Ps = r["f"], r["tau"], r["P"]
        best = 0.0
        for k in range(-50, 51):
            best = max(best, oracle.refine_eval(x, Lw, rec.fs, chips, fs_ + 0.01 * k, ts_)[0])
        for k in range(-100, 101):
            best = max(best, oracle.refine_eval(x, Lw, rec.fs, chips, fs_, ts_ + 1e-4 * k)[0])
        for a in range(-10, 11):
            for b in range(-10, 11):
                best = max(best, oracle.refine_eval(x, Lw, rec.fs, chips, fs_ + 0.05 * a, ts_ + 1e-3 * b)[0])
        assert best <= Ps * (1.0 + 5e-5), (prn, best / Ps - 1.0)
        assert Ps > oracle.refine_eval(x, Lw, rec.fs, chips, f0, tau0)[0], prn


def test_flat_acceptance_leaves_fp64_endpoints_unchanged():
    """The Doppler step's second acceptance clause (a trial that lowers
    |dP/df| while losing at most 1e-5 of P) exists for the FP32 kernel, where
    changes of P near the peak are below single precision.  In FP64 Armijo
    alone resolves the peak: with and without the clause the ascent ends at
    the same point (within its stopping tolerances) for every satellite of
    the 12 ms workload and for 40 seeded random off-peak starts."""
    rec, x, starts = _refine_12ms_starts()
    Lw = 10 * rec.N
    rprn, rf, rtau = siggen.refine_candidates(rec)
    cases = starts + list(zip(rprn[:40].tolist(), rf[:40].tolist(), rtau[:40].tolist()))
    for prn, f0, tau0 in cases:
        chips = oracle.ca_code(int(prn)).astype(float)
        a = oracle.refine(x, Lw, rec.fs, chips, f0, tau0, max_iter=100, search_hz=250.0, flat_accept=True)
        b = oracle.refine(x, Lw, rec.fs, chips, f0, tau0, max_iter=100, search_hz=250.0, flat_accept=False)
        assert abs(a["f"] - b["f"]) < 5e-3, (prn, f0, tau0, a, b)
        assert abs(a["tau"] - b["tau"]) < 5e-5, (prn, f0, tau0, a, b)
        assert abs(a["P"] - b["P"]) <= 1e-6 * max(a["P"], b["P"]), (prn, f0, tau0, a, b)
