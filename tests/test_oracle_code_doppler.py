"""Pins of the oracle's code-Doppler compensated non-coherent sum.

A signal at Doppler f has its code compressed by f / f_L1 with the carrier,
so its delay falls by f t fs / f_L1 samples after t seconds (f_L1 = 1540 x
1.023 MHz: 1540 carrier cycles per chip).  With compensation, block b enters
the sum as |R_b[(tau - sigma_b) mod N]|^2, sigma_b the nearest integer to
f b L / f_L1.

Pins:
  - a noise-free signal whose block b is delayed by exactly tau0 - sigma_b
    samples sums to the closed form B (A L)^2 at tau0 in every half-bit set,
    for positive and negative Doppler, while the plain sum spreads it;
  - with f = 0 or a single block the two sums are identical;
  - a physically synthesised signal (continuous code Doppler, generator of
    the workloads) gains power and peaks at its delay in the middle of
    block 0;
  - the shift rule itself at exact half-sample points (halves round up).
"""
import numpy as np
import pytest

import oracle
import siggen

F_L1 = 1540 * 1023000


def test_shift_rule_at_half_points():
    L = 2 * 1023000  # f L / f_L1 = f / 770: half-sample points at f = 385 (2k + 1)
    assert oracle.code_doppler_shift(385, 1, L) == 1       # 0.5 -> 1
    assert oracle.code_doppler_shift(385 * 3, 1, L) == 2   # 1.5 -> 2
    assert oracle.code_doppler_shift(-385, 1, L) == 0      # -0.5 -> 0
    assert oracle.code_doppler_shift(-385 * 3, 1, L) == -1  # -1.5 -> -1
    assert oracle.code_doppler_shift(384, 1, L) == 0       # just below 0.5
    assert oracle.code_doppler_shift(-386, 1, L) == -1     # just below -0.5
    assert oracle.code_doppler_shift(770, 7, L) == 7       # exact integers
    assert oracle.code_doppler_shift(12345, 0, L) == 0


def _block_delayed_signal(fs, coh, B, f, prn, tau0, A=0.5):
    """x[b L + n] = A c_s[(n - tau_b) mod N] exp(j 2 pi f (b L + n) / fs),
    tau_b = tau0 - sigma_b (the delay falls for positive Doppler)."""
    N = fs // 1000
    L = coh * N
    rep = oracle.replica(oracle.ca_code(prn), N)
    n = np.arange(L)
    x = np.zeros(B * L, np.complex128)
    sig = []
    for b in range(B):
        s = oracle.code_doppler_shift(f, b, L)
        sig.append(s)
        tb = tau0 - s
        x[b * L:(b + 1) * L] = A * rep[(n - tb) % N]
    t = np.arange(B * L)
    # exact carrier phase (f t mod fs) / fs, as the wipe-off uses
    x *= np.exp(2j * np.pi * ((f * t) % fs) / fs)
    return x, sig, A * L


@pytest.mark.parametrize("f", [9750, -9750])
@pytest.mark.parametrize("half", [False, True])
def test_closed_form_with_block_delays(f, half):
    fs, coh, B, prn, tau0 = 2_048_000, 1, 240, 5, 700
    x, sig, AL = _block_delayed_signal(fs, coh, B, f, prn, tau0)
    assert len(set(sig)) >= 3  # the delays really spread over several samples
    dopp = np.array([f], np.int64)
    Sc = oracle.surfaces(x, fs, coh, B, half, [prn], dopp, 4, code_doppler=True)
    Sp = oracle.surfaces(x, fs, coh, B, half, [prn], dopp, 4, code_doppler=False)
    sets = 2 if half else 1
    for s in range(sets):
        nb = len(range(s, B, sets))
        expect = nb * AL * AL
        assert Sc[s, 0, 0, tau0] == pytest.approx(expect, rel=1e-9)
        assert int(np.argmax(Sc[s, 0, 0])) == tau0
        # without compensation the blocks' peaks sit at tau0 - sigma_b, so no
        # cell of the plain surface reaches the closed form
        assert Sp[s, 0, 0].max() < 0.9 * expect


@pytest.mark.parametrize("case", ["zero_doppler", "one_block"])
def test_reduces_to_plain_sum(case):
    rec = siggen.plain_4ms()
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    prns = [s.prn for s in rec.sats][:2]
    if case == "zero_doppler":
        dopp, B = np.array([0], np.int64), rec.n_blocks
    else:
        dopp, B = rec.dopp_hz[::5], 1
    a = oracle.surfaces(x, rec.fs, rec.coh_ms, B, False, prns, dopp, 4, code_doppler=True)
    b = oracle.surfaces(x, rec.fs, rec.coh_ms, B, False, prns, dopp, 4, code_doppler=False)
    np.testing.assert_array_equal(a, b)


def test_physical_code_doppler_is_recovered():
    """Continuous code Doppler from the generator (noise-free, no data bits):
    9.5 kHz over 200 ms walks the code by 1.23 chips (4.9 samples at
    4.096 MHz).  Compensation must recover most of the coherent power and
    put the peak at the delay of the middle of block 0."""
    fs, coh, B = 4_096_000, 10, 20
    N = fs // 1000
    L = coh * N
    sat = siggen.Sat(prn=17, cn0_dbhz=45.0, dopp_hz=9500.0, code_phase_chips=311.4, carrier_phase=0.7,
                     bit_edge_ms=0.0)
    x = siggen.synthesize(np.random.default_rng(3), fs, B * L, [sat], noise=False, nav_bits=False,
                          code_doppler=True, amplitude=1.0)
    dopp = np.array([9500], np.int64)
    Sc = oracle.surfaces(x, fs, coh, B, False, [17], dopp, 4, code_doppler=True)[0, 0, 0]
    Sp = oracle.surfaces(x, fs, coh, B, False, [17], dopp, 4, code_doppler=False)[0, 0, 0]
    ideal = B * float(L) ** 2
    # residual misalignment stays within half a sample (0.82 of ideal here;
    # the plain sum keeps 0.53, the shift with the wrong sign 0.29)
    assert Sc.max() > 0.7 * ideal
    assert Sc.max() > 1.3 * Sp.max()
    # delay (samples) at the middle of block 0: tau0 - f (L / 2 / fs) / 1540 chips
    mid = (sat.code_phase_chips - sat.dopp_hz * (L / 2 / fs) / 1540.0) * N / 1023.0
    d = (int(np.argmax(Sc)) - mid + N / 2) % N - N / 2
    assert abs(d) <= 1.0, (int(np.argmax(Sc)), mid)
