"""Pins of the oracle's tracking channel (Section 3, Fig. 3): fixed-point
NCOs, early / prompt / late correlators, Costas PLL and carrier-aided DLL.

Pins:
  - open loop (both bandwidths 0) the NCOs follow their integer recurrences
    and, for a noise-free replica of the channel's own code and carrier, the
    prompt correlator is the closed form A L exp(j phi0) up to rounding;
  - the Costas discriminator returns the carrier phase offset (and its
    half-cycle alias beyond a quarter cycle), blind to a data-bit sign;
  - the DLL discriminator returns the code delay offset within the spacing
    (the triangle of the sampled correlation);
  - closed loop, a drifting noise-free signal (code Doppler, data bits) and
    a noisy one are pulled in and held: frequency, delay and prompt phase;
  - with a zero recording the discriminators are zero and the NCOs free-run.
"""
import numpy as np
import pytest

import oracle
import siggen

FS = 4_096_000
N = FS // 1000
TWO32 = 2.0 ** 32


def _words(f, f_code):
    wc = int(np.int64(np.round(f * TWO32 / FS))) & 0xFFFFFFFF
    wk = int(np.round(f_code * TWO32 / FS)) & 0xFFFFFFFF
    return wc, wk


def _replica_signal(prn, f, tau, phi0, n, amp=1.0, sign=None):
    """The tracking channel's own open-loop replica: carrier from the same
    32-bit NCO word, code at f_code = R_c (1 + f / f_L1), both from t = 0."""
    wc, wk = _words(f, 1.023e6 * (1.0 + f / (1540.0 * 1.023e6)))
    i = np.arange(n, dtype=np.int64)
    theta = (i * wc) & 0xFFFFFFFF
    P0 = int(np.round(-tau * TWO32)) % (1023 << 32)
    u = P0 + i * wk
    chips = oracle.ca_code(prn).astype(float)
    c = chips[(u >> 32) % 1023]
    x = amp * c * np.exp(2j * np.pi * theta / TWO32 + 1j * phi0)
    if sign is not None:
        x = x * sign
    return x, wc, wk, P0


def test_open_loop_nco_and_prompt_closed_form():
    f, tau, phi0 = 1317.0, 211.37, 0.4
    n_int = 6
    x, wc, wk, P0 = _replica_signal(5, f, tau, phi0, n_int * N)
    out = oracle.track(x, FS, 1, n_int, oracle.ca_code(5), f, tau, 1.0, 0.0, 0.0)
    for k in range(n_int):
        P = (P0 + k * N * wk) % (1023 << 32)
        assert out[k]["tau_chips"] == ((1023 << 32) - P) % (1023 << 32) / TWO32
        signed = wc - (1 << 32) if wc >= (1 << 31) else wc
        assert out[k]["f_hz"] == signed * FS / TWO32
        zp = complex(*out[k]["zp"])
        assert abs(zp - N * np.exp(1j * phi0)) < 1e-8 * N
        assert abs(out[k]["e_phi"] - phi0 / (2 * np.pi)) < 1e-12


@pytest.mark.parametrize("phi0", [-1.2, -0.3, 0.0, 0.7, 1.4, 2.0, -2.5])
def test_costas_discriminator(phi0):
    f, tau = -2250.0, 77.0
    x, *_ = _replica_signal(12, f, tau, phi0, N)
    out = oracle.track(x, FS, 1, 1, oracle.ca_code(12), f, tau, 1.0, 0.0, 0.0)
    want = phi0 / (2 * np.pi)
    want = (want + 0.25) % 0.5 - 0.25  # Costas: modulo half a cycle
    assert abs(out[0]["e_phi"] - want) < 1e-12
    # a data-bit sign flips I and Q together and leaves e_phi unchanged
    xs, *_ = _replica_signal(12, f, tau, phi0, N, sign=-1.0)
    assert abs(oracle.track(xs, FS, 1, 1, oracle.ca_code(12), f, tau, 1.0, 0.0, 0.0)[0]["e_phi"] - want) < 1e-12


@pytest.mark.parametrize("prn", [21, 3])
@pytest.mark.parametrize("err", [-0.4, -0.2, -0.05, 0.0, 0.1, 0.3])
def test_dll_discriminator_reads_the_delay_offset(prn, err):
    """Signal delayed by tau + err, replica at tau.  Over a code period the
    correlation of two rectangular-chip replicas offset by x chips is
    (1 - |x|) + |x| rho1, rho1 the code's lag-1 periodic autocorrelation / 1023
    (63, -1 or -65 over 1023 for C/A codes), so for |err| within half the
    spacing d the discriminator reads
        err * (1 - d/2) * 2 (1 - rho1) / (2 - d (1 - rho1))
    (err itself for rho1 = 0); sampling at ~4 samples per chip leaves up to
    about 0.006 (the plain triangle would miss by up to 0.045)."""
    f, tau = 500.0, 400.25
    c = oracle.ca_code(prn).astype(float)
    rho1 = float(np.dot(c, np.roll(c, -1))) / 1023.0
    x, *_ = _replica_signal(prn, f, tau + err, 0.0, N)
    for d in (1.0, 0.5):
        if abs(err) >= d / 2:
            continue
        out = oracle.track(x, FS, 1, 1, oracle.ca_code(prn), f, tau, d, 0.0, 0.0)
        want = err * (1 - d / 2) * 2 * (1 - rho1) / (2 - d * (1 - rho1))
        assert abs(out[0]["e_tau"] - want) < 1e-2, (prn, d, err, out[0]["e_tau"], want)


def _truth_tau(sat, t):
    return (sat.code_phase_chips - sat.dopp_hz * t / 1540.0) % 1023


@pytest.mark.parametrize("noise", [False, True])
def test_closed_loop_pull_in_and_hold(noise):
    sat = siggen.Sat(prn=7, cn0_dbhz=45.0, dopp_hz=1234.5, code_phase_chips=300.3, carrier_phase=1.0,
                     bit_edge_ms=5.0, dopp_rate=0.5)
    rng = np.random.default_rng(11)
    sat.bits = rng.choice(np.array([-1, 1], np.int8), size=40)
    n_int = 600
    x = siggen.synthesize(rng, FS, n_int * N, [sat], noise=noise, nav_bits=True, code_doppler=True)
    out = oracle.track(x, FS, 1, n_int, oracle.ca_code(7), sat.dopp_hz + 3.0, sat.code_phase_chips + 0.1,
                       1.0, 15.0, 2.0)
    last = out[-100:]
    t = np.arange(n_int - 100, n_int) * 1e-3
    f_true = sat.dopp_hz + sat.dopp_rate * t
    # noise-free the NCO sits on the truth; with noise the proportional path
    # passes the discriminator's jitter (about 2 zeta w_n 0.02 cycles = 0.8 Hz
    # rms at 45 dB-Hz), so its mean is checked
    if noise:
        assert abs(np.mean(last["f_hz"] - f_true)) < 0.2
    else:
        assert np.abs(last["f_hz"] - f_true).max() < 0.05
    dtau = (last["tau_chips"] - _truth_tau(sat, t) + 511.5) % 1023 - 511.5
    assert np.abs(dtau).mean() < (0.03 if noise else 0.01)
    I, Q = last["zp"][:, 0], last["zp"][:, 1]
    # phase lock: the prompt power sits in I (either sign: data bits)
    assert np.mean(Q ** 2) < (0.1 if noise else 1e-3) * np.mean(I ** 2)


def test_zero_input_free_runs():
    x = np.zeros(5 * N, complex)
    out = oracle.track(x, FS, 1, 5, oracle.ca_code(1), 100.0, 10.0, 1.0, 15.0, 1.0)
    assert np.all(out["e_phi"] == 0) and np.all(out["e_tau"] == 0)
    assert np.all(out["f_hz"] == out["f_hz"][0])
    step = (out["tau_chips"][0] - out["tau_chips"][1]) % 1023
    assert np.allclose((out["tau_chips"][:-1] - out["tau_chips"][1:]) % 1023, step)


def test_rejects_bad_arguments():
    x = np.zeros(N, complex)
    with pytest.raises(ValueError):
        oracle.track(x, FS, 1, 2, oracle.ca_code(1), 0.0, 0.0)  # more intervals than samples
    with pytest.raises(ValueError):
        oracle.track(x, FS, 1, 1, oracle.ca_code(1), 0.0, 0.0, spacing=0.0)
