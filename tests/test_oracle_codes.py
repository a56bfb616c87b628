"""Pins of the oracle's Gold codes and replica (code NCO of Section 3, Fig. 2).

The oracle builds codes from G2 delays; here they are checked against the
ICD's printed first-10-chip octals, a third derivation (two-tap phase
selectors, written below), and the algebraic invariants of Gold codes.
"""
import os

import numpy as np
import pytest

import oracle
import siggen

PRNS = list(range(1, 33))

# Phase-selector taps (IS-GPS-200 Table 3-Ia, "Code Phase Selection"):
# the G2i output is the XOR of these two G2 stages.
PHASE_SELECT = [(2, 6), (3, 7), (4, 8), (5, 9), (1, 9), (2, 10), (1, 8), (2, 9), (3, 10), (2, 3),
                (3, 4), (5, 6), (6, 7), (7, 8), (8, 9), (9, 10), (1, 4), (2, 5), (3, 6), (4, 7),
                (5, 8), (6, 9), (1, 3), (4, 6), (5, 7), (6, 8), (7, 9), (8, 10), (1, 6), (2, 7),
                (3, 8), (4, 9)]


def _phase_selector_code(prn):
    g1 = [1] * 10
    g2 = [1] * 10
    a, b = PHASE_SELECT[prn - 1]
    out = []
    for _ in range(1023):
        bit = g1[9] ^ g2[a - 1] ^ g2[b - 1]
        out.append(1 - 2 * bit)
        f1 = g1[2] ^ g1[9]
        f2 = g2[1] ^ g2[2] ^ g2[5] ^ g2[7] ^ g2[8] ^ g2[9]
        g1 = [f1] + g1[:9]
        g2 = [f2] + g2[:9]
    return np.array(out, np.int8)


@pytest.fixture(scope="module")
def codes():
    return np.stack([oracle.ca_code(p) for p in PRNS]).astype(np.int64)


def _circ_corr(a, b):
    """Periodic cross-correlation sum_i a[i] b[(i + k) mod 1023] for all k."""
    return np.rint(np.real(np.fft.ifft(np.conj(np.fft.fft(a)) * np.fft.fft(b)))).astype(np.int64)


def test_first_ten_chips_match_icd_octal(codes, golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "ca_first10_octal.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 32
    for prn, octal in rows:
        bits = (1 - codes[int(prn) - 1][:10]) // 2
        assert int("".join(str(b) for b in bits), 2) == int(octal, 8), prn


def test_phase_selector_derivation_agrees(codes):
    for p in PRNS:
        np.testing.assert_array_equal(_phase_selector_code(p), codes[p - 1])


def test_balance_512_511(codes):
    for c in codes:
        assert (c == -1).sum() == 512 and (c == 1).sum() == 511


def test_autocorrelation_three_valued(codes):
    for c in codes:
        r = _circ_corr(c, c)
        assert r[0] == 1023
        assert set(np.unique(r[1:]).tolist()) <= {-1, 63, -65}


def test_crosscorrelation_three_valued(codes):
    for i in range(32):
        for j in range(i + 1, 32):
            r = _circ_corr(codes[i], codes[j])
            assert set(np.unique(r).tolist()) <= {-1, 63, -65}, (i + 1, j + 1)


def test_bad_prn_rejected():
    with pytest.raises(ValueError):
        oracle.ca_code(0)
    with pytest.raises(ValueError):
        oracle.ca_code(33)


def test_signal_table_is_the_oracle_table(codes):
    np.testing.assert_array_equal(siggen.chip_table().astype(np.int64), codes)


@pytest.mark.parametrize("N", [256, 2048, 4096, 8192, 16384])
def test_replica_sampling(codes, N):
    rep = oracle.replica(codes[0].astype(np.int8), N)
    # every sample of chip k lies in [k N / 1023, (k+1) N / 1023)
    m = np.arange(N)
    k = (m * 1023) // N
    np.testing.assert_array_equal(rep, codes[0][k])
    # each chip spans floor or ceil of N/1023 samples, all chips present
    counts = np.bincount(k, minlength=1023)
    assert counts.min() >= N // 1023 and counts.max() <= -(-N // 1023)
    assert (counts > 0).all() == (N >= 1023)


def test_paper_sample_count_bookkeeping(golden_dir):
    rows = [l.split() for l in open(os.path.join(golden_dir, "paper_counts.txt"))
            if l.strip() and not l.startswith("#")]
    fs, ms, loop = (int(v) for v in rows[0])
    assert fs * ms // 1000 == loop  # replica / mixing loop length of Section 3
    n, mults = int(rows[1][0]), float(rows[1][1])
    assert abs(n * n - mults) / mults < 0.01  # brute-force shift-multiply count
