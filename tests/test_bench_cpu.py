"""The optimised CPU acquisition of bench.py (a reported baseline beside the
oracle) computes the same surfaces' per-PRN peaks as the FP64 oracle, within
FP32 rounding, on a sample of the 100 ms workload's Doppler bins."""
import os
import sys

import numpy as np

import oracle
import siggen

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_optimised_cpu_peaks_match_oracle():
    rec = siggen.weak_100ms()
    cells, best = bench.cpu_fft_acquire(rec, 4, every=27)
    dopp = rec.dopp_hz[::27]
    assert cells == 32 * len(dopp) * rec.N * rec.n_blocks * rec.coh_ms
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    S = oracle.surfaces(x, rec.fs, rec.coh_ms, rec.n_blocks, True, np.arange(1, 33), dopp, 4)
    ref = S.max(axis=(2, 3))
    assert best.shape == ref.shape
    assert np.abs(best / ref - 1).max() < 1e-5
