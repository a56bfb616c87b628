"""Comparison rules between the CUDA path (FP32) and the FP64 oracle.

Surfaces: per PRN and set, max |S_gpu - S_ref| <= 1e-4 * max S_ref and
||S_gpu - S_ref||_2 <= 1e-5 * ||S_ref||_2 (cell-wise relative error is
meaningless near zero).  Detections: PRN, detected flag, set, Doppler bin
and code phase identical, except where the oracle's decision is a near-tie
within 1e-5 relative (argmax runner-up, ratio vs threshold, set ratios);
such cases are counted as ambiguous and either answer is accepted.
"""
import numpy as np

SURF_MAX_REL = 1e-4
SURF_L2_REL = 1e-5
TIE_REL = 1e-5


def compare_surfaces(S_gpu, S_ref):
    S_gpu = np.asarray(S_gpu, np.float64)
    assert S_gpu.shape == S_ref.shape, (S_gpu.shape, S_ref.shape)
    sets, P = S_ref.shape[:2]
    worst = 0.0
    for s in range(sets):
        for p in range(P):
            a, b = S_gpu[s, p], S_ref[s, p]
            mx = np.abs(a - b).max() / b.max()
            l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
            worst = max(worst, mx)
            assert mx <= SURF_MAX_REL, ("surface max rel", s, p, mx)
            assert l2 <= SURF_L2_REL, ("surface l2 rel", s, p, l2)
    return worst


def _ambiguous(S_ref, det_ref, threshold, excl):
    """Near-tie flags per PRN from the oracle surfaces."""
    sets, P, D, N = S_ref.shape
    amb = np.zeros(P, bool)
    for p in range(P):
        ratios = []
        for s in range(sets):
            flat = S_ref[s, p].ravel()
            top2 = np.partition(flat, -2)[-2:]
            if (top2[1] - top2[0]) <= TIE_REL * top2[1]:
                amb[p] = True
            # the second peak enters only through its value, so its own ties do not matter
            d, t = np.unravel_index(np.argmax(S_ref[s, p]), (D, N))
            row = S_ref[s, p, d].copy()
            dist = np.abs(np.arange(N) - t)
            dist = np.minimum(dist, N - dist)
            row[dist <= excl] = -1
            ratios.append(flat.max() / row.max() if row.max() > 0 else np.inf)
        r = det_ref[p]["ratio"]
        if abs(r - threshold) <= TIE_REL * threshold:
            amb[p] = True
        if sets == 2 and abs(ratios[0] - ratios[1]) <= TIE_REL * max(ratios):
            amb[p] = True
    return amb


def compare_detections(det_gpu, det_ref, S_ref, threshold=2.0, excl=None):
    """det_gpu: structured array (library records); det_ref: oracle dicts.
    Returns the number of ambiguous PRNs (accepted either way)."""
    N = S_ref.shape[-1]
    if excl is None:
        excl = -(-N // 1023)
    amb = _ambiguous(S_ref, det_ref, threshold, excl)
    assert len(det_gpu) == len(det_ref)
    for p, (g, r) in enumerate(zip(det_gpu, det_ref)):
        assert int(g["prn"]) == r["prn"]
        if amb[p]:
            continue
        got = (bool(g["detected"]), int(g["set"]), int(g["dopp_bin"]), int(g["code_phase"]))
        want = (r["detected"], r["set"], r["dopp_bin"], r["code_phase"])
        assert got == want, ("PRN", r["prn"], got, want)
        assert abs(float(g["ratio"]) - r["ratio"]) <= 1e-3 * r["ratio"]
        assert abs(float(g["peak"]) - r["peak"]) <= 1e-4 * r["peak"]
    return int(amb.sum())
