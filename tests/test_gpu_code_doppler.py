"""GPU parity of the code-Doppler compensated non-coherent sum
(GNSS_CODE_DOPPLER) against the FP64 oracle.  The library rotates each
folded block by sigma_b samples before its forward FFT; the oracle shifts the
block's correlation instead.  Checked: the rotated spectra of the forward
stage (wrap-around and negative Doppler included), surfaces and detections of
the 400 ms weak-signal recording, and the batched and no-allocation entry
points with the flag."""
import numpy as np
import pytest

import oracle
import siggen
from parity import compare_detections, compare_surfaces

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def _dev(raw):
    return torch.from_numpy(np.ascontiguousarray(raw)).cuda()


@pytest.mark.parametrize("N,coh,B", [(2048, 10, 30), (4096, 1, 200), (16384, 2, 12)])
def test_stage_spectra_are_the_rotated_blocks(g, N, coh, B):
    """Y_{f,b} = FFT(y_{f,b} rotated by sigma_b): bins chosen so that shifts
    are several samples, of both signs, and wrap around the block."""
    fs = N * 1000
    L = coh * N
    n = B * L
    rng = np.random.default_rng(N + coh)
    lv = np.array([-3, -1, 1, 3], np.int8)
    raw = siggen.pack(rng.choice(lv, n), rng.choice(lv, n), siggen.FMT_2BIT_IQ)
    dopp = [-9875, -250, 0, 4125, 9750]
    plan = g.Plan(fs, coh, -9875, 125, 160, prns=[1], fmt=siggen.FMT_2BIT_IQ, code_doppler=True)
    Y = torch.zeros((160, B, N, 2), dtype=torch.float32, device="cuda")
    plan.stage_wipe_fft(_dev(raw), n, B, Y)
    torch.cuda.synchronize()
    x = oracle.unpack(raw, n, siggen.FMT_2BIT_IQ)
    shifts = set()
    for f in dopp:
        d = (f + 9875) // 125
        for b in (0, 1, B // 2, B - 1):
            sigma = oracle.code_doppler_shift(f, b, L)
            shifts.add(sigma)
            got = Y[d, b].cpu().numpy().astype(np.float64)
            got = got[:, 0] + 1j * got[:, 1]
            ref = oracle.fft(np.roll(oracle.wipe_fold(x, fs, coh, f, b), sigma))
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= 2e-5, (f, b, sigma, err)
    assert min(shifts) < 0 < max(shifts)


def test_long_400ms_parity(g):
    rec = siggen.long_400ms()
    prns = sorted({s.prn for s in rec.sats} | {1, 2, 3, 4})
    plan = g.Plan.for_recording(rec, prns, code_doppler=True)
    surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
    det = plan.acquire(_dev(rec.raw), rec.n_samples, surface=surf)
    torch.cuda.synchronize()
    dref, Sref = oracle.acquire(rec.raw, rec.n_samples, rec.fmt, rec.fs, rec.coh_ms, rec.dopp_hz, prns,
                                half_bit=True, nthreads=8, code_doppler=True)
    compare_surfaces(surf.cpu().numpy(), Sref)
    assert compare_detections(det, dref, Sref) == 0


def test_compensation_detects_more_satellites(g):
    """On the 400 ms recording the compensated search finds every satellite
    the plain one finds, and more, at the injected code phase."""
    rec = siggen.long_400ms()
    found = {}
    for cd in (False, True):
        plan = g.Plan.for_recording(rec, code_doppler=cd)
        det = plan.acquire(_dev(rec.raw), rec.n_samples)
        found[cd] = {int(d["prn"]): int(d["code_phase"]) for d in det if d["detected"]}
    truth = {s.prn: rec.truth_code_phase(s) for s in rec.sats}
    assert set(found[False]) <= set(found[True])
    assert len(found[True]) > len(found[False])
    for p, t in found[True].items():
        assert p in truth
        # block-0 delay: within 2 samples of the injected t = 0 phase
        assert abs((t - truth[p] + rec.N / 2) % rec.N - rec.N / 2) <= 2.0, (p, t, truth[p])


def test_batch_and_noalloc_with_flag(g):
    recs = siggen.batch_requests(4, ms_range=(100, 160))
    items, alone = [], []
    for r in recs:
        plan = g.Plan.for_recording(r, code_doppler=True)
        raw = _dev(r.raw)
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        items.append((plan, raw, r.n_samples, out, surf))
        a_out = torch.zeros_like(out)
        a_surf = torch.zeros_like(surf)
        plan.acquire_device(raw, r.n_samples, a_out, surface=a_surf)
        alone.append((a_out, a_surf))
    g.acquire_batch(items)
    torch.cuda.synchronize()
    for (plan, raw, n, out, surf), (a_out, a_surf) in zip(items, alone):
        np.testing.assert_array_equal(out.cpu().numpy(), a_out.cpu().numpy())
        np.testing.assert_array_equal(surf.cpu().numpy(), a_surf.cpu().numpy())
    # the oracle agrees on one of them
    r = recs[0]
    plan, raw, n, out, surf = items[0]
    prns = np.arange(1, 33)
    x = oracle.unpack(r.raw, r.n_samples, r.fmt)
    S = oracle.surfaces(x, r.fs, r.coh_ms, plan.n_blocks(n), r.half_bit, prns, r.dopp_hz, 8, code_doppler=True)
    compare_surfaces(surf.cpu().numpy(), S)
    compare_detections(g.detections_from_bytes(out.cpu().numpy()), oracle.detect(S, prns), S)


def test_noalloc_with_flag(g):
    """A request small enough for the fixed scratch (41 bins x 20 blocks x
    2048 x 8 bytes of spectra): same records and surfaces as the pool path."""
    r = siggen.make_recording(1309005299, 2_048_000, 2048 * 60, siggen.FMT_2BIT_IQ, 3, (40.0, 45.0),
                              (-9500.0, 9500.0), coh_ms=3, dopp_min_hz=-10000, dopp_step_hz=500, n_dopp=41)
    plan = g.Plan.for_recording(r, code_doppler=True)
    raw = _dev(r.raw)
    res = []
    for noalloc in (False, True):
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        if noalloc:
            g.check(g.lib.gnss_acquire_noalloc(plan.handle, raw.data_ptr(), r.n_samples, out.data_ptr(),
                                               surf.data_ptr(), None), "gnss_acquire_noalloc")
        else:
            plan.acquire_device(raw, r.n_samples, out, surface=surf)
        torch.cuda.synchronize()
        res.append((out.cpu().numpy(), surf.cpu().numpy()))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    np.testing.assert_array_equal(res[0][1], res[1][1])
