"""GPU parity of the acquisition path against the FP64 oracle, through the
C ABI (Section 3, Fig. 2): codes bit-exact, code spectra, the fused
wipe-off/fold/FFT stage, surfaces within 1e-4 (max) / 1e-5 (L2) relative,
detections identical up to near-ties, plus edge cases."""
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


def _gpu_acquire(plan, raw, n, with_surface=True):
    surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda") if with_surface else None
    det = plan.acquire(_dev(raw), n, surface=surf)
    torch.cuda.synchronize()
    return det, (surf.cpu().numpy() if with_surface else None)


def _oracle(rec_like, raw, n, prns, B, half_bit=False, whole=False, threshold=2.0):
    x = oracle.unpack(raw, n, rec_like["fmt"])
    S = oracle.surfaces(x, rec_like["fs"], rec_like["coh"], B, half_bit, prns, rec_like["dopp"], nthreads=8)
    return oracle.detect(S, prns, threshold, whole_surface=whole), S


def test_gold_codes_bit_exact(g):
    plan = g.Plan(2_048_000, 1, -5000, 500, 21, prns=range(1, 33), fmt=g.FMT_I8_IQ)
    want = np.stack([oracle.ca_code(p) for p in range(1, 33)])
    np.testing.assert_array_equal(plan.codes(), want)
    sub = g.Plan(2_048_000, 1, 0, 1, 1, prns=[3, 17, 32], fmt=g.FMT_I8_IQ)
    np.testing.assert_array_equal(sub.codes(), want[[2, 16, 31]])


@pytest.mark.parametrize("N", [256, 1024, 2048, 4096, 8192, 16384])
def test_code_spectra(g, N):
    prns = [1, 9, 32]
    plan = g.Plan(N * 1000, 1, 0, 1, 1, prns=prns)
    out = torch.zeros((len(prns), N, 2), dtype=torch.float32, device="cuda")
    plan.code_spectra(out)
    got = out.cpu().numpy().astype(np.float64)
    got = got[..., 0] + 1j * got[..., 1]
    for i, p in enumerate(prns):
        ref = oracle.fft(oracle.replica(oracle.ca_code(p), N))
        assert np.abs(got[i] - ref).max() <= 1e-5 * np.abs(ref).max()


def _random_recording(seed, n, fmt):
    rng = np.random.default_rng(seed)
    lv = np.array([-3, -1, 1, 3], np.int8)
    if fmt == siggen.FMT_I8_IQ:
        li = rng.integers(-100, 101, n).astype(np.int8)
        lq = rng.integers(-100, 101, n).astype(np.int8)
    else:
        li, lq = rng.choice(lv, n), rng.choice(lv, n)
    return siggen.pack(li, lq, fmt)


@pytest.mark.parametrize("N,coh,fmt", [(256, 3, 1), (2048, 1, 0), (2048, 2, 1), (4096, 3, 1), (8192, 1, 0),
                                       (16384, 2, 1), (16384, 1, 0)])
def test_stage_wipe_fold_fft(g, N, coh, fmt):
    fs = N * 1000
    B = 2
    n = B * coh * N + 123  # ragged tail ignored
    raw = _random_recording(N + coh, n, fmt)
    dopp = [-7250, 0, 3125]
    plan = g.Plan(fs, coh, -7250, 7250 + 3125, 2, prns=[1], fmt=fmt)  # bins -7250, 3125
    plan0 = g.Plan(fs, coh, 0, 1, 1, prns=[1], fmt=fmt)              # bin 0
    x = oracle.unpack(raw, n, fmt)
    for pl, fl in ((plan, [dopp[0], dopp[2]]), (plan0, [0])):
        Y = torch.zeros((len(fl), B, N, 2), dtype=torch.float32, device="cuda")
        pl.stage_wipe_fft(_dev(raw), n, B, Y)
        Yh = Y.cpu().numpy().astype(np.float64)
        Yh = Yh[..., 0] + 1j * Yh[..., 1]
        for d, f in enumerate(fl):
            for b in range(B):
                ref = oracle.fft(oracle.wipe_fold(x, fs, coh, f, b))
                err = np.abs(Yh[d, b] - ref).max() / np.abs(ref).max()
                assert err <= 2e-5, (f, b, err)


def _rec_dict(rec):
    return dict(fmt=rec.fmt, fs=rec.fs, coh=rec.coh_ms, dopp=rec.dopp_hz)


def test_acquire_plain_4ms_parity_and_truth(g):
    rec = siggen.plain_4ms()
    prns = list(range(1, 33))
    plan = g.Plan.for_recording(rec, prns)
    det, S = _gpu_acquire(plan, rec.raw, rec.n_samples)
    dref, Sref = _oracle(_rec_dict(rec), rec.raw, rec.n_samples, prns, rec.n_blocks)
    compare_surfaces(S, Sref)
    assert compare_detections(det, dref, Sref) == 0
    assert {int(d["prn"]) for d in det if d["detected"]} == {s.prn for s in rec.sats}


def test_acquire_weak_100ms_full_size_parity(g):
    """The 100 ms, 4.096 MHz, 81-bin, 10 ms x 10 half-bit workload at full
    size, in the launch configuration the benchmark times."""
    rec = siggen.weak_100ms()
    prns = list(range(1, 33))
    plan = g.Plan.for_recording(rec, prns)
    det, S = _gpu_acquire(plan, rec.raw, rec.n_samples)
    dref, Sref = _oracle(_rec_dict(rec), rec.raw, rec.n_samples, prns, rec.n_blocks, half_bit=True)
    compare_surfaces(S, Sref)
    assert compare_detections(det, dref, Sref) == 0
    # without a surface buffer the detections are the same records
    det2, _ = _gpu_acquire(plan, rec.raw, rec.n_samples, with_surface=False)
    np.testing.assert_array_equal(det2, det)


def test_class_by_class_tile_order_large_spectra(g):
    """Spectra above the L2 budget (24 MB) switch the correlate tiles to the
    class-by-class order: 60 ms at 16.384 MHz, 1 ms blocks, 81 bins of 250 Hz
    (8 spectrum classes, 63 MB of spectra), three PRNs; surfaces and
    detections against the oracle, and every (PRN, bin) row lands in its own
    place.  The same recording cut to 20 ms (21 MB, the bin-by-bin order)
    agrees too."""
    N, fs = 16384, 16_384_000
    prns = [3, 9, 30]
    dopp = np.arange(81) * 250 - 10000
    rng = np.random.default_rng(77)
    sats = [siggen.Sat(prn=9, cn0_dbhz=48.0, dopp_hz=-1750.0, code_phase_chips=100.7, carrier_phase=0.3,
                       bit_edge_ms=3.0),
            siggen.Sat(prn=30, cn0_dbhz=46.0, dopp_hz=3260.0, code_phase_chips=611.2, carrier_phase=1.1,
                       bit_edge_ms=9.0)]
    for ms in (60, 20):
        n = ms * N
        x = siggen.synthesize(rng, fs, n, sats)
        li, lq = siggen.quantize_2bit(x, sats, fs)
        raw = siggen.pack(li, lq, siggen.FMT_2BIT_IQ)
        plan = g.Plan(fs, 1, -10000, 250, 81, prns=prns, fmt=siggen.FMT_2BIT_IQ)
        det, S = _gpu_acquire(plan, raw, n)
        dref, Sref = _oracle(dict(fmt=siggen.FMT_2BIT_IQ, fs=fs, coh=1, dopp=dopp), raw, n, prns, ms)
        compare_surfaces(S, Sref)
        assert compare_detections(det, dref, Sref) == 0
        assert {int(d["prn"]) for d in det if d["detected"]} == {9, 30}


def test_host_device_and_async_paths_agree(g):
    rec = siggen.plain_4ms()
    plan = g.Plan.for_recording(rec)
    det_dev, _ = _gpu_acquire(plan, rec.raw, rec.n_samples, with_surface=False)
    det_host = plan.acquire(np.ascontiguousarray(rec.raw), rec.n_samples)
    out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    plan.acquire_device(_dev(rec.raw), rec.n_samples, out, stream=s)
    s.synchronize()
    det_async = g.detections_from_bytes(out.cpu().numpy())
    np.testing.assert_array_equal(det_host, det_dev)
    np.testing.assert_array_equal(det_async, det_dev)
    # caller-owned page-locked record buffer, filled by an asynchronous copy
    pin = torch.zeros(plan.n_prn * g.DETECTION_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    recs = pin.numpy().view(g.DETECTION_DTYPE)
    got = plan.acquire(torch.from_numpy(np.ascontiguousarray(rec.raw)).pin_memory().numpy(), rec.n_samples,
                       stream=s, out=recs)
    assert got is recs
    np.testing.assert_array_equal(recs, det_dev)
    with pytest.raises(ValueError):
        plan.acquire(np.ascontiguousarray(rec.raw), rec.n_samples, out=np.zeros(plan.n_prn + 1, g.DETECTION_DTYPE))


def test_traced_acquisition_same_records_and_ordered_events(g):
    """The traced entry point gives the untraced records and surfaces, and its
    four stage events are recorded in order on the launching stream."""
    rec = siggen.weak_100ms()
    plan = g.Plan.for_recording(rec)
    raw = _dev(rec.raw)
    s = torch.cuda.Stream()
    o1 = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    o2 = torch.zeros_like(o1)
    s1 = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
    s2 = torch.zeros_like(s1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    plan.acquire_device(raw, rec.n_samples, o1, surface=s1, stream=s)
    plan.acquire_device_traced(raw, rec.n_samples, o2, ev, surface=s2, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(o1.cpu().numpy(), o2.cpu().numpy())
    np.testing.assert_array_equal(s1.cpu().numpy(), s2.cpu().numpy())
    gaps = [ev[k].elapsed_time(ev[k + 1]) for k in range(3)]
    assert all(t > 0 for t in gaps), gaps
    assert gaps[2] > gaps[0] and gaps[2] > gaps[1]  # the correlate stage dominates


@pytest.mark.parametrize("extra,noncoh", [(0.5, 0), (0.0, 2), (2.7, 3)])
def test_ragged_tail_and_noncoh_cap(g, extra, noncoh):
    rec = siggen.plain_4ms()
    n = int((3 + extra) * rec.N)  # 3 whole blocks + a partial one
    B = 3 if not noncoh else min(3, noncoh)
    prns = [3, 5, 10, 21, 29]  # ascending, the order of the records
    plan = g.Plan(rec.fs, 1, rec.dopp_min_hz, rec.dopp_step_hz, rec.n_dopp, prns=prns, noncoh=noncoh,
                  fmt=rec.fmt)
    raw = rec.raw[: siggen.recording_bytes(n, rec.fmt)]
    det, S = _gpu_acquire(plan, raw, n)
    dref, Sref = _oracle(_rec_dict(rec), raw, n, prns, B)
    compare_surfaces(S, Sref)
    compare_detections(det, dref, Sref)


def test_too_short_and_misaligned_rejected(g):
    plan = g.Plan(2_048_000, 2, -500, 500, 3, prns=[1], fmt=g.FMT_I8_IQ)
    raw = _dev(np.zeros(2 * 4096 + 64, np.uint8))
    with pytest.raises(g.GnssError) as e:
        plan.acquire(raw, 4095)
    assert e.value.status == g.EINVAL
    with pytest.raises(g.GnssError) as e:
        plan.acquire(raw[2:], 4096)
    assert e.value.status == g.EINVAL


@pytest.mark.parametrize("N,coh,B,dopp,prns,fmt,half", [
    (256, 4, 3, (-2000, 1000, 5), [1, 2], 1, True),
    (16384, 1, 2, (-1000, 1000, 3), [7, 8], 1, False),
    (16384, 1, 3, (0, 1, 1), [5], 0, True),
    (8192, 2, 2, (-3000, 1500, 5), [12, 30, 31], 0, True),
    (4096, 20, 1, (-250, 250, 3), [4], 1, False),
    (1024, 1, 5, (2000, 1, 1), list(range(1, 33)), 0, False),
])
def test_edge_shapes(g, N, coh, B, dopp, prns, fmt, half):
    """Smallest and largest FFT sizes, a single Doppler bin, a single PRN, a
    long coherent block, one block, half-bit sets with an odd block count."""
    fs = N * 1000
    rng = np.random.default_rng(N + B)
    n = B * coh * N
    sats = [siggen.Sat(prn=prns[0], cn0_dbhz=50.0, dopp_hz=float(dopp[0] + dopp[1]), code_phase_chips=333.3,
                       carrier_phase=1.0, bit_edge_ms=7.0)]
    x = siggen.synthesize(rng, fs, n, sats, nav_bits=False)
    li, lq = siggen.quantize_2bit(x, sats, fs)
    raw = siggen.pack(li, lq, fmt)
    plan = g.Plan(fs, coh, dopp[0], dopp[1], dopp[2], prns=prns, half_bit=half, fmt=fmt)
    det, S = _gpu_acquire(plan, raw, n)
    dopp_hz = dopp[0] + dopp[1] * np.arange(dopp[2])
    dref, Sref = _oracle(dict(fmt=fmt, fs=fs, coh=coh, dopp=dopp_hz), raw, n, prns, B, half_bit=half)
    compare_surfaces(S, Sref)
    compare_detections(det, dref, Sref)


def test_second_peak_over_whole_surface(g):
    rec = siggen.plain_4ms()
    prns = list(range(1, 33))
    plan = g.Plan.for_recording(rec, prns, second_whole=True)
    det, S = _gpu_acquire(plan, rec.raw, rec.n_samples)
    dref, Sref = _oracle(_rec_dict(rec), rec.raw, rec.n_samples, prns, rec.n_blocks, whole=True)
    assert compare_detections(det, dref, Sref) == 0
    with pytest.raises(g.GnssError):
        plan.acquire(_dev(rec.raw), rec.n_samples)  # needs a surface buffer
