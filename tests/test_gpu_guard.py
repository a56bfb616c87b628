"""Guard words around every device output (a stand-in for a memory checker,
which this pool does not offer): each output buffer is the middle of a larger
allocation whose leading and trailing 4 KB hold a sentinel byte, and after the
call the sentinels must be intact -- no entry point writes outside the
buffers its caller passed."""
import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GUARD = 4096
SENTINEL = 0xA5


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


class Guarded:
    """nbytes of device memory between two guard regions."""

    def __init__(self, nbytes):
        self.n = nbytes
        self.whole = torch.full((nbytes + 2 * GUARD,), SENTINEL, dtype=torch.uint8, device="cuda")
        self.bytes = self.whole[GUARD:GUARD + nbytes]

    def floats(self, shape):
        return self.bytes.view(torch.float32).view(shape)

    def intact(self):
        w = self.whole.cpu().numpy()
        return bool((w[:GUARD] == SENTINEL).all() and (w[GUARD + self.n:] == SENTINEL).all())


def _dev(raw):
    return torch.from_numpy(np.ascontiguousarray(raw)).cuda()


@pytest.mark.parametrize("make", [siggen.plain_4ms, siggen.weak_100ms])
def test_acquire_device_and_stages_stay_inside_their_buffers(g, make):
    rec = make()
    plan = g.Plan.for_recording(rec)
    raw = _dev(rec.raw)
    out = Guarded(plan.n_prn * 28)
    shape = plan.surface_shape()
    surf = Guarded(int(np.prod(shape)) * 4)
    plan.acquire_device(raw, rec.n_samples, out.bytes, surface=surf.floats(shape))
    torch.cuda.synchronize()
    assert out.intact() and surf.intact()
    B = plan.n_blocks(rec.n_samples)
    spec = Guarded(plan.n_dopp * B * plan.N * 8)
    plan.stage_wipe_fft(raw, rec.n_samples, B, spec.floats((plan.n_dopp, B, plan.N, 2)))
    out2 = Guarded(plan.n_prn * 28)
    surf2 = Guarded(int(np.prod(shape)) * 4)
    plan.stage_correlate(spec.floats((plan.n_dopp, B, plan.N, 2)), B, out2.bytes, surface=surf2.floats(shape))
    torch.cuda.synchronize()
    assert spec.intact() and out2.intact() and surf2.intact()
    # per-bin stage spectra against shared class spectra: equal up to rounding
    a = g.detections_from_bytes(out2.bytes.cpu().numpy())
    b = g.detections_from_bytes(out.bytes.cpu().numpy())
    for f in ("prn", "detected", "dopp_bin", "code_phase"):
        np.testing.assert_array_equal(a[f], b[f])


def test_batch_and_graph_stay_inside_their_buffers(g):
    recs = siggen.batch_requests(4, ms_range=(20, 40)) + [siggen.plain_4ms()]
    guards, reqs = [], []
    for r in recs:
        plan = g.Plan.for_recording(r)
        out = Guarded(plan.n_prn * 28)
        shape = plan.surface_shape()
        surf = Guarded(int(np.prod(shape)) * 4)
        guards += [out, surf]
        reqs.append((plan, _dev(r.raw), r.n_samples, out.bytes, surf.floats(shape)))
    g.acquire_batch(reqs)
    torch.cuda.synchronize()
    assert all(x.intact() for x in guards)
    graph = g.BatchGraph(reqs)
    try:
        graph.launch()
        torch.cuda.synchronize()
    finally:
        graph.close()
    assert all(x.intact() for x in guards)


def test_zoom_refine_and_track_stay_inside_their_buffers(g):
    rec = siggen.plain_4ms()
    plan = g.Plan.for_recording(rec)
    raw = _dev(rec.raw)
    det = plan.acquire(raw, rec.n_samples)
    hits = det[det["detected"] == 1]
    assert len(hits) > 0
    zoom, span = 5, 1
    out = Guarded(len(hits) * 28)
    per = plan.n_sets * (2 * span * zoom + 1) * plan.N
    surf = Guarded(len(hits) * per * 4)
    dh = np.ascontiguousarray(hits, g.DETECTION_DTYPE)
    g.check(g.lib.gnss_acquire_zoom(plan.handle, raw.data_ptr(), rec.n_samples, dh.ctypes.data, len(dh), zoom, span,
                                    out.bytes.data_ptr(), surf.bytes.data_ptr(), None), "gnss_acquire_zoom")
    torch.cuda.synchronize()
    assert out.intact() and surf.intact()
    cands = g.candidates(hits["prn"], hits["dopp_hz"].astype(float), hits["code_phase"] * 1023.0 / plan.N)
    cdev = torch.from_numpy(cands.view(np.uint8).copy()).cuda()
    ref = Guarded(len(cands) * g.REFINED_DTYPE.itemsize)
    plan.refine_device(raw, rec.n_samples, cdev, len(cands), 1, 20, ref.bytes)
    torch.cuda.synchronize()
    assert ref.intact()
    n_int = 3
    trk = Guarded(len(cands) * n_int * g.TRACK_DTYPE.itemsize)
    plan.track(raw, rec.n_samples, cdev, len(cands), trk.bytes, n_int)
    torch.cuda.synchronize()
    assert trk.intact()


def test_noalloc_stays_inside_its_buffers(g):
    """The allocation-free entry point on the 100 ms request and then on the
    4 ms one (the shared fixed scratch keeps the larger call's contents): its
    records and surfaces stay inside the caller's buffers, and equal the
    pool-scratch entry point's."""
    for make in (siggen.weak_100ms, siggen.plain_4ms):
        rec = make()
        plan = g.Plan.for_recording(rec)
        raw = _dev(rec.raw)
        shape = plan.surface_shape()
        out, surf = Guarded(plan.n_prn * 28), Guarded(int(np.prod(shape)) * 4)
        plan.acquire_noalloc(raw, rec.n_samples, out.bytes, surface=surf.floats(shape))
        torch.cuda.synchronize()
        assert out.intact() and surf.intact()
        out2 = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        surf2 = torch.zeros(shape, dtype=torch.float32, device="cuda")
        plan.acquire_device(raw, rec.n_samples, out2, surface=surf2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.bytes.cpu().numpy(), out2.cpu().numpy())
        np.testing.assert_array_equal(surf.floats(shape).cpu().numpy(), surf2.cpu().numpy())
