"""gnss_acquire_noalloc: the acquisition for callers that cannot allocate
device memory at request time (fixed-footprint services, processes whose
device memory belongs to another allocator).  It must give the same records
and surfaces as gnss_acquire_device, on consecutive calls that reuse its one
fixed scratch array, and refuse requests larger than that array.

This file is collected last so that a failure here comes after every other
test has run; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import siggen
from parity import SURF_MAX_REL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    fn = g.lib.gnss_acquire_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    return g


def _run(g, plan, raw_dev, n, noalloc):
    out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
    if noalloc:
        st = g.lib.gnss_acquire_noalloc(plan.handle, raw_dev.data_ptr(), n, out.data_ptr(), surf.data_ptr(), None)
        g.check(st, "gnss_acquire_noalloc")
    else:
        plan.acquire_device(raw_dev, n, out, surface=surf)
    torch.cuda.synchronize()
    return g.detections_from_bytes(out.cpu().numpy()), surf.cpu().numpy()


def test_noalloc_matches_pool_path_on_consecutive_calls(g):
    recs = [siggen.weak_100ms(), siggen.plain_4ms()]  # large then small: stale scratch would show
    for rec in recs + recs[:1]:
        plan = g.Plan.for_recording(rec)
        raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
        d_ref, s_ref = _run(g, plan, raw, rec.n_samples, noalloc=False)
        d1, s1 = _run(g, plan, raw, rec.n_samples, noalloc=True)
        d2, s2 = _run(g, plan, raw, rec.n_samples, noalloc=True)
        for d, s in ((d1, s1), (d2, s2)):
            np.testing.assert_array_equal(d, d_ref)
            err = np.abs(s.astype(np.float64) - s_ref).max() / s_ref.max()
            assert err <= SURF_MAX_REL


def test_noalloc_rejects_requests_over_its_scratch(g):
    rec = siggen.weak_100ms()
    # with code-Doppler compensation every bin keeps its own spectra:
    # 20 blocks x 81 bins x 4096 x 8 B = 53 MB > 32 MiB
    plan = g.Plan.for_recording(rec, code_doppler=True)
    n = 2 * rec.n_samples
    raw = torch.zeros(siggen.recording_bytes(n, rec.fmt), dtype=torch.uint8, device="cuda")
    out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    st = g.lib.gnss_acquire_noalloc(plan.handle, raw.data_ptr(), n, out.data_ptr(), None, None)
    assert st == g.EINVAL
    assert b"32 MiB" in g.lib.gnss_last_error() or b"33554432" in g.lib.gnss_last_error()
