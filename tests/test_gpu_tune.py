"""Autotuner of the correlate kernel (gnss_autotune): every launch shape it
can choose gives oracle-exact detections and surfaces within tolerance, and
tuning picks one of the shapes it timed."""
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


def _recording(N, coh, B, fmt, seed):
    fs = N * 1000
    rng = np.random.default_rng(seed)
    n = B * coh * N
    sats = [siggen.Sat(prn=9, cn0_dbhz=50.0, dopp_hz=-1750.0 + 13.0, code_phase_chips=100.7, carrier_phase=0.3,
                       bit_edge_ms=3.0)]
    x = siggen.synthesize(rng, fs, n, sats)
    li, lq = siggen.quantize_2bit(x, sats, fs)
    return siggen.pack(li, lq, fmt), n


STAGED = 0x100
CLASS_LOCAL = 0x200
TMEM = 0x400
OCC = 0x800


def PRNS(k):
    return (k - 1) << 12


def BINS(m):
    return (m - 1) << 14


def _tm_codes(N):
    """Every TMEM shape the library is built with at N (whether the GPU can
    take it depends on its occupancy: see _tm_accepted)."""
    e = {2048: 16, 4096: 16, 8192: 16, 16384: 32}.get(N)
    if e is None:
        return []
    ks = (1, 2) if e == 16 else (1,)
    occ = [16 | TMEM | OCC] if N in (2048, 4096, 8192, 16384) else []
    return [e | TMEM | PRNS(k) | BINS(m) for k in ks for m in (1, 2)] + occ


def _tm_accepted(g, plan):
    """The TMEM shapes the library accepts for the plan's N on this GPU; the
    one-PRN, one-bin shape must be among them."""
    ok = []
    for code in _tm_codes(plan.N):
        try:
            assert plan.autotune(code)["chosen"] == code
            ok.append(code)
        except g.GnssError as e:
            assert e.status == g.EINVAL
    if plan.N in (2048, 4096, 8192, 16384):
        assert (16 if plan.N < 16384 else 32) | TMEM in ok
    return ok


def _default(N):
    """The library's default variant at N (the tensor-memory occupancy forms
    at 4096, 8192 and 16384, which every B300 can hold)."""
    if N in (4096, 8192, 16384):
        return 16 | TMEM | OCC
    return (16 | CLASS_LOCAL) if N == 8192 else 16


def _valid(N):
    v = [16] if N <= 16384 else []
    if N >= 1024:
        v.append(32)
    if N <= 8192:
        v.append(16 | STAGED)
    if N <= 8192:
        v.append(8)
    if N in (4096, 8192):
        v.append(16 | CLASS_LOCAL)
    if N == 16384:
        v.append(32 | CLASS_LOCAL)  # split over a two-CTA cluster
    return v


@pytest.mark.parametrize("N,half,B", [(256, True, 3), (2048, False, 4), (4096, True, 5), (8192, True, 4),
                                      (16384, False, 4), (16384, True, 4)])
def test_every_shape_matches_oracle(g, N, half, B):
    coh, fmt = 1, siggen.FMT_2BIT_IQ
    raw, n = _recording(N, coh, B, fmt, N)
    prns = [3, 9, 30]
    dopp = (-3000, 250, 9)
    plan = g.Plan(N * 1000, coh, dopp[0], dopp[1], dopp[2], prns=prns, half_bit=half, fmt=fmt)
    x = oracle.unpack(raw, n, fmt)
    S = oracle.surfaces(x, N * 1000, coh, B, half, prns, dopp[0] + dopp[1] * np.arange(dopp[2]), 8)
    ref = oracle.detect(S, prns)
    default = _default(N)
    try:
        valid = _valid(N) + _tm_accepted(g, plan)
        for elems in valid:
            assert plan.autotune(elems)["chosen"] == elems
            surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
            det = plan.acquire(torch.from_numpy(np.ascontiguousarray(raw)).cuda(), n, surface=surf)
            torch.cuda.synchronize()
            compare_surfaces(surf.cpu().numpy(), S)
            assert compare_detections(det, ref, S) == 0
        r = plan.autotune()
        assert r["chosen"] in r["timed"] and sorted(r["timed"]) == sorted(valid)
        assert (r["prns_per_cta"], r["bins_per_cta"]) == (
            ((r["chosen"] >> 12) & 3) + 1 if r["chosen"] & TMEM else 1,
            ((r["chosen"] >> 14) & 3) + 1 if r["chosen"] & TMEM else 1)
        assert all(ms > 0 for ms in r["timed"].values())
    finally:
        plan.autotune(default)


def test_invalid_shape_rejected(g):
    plan = g.Plan(512_000, 1, 0, 1, 1, prns=[1])
    with pytest.raises(g.GnssError) as e:
        plan.autotune(32)  # N = 512 has too few elements for 32 per thread
    assert e.value.status == g.EINVAL
    big = g.Plan(16_384_000, 1, 0, 1, 1, prns=[1])
    with pytest.raises(g.GnssError) as e:
        big.autotune(16 | STAGED)  # the stage does not fit beside the 16384-point exchange buffer
    assert e.value.status == g.EINVAL
    with pytest.raises(g.GnssError) as e:
        big.autotune(16 | CLASS_LOCAL)  # the class-local schedule is built for N = 4096 and 8192
    assert e.value.status == g.EINVAL
    with pytest.raises(g.GnssError) as e:
        g.Plan(8_192_000, 1, 0, 1, 1, prns=[1]).autotune(32 | CLASS_LOCAL)  # the split is for N = 16384
    assert e.value.status == g.EINVAL
    for N, code in ((1024, 16 | TMEM),              # not built below 2048
                    (4096, 32 | TMEM),              # 16 per thread below 16384
                    (16384, 32 | TMEM | PRNS(2)),   # one PRN per CTA at 16384
                    (4096, 16 | TMEM | PRNS(3)),    # 1 or 2 PRNs per CTA
                    (4096, 16 | TMEM | BINS(4)),    # 1 or 2 bins per CTA
                    (16384, 32 | TMEM | OCC),       # the occupancy form: 2048, 4096 and 8192 only
                    (4096, 16 | TMEM | OCC | PRNS(2)),  # one PRN and bin per CTA
                    (4096, 16 | OCC),               # a form of the TMEM variant
                    (4096, 16 | TMEM | 0x10000)):   # unknown bits
        with pytest.raises(g.GnssError) as e:
            g.Plan(N * 1000, 1, 0, 1, 1, prns=[1]).autotune(code)
        assert e.value.status == g.EINVAL, (N, hex(code))


def test_staged_full_size_and_batch(g):
    """The staged variant on the 100 ms benchmark workload at full size and
    inside a batch of uneven requests: oracle parity at full size, and the
    batch gives the register variant's records and surfaces (1e-6)."""
    from parity import compare_detections as cd, compare_surfaces as cs
    rec = siggen.weak_100ms()
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    prns = np.arange(1, 33)
    S = oracle.surfaces(x, rec.fs, rec.coh_ms, rec.n_blocks, True, prns, rec.dopp_hz, 8)
    ref = oracle.detect(S, prns)
    try:
        plan.autotune(16 | STAGED)
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        det = plan.acquire(raw, rec.n_samples, surface=surf)
        cs(surf.cpu().numpy(), S)
        assert cd(det, ref, S) == 0
        recs = siggen.batch_requests(6, ms_range=(20, 60), fs_choices=(4_096_000,))
        items, alone = [], []
        for r in recs:
            p = g.Plan.for_recording(r)
            rr = torch.from_numpy(np.ascontiguousarray(r.raw)).cuda()
            out = torch.zeros(p.n_prn * 28, dtype=torch.uint8, device="cuda")
            sf = torch.zeros(p.surface_shape(), dtype=torch.float32, device="cuda")
            items.append((p, rr, r.n_samples, out, sf))
        g.acquire_batch(items)
        torch.cuda.synchronize()
        plan.autotune(16 | CLASS_LOCAL)  # the register form's class-local schedule
        for p, rr, n, out, sf in items:
            o2 = torch.zeros_like(out)
            s2 = torch.zeros_like(sf)
            p.acquire_device(rr, n, o2, surface=s2)
            torch.cuda.synchronize()
            a = g.detections_from_bytes(out.cpu().numpy())
            b = g.detections_from_bytes(o2.cpu().numpy())
            for f in ("prn", "detected", "set", "dopp_bin", "code_phase"):
                np.testing.assert_array_equal(a[f], b[f])
            np.testing.assert_allclose(a["peak"], b["peak"], rtol=1e-6)
            A, Bs = sf.cpu().numpy(), s2.cpu().numpy()
            assert np.abs(A - Bs).max() <= 1e-6 * np.abs(Bs).max()
    finally:
        plan.autotune(_default(4096))


def _weak_100ms(g):
    rec = siggen.weak_100ms()
    return g.Plan.for_recording(rec), rec.raw, rec.n_samples


def _fs_8192(g):
    raw, n = _recording(8192, 2, 10, siggen.FMT_2BIT_IQ, 8192)
    return g.Plan(8_192_000, 2, -10000, 500, 41, prns=range(1, 33), half_bit=False, fmt=siggen.FMT_2BIT_IQ), raw, n


@pytest.mark.parametrize("make", [_weak_100ms, _fs_8192])
def test_class_local_matches_two_barrier_schedule(g, make):
    """The class-local schedule (the register form's at N = 4096 and 8192) runs the
    same butterflies with the same operands as the two-barrier schedule, only
    on other threads -- at 8192 the last radix-2 pass across lane pairs by
    shuffle -- so both give identical surfaces and records: the full 100 ms
    workload at 4096, 20 ms at 8.192 MHz with 32 PRNs and 41 bins."""
    plan, raw_np, n = make(g)
    raw = torch.from_numpy(np.ascontiguousarray(raw_np)).cuda()
    res = {}
    try:
        for code in (16, 16 | CLASS_LOCAL):
            plan.autotune(code)
            surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
            det = plan.acquire(raw, n, surface=surf)
            res[code] = (det, surf.cpu().numpy())
    finally:
        plan.autotune(_default(plan.N))
    (d0, s0), (d1, s1) = res[16], res[16 | CLASS_LOCAL]
    np.testing.assert_array_equal(s0, s1)
    for f in ("prn", "detected", "set", "dopp_bin", "code_phase", "peak", "second", "ratio"):
        np.testing.assert_array_equal(d0[f], d1[f])


def test_split_cluster_batch_equals_alone_and_whole_surface(g):
    """The 16384-point split (two CTAs per tile in a cluster, merging their row
    statistics through distributed shared memory): a batch of uneven
    16.384 MHz requests gives each request's single-launch records and
    surfaces bit for bit, both agree with the 32-per-thread form within
    1e-6, and with GNSS_SECOND_WHOLE (the other CTA's surface half read by
    the detecting CTA) the second peak matches that form too."""
    recs = siggen.batch_requests(3, ms_range=(10, 30), fs_choices=(16_384_000,))
    try:
        res = {}
        for code in (32 | CLASS_LOCAL, 32):
            items = []
            for r in recs:
                p = g.Plan.for_recording(r)
                p.autotune(code)
                rr = torch.from_numpy(np.ascontiguousarray(r.raw)).cuda()
                out = torch.zeros(p.n_prn * 28, dtype=torch.uint8, device="cuda")
                sf = torch.zeros(p.surface_shape(), dtype=torch.float32, device="cuda")
                items.append((p, rr, r.n_samples, out, sf))
            g.acquire_batch(items)
            torch.cuda.synchronize()
            batch = [(g.detections_from_bytes(o.cpu().numpy()), sf.cpu().numpy()) for _, _, _, o, sf in items]
            alone = []
            for p, rr, n, out, sf in items:
                o2, s2 = torch.zeros_like(out), torch.zeros_like(sf)
                p.acquire_device(rr, n, o2, surface=s2)
                torch.cuda.synchronize()
                alone.append((g.detections_from_bytes(o2.cpu().numpy()), s2.cpu().numpy()))
            for (da, sa), (db, sb) in zip(batch, alone):
                np.testing.assert_array_equal(sa, sb)
                for f in ("prn", "detected", "set", "dopp_bin", "code_phase", "peak", "second", "ratio"):
                    np.testing.assert_array_equal(da[f], db[f])
            res[code] = alone
        for (da, sa), (db, sb) in zip(res[32 | CLASS_LOCAL], res[32]):
            assert np.abs(sa - sb).max() <= 1e-6 * np.abs(sb).max()
            for f in ("prn", "detected", "set", "dopp_bin", "code_phase"):
                np.testing.assert_array_equal(da[f], db[f])
            np.testing.assert_allclose(da["second"], db["second"], rtol=1e-5)
        r = recs[0]
        whole = {}
        for code in (32 | CLASS_LOCAL, 32):
            p = g.Plan.for_recording(r, second_whole=True)
            p.autotune(code)
            rr = torch.from_numpy(np.ascontiguousarray(r.raw)).cuda()
            sf = torch.zeros(p.surface_shape(), dtype=torch.float32, device="cuda")
            whole[code] = p.acquire(rr, r.n_samples, surface=sf)
        a, b = whole[32 | CLASS_LOCAL], whole[32]
        for f in ("prn", "detected", "dopp_bin", "code_phase"):
            np.testing.assert_array_equal(a[f], b[f])
        np.testing.assert_allclose(a["second"], b["second"], rtol=1e-5)
    finally:
        g.Plan(16_384_000, 1, 0, 1, 1, prns=[1]).autotune(_default(16384))


def _case_weak_100ms(g):
    rec = siggen.weak_100ms()
    return [(g.Plan.for_recording(rec), rec.raw, rec.n_samples)]


def _case_8192_odd(g):
    # 3 PRNs and 41 bins: the last CTA of a two-PRN or two-bin shape holds one
    raw, n = _recording(8192, 2, 10, siggen.FMT_2BIT_IQ, 8192)
    return [(g.Plan(8_192_000, 2, -10000, 500, 41, prns=[3, 9, 30], half_bit=True, fmt=siggen.FMT_2BIT_IQ), raw, n)]


def _case_2048_whole(g):
    # 5 PRNs, 9 bins, 1 ms x 7 blocks; the second variant scans the whole surface
    raw, n = _recording(2048, 1, 7, siggen.FMT_2BIT_IQ, 2048)
    return [(g.Plan(2_048_000, 1, -3000, 250, 9, prns=[1, 3, 9, 17, 30], half_bit=hb, fmt=siggen.FMT_2BIT_IQ,
                    second_whole=sw), raw, n) for hb, sw in ((False, False), (True, True))]


def _case_16384(g):
    raw, n = _recording(16384, 1, 3, siggen.FMT_2BIT_IQ, 16384)
    return [(g.Plan(16_384_000, 1, -3000, 250, 9, prns=[3, 9, 30], half_bit=True, fmt=siggen.FMT_2BIT_IQ), raw, n)]


@pytest.mark.parametrize("make", [_case_weak_100ms, _case_8192_odd, _case_2048_whole, _case_16384])
def test_tmem_matches_register_form(g, make):
    """The TMEM variant (code spectra and sums in tensor memory, the next
    block's spectrum prefetched) runs each block's products, transform and
    sums operation for operation as the register form: every shape the GPU
    accepts (1-2 PRNs and 1-2 bins per CTA) gives the default variant's
    surfaces and records bit for bit -- the full 100 ms workload, odd PRN and
    bin counts that leave a CTA one PRN or bin short, half-bit sets and the
    whole-surface second peak.  (At 16384 the reference is the 32-per-thread
    register form; the occupancy form there factors the transform
    differently, so it is held to the oracle in
    test_every_shape_matches_oracle instead.)"""
    for plan, raw_np, n in make(g):
        raw = torch.from_numpy(np.ascontiguousarray(raw_np)).cuda()
        default = _default(plan.N)
        # at 16384 the reference is the 32-per-thread register form
        ref_code = 32 if plan.N == 16384 else default
        try:
            plan.autotune(ref_code)
            surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
            d0 = plan.acquire(raw, n, surface=surf)
            s0 = surf.cpu().numpy()
            for code in _tm_accepted(g, plan):
                if plan.N == 16384 and code & OCC:
                    continue  # another factorisation (16 per thread, radix 16-16-16-4): against the oracle instead
                plan.autotune(code)
                surf = torch.full(plan.surface_shape(), -1.0, dtype=torch.float32, device="cuda")
                d1 = plan.acquire(raw, n, surface=surf)
                np.testing.assert_array_equal(surf.cpu().numpy(), s0, err_msg=hex(code))
                for f in ("prn", "detected", "set", "dopp_bin", "code_phase", "peak", "second", "ratio"):
                    np.testing.assert_array_equal(d1[f], d0[f], err_msg=hex(code))
        finally:
            plan.autotune(default)


def test_tmem_batch_equals_alone(g):
    """A batch of uneven requests (2.048, 4.096 and 8.192 MHz, 20-60 ms) under
    the two-PRN, two-bin TMEM shape: each request's records and surfaces equal
    its single launch under the same shape and under the default variant, bit
    for bit (the batch counts its CTA offsets per request by the shape)."""
    recs = siggen.batch_requests(8, ms_range=(20, 60))
    sizes = sorted({r.fs // 1000 for r in recs})
    probe = {N: g.Plan(N * 1000, 1, 0, 1, 1, prns=[1]) for N in sizes}
    try:
        res = {}
        for which in ("tm", "default"):
            for N, p in probe.items():
                if which == "default":
                    p.autotune(_default(N))
                else:
                    acc = _tm_accepted(g, p)
                    p.autotune(max(acc, key=lambda c: (c >> 12) & 15))  # the most PRNs and bins accepted
            items = []
            for r in recs:
                p = g.Plan.for_recording(r)
                rr = torch.from_numpy(np.ascontiguousarray(r.raw)).cuda()
                out = torch.zeros(p.n_prn * 28, dtype=torch.uint8, device="cuda")
                sf = torch.zeros(p.surface_shape(), dtype=torch.float32, device="cuda")
                items.append((p, rr, r.n_samples, out, sf))
            g.acquire_batch(items)
            torch.cuda.synchronize()
            batch = [(o.cpu().numpy(), sf.cpu().numpy()) for _, _, _, o, sf in items]
            alone = []
            for p, rr, n, out, sf in items:
                o2, s2 = torch.zeros_like(out), torch.zeros_like(sf)
                p.acquire_device(rr, n, o2, surface=s2)
                torch.cuda.synchronize()
                alone.append((o2.cpu().numpy(), s2.cpu().numpy()))
            for (oa, sa), (ob, sb) in zip(batch, alone):
                np.testing.assert_array_equal(oa, ob)
                np.testing.assert_array_equal(sa, sb)
            res[which] = alone
        for (oa, sa), (ob, sb) in zip(res["tm"], res["default"]):
            np.testing.assert_array_equal(oa, ob)
            np.testing.assert_array_equal(sa, sb)
    finally:
        for N, p in probe.items():
            p.autotune(_default(N))


def test_staged_wait_gives_up_safely(g):
    """The staged variant's bounded waits, made to give up at once by the
    testing hook (every wait polls zero times; the final drain keeps its full
    bound): each CTA stops issuing copies, reads its spectra from global
    memory, drains the one copy in flight and flags its call.  The
    synchronous call returns GNSS_ETIMEOUT, the device-resident and batched
    calls flag every record with GNSS_DET_STAGE_TIMEOUT, and the records and
    surfaces themselves are those of a run whose waits all succeed, bit for
    bit.  With the limit back, the next call carries no flag."""
    raw_np, n = _recording(4096, 1, 5, siggen.FMT_2BIT_IQ, 4096)
    plan = g.Plan(4_096_000, 1, -3000, 250, 9, prns=[3, 9, 30], half_bit=True, fmt=siggen.FMT_2BIT_IQ)
    raw = torch.from_numpy(np.ascontiguousarray(raw_np)).cuda()
    try:
        plan.autotune(16 | STAGED)
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        ref = plan.acquire(raw, n, surface=surf)
        ref_s = surf.cpu().numpy()
        assert not (ref["flags"] & g.STAGE_TIMEOUT).any()
        g.set_stage_wait_limit(0)
        try:
            out = np.zeros(plan.n_prn, g.DETECTION_DTYPE)
            with pytest.raises(g.GnssError) as e:
                plan.acquire(raw, n, out=out)
            assert e.value.status == g.ETIMEOUT
            assert (out["flags"] & g.STAGE_TIMEOUT).all()
            od = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
            s2 = torch.zeros_like(surf)
            plan.acquire_device(raw, n, od, surface=s2)
            torch.cuda.synchronize()
            d2 = g.detections_from_bytes(od.cpu().numpy())
            assert (d2["flags"] & g.STAGE_TIMEOUT).all()
            np.testing.assert_array_equal(s2.cpu().numpy(), ref_s)
            for f in ("prn", "detected", "set", "dopp_bin", "code_phase", "peak", "second", "ratio"):
                np.testing.assert_array_equal(d2[f], ref[f])
            ob = torch.zeros_like(od)
            g.acquire_batch([(plan, raw, n, ob, None)])
            torch.cuda.synchronize()
            db = g.detections_from_bytes(ob.cpu().numpy())
            assert (db["flags"] & g.STAGE_TIMEOUT).all()
            np.testing.assert_array_equal(db["code_phase"], ref["code_phase"])
        finally:
            g.set_stage_wait_limit(g.STAGE_WAIT_DEFAULT)
        again = plan.acquire(raw, n)
        assert not (again["flags"] & g.STAGE_TIMEOUT).any()
        np.testing.assert_array_equal(again["peak"], ref["peak"])
    finally:
        plan.autotune(_default(4096))


@pytest.mark.parametrize("N", [2048, 4096, 8192, 16384])
def test_buffer_release_wait_gives_up_safely(g, N):
    """The class-local occupancy forms keep one exchange buffer per CTA; the
    next transform's stores wait (bounded) for every warp's release of it.
    With the testing hook every such wait gives up at once: the warps then
    race on the buffer (shared memory, in bounds), and every call reports it
    -- the synchronous call returns GNSS_ETIMEOUT, the device-resident and
    batched calls flag every record with GNSS_DET_WAIT_TIMEOUT.  With the
    limit back, the next call carries no flag and equals the reference."""
    raw_np, n = _recording(N, 1, 5, siggen.FMT_2BIT_IQ, N)
    plan = g.Plan(N * 1000, 1, -3000, 250, 9, prns=[3, 9, 30], half_bit=True, fmt=siggen.FMT_2BIT_IQ)
    raw = torch.from_numpy(np.ascontiguousarray(raw_np)).cuda()
    occ = 16 | TMEM | OCC
    try:
        plan.autotune(occ)
        ref = plan.acquire(raw, n)
        assert not (ref["flags"] & (g.WAIT_TIMEOUT | g.STAGE_TIMEOUT)).any()
        g.set_buf_wait_limit(0)
        try:
            out = np.zeros(plan.n_prn, g.DETECTION_DTYPE)
            with pytest.raises(g.GnssError) as e:
                plan.acquire(raw, n, out=out)
            assert e.value.status == g.ETIMEOUT
            assert (out["flags"] & g.WAIT_TIMEOUT).all()
            od = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
            plan.acquire_device(raw, n, od)
            torch.cuda.synchronize()
            assert (g.detections_from_bytes(od.cpu().numpy())["flags"] & g.WAIT_TIMEOUT).all()
            ob = torch.zeros_like(od)
            g.acquire_batch([(plan, raw, n, ob, None)])
            torch.cuda.synchronize()
            assert (g.detections_from_bytes(ob.cpu().numpy())["flags"] & g.WAIT_TIMEOUT).all()
        finally:
            g.set_buf_wait_limit(g.STAGE_WAIT_DEFAULT)
        again = plan.acquire(raw, n)
        assert not (again["flags"] & g.WAIT_TIMEOUT).any()
        for f in ("prn", "detected", "set", "dopp_bin", "code_phase", "peak", "second", "ratio"):
            np.testing.assert_array_equal(again[f], ref[f])
    finally:
        plan.autotune(_default(N))
