"""GPU parity of the tracking channels (gnss_track) against the FP64 oracle
(Section 3, Fig. 3): the 1 s tracking recording with its 8 satellites started
from perturbed truth, int8 recordings at 2.048 and 16.384 MHz with 2 ms
intervals, channels for absent PRNs, and the status of bad channels.

Both sides run the same fixed-point NCOs; only the correlator sums (FP32 vs
FP64) and hence, through the loops, the NCO words' last bits can differ.  A
locked channel is compared record by record: NCO frequency within 2e-3 Hz
(two steps of the 32-bit carrier word), delay within 1e-4 chip, correlators
within 1e-4 of the channel's prompt scale, discriminators within 1e-4.  A
channel on an absent PRN tracks noise, where FP32 and FP64 can take
different near-zero decisions: only its first interval (same NCO words on
both sides) is compared, the rest checked for validity."""
import numpy as np
import pytest

import oracle
import siggen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def _run(g, rec, prn, f, tau, n_int, coh=1, spacing=1.0, bpll=15.0, bdll=2.0):
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    cands = g.candidates(prn, f, tau)
    cdev = torch.from_numpy(cands.view(np.uint8)).cuda()
    out = torch.zeros(len(cands) * n_int * g.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    plan.track(raw, rec.n_samples, cdev, len(cands), out, n_int, coh, spacing, bpll, bdll)
    torch.cuda.synchronize()
    return g.track_records(out.cpu().numpy()).reshape(len(cands), n_int)


def _compare(gpu, ref, n=None):
    n = len(ref) if n is None else n
    gpu, ref = gpu[:n], ref[:n]
    assert np.all(gpu["status"] == 0)
    scale = max(np.abs(ref["zp"]).max(), 1.0)
    assert np.abs(gpu["f_hz"] - ref["f_hz"]).max() <= 2e-3
    dt = (gpu["tau_chips"] - ref["tau_chips"] + 511.5) % 1023 - 511.5
    assert np.abs(dt).max() <= 1e-4
    for z in ("ze", "zp", "zl"):
        assert np.abs(gpu[z] - ref[z]).max() <= 1e-4 * scale, z
    assert np.abs(gpu["e_phi"] - ref["e_phi"]).max() <= 1e-4
    assert np.abs(gpu["e_tau"] - ref["e_tau"]).max() <= 1e-4


def test_track_1s_parity_and_lock(g):
    rec = siggen.track_1s()
    prn, f, tau = siggen.track_starts(rec)
    n_int = 400
    out = _run(g, rec, prn, f, tau, n_int)
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    for k in range(len(prn)):
        ref = oracle.track(x, rec.fs, 1, n_int, oracle.ca_code(int(prn[k])), f[k], tau[k], 1.0, 15.0, 2.0)
        _compare(out[k], ref)
        # locked: prompt power in I
        last = out[k][-100:]
        assert np.mean(last["zp"][:, 1] ** 2) < 0.1 * np.mean(last["zp"][:, 0] ** 2)


@pytest.mark.parametrize("tpc", [32, 64, 128, 256])
def test_threads_per_channel_launch(g, tpc):
    """Channels take the smallest group of 32 .. 256 threads that gives them
    together the GPU's resident threads (1024 per SM), so the channel count
    picks the group: copies of the 8 satellites' channels, as many as select
    a group of tpc threads, give identical records copy to copy and match the
    oracle."""
    rec = siggen.track_1s()
    prn, f, tau = siggen.track_starts(rec)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # tpc < 256: the fewest channels for which tpc threads each suffice
    n_chan = 80 * len(prn) if tpc == 256 else -(-sms * 1024 // tpc)
    reps = -(-n_chan // len(prn))
    assert tpc == 256 or reps * len(prn) < 2 * n_chan  # still in tpc's range
    n_int = 200
    out = _run(g, rec, np.tile(prn, reps), np.tile(f, reps), np.tile(tau, reps), n_int)
    for r in range(1, reps):
        np.testing.assert_array_equal(out[r * len(prn):(r + 1) * len(prn)], out[:len(prn)])
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    for k in range(len(prn)):
        ref = oracle.track(x, rec.fs, 1, n_int, oracle.ca_code(int(prn[k])), f[k], tau[k], 1.0, 15.0, 2.0)
        _compare(out[k], ref)


@pytest.mark.parametrize("fs,coh", [(2_048_000, 2), (16_384_000, 1)])
def test_int8_rates_and_intervals(g, fs, coh):
    N = fs // 1000
    n_int = 120
    rng = np.random.default_rng(fs + coh)
    sats = siggen.draw_sats(rng, 3, (44.0, 48.0), (-4000.0, 4000.0), n_int * coh, rate=0.5)
    x = siggen.synthesize(rng, fs, n_int * coh * N, sats)
    li, lq = siggen.quantize_2bit(x, sats, fs)
    rec = siggen.Recording(raw=siggen.pack(li, lq, siggen.FMT_I8_IQ), fmt=siggen.FMT_I8_IQ, fs=fs,
                           n_samples=n_int * coh * N, sats=sats)
    prn = np.array([s.prn for s in sats])
    f = np.array([s.dopp_hz + 2.0 for s in sats])
    tau = np.array([(s.code_phase_chips - 0.05) % 1023 for s in sats])
    out = _run(g, rec, prn, f, tau, n_int, coh=coh, spacing=0.5, bpll=10.0, bdll=1.0)
    xx = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    for k in range(len(prn)):
        ref = oracle.track(xx, fs, coh, n_int, oracle.ca_code(int(prn[k])), f[k], tau[k], 0.5, 10.0, 1.0)
        _compare(out[k], ref)


def test_absent_prn_and_bad_channels(g):
    rec = siggen.track_1s()
    present = {s.prn for s in rec.sats}
    absent = [p for p in range(1, 33) if p not in present][:3]
    n_int = 50
    prn = absent + [absent[0], absent[0]]
    f = [100.0, -2000.0, 3000.0, 0.6 * rec.fs, 0.0]
    tau = [10.0, 500.0, 900.0, 0.0, 0.0]
    plan = g.Plan.for_recording(rec, prns=[p for p in range(1, 33) if p != 32])
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    cands = g.candidates(prn + [32], f + [0.0], tau + [0.0])
    cdev = torch.from_numpy(cands.view(np.uint8)).cuda()
    out_dev = torch.zeros(len(cands) * n_int * g.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    plan.track(raw, rec.n_samples, cdev, len(cands), out_dev, n_int)
    torch.cuda.synchronize()
    out = g.track_records(out_dev.cpu().numpy()).reshape(len(cands), n_int)
    x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
    for k in range(3):  # noise channels: first interval exact, then valid
        ref = oracle.track(x, rec.fs, 1, 1, oracle.ca_code(prn[k]), f[k], tau[k], 1.0, 15.0, 1.0)
        _compare(out[k], ref, n=1)
        assert np.all(out[k]["status"] == 0) and np.all(np.isfinite(out[k]["f_hz"]))
    assert np.all(out[3]["status"] == -2)  # carrier beyond fs / 2: stopped at once
    assert np.all(out[4]["status"] == 0)
    assert np.all(out[5]["status"] == -1)  # PRN 32 is not in this plan


def test_rejects_bad_configuration(g):
    rec = siggen.track_1s()
    plan = g.Plan.for_recording(rec)
    raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
    cdev = torch.from_numpy(g.candidates([1], [0.0], [0.0]).view(np.uint8)).cuda()
    out = torch.zeros(10 * g.TRACK_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    for kw in (dict(n_int=1001), dict(n_int=1, spacing=0.0), dict(n_int=1, spacing=1.5),
               dict(n_int=1, pll_bw_hz=-1.0)):
        with pytest.raises(g.GnssError) as e:
            plan.track(raw, rec.n_samples, cdev, 1, out, **kw)
        assert e.value.status == g.EINVAL
    low = g.Plan(1_024_000, 1, 0, 1, 1, prns=[1])
    with pytest.raises(g.GnssError):
        low.track(raw, 1024 * 10, cdev, 1, out, 1)  # under 2.048 MHz
