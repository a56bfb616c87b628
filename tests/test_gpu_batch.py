"""Batched acquisition (gnss_acquire_batch): recordings of uneven length,
sample rate, Doppler grid and coherent length in one launch triple per
(FFT size, format, half-bit) group.  Each request must give exactly the
records and surfaces it gets alone (gnss_acquire_device), whatever the wave
split, and match the FP64 oracle."""
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


@pytest.fixture(scope="module")
def mix(g):
    """Short uneven 2-bit recordings at 2.048 / 4.096 / 8.192 MHz with 250 / 500 Hz
    grids, plus an int8 4 ms recording and a half-bit 100 ms recording, so the
    batch spans several groups."""
    recs = siggen.batch_requests(10, ms_range=(20, 40))
    recs += [siggen.plain_4ms(), siggen.weak_100ms()]
    items = []
    for rec in recs:
        plan = g.Plan.for_recording(rec)
        raw = torch.from_numpy(np.ascontiguousarray(rec.raw)).cuda()
        items.append((rec, plan, raw))
    return items


def _alone(g, plan, raw, n):
    out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
    plan.acquire_device(raw, n, out, surface=surf)
    return out, surf


def _batched(g, mix, budget):
    outs, surfs, reqs = [], [], []
    for rec, plan, raw in mix:
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        outs.append(out)
        surfs.append(surf)
        reqs.append((plan, raw, rec.n_samples, out, surf))
    g.acquire_batch(reqs, scratch_budget=budget)
    torch.cuda.synchronize()
    return outs, surfs


@pytest.mark.parametrize("budget", [0, 1, 200 << 20])
def test_batch_equals_alone(g, mix, budget):
    """budget 0: default (one wave per group); 1 byte: every request in a wave
    of its own; 200 MB: groups split into several waves."""
    outs, surfs = _batched(g, mix, budget)
    for (rec, plan, raw), out, surf in zip(mix, outs, surfs):
        a_out, a_surf = _alone(g, plan, raw, rec.n_samples)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), a_out.cpu().numpy())
        np.testing.assert_array_equal(surf.cpu().numpy(), a_surf.cpu().numpy())


def test_batch_matches_oracle(g, mix):
    outs, surfs = _batched(g, mix, 0)
    for k in (0, 3, 7, 10):  # 2-bit at three rates and grids, and int8
        rec, plan, raw = mix[k]
        x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
        prns = np.arange(1, 33)
        S = oracle.surfaces(x, rec.fs, rec.coh_ms, rec.n_blocks, rec.half_bit, prns, rec.dopp_hz, 8)
        det = oracle.detect(S, prns)
        compare_surfaces(surfs[k].cpu().numpy(), S)
        compare_detections(g.detections_from_bytes(outs[k].cpu().numpy()), det, S)


def test_batch_rejects_invalid_request_before_launching(g, mix):
    rec, plan, raw = mix[0]
    out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
    good = (plan, raw, rec.n_samples, out, None)
    short = (plan, raw, plan.block_len - 1, out, None)
    with pytest.raises(g.GnssError) as e:
        g.acquire_batch([good, short])
    assert e.value.status == g.EINVAL
    assert b"request 1" in g.lib.gnss_last_error()
    g.acquire_batch([])  # empty batch is a no-op


@pytest.mark.parametrize("budget", [0, 200 << 20])
def test_batch_graph_replays_the_batch(g, mix, budget):
    """The batch captured into a CUDA graph: each replay gives exactly the
    records and surfaces of gnss_acquire_batch, with one wave per group or
    several waves sharing the graph's scratch; two replays in a row on one
    stream give the same results again."""
    ref_outs, ref_surfs = _batched(g, mix, budget)
    outs, surfs, reqs = [], [], []
    for rec, plan, raw in mix:
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
        outs.append(out)
        surfs.append(surf)
        reqs.append((plan, raw, rec.n_samples, out, surf))
    graph = g.BatchGraph(reqs, scratch_budget=budget)
    s = torch.cuda.Stream()
    try:
        for _ in range(2):
            for o, sf in zip(outs, surfs):
                o.zero_()
                sf.zero_()
            torch.cuda.synchronize()
            graph.launch(stream=s)
            s.synchronize()
            for o, sf, ro, rs in zip(outs, surfs, ref_outs, ref_surfs):
                np.testing.assert_array_equal(o.cpu().numpy(), ro.cpu().numpy())
                np.testing.assert_array_equal(sf.cpu().numpy(), rs.cpu().numpy())
    finally:
        graph.close()


def test_batch_graph_follows_new_recordings_in_the_same_buffers(g):
    """Slots refilled with other recordings of the same size: a replay of the
    unchanged graph acquires the new contents (here, the bytes of each
    recording shuffled), as gnss_acquire_device does on them."""
    first = siggen.batch_requests(4, ms_range=(20, 40), seed=7)
    rng = np.random.default_rng(11)
    items = []
    for r1 in first:
        plan = g.Plan.for_recording(r1)
        raw = torch.from_numpy(np.ascontiguousarray(r1.raw)).cuda()
        out = torch.zeros(plan.n_prn * 28, dtype=torch.uint8, device="cuda")
        items.append((plan, raw, r1.n_samples, out, None))
    graph = g.BatchGraph(items)
    try:
        graph.launch()
        torch.cuda.synchronize()
        for (plan, raw, n, out, _), r1 in zip(items, first):
            new = np.ascontiguousarray(r1.raw).copy()
            rng.shuffle(new)  # a different recording of the same size and format
            raw.copy_(torch.from_numpy(new))
        graph.launch()
        torch.cuda.synchronize()
        for plan, raw, n, out, _ in items:
            ref = torch.zeros_like(out)
            plan.acquire_device(raw, n, ref)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    finally:
        graph.close()
