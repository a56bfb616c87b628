"""Served requests at the serving workload's largest sample rate against the
FP64 oracle: two requests of the serving pool (64 recordings, the benchmark's
seed) -- the shortest at 16.384 MHz (57 ms, 2 ms coherent blocks, 81 bins:
the 16384-point occupancy form) and the shortest at 8.192 MHz (20 ms) -- go
through the server together; the records of the satellites each recording
holds (up to four) and of two PRNs it does not hold are compared with the
oracle's detections for those PRNs (a PRN's record depends on its own
surfaces only)."""
import numpy as np
import pytest

import oracle
import siggen
from parity import compare_detections

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

POOL = 64


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


def _shortest(fs):
    params = siggen._batch_params(POOL, siggen.SEED_BASE + 5, (2_048_000, 4_096_000, 8_192_000, 16_384_000),
                                  (10, 500), (2, 12))
    return min((p[1], i) for i, p in enumerate(params) if p[0] == fs)[1]


def test_served_requests_match_the_oracle(g):
    idx = [_shortest(16_384_000), _shortest(8_192_000)]
    recs = siggen.serving_requests_subset((POOL, idx))
    assert [r.fs for r in recs] == [16_384_000, 8_192_000]
    srv = g.Server(max_batch=64, streams=2)
    try:
        tickets = [srv.submit(g.Server.desc_for(r), r.raw, r.n_samples) for r in recs]
        served = [srv.wait(t, 600000) for t in tickets]
    finally:
        srv.close()
    for rec, out in zip(recs, served):
        assert len(out) == 32 and list(out["prn"]) == list(range(1, 33))
        present = sorted({s.prn for s in rec.sats})[:4]
        absent = [p for p in range(1, 33) if p not in {s.prn for s in rec.sats}][:2]
        prns = sorted(present + absent)
        x = oracle.unpack(rec.raw, rec.n_samples, rec.fmt)
        S = oracle.surfaces(x, rec.fs, rec.coh_ms, rec.n_blocks, rec.half_bit, prns, rec.dopp_hz, nthreads=8)
        ref = oracle.detect(S, prns)
        got = out[np.isin(out["prn"], prns)]
        assert compare_detections(got, ref, S) == 0, rec.fs
        for s in rec.sats:  # strong satellites are found within a bin of their injected Doppler
            if s.prn in present and s.cn0_dbhz >= 42.0:
                r = out[out["prn"] == s.prn][0]
                assert r["detected"], (rec.fs, s.prn)
                assert abs(float(r["dopp_hz"]) - s.dopp_hz) <= rec.dopp_step_hz, (rec.fs, s.prn, r["dopp_hz"])
