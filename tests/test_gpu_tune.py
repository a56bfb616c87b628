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


@pytest.mark.parametrize("N,half", [(2048, False), (8192, True), (16384, False)])
def test_every_shape_matches_oracle(g, N, half):
    coh, B, fmt = 1, 4, siggen.FMT_2BIT_IQ
    raw, n = _recording(N, coh, B, fmt, N)
    prns = [3, 9, 30]
    dopp = (-3000, 250, 9)
    plan = g.Plan(N * 1000, coh, dopp[0], dopp[1], dopp[2], prns=prns, half_bit=half, fmt=fmt)
    x = oracle.unpack(raw, n, fmt)
    S = oracle.surfaces(x, N * 1000, coh, B, half, prns, dopp[0] + dopp[1] * np.arange(dopp[2]), 8)
    ref = oracle.detect(S, prns)
    default = 32 if N >= 16384 else 16
    try:
        for elems in (16, 32):
            if (elems == 32 and N < 1024) or (elems == 16 and N > 16384):
                continue
            assert plan.autotune(elems)["chosen"] == elems
            surf = torch.zeros(plan.surface_shape(), dtype=torch.float32, device="cuda")
            det = plan.acquire(torch.from_numpy(np.ascontiguousarray(raw)).cuda(), n, surface=surf)
            torch.cuda.synchronize()
            compare_surfaces(surf.cpu().numpy(), S)
            assert compare_detections(det, ref, S) == 0
        r = plan.autotune()
        assert r["chosen"] in r["timed"] and len(r["timed"]) == 2
        assert all(ms > 0 for ms in r["timed"].values())
    finally:
        plan.autotune(default)


def test_invalid_shape_rejected(g):
    plan = g.Plan(512_000, 1, 0, 1, 1, prns=[1])
    with pytest.raises(g.GnssError) as e:
        plan.autotune(32)  # N = 512 has too few elements for 32 per thread
    assert e.value.status == g.EINVAL
