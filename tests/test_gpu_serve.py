"""Request server with continuous batching (gnss_server_*): results in the mix
equal the results alone; admission by device memory; back-pressure,
cancellation, waits with a limit, queue timeout and an injected allocation
failure -- all made on the host, nothing is faulted on the device."""
import threading
import time

import numpy as np
import pytest

import siggen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    import paper_1309_0052_b300 as g
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return g


@pytest.fixture(scope="module")
def recs():
    return siggen.batch_requests(12, ms_range=(20, 60)) + [siggen.plain_4ms(), siggen.weak_100ms()]


@pytest.fixture(scope="module")
def alone(g, recs):
    """Records of every recording acquired on its own (gnss_acquire)."""
    out = []
    for rec in recs:
        plan = g.Plan.for_recording(rec)
        out.append(plan.acquire(np.ascontiguousarray(rec.raw), rec.n_samples))
    return out


def test_results_in_the_mix_equal_results_alone(g, recs, alone):
    srv = g.Server(max_batch=8, streams=2)
    tickets = []
    lock = threading.Lock()

    def client(chunk):
        for k in chunk:
            t = srv.submit(g.Server.desc_for(recs[k]), recs[k].raw, recs[k].n_samples)
            with lock:
                tickets.append((k, t))
            time.sleep(0.002)

    threads = [threading.Thread(target=client, args=(range(i, len(recs), 3),)) for i in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for k, t in tickets:
        np.testing.assert_array_equal(srv.wait(t, 60000), alone[k])
    st = srv.stats()
    assert st["completed"] == len(recs) and st["failed"] == 0 and st["queued"] == 0
    # a burst: the requests submitted while the first one is on the GPU are
    # admitted together (continuous batching), whatever the kernels' speed
    burst = [srv.submit(g.Server.desc_for(r), r.raw, r.n_samples) for r in recs]
    for k, t in enumerate(burst):
        np.testing.assert_array_equal(srv.wait(t, 60000), alone[k])
    st2 = srv.stats()
    assert st2["completed"] == 2 * len(recs) and st2["failed"] == 0
    assert st2["batches"] - st["batches"] < len(recs)  # requests shared launches
    srv.close()


def test_admission_by_device_memory(g, recs, alone):
    # each of these requests holds at most ~20 MB in flight (folded blocks and
    # the spectra shared by bins a whole kHz apart), the 14 together ~150 MB
    budget = 40 << 20
    srv = g.Server(device_mem_budget=budget, max_batch=64)
    tickets = [srv.submit(g.Server.desc_for(r), r.raw, r.n_samples) for r in recs]
    seen = 0
    while True:
        s = srv.stats()
        assert s["device_bytes_reserved"] <= budget
        seen = max(seen, s["batches_in_flight"])
        if s["completed"] + s["failed"] == len(recs):
            break
        time.sleep(0.001)
    for k, t in enumerate(tickets):
        np.testing.assert_array_equal(srv.poll(t), alone[k])
    assert srv.stats()["batches"] > 1
    srv.close()


def test_request_larger_than_budget_is_refused(g, recs):
    # the 100 ms request holds about 3 MB in flight (recording, 1.3 MB of
    # folded blocks, 1.3 MB of shared spectra, row statistics)
    srv = g.Server(device_mem_budget=1 << 20)
    with pytest.raises(g.GnssError) as e:
        srv.submit(g.Server.desc_for(recs[-1]), recs[-1].raw, recs[-1].n_samples)
    assert e.value.status == g.EBUSY
    srv.close()


def test_host_staging_back_pressure(g, recs):
    srv = g.Server(host_staging_bytes=300 << 10, device_mem_budget=8 << 30)
    rec = recs[-1]  # 204,800 bytes of recording
    t1 = srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples)
    busy = 0
    for _ in range(3):
        try:
            srv.wait(srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples), 60000)
        except g.GnssError as e:
            assert e.status == g.EBUSY
            busy += 1
    srv.wait(t1, 60000)
    assert busy >= 1
    srv.close()


def test_cancel_wait_limit_and_unknown_ticket(g, recs):
    srv = g.Server(max_batch=1, streams=1)
    rec = recs[-1]
    ts = [srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples) for _ in range(6)]
    srv.cancel(ts[-1])  # still queued behind the others
    with pytest.raises(g.GnssError) as e:
        srv.wait(ts[-1], 60000)
    assert e.value.status == g.ECANCELLED
    with pytest.raises(g.GnssError) as e:
        srv.wait(ts[-2], 0)  # not done yet
    assert e.value.status == g.ETIMEOUT
    for t in ts[:-1]:
        assert len(srv.wait(t, 60000)) == 32
    with pytest.raises(g.GnssError) as e:
        srv.poll(ts[0])  # handed out already
    assert e.value.status == g.EINVAL
    srv.close()


def test_queue_timeout(g, recs):
    srv = g.Server(max_batch=1, streams=1, queue_timeout_ms=1)
    rec = recs[-1]
    ts = [srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples) for _ in range(8)]
    codes = []
    for t in ts:
        try:
            srv.wait(t, 60000)
            codes.append(g.OK)
        except g.GnssError as e:
            codes.append(e.status)
    assert set(codes) <= {g.OK, g.ETIMEOUT}
    assert g.ETIMEOUT in codes
    srv.close()


def test_injected_allocation_failure(g, recs, alone):
    srv = g.Server(max_batch=64, streams=1)
    srv.inject_alloc_failure(0)
    rec = recs[0]
    t_fail = srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples)
    with pytest.raises(g.GnssError) as e:
        srv.wait(t_fail, 60000)
    assert e.value.status == g.ENOMEM
    t_ok = srv.submit(g.Server.desc_for(rec), rec.raw, rec.n_samples)
    np.testing.assert_array_equal(srv.wait(t_ok, 60000), alone[0])
    s = srv.stats()
    assert s["failed"] == 1 and s["device_bytes_reserved"] == 0
    srv.close()


def test_admission_bound_refuses_on_the_host(g, recs, alone):
    """The admission bound (max_queue_wait_ms): once a batch has completed and
    the server knows its throughput, a submission whose projected wait -- the
    work queued and in flight ahead of it plus its own, over that throughput
    -- exceeds the bound is refused at once with GNSS_EBUSY (counted in the
    stats); every accepted request still completes with its records alone.
    The decision is made on the host; nothing is faulted on the device."""
    rec, ref = recs[-1], alone[-1]  # the 100 ms request
    srv = g.Server(max_batch=4, streams=2, max_queue_wait_ms=20)
    desc = g.Server.desc_for(rec)
    try:
        np.testing.assert_array_equal(srv.wait(srv.submit(desc, rec.raw, rec.n_samples), 60000), ref)
        tickets, refused = [], 0
        for _ in range(300):
            try:
                tickets.append(srv.submit(desc, rec.raw, rec.n_samples))
            except g.GnssError as e:
                assert e.status == g.EBUSY and "admission bound" in str(e)
                refused += 1
        assert refused > 0 and len(tickets) > 0
        for t in tickets:
            np.testing.assert_array_equal(srv.wait(t, 60000), ref)
        st = srv.stats()
        assert st["refused"] == refused
        assert st["completed"] == len(tickets) + 1 and st["failed"] == 0
    finally:
        srv.close()


def test_no_admission_bound_by_default(g, recs, alone):
    """Without a bound a burst queues up in full (only memory and staging
    limit admission) and nothing is refused."""
    rec, ref = recs[-1], alone[-1]
    srv = g.Server(max_batch=4, streams=2)
    desc = g.Server.desc_for(rec)
    try:
        tickets = [srv.submit(desc, rec.raw, rec.n_samples) for _ in range(40)]
        for t in tickets:
            np.testing.assert_array_equal(srv.wait(t, 60000), ref)
        assert srv.stats()["refused"] == 0
    finally:
        srv.close()
