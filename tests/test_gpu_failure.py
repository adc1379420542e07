"""Failure detection without a GPU fault: a bounded wait that nothing
completes gives up, the status word reports EC_ETIMEOUT, and the context
keeps working."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch.cuda.set_device(0)
    xo.ec_device_status(reset=True)
    xo.ec_selftest_wait_timeout(torch.cuda.current_stream().cuda_stream)
    assert xo.ec_device_status(reset=True) == xo.EC_ETIMEOUT
    assert xo.ec_device_status() == 0
    # the context is still usable: an encode afterwards is correct
    k, m, B = 4, 2, 4096
    plan = xo.ec_plan_create(k, m)
    try:
        data = [synth.block_bytes(61, 0, j, B) for j in range(k)]
        d = [torch.from_numpy(x).cuda() for x in data]
        par = [torch.empty(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(plan, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B,
                     torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref = oracle.encode(oracle.cauchy(k, m), data)
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), ref[i])
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)


def test_injected_allocation_failures_are_reported_and_recover():
    """Host-side fault injection: allocations made by the library fail as if
    memory ran out; each call reports EC_ENOMEM and the next ones work."""
    import oracle
    from paper_2108_02692_gb300 import synth
    torch.cuda.set_device(0)
    k, m, B = 4, 2, 8 * 528
    plan = xo.ec_plan_create(k, m)
    st = torch.cuda.current_stream().cuda_stream
    try:
        data = [synth.block_bytes(93, 0, j, B) for j in range(k)]
        ref = oracle.encode(oracle.cauchy(k, m), data)
        d = [torch.from_numpy(x).cuda() for x in data]
        par = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        job = {"plan": plan, "op": xo.EC_OP_ENCODE, "blocks": [t.data_ptr() for t in d],
               "out": [t.data_ptr() for t in par], "block_bytes": B}
        xo.ec_debug_fail_alloc(1)
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode(plan, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, st)
        assert e.value.status == xo.EC_ENOMEM
        # a batch makes four allocations (descriptors, queues, block table,
        # tensor maps): fail each in turn
        for nth in (1, 2, 3, 4):
            xo.ec_debug_fail_alloc(nth)
            with pytest.raises(xo.XorecError) as e:
                xo.ec_batch_create([job])
            assert e.value.status == xo.EC_ENOMEM
        # a server makes three per slot (its status word in mapped host
        # memory, the device table, the pinned staging): fail the first and
        # the last
        for nth in (1, 12):
            xo.ec_debug_fail_alloc(nth)
            with pytest.raises(xo.XorecError) as e:
                xo.ec_server_create()
            assert e.value.status == xo.EC_ENOMEM
        xo.ec_debug_fail_alloc(0)
        xo.ec_encode(plan, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, st)
        b = xo.ec_batch_create([job])
        xo.ec_batch_run(b, st)
        torch.cuda.synchronize()
        xo.ec_batch_destroy(b)
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), ref[i])
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_debug_fail_alloc(0)
        xo.ec_plan_destroy(plan)


def _encode_job(plan, k, m, B, seed):
    data = [synth.block_bytes(seed, 0, j, B) for j in range(k)]
    ref = oracle.encode(oracle.cauchy(k, m), data)
    d = [torch.from_numpy(x).cuda() for x in data]
    par = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
    job = {"plan": plan, "op": xo.EC_OP_ENCODE, "blocks": [t.data_ptr() for t in d],
           "out": [t.data_ptr() for t in par], "block_bytes": B}
    return job, d, par, ref


def test_batch_reports_a_timeout_in_its_own_status_word():
    """A bounded wait that gives up during a batch run (injected on the host:
    the self-test wait runs first on the run's stream, aimed at the batch's
    words) shows in the batch's own status word and in the device's word;
    ec_run_batch returns EC_ETIMEOUT; later runs are clean and correct."""
    torch.cuda.set_device(0)
    k, m, B = 4, 2, 8 * 528
    plan = xo.ec_plan_create(k, m)
    st = torch.cuda.current_stream().cuda_stream
    try:
        job, d, par, ref = _encode_job(plan, k, m, B, 95)
        xo.ec_device_status(reset=True)
        b = xo.ec_batch_create([job])
        try:
            assert xo.ec_batch_status(b) == 0
            xo.ec_debug_inject_timeout(1)
            xo.ec_batch_run(b, st)
            assert xo.ec_batch_status(b) == xo.EC_ETIMEOUT
            assert xo.ec_batch_status(b, reset=True) == xo.EC_ETIMEOUT
            assert xo.ec_batch_status(b) == 0
            assert xo.ec_device_status(reset=True) == xo.EC_ETIMEOUT
            for t in par:
                t.zero_()
            xo.ec_batch_run(b, st)
            assert xo.ec_batch_status(b) == 0
            for i in range(m):
                assert np.array_equal(par[i].cpu().numpy(), ref[i])
        finally:
            xo.ec_batch_destroy(b)
        xo.ec_debug_inject_timeout(1)
        with pytest.raises(xo.XorecError) as e:
            xo.ec_run_batch([job], st)
        assert e.value.status == xo.EC_ETIMEOUT
        assert xo.ec_device_status(reset=True) == xo.EC_ETIMEOUT
        xo.ec_run_batch([job], st)
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_debug_inject_timeout(0)
        xo.ec_plan_destroy(plan)


def _poll_until(server, n, timeout=30.0):
    import time
    got, t0 = [], time.time()
    while len(got) < n and time.time() - t0 < timeout:
        got += xo.ec_server_poll_ex(server)
        time.sleep(0.001)
    assert len(got) == n, got
    return got


def test_server_fails_the_requests_of_a_timed_out_batch():
    """Each serving slot has its own status word: when a bounded wait of its
    batch gives up (injected), that batch's requests come back with
    EC_ETIMEOUT, their admitted bytes return, and the next request on the
    same slot completes normally and bit-exact."""
    torch.cuda.set_device(0)
    k, m, B = 4, 2, 8 * 528
    plan = xo.ec_plan_create(k, m)
    sv = xo.ec_server_create(slots=1, max_batch=1, background_compile=False)
    try:
        xo.ec_server_warm(sv, plan, 0)
        xo.ec_device_status(reset=True)
        job, d, par, ref = _encode_job(plan, k, m, B, 96)
        xo.ec_debug_inject_timeout(1)
        t1 = xo.ec_server_submit(sv, job)
        (got,) = _poll_until(sv, 1)
        assert got[0] == t1 and got[2] == xo.EC_ETIMEOUT
        st = xo.ec_server_stats_get(sv)
        assert st["failed"] == 1 and st["admitted_bytes"] == 0
        assert xo.ec_device_status(reset=True) == xo.EC_ETIMEOUT
        for t in par:
            t.zero_()
        t2 = xo.ec_server_submit(sv, job)
        (got,) = _poll_until(sv, 1)
        assert got[0] == t2 and got[2] == xo.EC_OK
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), ref[i])
        st = xo.ec_server_stats_get(sv)
        assert st["failed"] == 1 and st["completed"] == 2 and st["admitted_bytes"] == 0
    finally:
        xo.ec_debug_inject_timeout(0)
        xo.ec_server_destroy(sv)
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0


def test_server_dispatch_failure_fails_tickets_and_releases_bytes():
    """A batch that cannot be launched (its slot's table cannot grow: the
    allocation fails, injected on the host) returns its requests with
    EC_ENOMEM and gives their admitted bytes back; the server recovers."""
    torch.cuda.set_device(0)
    k, m, B = 40, 8, 8 * 256
    plan = xo.ec_plan_create(k, m)
    # one request per batch; a wide code's block table (48 pointers) is
    # larger than a slot's initial table, so the dispatch must grow it
    sv = xo.ec_server_create(slots=1, max_batch=1, background_compile=False)
    try:
        xo.ec_server_warm(sv, plan, 0)
        job, d, par, ref = _encode_job(plan, k, m, B, 97)
        xo.ec_debug_fail_alloc(1)
        t1 = xo.ec_server_submit(sv, job)
        (got,) = _poll_until(sv, 1)
        assert got[0] == t1 and got[2] == xo.EC_ENOMEM
        st = xo.ec_server_stats_get(sv)
        assert st["failed"] == 1 and st["admitted_bytes"] == 0 and st["pending"] == 0
        xo.ec_debug_fail_alloc(0)
        t2 = xo.ec_server_submit(sv, job)
        (got,) = _poll_until(sv, 1)
        assert got[0] == t2 and got[2] == xo.EC_OK
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), ref[i])
    finally:
        xo.ec_debug_fail_alloc(0)
        xo.ec_server_destroy(sv)
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0
