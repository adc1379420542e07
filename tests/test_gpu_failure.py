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
        # a server makes two per slot (device table, pinned staging): fail the
        # first and the last
        for nth in (1, 8):
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
