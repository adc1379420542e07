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
