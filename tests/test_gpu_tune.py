"""Autotuner: picks a launch shape and register budget, keeps the results
bit-exact."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def test_autotune_then_encode_and_decode():
    torch.cuda.set_device(0)
    k, m = 10, 4
    plan = xo.ec_plan_create(k, m)
    try:
        st = torch.cuda.current_stream().cuda_stream
        r = xo.ec_plan_autotune(plan, 1 << 20, 8, st)
        assert r["candidates"] >= 2 and r["threads"] in (128, 256) and r["gbps_in"] > 0
        B = 8 * 1552
        data = [synth.block_bytes(71, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(oracle.cauchy(k, m), data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        par = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(plan, [t.data_ptr() for t in d[:k]], [t.data_ptr() for t in par], B, st)
        er = [1, 7, 11]
        outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
        xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                     [t.data_ptr() for t in outs], B, st)
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), blocks[k + i])
        for t, e in zip(outs, er):
            assert np.array_equal(t.cpu().numpy(), blocks[e])
    finally:
        xo.ec_plan_destroy(plan)
