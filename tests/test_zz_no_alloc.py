"""ec_encode_noalloc: the encode entry point for callers that may not
allocate device memory while they encode.  Its output must equal that of
ec_encode and the oracle's encode (bit for bit, the tolerance of every
parity test here) on two calls in a row, whose second call reuses the
shared static scratch array; a bounded wait of its kernel that gives up is
visible through ec_device_status.  Kept in a file that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,m,B", [(10, 4, 8 * 3152), (4, 2, 64 * 1024)])
def test_noalloc_encode_matches_ec_encode_twice(k, m, B):
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    plan = xo.ec_plan_create(k, m)
    try:
        outs = []
        for call in range(2):
            host = [synth.block_bytes(40 + call, k, j, B) for j in range(k)]
            expect = oracle.encode(oracle.cauchy(k, m), host)
            data = [torch.from_numpy(x).cuda() for x in host]
            ref = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
            got = [torch.full((B,), 0x77, dtype=torch.uint8, device="cuda") for _ in range(m)]
            xo.ec_encode(plan, [t.data_ptr() for t in data], [t.data_ptr() for t in ref], B, st)
            xo.ec_encode_noalloc(plan, [t.data_ptr() for t in data],
                                 [t.data_ptr() for t in got], B, st)
            torch.cuda.synchronize()
            for i in range(m):
                g = got[i].cpu().numpy()
                assert np.array_equal(g, ref[i].cpu().numpy()), (call, i)
                assert np.array_equal(g, expect[i]), (call, i)
            outs.append([g.cpu().numpy() for g in got])
        # the two calls encoded different data
        assert not np.array_equal(outs[0][0], outs[1][0])
        # no bounded wait gave up, in the device's word or the array's
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)


def test_noalloc_timeout_is_reported_by_ec_device_status():
    """The kernels of ec_encode_noalloc record a timed-out wait in the status
    word of the static array; ec_device_status reads and clears it.  The
    timeout is injected on the host: the self-test wait, aimed at that word,
    runs on the call's stream before the encode (which still runs and is
    bit-exact)."""
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    k, m, B = 4, 2, 8 * 528
    plan = xo.ec_plan_create(k, m)
    try:
        host = [synth.block_bytes(42, k, j, B) for j in range(k)]
        expect = oracle.encode(oracle.cauchy(k, m), host)
        data = [torch.from_numpy(x).cuda() for x in host]
        got = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode_noalloc(plan, [t.data_ptr() for t in data], [t.data_ptr() for t in got], B, st)
        xo.ec_device_status(reset=True)
        xo.ec_debug_inject_timeout(1)
        xo.ec_encode_noalloc(plan, [t.data_ptr() for t in data], [t.data_ptr() for t in got], B, st)
        assert xo.ec_device_status(reset=True) == xo.EC_ETIMEOUT
        assert xo.ec_device_status() == 0
        for i in range(m):
            assert np.array_equal(got[i].cpu().numpy(), expect[i])
    finally:
        xo.ec_debug_inject_timeout(0)
        xo.ec_plan_destroy(plan)


def test_noalloc_rejects_bad_arguments():
    torch.cuda.set_device(0)
    plan = xo.ec_plan_create(4, 2)
    try:
        B = 1024
        bufs = [torch.zeros(B + 16, dtype=torch.uint8, device="cuda") for _ in range(6)]
        ptrs = [b.data_ptr() for b in bufs]
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode_noalloc(plan, ptrs[:4], ptrs[4:], 1000, 0)
        assert e.value.status == xo.EC_EINVAL
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode_noalloc(plan, [ptrs[0] + 8] + ptrs[1:4], ptrs[4:], B, 0)
        assert e.value.status == xo.EC_EINVAL
    finally:
        xo.ec_plan_destroy(plan)
