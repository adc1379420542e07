"""Degenerate and empty inputs on the GPU, and a closed-form check that does
not use the oracle: with one parity block the scaled Cauchy matrix is the
all-ones row, so the parity is the XOR of the data blocks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan():
    torch.cuda.set_device(0)
    h = xo.ec_plan_create(10, 4)
    yield h
    xo.ec_plan_destroy(h)


def stream():
    return torch.cuda.current_stream().cuda_stream


def test_zero_stripes_write_nothing(plan):
    k, m, B = 10, 4, 4096
    data = torch.zeros((1, k, B), dtype=torch.uint8, device="cuda")
    par = torch.full((1, m, B), 0x77, dtype=torch.uint8, device="cuda")
    xo.ec_encode_strided(plan, data.data_ptr(), k * B, B, par.data_ptr(), m * B, B, 0, B, stream())
    h_data = torch.zeros((1, k, B), dtype=torch.uint8, pin_memory=True)
    h_par = torch.full((1, m, B), 0x77, dtype=torch.uint8, pin_memory=True)
    xo.ec_encode_host_strided(plan, h_data.data_ptr(), k * B, B, h_par.data_ptr(), m * B, B, 0, B,
                              0, stream())
    torch.cuda.synchronize()
    assert bool((par == 0x77).all()) and bool((h_par == 0x77).all())


def test_empty_batch_runs_and_captures(plan):
    b = xo.ec_batch_create([])
    try:
        info = xo.ec_batch_info_get(b)
        assert info["stripes"] == 0 and info["launches"] == 0
        xo.ec_batch_run(b, stream())
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            xo.ec_batch_run(b, s.cuda_stream)
        g.replay()
        torch.cuda.synchronize()
    finally:
        xo.ec_batch_destroy(b)
    xo.ec_run_batch([], stream())
    torch.cuda.synchronize()
    assert xo.ec_device_status() == 0


@pytest.mark.parametrize("executor", [xo.EC_EXEC_INTERP, xo.EC_EXEC_COMPILED, xo.EC_EXEC_DENSE],
                         ids=["interp", "compiled", "dense"])
@pytest.mark.parametrize("k", [1, 7, 32])
def test_single_scaled_parity_is_xor_of_data(k, executor):
    B = 8 * 1040
    h = xo.ec_plan_create_ex(k, 1, matrix_kind=xo.EC_MATRIX_CAUCHY_MIN, executor=executor)
    try:
        data = [synth.block_bytes(81, k, j, B) for j in range(k)]
        expect = np.bitwise_xor.reduce(np.stack(data), axis=0)
        d = [torch.from_numpy(x).cuda() for x in data]
        par = torch.zeros(B, dtype=torch.uint8, device="cuda")
        xo.ec_encode(h, [t.data_ptr() for t in d], [par.data_ptr()], B, stream())
        # recover a lost data block from the other blocks and the parity
        lost = k // 2
        rec = torch.zeros(B, dtype=torch.uint8, device="cuda")
        blocks = [None if j == lost else d[j].data_ptr() for j in range(k)] + [par.data_ptr()]
        xo.ec_decode(h, [lost], blocks, [rec.data_ptr()], B, stream())
        torch.cuda.synchronize()
        assert np.array_equal(par.cpu().numpy(), expect)
        assert np.array_equal(rec.cpu().numpy(), data[lost])
    finally:
        xo.ec_plan_destroy(h)


def test_erasure_order_is_the_callers(plan):
    # outputs follow the caller's erasure order, whatever it is
    k, m, B = 10, 4, 8 * 528
    data = [synth.block_bytes(82, 0, j, B) for j in range(k)]
    blocks = data + oracle.encode(oracle.cauchy(k, m), data)
    d = [torch.from_numpy(x).cuda() for x in blocks]
    for er in ([13, 2, 7, 0], [5, 11], [12, 3, 10]):
        outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
        xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                     [t.data_ptr() for t in outs], B, stream())
        torch.cuda.synchronize()
        for t, e in zip(outs, er):
            assert np.array_equal(t.cpu().numpy(), blocks[e]), (er, e)
