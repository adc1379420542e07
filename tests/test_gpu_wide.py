"""Wide codes (more than 96 input strips, k >= 13): the two-level program
(partial sums in registers, each input word read from the shared-memory tile
once per group; with or without XorRePair temporals per window) and the
one-statement-per-row form (stream_window = -1) against the oracle: single
launches, strided launches with ragged strip tails, decoders, and batches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("k,m", [(13, 4), (16, 4), (20, 4), (32, 4), (24, 8)])
def test_two_level_strided_encode_matches_oracle(k, m):
    torch.cuda.set_device(0)
    B, n = 8 * 1552, 3                       # 1552 = 3 x 512 + 16: ragged tile
    data = np.stack([np.stack([synth.block_bytes(91, s, j, B) for j in range(k)])
                     for s in range(n)])
    d = torch.from_numpy(data).cuda()
    P = oracle.cauchy(k, m)
    outs = {}
    # (window, temporals per window): automatic, plain two-level, row form
    for window, temps in ((0, 0), (0, -1), (-1, 0)):
        plan = xo.ec_plan_create_ex(k, m, executor=xo.EC_EXEC_COMPILED, stream_window=window,
                                    stream_temps=temps)
        try:
            info = xo.ec_plan_info(plan)
            assert info["window"] == (32 if window == 0 else 0)
            par = torch.full((n, m, B), 0xA5, dtype=torch.uint8, device="cuda")
            xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                                 stream())
            torch.cuda.synchronize()
            assert xo.ec_plan_info(plan)["compiled"]
            outs[(window, temps)] = par.cpu().numpy()
        finally:
            xo.ec_plan_destroy(plan)
    for s in range(n):
        ref = oracle.encode(P, list(data[s]))
        for key, got in outs.items():
            for i in range(m):
                assert np.array_equal(got[s, i], ref[i]), (key, s, i)
    assert xo.ec_device_status() == 0


@pytest.mark.parametrize("executor", [xo.EC_EXEC_INTERP, xo.EC_EXEC_COMPILED, xo.EC_EXEC_DENSE],
                         ids=["interp", "compiled", "dense"])
def test_two_level_decode_patterns(executor):
    torch.cuda.set_device(0)
    k, m, B = 16, 4, 8 * 1040
    data = [synth.block_bytes(92, 0, j, B) for j in range(k)]
    blocks = data + oracle.encode(oracle.cauchy(k, m), data)
    d = [torch.from_numpy(x).cuda() for x in blocks]
    plan = xo.ec_plan_create_ex(k, m, executor=executor)
    try:
        rng = np.random.default_rng(92)
        pats = [[0], [19], [3, 17], [0, 1, 2, 3], [5, 16, 18, 19], [15, 2, 9]]
        pats += [sorted(int(x) for x in rng.choice(k + m, size=4, replace=False))
                 for _ in range(4)]
        for er in pats:
            assert xo.ec_plan_info(plan, er)["window"] == 32
            outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
            xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         [t.data_ptr() for t in outs], B, stream())
            torch.cuda.synchronize()
            for t, e in zip(outs, er):
                assert np.array_equal(t.cpu().numpy(), blocks[e]), (er, e)
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)


def test_two_level_batch_mixed_with_narrow_codes():
    torch.cuda.set_device(0)
    codes = [(16, 4), (20, 4), (10, 4)]
    plans = {c: xo.ec_plan_create(*c) for c in codes}
    try:
        rng = np.random.default_rng(93)
        jobs, outs, expect, keep = [], [], [], []
        for s in range(24):
            k, m = codes[s % len(codes)]
            B = int(rng.choice([128, 4096, 8 * 1552]))
            data = [synth.block_bytes(93, s, j, B) for j in range(k)]
            blocks = data + oracle.encode(oracle.cauchy(k, m), data)
            dd = [torch.from_numpy(x).cuda() for x in blocks]
            keep += dd
            if s % 2:
                o = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
                             "blocks": [t.data_ptr() for t in dd[:k]],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append(blocks[k:])
            else:
                er = sorted(int(x) for x in rng.choice(k + m, size=int(rng.integers(1, m + 1)),
                                                       replace=False))
                o = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                             "blocks": [None if i in er else dd[i].data_ptr()
                                        for i in range(k + m)],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append([blocks[e] for e in er])
            outs.append(o)
        b = xo.ec_batch_create(jobs)
        try:
            xo.ec_batch_run(b, stream())
            torch.cuda.synchronize()
        finally:
            xo.ec_batch_destroy(b)
        for o, ref in zip(outs, expect):
            for t, r in zip(o, ref):
                assert np.array_equal(t.cpu().numpy(), r)
        assert xo.ec_device_status() == 0
    finally:
        for h in plans.values():
            xo.ec_plan_destroy(h)
