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


def test_set_launch_shape_runs_plain_batched_and_served():
    """A plan pinned to 256 threads per CTA (1 KiB strip tiles) and a
    register budget of 112 next to a default plan: plain calls, one batch
    and the serving loop all stay bit-exact."""
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    tuned = xo.ec_plan_create(6, 3)
    plain = xo.ec_plan_create(4, 2)
    xo.ec_plan_set_launch(tuned, 256, 112)
    keep, jobs, expect = [], [], []
    try:
        assert xo.ec_plan_info(tuned)["threads"] == 256
        assert xo.ec_plan_info(tuned, [0, 5])["threads"] == 256
        assert xo.ec_plan_info(plain)["threads"] == 128
        rng = np.random.default_rng(5)
        for s in range(24):
            plan, (k, m) = (tuned, (6, 3)) if s % 3 else (plain, (4, 2))
            B = int(rng.choice([128, 1024, 8 * 1040, 8 * 4112]))
            data = [synth.block_bytes(72, s, j, B) for j in range(k)]
            blocks = data + oracle.encode(oracle.cauchy(k, m), data)
            d = [torch.from_numpy(x).cuda() for x in blocks]
            keep += d
            if s % 2:
                o = [torch.full((B,), 0x5A, dtype=torch.uint8, device="cuda") for _ in range(m)]
                jobs.append({"plan": plan, "op": xo.EC_OP_ENCODE,
                             "blocks": [t.data_ptr() for t in d[:k]],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, blocks[k:]))
            else:
                er = sorted(int(x) for x in rng.choice(k + m, size=int(rng.integers(1, m + 1)),
                                                       replace=False))
                o = [torch.full((B,), 0x5A, dtype=torch.uint8, device="cuda") for _ in er]
                jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er,
                             "blocks": [None if i in er else d[i].data_ptr()
                                        for i in range(k + m)],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, [blocks[e] for e in er]))
            keep += o

        def check_and_reset():
            torch.cuda.synchronize()
            for o, ref in expect:
                for t, r in zip(o, ref):
                    assert np.array_equal(t.cpu().numpy(), r)
                    t.fill_(0x5A)
            torch.cuda.synchronize()

        # plain single-stripe calls
        for j, (o, _) in zip(jobs, expect):
            if j["op"] == xo.EC_OP_ENCODE:
                xo.ec_encode(j["plan"], j["blocks"], j["out"], j["block_bytes"], st)
            else:
                xo.ec_decode(j["plan"], j["erasures"], j["blocks"], j["out"], j["block_bytes"], st)
        check_and_reset()
        # one batch: the tuned plan's modules run 256-thread CTAs
        b = xo.ec_batch_create(jobs, xo.EC_EXEC_COMPILED)
        try:
            xo.ec_batch_run(b, st)
            check_and_reset()
        finally:
            xo.ec_batch_destroy(b)
        # the serving loop
        server = xo.ec_server_create()
        try:
            arr, hold = xo.make_jobs(jobs)
            tickets = set(xo.ec_server_submit_raw(server, arr[i]) for i in range(len(jobs)))
            import time
            t0 = time.time()
            while tickets:
                for t, _ in xo.ec_server_poll(server):
                    tickets.discard(t)
                assert time.time() - t0 < 60
                time.sleep(0.001)
            check_and_reset()
        finally:
            xo.ec_server_destroy(server)
    finally:
        xo.ec_plan_destroy(tuned)
        xo.ec_plan_destroy(plain)


def test_autotune_wide_code_keeps_parity():
    """RS(32,4): the candidates include the 64-thread tiles that keep two CTAs
    per SM; whichever shape wins, encode and decode stay bit-exact."""
    torch.cuda.set_device(0)
    k, m = 32, 4
    plan = xo.ec_plan_create(k, m)
    try:
        st = torch.cuda.current_stream().cuda_stream
        r = xo.ec_plan_autotune(plan, 64 << 10, 8, st)
        assert r["candidates"] >= 7 and r["threads"] in (64, 128, 256)
        assert xo.ec_plan_info(plan)["threads"] == r["threads"]
        B = 8 * 1552
        data = [synth.block_bytes(73, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(oracle.cauchy(k, m), data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        par = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(plan, [t.data_ptr() for t in d[:k]], [t.data_ptr() for t in par], B, st)
        er = [0, 13, 31, 34]
        outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
        xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                     [t.data_ptr() for t in outs], B, st)
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), blocks[k + i])
        for t, e in zip(outs, er):
            assert np.array_equal(t.cpu().numpy(), blocks[e])
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)
