"""Batched launches (mixed codes, block sizes, encode and decode jobs)
against the oracle, alone-versus-in-the-mix identity, and CUDA-graph
capture of ec_batch_run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu

CODES = [(4, 2), (6, 3), (10, 4), (12, 4)]


@pytest.fixture(scope="module")
def plans():
    torch.cuda.set_device(0)
    ps = {c: xo.ec_plan_create(*c) for c in CODES}
    yield ps
    for h in ps.values():
        xo.ec_plan_destroy(h)


def make_jobs(plans, n, seed, sizes=(128, 1024, 4096, 8 * 1552, 64 * 1024)):
    """Random mix; returns jobs, device buffers to keep, and expected bytes."""
    rng = np.random.default_rng(seed)
    jobs, keep, expect = [], [], []
    for s in range(n):
        k, m = CODES[int(rng.integers(0, len(CODES)))]
        B = int(sizes[int(rng.integers(0, len(sizes)))])
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(31, seed * 1000 + s, j, B) for j in range(k)]
        par = oracle.encode(P, data)
        if rng.uniform() < 0.5:
            d = [torch.from_numpy(x).cuda() for x in data]
            o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in range(m)]
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
                         "blocks": [t.data_ptr() for t in d], "out": [t.data_ptr() for t in o],
                         "block_bytes": B})
            keep += d + o
            expect.append((o, par))
        else:
            ne = int(rng.integers(1, m + 1))
            er = [int(x) for x in rng.choice(k + m, size=ne, replace=False)]
            blocks = data + par
            d = [torch.from_numpy(x).cuda() for x in blocks]
            o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in er]
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                         "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         "out": [t.data_ptr() for t in o], "block_bytes": B})
            keep += d + o
            expect.append((o, [blocks[e] for e in er]))
    return jobs, keep, expect


def check(expect):
    for o, ref in expect:
        for t, r in zip(o, ref):
            assert np.array_equal(t.cpu().numpy(), r)


@pytest.mark.parametrize("executor", [xo.EC_EXEC_INTERP, xo.EC_EXEC_COMPILED, xo.EC_EXEC_DENSE],
                         ids=["interp", "compiled", "dense"])
def test_mixed_batch_matches_oracle(plans, executor):
    jobs, keep, expect = make_jobs(plans, 40, seed=1 + executor)
    b = xo.ec_batch_create(jobs, executor)
    try:
        info = xo.ec_batch_info_get(b)
        assert info["stripes"] == 40
        if executor == xo.EC_EXEC_COMPILED:
            assert info["compiled_programs"] == info["programs"]
        xo.ec_batch_run(b, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        check(expect)
    finally:
        xo.ec_batch_destroy(b)


@pytest.mark.parametrize("ranges", [2, 7, 152, 4096])
@pytest.mark.parametrize("executor", [xo.EC_EXEC_INTERP, xo.EC_EXEC_COMPILED, xo.EC_EXEC_DENSE],
                         ids=["interp", "compiled", "dense"])
def test_batch_item_ranges_match_oracle(plans, executor, ranges, monkeypatch):
    """Items split into per-SM ranges (forced here; a batch only chooses them
    when it has enough items): CTAs start on their SM's range and move to the
    others, so every item of a mixed batch is still computed exactly once,
    whatever the number of ranges (more ranges than SMs are capped)."""
    monkeypatch.setenv("EC_BATCH_RANGES", str(ranges))
    jobs, keep, expect = make_jobs(plans, 40, seed=50 + ranges + executor,
                                   sizes=(128, 4096, 8 * 1552, 64 * 1024, 8 * 32784))
    b = xo.ec_batch_create(jobs, executor)
    try:
        st = torch.cuda.current_stream().cuda_stream
        for _ in range(2):   # the queue heads are reset at every run
            for o, _ in expect:
                for t in o:
                    t.fill_(0xEE)
            xo.ec_batch_run(b, st)
            torch.cuda.synchronize()
            check(expect)
    finally:
        xo.ec_batch_destroy(b)
    assert xo.ec_device_status() == 0


def test_alone_and_in_mix_give_identical_bytes(plans):
    jobs, keep, expect = make_jobs(plans, 30, seed=7)
    st = torch.cuda.current_stream().cuda_stream
    xo.ec_run_batch(jobs, st)
    mixed = [[t.cpu().numpy().copy() for t in o] for o, _ in expect]
    for o, _ in expect:
        for t in o:
            t.fill_(0x11)
    for j in jobs:
        xo.ec_run_batch([j], st)
    alone = [[t.cpu().numpy().copy() for t in o] for o, _ in expect]
    for a, b in zip(mixed, alone):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    check(expect)


def test_batch_run_in_cuda_graph(plans):
    jobs, keep, expect = make_jobs(plans, 12, seed=9, sizes=(4096, 8 * 1040))
    b = xo.ec_batch_create(jobs)
    try:
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            xo.ec_batch_run(b, s.cuda_stream)
        for o, _ in expect:
            for t in o:
                t.fill_(0x22)
        torch.cuda.synchronize()
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        check(expect)
    finally:
        xo.ec_batch_destroy(b)


def test_batch_argument_errors(plans):
    with pytest.raises(xo.XorecError):
        xo.ec_batch_create([{"plan": plans[(4, 2)], "op": 7, "blocks": [0] * 4,
                             "out": [0] * 2, "block_bytes": 1024}])
    buf = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    with pytest.raises(xo.XorecError) as e:
        xo.ec_batch_create([{"plan": plans[(4, 2)], "op": xo.EC_OP_DECODE, "erasures": [0, 1, 2],
                             "blocks": [p] * 6, "out": [p] * 3, "block_bytes": 1024}])
    assert e.value.status == xo.EC_ETOOMANY


def test_batch_with_wide_codes():
    torch.cuda.set_device(0)
    codes = [(40, 8), (10, 4), (20, 4)]
    plans = {c: xo.ec_plan_create(*c) for c in codes}
    try:
        rng = np.random.default_rng(12)
        jobs, keep, expect = [], [], []
        for s in range(9):
            k, m = codes[s % 3]
            B = int(rng.choice([1024, 4096, 8 * 1040]))
            P = oracle.cauchy(k, m)
            data = [synth.block_bytes(33, s, j, B) for j in range(k)]
            blocks = data + oracle.encode(P, data)
            d = [torch.from_numpy(x).cuda() for x in blocks]
            keep += d
            if s % 2 == 0:
                o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in range(m)]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
                             "blocks": [t.data_ptr() for t in d[:k]],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, blocks[k:]))
            else:
                er = [0, k + 1]
                o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in er]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                             "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, [blocks[e] for e in er]))
            keep += o
        xo.ec_run_batch(jobs, torch.cuda.current_stream().cuda_stream)
        check(expect)
    finally:
        for h in plans.values():
            xo.ec_plan_destroy(h)
