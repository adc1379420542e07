"""Serving loop: continuous batching of encode/decode requests.  Results
are checked against the oracle, and every request's bytes are the same
when it runs alone and when it runs in the mix (tolerance: zero bytes)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu

CODES = [(10, 4), (6, 3)]


@pytest.fixture(scope="module")
def plans():
    torch.cuda.set_device(0)
    ps = {c: xo.ec_plan_create(*c) for c in CODES}
    yield ps
    for h in ps.values():
        xo.ec_plan_destroy(h)


def requests(plans, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n):
        k, m = CODES[int(rng.integers(0, 2))]
        B = int(rng.choice([128, 4096, 8 * 1552, 64 * 1024]))
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(51, seed * 1000 + s, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        if rng.uniform() < 0.5:
            o = [torch.full((B,), 0xAB, dtype=torch.uint8, device="cuda") for _ in range(m)]
            job = {"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
                   "blocks": [t.data_ptr() for t in d[:k]], "out": [t.data_ptr() for t in o],
                   "block_bytes": B}
            expect = blocks[k:]
        else:
            ne = int(rng.integers(1, m + 1))
            er = [int(x) for x in rng.choice(k + m, size=ne, replace=False)]
            o = [torch.full((B,), 0xAB, dtype=torch.uint8, device="cuda") for _ in er]
            job = {"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                   "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                   "out": [t.data_ptr() for t in o], "block_bytes": B}
            expect = [blocks[e] for e in er]
        out.append({"job": job, "keep": d, "out": o, "expect": expect})
    return out


def wait_all(server, tickets, timeout=60.0):
    left = set(tickets)
    t0 = time.time()
    while left:
        for t, _ in xo.ec_server_poll(server):
            left.discard(t)
        assert time.time() - t0 < timeout, "requests did not complete"
        time.sleep(0.001)


def test_served_mix_matches_oracle_and_alone(plans):
    server = xo.ec_server_create()
    try:
        reqs = requests(plans, 60, seed=3)
        arr, keep = xo.make_jobs([r["job"] for r in reqs])
        tickets = [xo.ec_server_submit_raw(server, arr[i]) for i in range(len(reqs))]
        assert all(tickets)
        wait_all(server, tickets)
        mixed = []
        for r in reqs:
            got = [t.cpu().numpy().copy() for t in r["out"]]
            for g, e in zip(got, r["expect"]):
                assert np.array_equal(g, e)
            mixed.append(got)
        st = xo.ec_server_stats_get(server)
        assert st["completed"] == 60 and st["failed"] == 0
        # alone: one request at a time
        for i, r in enumerate(reqs):
            for t in r["out"]:
                t.fill_(0x5C)
            tk = xo.ec_server_submit_raw(server, arr[i])
            wait_all(server, [tk])
            for t, g in zip(r["out"], mixed[i]):
                assert np.array_equal(t.cpu().numpy(), g)
    finally:
        xo.ec_server_destroy(server)


def test_admission_budget(plans):
    B = 64 * 1024
    server = xo.ec_server_create(hbm_budget=14 * B + 1)     # room for one RS(10,4) stripe
    try:
        reqs = requests(plans, 1, seed=5)
        k, m = 10, 4
        data = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(k + m)]
        job = {"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
               "blocks": [t.data_ptr() for t in data[:k]],
               "out": [t.data_ptr() for t in data[k:]], "block_bytes": B}
        arr, keep = xo.make_jobs([job, job])
        t1 = xo.ec_server_submit_raw(server, arr[0])
        assert t1
        t2 = xo.ec_server_submit_raw(server, arr[1])
        if t2 == 0:                      # over budget until the first finishes
            wait_all(server, [t1])
            t2 = xo.ec_server_submit_raw(server, arr[1])
            assert t2
            wait_all(server, [t2])
        else:
            wait_all(server, [t1, t2])
        assert xo.ec_server_stats_get(server)["admitted_bytes"] == 0
    finally:
        xo.ec_server_destroy(server)


def test_warm_compiles_every_pattern(plans):
    server = xo.ec_server_create()
    try:
        xo.ec_server_warm(server, plans[(6, 3)], 3)
        reqs = [r for r in requests(plans, 20, seed=8)]
        arr, keep = xo.make_jobs([r["job"] for r in reqs])
        tickets = [xo.ec_server_submit_raw(server, arr[i]) for i in range(len(reqs))]
        wait_all(server, tickets)
        for r in reqs:
            for t, e in zip(r["out"], r["expect"]):
                assert np.array_equal(t.cpu().numpy(), e)
    finally:
        xo.ec_server_destroy(server)


@pytest.mark.parametrize("background", [True, False], ids=["background", "interp-only"])
def test_new_patterns_run_then_get_compiled(background):
    """Requests whose decode programs were never compiled run on the
    interpreter at once; with background compilation the programs then get
    compiled kernels and later requests use them.  Bit-exact throughout."""
    import itertools
    k, m, B = 6, 3, 8 * 1552
    plan = xo.ec_plan_create(k, m)      # fresh: no compiled module yet
    server = xo.ec_server_create(background_compile=background)
    try:
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(53, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        pats = [list(e) for e in itertools.combinations(range(k + m), 2)][:12]
        outs = [[torch.full((B,), 0xAB, dtype=torch.uint8, device="cuda") for _ in er]
                for er in pats]
        jobs = [{"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er,
                 "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                 "out": [t.data_ptr() for t in o], "block_bytes": B}
                for er, o in zip(pats, outs)]
        arr, keep = xo.make_jobs(jobs)

        def run_and_check():
            tickets = [xo.ec_server_submit_raw(server, arr[i]) for i in range(len(jobs))]
            wait_all(server, tickets)
            for er, o in zip(pats, outs):
                for t, e in zip(o, er):
                    assert np.array_equal(t.cpu().numpy(), blocks[e])
                    t.fill_(0xAB)
            torch.cuda.synchronize()

        run_and_check()
        t0 = time.time()
        while background and xo.ec_server_stats_get(server)["compiled_in_background"] < len(pats):
            assert time.time() - t0 < 120, "background compilation did not finish"
            time.sleep(0.05)
        run_and_check()
        n = xo.ec_server_stats_get(server)["compiled_in_background"]
        assert n == (len(pats) if background else 0)
    finally:
        xo.ec_server_destroy(server)
        xo.ec_plan_destroy(plan)


def test_cancel_queued_requests(plans):
    """One slot and one request per batch, so requests queue behind each
    other; cancelling from the back of the queue drops requests that were
    still waiting (their outputs stay untouched and their tickets never
    complete) while everything else completes bit-exact."""
    server = xo.ec_server_create(max_batch=1, slots=1)
    try:
        reqs = requests(plans, 40, seed=11)
        arr, keep = xo.make_jobs([r["job"] for r in reqs])
        tickets = [xo.ec_server_submit_raw(server, arr[i]) for i in range(len(reqs))]
        assert all(tickets)
        cancelled = {t for t in reversed(tickets[-10:]) if xo.ec_server_cancel(server, t)}
        assert cancelled, "no request was still queued"
        with pytest.raises(xo.XorecError) as e:
            xo.ec_server_cancel(server, max(tickets) + 100)
        assert e.value.status == xo.EC_EINVAL
        left = [t for t in tickets if t not in cancelled]
        wait_all(server, left)
        time.sleep(0.05)
        assert not [t for t, _ in xo.ec_server_poll(server) if t in cancelled]
        for t, r in zip(tickets, reqs):
            for o, ex in zip(r["out"], r["expect"]):
                got = o.cpu().numpy()
                if t in cancelled:
                    assert (got == 0xAB).all()
                else:
                    assert np.array_equal(got, ex)
        st = xo.ec_server_stats_get(server)
        assert st["cancelled"] == len(cancelled) and st["admitted_bytes"] == 0
        assert not xo.ec_server_cancel(server, left[0])      # already done
    finally:
        xo.ec_server_destroy(server)
