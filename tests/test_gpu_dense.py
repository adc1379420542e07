"""The dense bitmatrix executor (EC_EXEC_DENSE, and EC_EXEC_AUTO's tier for
programs without a compiled kernel) against the oracle, bit for bit: output
strip r is the XOR of the input strips whose bit (r, c) of the bitmatrix is
set (Sec. 1, property (ii)).  Covers both forms (column masks, and subset
tables of four strips), both widths of a consumer's column (two and four
words), more than 32 output strips (groups of rows), inputs
streamed by tensor copies and by per-strip copies, single launches, batches
of mixed codes, the serving loop before any module exists, and a code of
1024 input strips."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu

DENSE = xo.EC_EXEC_DENSE


@pytest.fixture(autouse=True)
def _device():
    torch.cuda.set_device(0)
    yield
    assert xo.ec_device_status() == 0


def stream():
    return torch.cuda.current_stream().cuda_stream


def _codeword(k, m, B, cfg, stripe=0):
    data = [synth.block_bytes(cfg, stripe, j, B) for j in range(k)]
    return data + oracle.encode(oracle.cauchy(k, m), data)


@pytest.mark.parametrize("kind", ["mask", "table"])
@pytest.mark.parametrize("words", ["2", "4"])
@pytest.mark.parametrize("tensor", ["1", "0"], ids=["tensor-copies", "strip-copies"])
@pytest.mark.parametrize("k,m", [(10, 4), (3, 5), (24, 8)])
def test_strided_encode(k, m, words, tensor, kind, monkeypatch):
    """ec_encode_strided: windows of one block by one tiled tensor copy (8- or
    4-byte elements) or by eight 1-D copies; strips of 2064 B end in a ragged
    tile; RS(3,5) and RS(24,8) have 40 and 64 output strips (two groups)."""
    monkeypatch.setenv("EC_DENSE_WORDS", words)
    monkeypatch.setenv("EC_DENSE_KIND", kind)
    monkeypatch.setenv("EC_TMA_TENSOR", tensor)
    B, n = 8 * 2064, 3
    data = np.stack([np.stack([synth.block_bytes(111, s, j, B) for j in range(k)])
                     for s in range(n)])
    d = torch.from_numpy(data).cuda()
    plan = xo.ec_plan_create_ex(k, m, executor=DENSE)
    try:
        par = torch.full((n, m, B), 0x5A, dtype=torch.uint8, device="cuda")
        xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                             stream())
        torch.cuda.synchronize()
        got = par.cpu().numpy()
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, list(data[s]))
            for i in range(m):
                assert np.array_equal(got[s, i], ref[i]), (s, i)
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("kind", ["mask", "table"])
@pytest.mark.parametrize("words", ["2", "4"])
def test_decode_more_than_32_rows(words, kind, monkeypatch):
    """RS(12,8): every set of 5 to 8 erasures among a spread sample (40 to 64
    output strips, two groups of rows), block pointer tables."""
    monkeypatch.setenv("EC_DENSE_WORDS", words)
    monkeypatch.setenv("EC_DENSE_KIND", kind)
    k, m, B = 12, 8, 8 * 1040
    blocks = _codeword(k, m, B, 112)
    d = [torch.from_numpy(b).cuda() for b in blocks]
    rng = np.random.default_rng(5)
    pats = [tuple(sorted(int(x) for x in rng.choice(k + m, size=ne, replace=False)))
            for ne in (5, 6, 7, 8) for _ in range(6)]
    plan = xo.ec_plan_create_ex(k, m, executor=DENSE)
    try:
        for er in pats:
            outs = [torch.full((B,), 0x21, dtype=torch.uint8, device="cuda") for _ in er]
            xo.ec_decode(plan, list(er), [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         [o.data_ptr() for o in outs], B, stream())
            torch.cuda.synchronize()
            for o, e in zip(outs, er):
                assert np.array_equal(o.cpu().numpy(), blocks[e]), (er, e)
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("kind", ["mask", "table"])
def test_every_rs6_3_pattern_four_words(kind, monkeypatch):
    """All 129 erasure sets of RS(6,3) with four words per column (2 KiB
    tiles): strips of 4224 B give two full tiles and a ragged one."""
    monkeypatch.setenv("EC_DENSE_WORDS", "4")
    monkeypatch.setenv("EC_DENSE_KIND", kind)
    k, m, B = 6, 3, 8 * 4224
    blocks = _codeword(k, m, B, 113)
    d = [torch.from_numpy(b).cuda() for b in blocks]
    plan = xo.ec_plan_create_ex(k, m, executor=DENSE)
    try:
        pats = [e for ne in range(1, 4) for e in itertools.combinations(range(k + m), ne)]
        assert len(pats) == 129
        outs = torch.empty((3, B), dtype=torch.uint8, device="cuda")
        for er in pats:
            xo.ec_decode(plan, list(er), [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         [outs[i].data_ptr() for i in range(len(er))], B, stream())
            got = outs.cpu().numpy()
            for i, e in enumerate(er):
                assert np.array_equal(got[i], blocks[e]), (er, e)
    finally:
        xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("kind", ["mask", "table"])
@pytest.mark.parametrize("words", ["2", "4"])
@pytest.mark.parametrize("tensor", ["1", "0"], ids=["tensor-copies", "strip-copies"])
def test_batch_of_mixed_codes(words, tensor, kind, monkeypatch):
    """One batch with EC_EXEC_DENSE: encodes and decodes of four codes (8 to
    64 output strips) and five block sizes in one launch, each item's windows
    and groups following its stripe; run twice (the queue resets)."""
    monkeypatch.setenv("EC_DENSE_WORDS", words)
    monkeypatch.setenv("EC_DENSE_KIND", kind)
    monkeypatch.setenv("EC_TMA_TENSOR", tensor)
    codes = [(4, 2), (10, 4), (3, 5), (12, 8)]
    plans = {c: xo.ec_plan_create(*c) for c in codes}
    try:
        rng = np.random.default_rng(114)
        jobs, keep, expect = [], [], []
        for s in range(24):
            k, m = codes[s % len(codes)]
            B = int(rng.choice([128, 1024, 8 * 528, 8 * 2064, 64 * 1024]))
            blocks = _codeword(k, m, B, 114, s)
            d = [torch.from_numpy(x).cuda() for x in blocks]
            keep += d
            if s % 3 == 0:
                o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in range(m)]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_ENCODE,
                             "blocks": [t.data_ptr() for t in d[:k]],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, blocks[k:]))
            else:
                ne = int(rng.integers(1, m + 1))
                er = [int(x) for x in rng.choice(k + m, size=ne, replace=False)]
                o = [torch.full((B,), 0xEE, dtype=torch.uint8, device="cuda") for _ in er]
                jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                             "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                             "out": [t.data_ptr() for t in o], "block_bytes": B})
                expect.append((o, [blocks[e] for e in er]))
            keep += o
        b = xo.ec_batch_create(jobs, DENSE)
        try:
            info = xo.ec_batch_info_get(b)
            assert info["compiled_programs"] == 0 and info["launches"] == 1
            for _ in range(2):
                for o, _ in expect:
                    for t in o:
                        t.fill_(0xEE)
                xo.ec_batch_run(b, stream())
                torch.cuda.synchronize()
                for o, ref in expect:
                    for t, r in zip(o, ref):
                        assert np.array_equal(t.cpu().numpy(), r)
            assert xo.ec_batch_status(b) == 0
        finally:
            xo.ec_batch_destroy(b)
    finally:
        for h in plans.values():
            xo.ec_plan_destroy(h)


def test_very_wide_code():
    """RS(128,4) (1024 input strips, 128 windows per item): encode and two
    decodes."""
    k, m, B = 128, 4, 8 * 1040
    blocks = _codeword(k, m, B, 115)
    d = [torch.from_numpy(x).cuda() for x in blocks]
    plan = xo.ec_plan_create_ex(k, m, executor=DENSE)
    try:
        par = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(plan, [t.data_ptr() for t in d[:k]], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), blocks[k + i])
        for er in ([0, 77, k + 1], [k - 1]):
            outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
            xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         [o.data_ptr() for o in outs], B, stream())
            torch.cuda.synchronize()
            for o, e in zip(outs, er):
                assert np.array_equal(o.cpu().numpy(), blocks[e])
    finally:
        xo.ec_plan_destroy(plan)


def test_served_before_any_module():
    """A server without background compiles and without warm-up: every
    request runs on the dense executor; all bit-exact and successful."""
    import time
    k, m, B = 10, 4, 8 * 2064
    plan = xo.ec_plan_create(k, m)
    sv = xo.ec_server_create(slots=2, max_batch=8, background_compile=False)
    try:
        blocks = _codeword(k, m, B, 116)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        reqs = []
        for er in (None, [2], [0, 11], [1, 3, 5, 13]):
            if er is None:
                o = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
                job = {"plan": plan, "op": xo.EC_OP_ENCODE, "blocks": [t.data_ptr() for t in d[:k]],
                       "out": [t.data_ptr() for t in o], "block_bytes": B}
                want = blocks[k:]
            else:
                o = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
                job = {"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er,
                       "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                       "out": [t.data_ptr() for t in o], "block_bytes": B}
                want = [blocks[e] for e in er]
            reqs.append((xo.ec_server_submit(sv, job), o, want))
        got, t0 = {}, time.time()
        while len(got) < len(reqs) and time.time() - t0 < 30:
            for tk, _, st in xo.ec_server_poll_ex(sv):
                got[tk] = st
            time.sleep(0.001)
        for tk, o, want in reqs:
            assert got.get(tk) == xo.EC_OK, tk
            for t, w in zip(o, want):
                assert np.array_equal(t.cpu().numpy(), w)
    finally:
        xo.ec_server_destroy(sv)
        xo.ec_plan_destroy(plan)
