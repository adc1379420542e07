"""Every decode program of a code, on the path the decode benchmark times:
one batch of compiled multi-program modules (ec_batch_create with the
compiled executor, then ec_batch_run), one stripe per erasure set.  Each
stripe's survivors come from a codeword the oracle encoded, so every byte
of every output block must equal the erased block it recovers (Sec. 1:
decoding returns the original data and parity).  Blocks of 8 x 528 bytes
give every strip one full 512-byte tile and a ragged 16-byte tail.

RS(10,4): all 1470 sets of 1-4 erasures, at the default launch shape (the
one the decode benchmark uses), with one queue and with the items split into
per-SM ranges, and at the autotuner's GB300 shape (128 threads, register
budget 160).  RS(6,3): all 129.  RS(12,4): all 2516."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu

B = 8 * 528
N_CODEWORDS = 4


@pytest.fixture(scope="module")
def rs10_4():
    """One RS(10,4) plan for both queue forms: its compiled modules are built
    by the first batch and reused by the second."""
    torch.cuda.set_device(0)
    plan = xo.ec_plan_create(10, 4)
    yield plan
    xo.ec_plan_destroy(plan)


def _sweep(k, m, shape=None, plan=None):
    torch.cuda.set_device(0)
    own = plan is None
    if own:
        plan = xo.ec_plan_create(k, m)
    try:
        if shape:
            xo.ec_plan_set_launch(plan, *shape)
        P = oracle.cauchy(k, m)
        words = []
        for w in range(N_CODEWORDS):
            data = [synth.block_bytes(71, 100 * k + w, j, B) for j in range(k)]
            words.append(data + oracle.encode(P, data))
        dwords = [torch.from_numpy(np.stack(cw)).cuda() for cw in words]
        pats = synth.all_erasure_patterns(k + m, m)
        n_out = sum(len(er) for er in pats)
        out = torch.full((n_out, B), 0xEE, dtype=torch.uint8, device="cuda")
        jobs, expect, row = [], [], 0
        rng = np.random.default_rng(k * 100 + m)
        for s, er in enumerate(pats):
            w = s % N_CODEWORDS
            order = [int(x) for x in rng.permutation(list(er))]   # caller order kept
            jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": order,
                         "blocks": [None if i in er else dwords[w][i].data_ptr()
                                    for i in range(k + m)],
                         "out": [out[row + i].data_ptr() for i in range(len(order))],
                         "block_bytes": B})
            expect += [(w, e) for e in order]
            row += len(order)
        b = xo.ec_batch_create(jobs, xo.EC_EXEC_COMPILED)
        try:
            info = xo.ec_batch_info_get(b)
            assert info["programs"] == len(pats)
            assert info["compiled_programs"] == len(pats)
            xo.ec_batch_run(b, torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            assert xo.ec_batch_status(b) == 0
        finally:
            xo.ec_batch_destroy(b)
        got = out.cpu().numpy()
        bad = [r for r, (w, e) in enumerate(expect) if not np.array_equal(got[r], words[w][e])]
        assert not bad, [expect[r] for r in bad[:5]]
        return len(pats)
    finally:
        if own:
            xo.ec_plan_destroy(plan)


@pytest.mark.parametrize("ranges", [1, 152], ids=["one-queue", "per-sm-ranges"])
def test_rs10_4_every_compiled_decode_program(rs10_4, ranges, monkeypatch):
    monkeypatch.setenv("EC_BATCH_RANGES", str(ranges))
    assert _sweep(10, 4, plan=rs10_4) == 1470


def test_rs10_4_every_compiled_decode_program_tuned_shape():
    assert _sweep(10, 4, shape=(128, 160)) == 1470


def test_rs6_3_every_compiled_decode_program():
    assert _sweep(6, 3) == 129


def test_rs12_4_every_compiled_decode_program():
    assert _sweep(12, 4) == 2516
