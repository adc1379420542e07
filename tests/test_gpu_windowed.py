"""The windowed pipeline of two-level programs (multilevel pebble game,
Sec. 8, with inputs streamed window by window through a ring of shared
memory): a producer warp copies one window of 32 input strips per phase,
the program consumes the windows in phase order.  Checked against the
oracle with the pipeline forced on (EC_WINDOWED=1) for codes it would not
take by default, and at its default for the widest ones: tensor copies with
a partial last window (RS(13,4): 104 strips), two groups of rows (RS(24,8)),
per-strip copies from block pointer tables, ragged strip tails, decoders,
the widest code of the benchmark (RS(100,4)), batched decodes as windowed
modules, and the serving loop running those modules."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


def _windowed_source(plan, erasures=None):
    return "xk::run_window_pipeline(p, smem, SlpBody()" in xo.ec_plan_kernel_source(plan, erasures)


@pytest.mark.parametrize("k,m,force", [(13, 4, True), (16, 4, True), (24, 8, True),
                                       (48, 4, False), (100, 4, False)])
def test_windowed_strided_encode(k, m, force, monkeypatch):
    """ec_encode_strided: one tiled tensor copy per window (a box of 32
    strips; past the last strip the box is zero-filled); strips of 1552 B
    end in a ragged 16-byte tile."""
    if force:
        monkeypatch.setenv("EC_WINDOWED", "1")
    torch.cuda.set_device(0)
    B, n = 8 * 1552, 3
    data = np.stack([np.stack([synth.block_bytes(97, s, j, B) for j in range(k)])
                     for s in range(n)])
    d = torch.from_numpy(data).cuda()
    plan = xo.ec_plan_create_ex(k, m, executor=xo.EC_EXEC_COMPILED)
    try:
        assert _windowed_source(plan)
        par = torch.full((n, m, B), 0x5A, dtype=torch.uint8, device="cuda")
        xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B, stream())
        torch.cuda.synchronize()
        got = par.cpu().numpy()
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, list(data[s]))
            for i in range(m):
                assert np.array_equal(got[s, i], ref[i]), (s, i)
    finally:
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0


@pytest.mark.parametrize("k,m", [(13, 4), (24, 8), (48, 4)])
def test_windowed_table_encode_and_decode(k, m, monkeypatch):
    """ec_encode and ec_decode (block pointer tables: one 1-D bulk copy per
    strip of the window) through the windowed pipeline."""
    monkeypatch.setenv("EC_WINDOWED", "1")
    torch.cuda.set_device(0)
    B = 8 * 2064                                    # 4 tiles of 512 B and a 16-byte tail
    plan = xo.ec_plan_create_ex(k, m, executor=xo.EC_EXEC_COMPILED)
    try:
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(98, k, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        par = [torch.full((B,), 0x3C, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(plan, [t.data_ptr() for t in d[:k]], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(par[i].cpu().numpy(), blocks[k + i]), i
        for er in ([0, 5, k + 1], [1, 2, 3, k + m - 1], [k - 1]):
            assert _windowed_source(plan, er)
            out = [torch.full((B,), 0x3C, dtype=torch.uint8, device="cuda") for _ in er]
            xo.ec_decode(plan, er, [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         [t.data_ptr() for t in out], B, stream())
            torch.cuda.synchronize()
            for t, e in zip(out, er):
                assert np.array_equal(t.cpu().numpy(), blocks[e]), (er, e)
    finally:
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0


def test_windowed_and_full_stage_kernels_agree():
    """RS(32,4) (256 strips: the full-stage kernel by default) encoded by both
    forms on arbitrary bytes gives identical parity."""
    torch.cuda.set_device(0)
    k, m, B, n = 32, 4, 8 * 4096, 4
    d = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
    for s in range(n):
        for j in range(k):
            xo.ec_synth_fill(d[s, j].data_ptr(), B, synth.block_seed(99, s, j), 0, stream())
    outs = []
    for force in ("0", "1"):
        import os
        os.environ["EC_WINDOWED"] = force
        try:
            plan = xo.ec_plan_create_ex(k, m, executor=xo.EC_EXEC_COMPILED)
            try:
                assert _windowed_source(plan) == (force == "1")
                par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
                xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                                     stream())
                torch.cuda.synchronize()
                outs.append(par.cpu().numpy())
            finally:
                xo.ec_plan_destroy(plan)
        finally:
            del os.environ["EC_WINDOWED"]
    assert np.array_equal(outs[0], outs[1])
    assert xo.ec_device_status() == 0


def test_batch_of_a_very_wide_code():
    """RS(128,4) decodes in a batch: 1024 input strips do not fit a stage of
    512-byte tiles in one CTA, so the batch's interpreter launch takes
    smaller tiles; bit-exact against the codeword."""
    torch.cuda.set_device(0)
    k, m, B = 128, 4, 8 * 1040
    plan = xo.ec_plan_create(k, m)
    try:
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(100, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        jobs, outs, want = [], [], []
        for er in ([0, 1, 2, 3], [5, k + 2], [k + 3]):
            o = [torch.full((B,), 0x77, dtype=torch.uint8, device="cuda") for _ in er]
            jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er,
                         "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         "out": [t.data_ptr() for t in o], "block_bytes": B})
            outs += o
            want += [blocks[e] for e in er]
        xo.ec_run_batch(jobs, stream())
        for t, w in zip(outs, want):
            assert np.array_equal(t.cpu().numpy(), w)
    finally:
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0


@pytest.mark.parametrize("tensor_copies", ["1", "0"], ids=["tensor-copies", "strip-copies"])
def test_windowed_batch_decodes(tensor_copies, monkeypatch):
    """Batches of wide decoders run as windowed modules (a producer warp pops
    items and streams their windows; the first slot of an item carries its
    index; a last slot ends the launch), beside a narrow code in the same
    batch; one 2-D tensor copy per input block of a window, or one 1-D copy
    per strip.  Bit-exact against the codewords, including a ragged tile."""
    monkeypatch.setenv("EC_WINDOWED", "1")
    monkeypatch.setenv("EC_TMA_TENSOR", tensor_copies)
    torch.cuda.set_device(0)
    codes = [(13, 4), (48, 4), (10, 4)]
    plans = {c: xo.ec_plan_create(*c) for c in codes}
    try:
        rng = np.random.default_rng(101)
        jobs, outs, want, keep = [], [], [], []
        for s in range(12):
            k, m = codes[s % 3]
            B = int(rng.choice([8 * 528, 8 * 2064, 4096]))
            P = oracle.cauchy(k, m)
            data = [synth.block_bytes(102, s, j, B) for j in range(k)]
            blocks = data + oracle.encode(P, data)
            d = [torch.from_numpy(x).cuda() for x in blocks]
            keep += d
            ne = int(rng.integers(1, m + 1))
            er = [int(x) for x in rng.choice(k + m, size=ne, replace=False)]
            o = [torch.full((B,), 0x66, dtype=torch.uint8, device="cuda") for _ in er]
            jobs.append({"plan": plans[(k, m)], "op": xo.EC_OP_DECODE, "erasures": er,
                         "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                         "out": [t.data_ptr() for t in o], "block_bytes": B})
            outs += o
            want += [blocks[e] for e in er]
        b = xo.ec_batch_create(jobs, xo.EC_EXEC_COMPILED)
        try:
            src = xo.ec_plan_module_source(plans[(48, 4)], [[0, 1]])
            assert "xk::run_batch_window_pipeline(p, smem, ModBody())" in src
            for _ in range(2):
                for t in outs:
                    t.fill_(0x66)
                xo.ec_batch_run(b, stream())
                torch.cuda.synchronize()
                for t, w in zip(outs, want):
                    assert np.array_equal(t.cpu().numpy(), w)
            assert xo.ec_batch_status(b) == 0
        finally:
            xo.ec_batch_destroy(b)
    finally:
        for h in plans.values():
            xo.ec_plan_destroy(h)
    assert xo.ec_device_status() == 0


def test_server_runs_windowed_modules():
    """Requests of a wide code through the serving loop: after ec_server_warm
    its programs run as windowed modules (the server's batches use the same
    batched windowed pipeline); every request bit-exact and successful."""
    import time
    torch.cuda.set_device(0)
    k, m, B = 48, 4, 8 * 2064
    plan = xo.ec_plan_create(k, m)
    sv = xo.ec_server_create(slots=2, max_batch=8, background_compile=False)
    try:
        xo.ec_server_warm(sv, plan, 2)
        assert "xk::run_batch_window_pipeline(p, smem, ModBody())" in \
            xo.ec_plan_module_source(plan, [[3, 50]])
        P = oracle.cauchy(k, m)
        data = [synth.block_bytes(103, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        reqs = []
        for er in (None, [3, 50], [0], [k, k + 1]):
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
    assert xo.ec_device_status() == 0


def _wide_decode_batch(k, sets, B, n_stripes, seed):
    m = 4
    plan = xo.ec_plan_create(k, m)
    P = oracle.cauchy(k, m)
    jobs, outs, want, keep = [], [], [], []
    for s in range(n_stripes):
        data = [synth.block_bytes(seed, s, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [torch.from_numpy(x).cuda() for x in blocks]
        keep += d
        er = sets[s % len(sets)]
        o = [torch.full((B,), 0x4B, dtype=torch.uint8, device="cuda") for _ in er]
        jobs.append({"plan": plan, "op": xo.EC_OP_DECODE, "erasures": er,
                     "blocks": [None if i in er else d[i].data_ptr() for i in range(k + m)],
                     "out": [t.data_ptr() for t in o], "block_bytes": B})
        outs += o
        want += [blocks[e] for e in er]
    return plan, jobs, outs, want, keep


@pytest.mark.parametrize("k", [100, 128])
def test_wide_decoders_of_one_module(k):
    """RS(100,4) and RS(128,4) decoders of 1, 3 and 4 erasures (8 to 32
    output strips, about 1.9 K to 11.5 K XORs) in one windowed module, with
    a ragged tile; bit-exact."""
    torch.cuda.set_device(0)
    sets = [[0, 7, 50, k + 1], [5], [3, k - 1, k + 2], [k, k + 1, k + 2, k + 3]]
    plan, jobs, outs, want, keep = _wide_decode_batch(k, sets, 8 * 1040, 8, 121 + k)
    try:
        b = xo.ec_batch_create(jobs, xo.EC_EXEC_COMPILED)
        try:
            assert xo.ec_batch_info_get(b)["programs"] == len(sets)
            xo.ec_batch_run(b, stream())
            torch.cuda.synchronize()
            for t, w in zip(outs, want):
                assert np.array_equal(t.cpu().numpy(), w)
        finally:
            xo.ec_batch_destroy(b)
    finally:
        xo.ec_plan_destroy(plan)
    assert xo.ec_device_status() == 0
