"""TMA tensor copies against per-strip bulk copies: the same bytes, both
equal to the oracle.  EC_TMA_TENSOR=0 makes the library stage every input
strip with its own 1-D copy; covered: strided launches (one 3-D copy per
tile), the largest box (32 data blocks = 256 strips), stages of more strips
than a box holds (several boxes per tile, down to 8 strips per box when k is
prime), ragged strip tails (zero-filled boxes), and batches (one 2-D copy
per input block and tile)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def stream():
    return torch.cuda.current_stream().cuda_stream


class tensor_copies:
    def __init__(self, on):
        self.on = on

    def __enter__(self):
        self.old = os.environ.get("EC_TMA_TENSOR")
        os.environ["EC_TMA_TENSOR"] = "1" if self.on else "0"

    def __exit__(self, *a):
        if self.old is None:
            os.environ.pop("EC_TMA_TENSOR", None)
        else:
            os.environ["EC_TMA_TENSOR"] = self.old


@pytest.mark.parametrize("k,m,B,n", [(10, 4, 8 * 1552, 5),     # ragged tail (1552 = 3 x 512 + 16)
                                     (32, 4, 8 * 528, 3),      # box of 256 strips
                                     (40, 4, 8 * 528, 2),      # two boxes of 160 strips
                                     (48, 4, 8 * 1552, 2),     # two boxes of 192, ragged tail
                                     (37, 3, 8 * 528, 2),      # k prime: 37 boxes of 8 strips
                                     (100, 4, 8 * 400, 2),     # four boxes of 200 strips
                                     (6, 3, 8 * 2048, 4)])
def test_strided_encode_same_bytes_with_and_without_tensor_copies(k, m, B, n):
    torch.cuda.set_device(0)
    plan = xo.ec_plan_create(k, m)
    try:
        data = np.stack([np.stack([synth.block_bytes(61, s, j, B) for j in range(k)])
                         for s in range(n)])
        d = torch.from_numpy(data).cuda()
        outs = []
        for on in (True, False):
            par = torch.full((n, m, B), 0x5C, dtype=torch.uint8, device="cuda")
            with tensor_copies(on):
                xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                                     stream())
                torch.cuda.synchronize()
            outs.append(par.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, list(data[s]))
            for i in range(m):
                assert np.array_equal(outs[0][s, i], ref[i]), (s, i)
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)


def test_batch_same_bytes_with_and_without_tensor_copies():
    torch.cuda.set_device(0)
    codes = [(4, 2), (10, 4), (12, 4)]
    plans = {c: xo.ec_plan_create(*c) for c in codes}
    try:
        rng = np.random.default_rng(62)
        jobs, outs, expect, keep = [], [], [], []
        for s in range(30):
            k, m = codes[s % len(codes)]
            B = int(rng.choice([128, 4096, 8 * 1040, 8 * 4112]))
            data = [synth.block_bytes(62, s, j, B) for j in range(k)]
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
        got = []
        for on in (True, False):
            with tensor_copies(on):
                b = xo.ec_batch_create(jobs)
            try:
                xo.ec_batch_run(b, stream())
                torch.cuda.synchronize()
            finally:
                xo.ec_batch_destroy(b)
            got.append([[t.cpu().numpy().copy() for t in o] for o in outs])
            for o in outs:
                for t in o:
                    t.zero_()
        for a, b2, ref in zip(got[0], got[1], expect):
            for x, y, r in zip(a, b2, ref):
                assert np.array_equal(x, y)
                assert np.array_equal(x, r)
        assert xo.ec_device_status() == 0
    finally:
        for h in plans.values():
            xo.ec_plan_destroy(h)


@pytest.mark.parametrize("pad_stripe,block_gap", [(4096, 0),       # padded stripes: tensor copies
                                                  (0, 1024),       # gaps between blocks: per-strip
                                                  (8192, 2048)])
def test_strided_layouts_with_padding(pad_stripe, block_gap):
    torch.cuda.set_device(0)
    k, m, B, n = 10, 4, 8 * 1040, 4
    bstride = B + block_gap
    sstride = k * bstride + pad_stripe
    plan = xo.ec_plan_create(k, m)
    try:
        buf = torch.zeros(n * sstride, dtype=torch.uint8, device="cuda")
        data = [[synth.block_bytes(63, s, j, B) for j in range(k)] for s in range(n)]
        for s in range(n):
            for j in range(k):
                o = s * sstride + j * bstride
                buf[o:o + B] = torch.from_numpy(data[s][j]).cuda()
        outs = []
        for on in (True, False):
            par = torch.full((n, m, B), 0x11, dtype=torch.uint8, device="cuda")
            with tensor_copies(on):
                xo.ec_encode_strided(plan, buf.data_ptr(), sstride, bstride, par.data_ptr(), m * B, B,
                                     n, B, stream())
                torch.cuda.synchronize()
            outs.append(par.cpu().numpy())
        assert np.array_equal(outs[0], outs[1])
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, data[s])
            for i in range(m):
                assert np.array_equal(outs[0][s, i], ref[i]), (s, i)
    finally:
        xo.ec_plan_destroy(plan)


def test_large_blocks_strided_sampled():
    # 64 MiB blocks: strips of 8 MiB, tile coordinates up to 2^21 words
    torch.cuda.set_device(0)
    k, m, B, n = 4, 2, 64 << 20, 2
    S = B // 8
    plan = xo.ec_plan_create(k, m)
    try:
        data = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
        for s in range(n):
            for j in range(k):
                xo.ec_synth_fill(data[s, j].data_ptr(), B, synth.block_seed(65, s, j), 0, stream())
        par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
        xo.ec_encode_strided(plan, data.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B, stream())
        torch.cuda.synchronize()
        P = oracle.cauchy(k, m)
        for s in range(n):
            for w0 in (0, S // 2 + 4096, S - 64):
                mini = [synth.strip_slice(65, s, j, B, w0, 64) for j in range(k)]
                ref = oracle.encode(P, mini)
                got = par[s].view(m, 8, S)[:, :, w0:w0 + 64].cpu().numpy()
                for i in range(m):
                    assert np.array_equal(got[i].reshape(-1), ref[i]), (s, w0, i)
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)


def test_many_tiny_stripes_strided():
    # 128-byte blocks: 16-byte strips inside 512-byte boxes (mostly zero fill)
    torch.cuda.set_device(0)
    k, m, B, n = 10, 4, 128, 5000
    plan = xo.ec_plan_create(k, m)
    try:
        data = np.stack([np.stack([synth.block_bytes(66, s, j, B) for j in range(k)])
                         for s in range(n)])
        d = torch.from_numpy(data).cuda()
        par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
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
