"""Several host threads on one plan at once: encodes (pointer table,
strided, from host memory) and decodes whose programs are built and
compiled on first use, each thread on its own stream; every result equal
to the oracle."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu


def test_threads_share_one_plan():
    torch.cuda.set_device(0)
    k, m, B, n = 10, 4, 8 * 1040, 3
    plan = xo.ec_plan_create(k, m)
    P = oracle.cauchy(k, m)
    errors = []

    def worker(t):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            st = s.cuda_stream
            rng = np.random.default_rng(100 + t)
            for it in range(3):
                data = np.stack([np.stack([synth.block_bytes(64, 100 * t + 10 * it + i, j, B)
                                           for j in range(k)]) for i in range(n)])
                ref = [oracle.encode(P, list(data[i])) for i in range(n)]
                d = torch.from_numpy(data).cuda()
                # strided encode (tensor copies)
                par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
                xo.ec_encode_strided(plan, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B, st)
                # from host memory (shared staging, enqueued one call at a time)
                h_data = torch.from_numpy(data).pin_memory()
                h_par = torch.zeros((n, m, B), dtype=torch.uint8).pin_memory()
                xo.ec_encode_host_strided(plan, h_data.data_ptr(), k * B, B, h_par.data_ptr(), m * B,
                                          B, n, B, 0, st)
                # a decode with a pattern of this thread (built on first use)
                er = sorted(int(x) for x in rng.choice(k + m, size=int(rng.integers(1, m + 1)),
                                                       replace=False))
                blocks = [d[0, j] for j in range(k)] + [par[0, i] for i in range(m)]
                outs = [torch.zeros(B, dtype=torch.uint8, device="cuda") for _ in er]
                s.synchronize()
                xo.ec_decode(plan, er, [None if i in er else blocks[i].data_ptr()
                                        for i in range(k + m)],
                             [o.data_ptr() for o in outs], B, st)
                s.synchronize()
                g = par.cpu().numpy()
                for i in range(n):
                    for j in range(m):
                        assert np.array_equal(g[i, j], ref[i][j])
                        assert np.array_equal(h_par.numpy()[i, j], ref[i][j])
                truth = list(data[0]) + ref[0]
                for o, e in zip(outs, er):
                    assert np.array_equal(o.cpu().numpy(), truth[e])
        except Exception as e:      # reported by the main thread
            errors.append(f"thread {t}: {e!r}")

    try:
        threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(timeout=300)
        assert not errors, errors
        assert xo.ec_device_status() == 0
    finally:
        xo.ec_plan_destroy(plan)
