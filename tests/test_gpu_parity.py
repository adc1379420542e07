"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle,
bit for bit.  Inputs come from the seeded generator; expected values come
only from the oracle (or are the generated originals, for decoding)."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import paper_2108_02692_gb300 as xo
from paper_2108_02692_gb300 import synth

pytestmark = pytest.mark.gpu

EXECS = [xo.EC_EXEC_INTERP, xo.EC_EXEC_COMPILED, xo.EC_EXEC_DENSE]
EXEC_IDS = ["interp", "compiled", "dense"]


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.set_device(0)
    xo.ec_device_status(reset=True)
    yield
    assert xo.ec_device_status() == 0


def dev(arr: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy()


def stream():
    return torch.cuda.current_stream().cuda_stream


class Plan:
    def __init__(self, k, m, executor=xo.EC_EXEC_AUTO, **kw):
        self.k, self.m = k, m
        self.h = xo.ec_plan_create_ex(k, m, executor=executor, **kw)

    def close(self):
        xo.ec_plan_destroy(self.h)


def test_device_generator_matches_host_generator():
    n = 1 << 20
    buf = torch.empty(n + 64, dtype=torch.uint8, device="cuda")
    for seed, off, length in [(0, 0, n), (12345, 8, 4096), (7, 3, 1001), (99, 13, 50)]:
        xo.ec_synth_fill(buf.data_ptr(), length, seed, off, stream())
        torch.cuda.synchronize()
        assert np.array_equal(host(buf[:length]), synth.stream_bytes(seed, off, length))
    # unaligned destination
    xo.ec_synth_fill(buf.data_ptr() + 3, 100, 5, 0, stream())
    torch.cuda.synchronize()
    assert np.array_equal(host(buf[3:103]), synth.stream_bytes(5, 0, 100))


ENC_CASES = [
    (4, 2, 64 * 1024),          # RS(4,2), 64 KiB blocks (8 KiB strips)
    (10, 4, 8 * 3152),          # strips of 3152 B: several tiles and a ragged tail
    (6, 3, 128),                # smallest block: 16-byte strips
    (12, 4, 8 * 1040),
    (1, 1, 1024),               # k = 1: parity is a scaled copy
    (2, 1, 4096),
    (3, 5, 2048),               # more parity than data
]


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
@pytest.mark.parametrize("k,m,B", ENC_CASES)
def test_encode_matches_oracle(k, m, B, executor):
    p = Plan(k, m, executor)
    try:
        data = [synth.block_bytes(21, 0, j, B) for j in range(k)]
        ref = oracle.encode(oracle.cauchy(k, m), data)
        d = [dev(x) for x in data]
        par = [torch.full((B,), 0xA5, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(p.h, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(host(par[i]), ref[i]), f"parity {i}"
    finally:
        p.close()


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
@pytest.mark.parametrize("opt", [xo.EC_OPT_RAW, xo.EC_OPT_REPAIR, xo.EC_OPT_XORREPAIR,
                                 xo.EC_OPT_TRIPLE])
def test_encode_opt_levels_and_matrices(opt, executor):
    k, m, B = 10, 4, 8 * 2064
    for kind, P in [(xo.EC_MATRIX_CAUCHY, oracle.cauchy(k, m)),
                    (xo.EC_MATRIX_POWER, oracle.power(k, m)),
                    (xo.EC_MATRIX_CAUCHY_MIN, oracle.cauchy_min(k, m))]:
        h = xo.ec_plan_create_ex(k, m, matrix_kind=kind, opt_level=opt, executor=executor)
        try:
            data = [synth.block_bytes(22, kind, j, B) for j in range(k)]
            ref = oracle.encode(P, data)
            d = [dev(x) for x in data]
            par = [torch.empty(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
            xo.ec_encode(h, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, stream())
            torch.cuda.synchronize()
            for i in range(m):
                assert np.array_equal(host(par[i]), ref[i])
        finally:
            xo.ec_plan_destroy(h)


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
def test_user_matrix_encode(executor):
    k, m, B = 5, 3, 1024
    rng = np.random.default_rng(3)
    P = rng.integers(0, 256, size=(m, k), dtype=np.uint8)
    P[1, 2] = 0                          # a zero coefficient
    P[2] = 0                             # an all-zero parity row
    h = xo.ec_plan_create_ex(k, m, matrix_kind=xo.EC_MATRIX_USER, matrix=P, executor=executor)
    try:
        data = [synth.block_bytes(23, 0, j, B) for j in range(k)]
        ref = oracle.encode(P, data)
        d = [dev(x) for x in data]
        par = [torch.full((B,), 0x5A, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(h, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(host(par[i]), ref[i])
    finally:
        xo.ec_plan_destroy(h)


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
def test_encode_strided_many_stripes(executor):
    k, m, B, n = 10, 4, 8 * 1552, 7
    p = Plan(k, m, executor)
    try:
        data = np.stack([np.stack([synth.block_bytes(24, s, j, B) for j in range(k)])
                         for s in range(n)])              # [n, k, B]
        d = dev(data)
        par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
        xo.ec_encode_strided(p.h, d.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                             stream())
        torch.cuda.synchronize()
        got = host(par)
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, list(data[s]))
            for i in range(m):
                assert np.array_equal(got[s, i], ref[i]), (s, i)
    finally:
        p.close()


def _codeword(k, m, B, cfg, stripe):
    data = [synth.block_bytes(cfg, stripe, j, B) for j in range(k)]
    return data + oracle.encode(oracle.cauchy(k, m), data)


def _decode_check(p, blocks, er, B, order=None):
    k, m = p.k, p.m
    dblocks = [dev(b) for b in blocks]
    ptrs = [None if i in er else dblocks[i].data_ptr() for i in range(k + m)]
    er_call = list(order) if order is not None else list(er)
    outs = [torch.full((B,), 0x33, dtype=torch.uint8, device="cuda") for _ in er_call]
    xo.ec_decode(p.h, er_call, ptrs, [o.data_ptr() for o in outs], B, stream())
    torch.cuda.synchronize()
    for o, e in zip(outs, er_call):
        assert np.array_equal(host(o), blocks[e]), (er_call, e)


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
def test_decode_rs4_2_every_pattern(executor):
    """RS(4,2), 64 KiB blocks: every erasure pattern of 1 and 2 blocks."""
    k, m, B = 4, 2, 64 * 1024
    p = Plan(k, m, executor)
    try:
        blocks = _codeword(k, m, B, 1, 0)
        n = 0
        for ne in (1, 2):
            for er in itertools.combinations(range(k + m), ne):
                _decode_check(p, blocks, er, B)
                n += 1
        assert n == 21
        _decode_check(p, blocks, (1, 4), B, order=(4, 1))   # caller order kept
    finally:
        p.close()


@pytest.mark.parametrize("executor", [xo.EC_EXEC_INTERP, xo.EC_EXEC_DENSE],
                         ids=["interp", "dense"])
def test_decode_rs6_3_every_pattern(executor):
    k, m, B = 6, 3, 8 * 528
    p = Plan(k, m, executor)
    try:
        blocks = _codeword(k, m, B, 25, 0)
        pats = [e for ne in range(1, 4) for e in itertools.combinations(range(9), ne)]
        assert len(pats) == 129
        for er in pats:
            _decode_check(p, blocks, er, B)
    finally:
        p.close()


def test_decode_rs6_3_sample_compiled():
    k, m, B = 6, 3, 8 * 528
    p = Plan(k, m, xo.EC_EXEC_COMPILED)
    try:
        blocks = _codeword(k, m, B, 25, 1)
        for er in [(0,), (8,), (0, 5), (2, 7), (6, 7, 8), (0, 1, 2), (1, 4, 8)]:
            _decode_check(p, blocks, er, B)
    finally:
        p.close()


@pytest.mark.parametrize("executor,B", [(xo.EC_EXEC_INTERP, 256), (xo.EC_EXEC_DENSE, 256),
                                        (xo.EC_EXEC_DENSE, 8 * 2064)],
                         ids=["interp", "dense", "dense-3-tiles"])
def test_decode_rs10_4_all_1470_patterns(executor, B):
    """Every erasure set of 1-4 blocks of RS(10,4) (C(14,<=4) = 1470); with
    strips of 2064 B the dense executor's 1 KiB tiles end in a ragged one."""
    k, m = 10, 4
    p = Plan(k, m, executor)
    try:
        pats = synth.all_erasure_patterns(14, 4)
        assert len(pats) == 1470
        xo.ec_decode_prepare(p.h, pats)
        blocks = _codeword(k, m, B, 26, 0)
        dblocks = [dev(b) for b in blocks]
        outs = torch.empty((4, B), dtype=torch.uint8, device="cuda")
        bad = []
        for er in pats:
            ptrs = [None if i in er else dblocks[i].data_ptr() for i in range(14)]
            xo.ec_decode(p.h, list(er), ptrs, [outs[i].data_ptr() for i in range(len(er))], B,
                         stream())
            got = host(outs)
            for i, e in enumerate(er):
                if not np.array_equal(got[i], blocks[e]):
                    bad.append(er)
        assert not bad, bad[:5]
    finally:
        p.close()


def test_decode_argument_errors():
    p = Plan(4, 2)
    try:
        B = 1024
        blocks = [torch.zeros(B + 16, dtype=torch.uint8, device="cuda") for _ in range(6)]
        ptrs = [b.data_ptr() for b in blocks]
        out = torch.zeros(B, dtype=torch.uint8, device="cuda")
        with pytest.raises(xo.XorecError) as e:
            xo.ec_decode(p.h, [0, 1, 2], ptrs, [out.data_ptr()] * 3, B, stream())
        assert e.value.status == xo.EC_ETOOMANY
        with pytest.raises(xo.XorecError) as e:
            xo.ec_decode(p.h, [0], ptrs, [out.data_ptr()], 1000, stream())
        assert e.value.status == xo.EC_EINVAL
        mis = list(ptrs)
        mis[1] = ptrs[1] + 8
        with pytest.raises(xo.XorecError) as e:
            xo.ec_decode(p.h, [0], mis, [out.data_ptr()], B, stream())
        assert e.value.status == xo.EC_EINVAL
        with pytest.raises(xo.XorecError) as e:
            xo.ec_encode(p.h, ptrs[:4], [ptrs[4] + 4, ptrs[5]], B, stream())
        assert e.value.status == xo.EC_EINVAL
    finally:
        p.close()


# ------------------------------------------------------------ full sizes

FULL_K, FULL_M, FULL_B, FULL_N = 10, 4, 1 << 20, 256


def _fill_stripes(buf, cfg, n, nblk, B):
    for s in range(n):
        for j in range(nblk):
            xo.ec_synth_fill(buf[s, j].data_ptr(), B, synth.block_seed(cfg, s, j), 0, stream())


@pytest.mark.parametrize("shape", [None, (128, 160), (256, 128)],
                         ids=["default", "128x160", "256x128"])
def test_full_size_encode_rs10_4_sampled(shape):
    """The benchmark's encode launch: 256 stripes x 10 x 1 MiB in one call,
    checked on sampled windows of every stripe against the oracle, under the
    default launch shape and the shapes the autotuner picks on GB300."""
    k, m, B, n = FULL_K, FULL_M, FULL_B, FULL_N
    p = Plan(k, m)
    if shape:
        xo.ec_plan_set_launch(p.h, *shape)
    try:
        data = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
        _fill_stripes(data, 2, n, k, B)
        par = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
        xo.ec_encode_strided(p.h, data.data_ptr(), k * B, B, par.data_ptr(), m * B, B, n, B,
                             stream())
        torch.cuda.synchronize()
        P = oracle.cauchy(k, m)
        rng = np.random.default_rng(2)
        S, L = B // 8, 64
        for s in range(n):
            w0 = int(rng.integers(0, (S - L) // 16)) * 16
            if s == n - 1:
                w0 = S - L                        # last bytes of every strip
            mini = [synth.strip_slice(2, s, j, B, w0, L) for j in range(k)]
            ref = oracle.encode(P, mini)
            got = host(par[s, :, :].view(m, 8, S)[:, :, w0:w0 + L])
            for i in range(m):
                assert np.array_equal(got[i].reshape(-1), ref[i]), (s, i, w0)
    finally:
        p.close()
        del data, par
        torch.cuda.empty_cache()


def test_full_size_decode_rs10_4_sampled():
    """256 stripes x 1 MiB blocks, one erasure set per stripe drawn from all
    1470 patterns.  The survivors are arbitrary bytes, so the check is the
    decode map itself: out = R * survivors with R = G[E] G[S]^{-1} computed
    by the oracle."""
    k, m, B, n = FULL_K, FULL_M, FULL_B, FULL_N
    p = Plan(k, m)
    try:
        pats = synth.decode_patterns(k, m, n)
        xo.ec_decode_prepare(p.h, sorted(set(pats)))
        xo.ec_plan_compile(p.h, sorted(set(pats)))     # compile in parallel up front
        surv = torch.empty((n, k, B), dtype=torch.uint8, device="cuda")
        _fill_stripes(surv, 3, n, k, B)
        outs = torch.zeros((n, m, B), dtype=torch.uint8, device="cuda")
        for s, er in enumerate(pats):
            ids = [i for i in range(k + m) if i not in er][:k]
            ptrs = [None] * (k + m)
            for j, bid in enumerate(ids):
                ptrs[bid] = surv[s, j].data_ptr()
            xo.ec_decode(p.h, list(er), ptrs, [outs[s, i].data_ptr() for i in range(len(er))],
                         B, stream())
        torch.cuda.synchronize()
        P = oracle.cauchy(k, m)
        rng = np.random.default_rng(3)
        S, L = B // 8, 32
        for s in range(0, n, 4):
            er = pats[s]
            R = oracle.decode_matrix(P, list(er))
            w0 = int(rng.integers(0, (S - L) // 16)) * 16
            mini = [synth.strip_slice(3, s, j, B, w0, L) for j in range(k)]
            ref = oracle.apply(R, mini)
            got = host(outs[s, :len(er)].view(len(er), 8, S)[:, :, w0:w0 + L])
            for i in range(len(er)):
                assert np.array_equal(got[i].reshape(-1), ref[i]), (s, er, i)
    finally:
        p.close()
        del surv, outs
        torch.cuda.empty_cache()


@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
def test_encode_from_host_memory(pinned):
    k, m, B, n = 10, 4, 8 * 1040, 9
    p = Plan(k, m)
    try:
        data = np.stack([np.stack([synth.block_bytes(27, s, j, B) for j in range(k)])
                         for s in range(n)])
        h_data = torch.from_numpy(data)
        h_par = torch.zeros((n, m, B), dtype=torch.uint8)
        if pinned:
            h_data = h_data.pin_memory()
            h_par = h_par.pin_memory()
        xo.ec_encode_host_strided(p.h, h_data.data_ptr(), k * B, B, h_par.data_ptr(), m * B, B,
                                  n, B, 4, stream())
        torch.cuda.synchronize()
        P = oracle.cauchy(k, m)
        for s in range(n):
            ref = oracle.encode(P, list(data[s]))
            for i in range(m):
                assert np.array_equal(h_par[s, i].numpy(), ref[i]), (s, i)
        # non-dense host layout: parity blocks interleaved with a gap
        h_par2 = torch.zeros((n, m, B + 128), dtype=torch.uint8)
        xo.ec_encode_host_strided(p.h, h_data.data_ptr(), k * B, B, h_par2.data_ptr(),
                                  m * (B + 128), B + 128, n, B, 3, stream())
        torch.cuda.synchronize()
        for s in range(n):
            for i in range(m):
                assert np.array_equal(h_par2[s, i, :B].numpy(), h_par[s, i].numpy())
    finally:
        p.close()


WIDE = [(20, 4, 8 * 1040), (40, 8, 4096), (100, 4, 2048), (1, 255, 1024), (128, 128, 256)]


@pytest.mark.parametrize("k,m,B", WIDE)
def test_wide_and_extreme_codes_encode(k, m, B):
    """Wide codes (more input strips than registers) run from the shared-
    memory stage or, when the tile does not fit, in the interpreter;
    k + m = 256 is the largest code."""
    p = Plan(k, m)
    try:
        data = [synth.block_bytes(28, k, j, B) for j in range(k)]
        ref = oracle.encode(oracle.cauchy(k, m), data)
        d = [dev(x) for x in data]
        par = [torch.full((B,), 0x3C, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(p.h, [t.data_ptr() for t in d], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(host(par[i]), ref[i]), i
    finally:
        p.close()


def test_wide_code_decode():
    k, m, B = 20, 4, 8 * 528
    p = Plan(k, m)
    try:
        blocks = _codeword(k, m, B, 29, 0)
        for er in [(0, 5, 21, 23), (19,), (20, 21, 22, 23), (3, 22)]:
            _decode_check(p, blocks, er, B)
    finally:
        p.close()


@pytest.mark.parametrize("executor", EXECS, ids=EXEC_IDS)
def test_cauchy_min_every_decode_pattern_rs6_3(executor):
    # scaled Cauchy: all 129 erasure sets of RS(6,3) recover the original
    # blocks bit for bit (strips of 528 bytes: one 512-byte tile and a
    # ragged 16-byte tail)
    k, m, B = 6, 3, 8 * 528
    P = oracle.cauchy_min(k, m)
    h = xo.ec_plan_create_ex(k, m, matrix_kind=xo.EC_MATRIX_CAUCHY_MIN, executor=executor)
    try:
        data = [synth.block_bytes(23, 0, j, B) for j in range(k)]
        blocks = data + oracle.encode(P, data)
        d = [dev(x) for x in blocks]
        par = [torch.empty(B, dtype=torch.uint8, device="cuda") for _ in range(m)]
        xo.ec_encode(h, [t.data_ptr() for t in d[:k]], [t.data_ptr() for t in par], B, stream())
        torch.cuda.synchronize()
        for i in range(m):
            assert np.array_equal(host(par[i]), blocks[k + i])
        for ne in range(1, m + 1):
            for er in itertools.combinations(range(k + m), ne):
                out = [torch.empty(B, dtype=torch.uint8, device="cuda") for _ in er]
                ptrs = [None if i in er else d[i].data_ptr() for i in range(k + m)]
                xo.ec_decode(h, list(er), ptrs, [t.data_ptr() for t in out], B, stream())
                torch.cuda.synchronize()
                for i, e in enumerate(er):
                    assert np.array_equal(host(out[i]), blocks[e]), (er, e)
    finally:
        xo.ec_plan_destroy(h)
