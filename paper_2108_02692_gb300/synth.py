"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds input generation only: no GF(2^8) arithmetic, no bitmatrix
and no XOR program.  Bytes come from the SplitMix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) in
its counter form: output i of the stream with seed s is
``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` and byte n of the stream is byte
``n % 8`` (little-endian) of output ``n // 8``.  The CUDA library implements
the same definition in its device generator so that full-size inputs never
cross the PCIe/C2C link; the two are checked against each other and against
the published seed-0 outputs.

The paper's workloads are "randomly generated arrays" (Sec. 7.2); the
recipes below reproduce their shapes (block sizes, codes, erasure patterns).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
BASE_SEED = 0x210802692
_M64 = (1 << 64) - 1


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream_words(seed: int, start_word: int, n_words: int) -> np.ndarray:
    """Outputs start_word .. start_word+n_words-1 of the stream ``seed``."""
    idx = np.arange(start_word + 1, start_word + n_words + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + idx * np.uint64(GAMMA)
    return mix64(z)


def stream_bytes(seed: int, offset: int, n: int) -> np.ndarray:
    """Bytes [offset, offset+n) of the stream ``seed``."""
    w0 = offset // 8
    w1 = (offset + n + 7) // 8
    words = stream_words(seed, w0, w1 - w0)
    b = words.view(np.uint8)  # little-endian hosts (x86_64, aarch64)
    s = offset - 8 * w0
    return b[s:s + n].copy()


def block_seed(workload_id: int, stripe: int, block: int) -> int:
    """Seed of block ``block`` of stripe ``stripe`` in workload ``workload_id``."""
    return (BASE_SEED ^ (workload_id << 40) ^ (stripe << 12) ^ block) & _M64


def block_bytes(workload_id: int, stripe: int, block: int, B: int,
                offset: int = 0, n: int | None = None) -> np.ndarray:
    if n is None:
        n = B - offset
    return stream_bytes(block_seed(workload_id, stripe, block), offset, n)


def strip_slice(workload_id: int, stripe: int, block: int, B: int, w0: int,
                L: int) -> np.ndarray:
    """Bytes [w0, w0+L) of each of the 8 strips of one block, as a block of
    8*L bytes in the same strip layout (columns are independent, so this is a
    valid small block for the oracle)."""
    S = B // 8
    parts = [block_bytes(workload_id, stripe, block, B, t * S + w0, L)
             for t in range(8)]
    return np.concatenate(parts)


# ---------------------------------------------------------------- workloads
#
# Config ids: 1 = RS(4,2) single stripe, 2 = RS(10,4) encode 256 stripes,
# 3 = RS(10,4) decode 256 stripes, 4 = batched mix, 5 = served stream.

def all_erasure_patterns(n: int, max_e: int, min_e: int = 1):
    out = []
    for e in range(min_e, max_e + 1):
        out.extend(itertools.combinations(range(n), e))
    return out


def decode_patterns(k: int, m: int, n_stripes: int, seed: int = 3):
    """One erasure set per stripe, uniform over all C(k+m, <= m) patterns."""
    pats = all_erasure_patterns(k + m, m)
    rng = np.random.Generator(np.random.PCG64(BASE_SEED ^ seed))
    idx = rng.integers(0, len(pats), size=n_stripes)
    return [tuple(pats[i]) for i in idx]


BATCH_CODES = [(6, 3), (8, 4), (10, 4), (12, 4)]


def batched_mix(n_stripes: int, min_b: int = 4096, max_b: int = 8 << 20,
                seed: int = 4, decode_frac: float = 0.5):
    """Stripes of the batched workload: code uniform over BATCH_CODES, block
    size log-uniform in [min_b, max_b] rounded to 128 B, and for a fraction
    of the stripes an erasure set of 1..m blocks."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED ^ seed))
    out = []
    for s in range(n_stripes):
        k, m = BATCH_CODES[int(rng.integers(0, len(BATCH_CODES)))]
        B = math.exp(rng.uniform(math.log(min_b), math.log(max_b)))
        B = max(128, int(round(B / 128.0)) * 128)
        er = None
        if rng.uniform() < decode_frac:
            ne = int(rng.integers(1, m + 1))
            er = tuple(sorted(int(x) for x in
                              rng.choice(k + m, size=ne, replace=False)))
        out.append({"k": k, "m": m, "B": B, "erasures": er})
    return out


def served_requests(duration_s: float, rate: float, seed: int = 5,
                    min_obj: int = 4096, max_obj: int = 16 << 20,
                    codes=((10, 4), (6, 3))):
    """Poisson arrivals of encode/decode requests with log-uniform object
    sizes; an object of L bytes becomes k blocks of
    B = roundup(ceil(L/k), 128) bytes (zero-padded tail)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED ^ seed))
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        k, m = codes[int(rng.integers(0, len(codes)))]
        L = int(math.exp(rng.uniform(math.log(min_obj), math.log(max_obj))))
        B = ((L + k - 1) // k + 127) // 128 * 128
        dec = bool(rng.uniform() < 0.5)
        er = None
        if dec:
            ne = int(rng.integers(1, m + 1))
            er = tuple(sorted(int(x) for x in
                              rng.choice(k + m, size=ne, replace=False)))
        reqs.append({"t": t, "k": k, "m": m, "L": L, "B": B,
                     "erasures": er})
    return reqs
