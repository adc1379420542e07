"""Python access to the plain C oracle (``xorec_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product path never
imports this package.

The oracle computes the plain definitions of the paper (GF(2^8) matrix
products on bit-sliced blocks, Sec. 1 and Sec. 6.1); see the C file header
for the exact reading of the layout.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xorec_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lib = None
_lock = threading.Lock()

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u8pp = ctypes.POINTER(_u8p)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liborc.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_gf_mul.restype = ctypes.c_uint8
            L.orc_gf_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
            L.orc_gf_inv.restype = ctypes.c_uint8
            L.orc_gf_inv.argtypes = [ctypes.c_uint8]
            L.orc_gf_pow2.restype = ctypes.c_uint8
            L.orc_gf_pow2.argtypes = [ctypes.c_long]
            L.orc_gf_tables.argtypes = [_u8p, _u8p]
            L.orc_cauchy.argtypes = [ctypes.c_int, ctypes.c_int, _u8p]
            L.orc_power.argtypes = [ctypes.c_int, ctypes.c_int, _u8p]
            L.orc_cauchy_min.argtypes = [ctypes.c_int, ctypes.c_int, _u8p]
            L.orc_get_elem.restype = ctypes.c_uint8
            L.orc_get_elem.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_size_t]
            L.orc_set_elem.argtypes = [_u8p, ctypes.c_size_t, ctypes.c_size_t,
                                       ctypes.c_uint8]
            L.orc_apply.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, _u8pp,
                                    _u8pp, ctypes.c_size_t]
            L.orc_encode.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, _u8pp,
                                     _u8pp, ctypes.c_size_t]
            L.orc_invert.argtypes = [ctypes.c_int, _u8p, _u8p]
            L.orc_decode.argtypes = [ctypes.c_int, ctypes.c_int, _u8p,
                                     ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                     _u8pp, _u8pp, ctypes.c_size_t]
            L.orc_bitmatrix.argtypes = [ctypes.c_int, ctypes.c_int, _u8p, _u8p]
            L.orc_apply_bitmatrix.argtypes = [ctypes.c_int, ctypes.c_int, _u8p,
                                              _u8pp, _u8pp, ctypes.c_size_t]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint8 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u8p)


def _pp(blocks):
    arr = (_u8p * max(1, len(blocks)))()
    for i, b in enumerate(blocks):
        arr[i] = _p(b) if b is not None else None
    return arr


def gf_mul(a: int, b: int) -> int:
    return int(lib().orc_gf_mul(a, b))


def gf_inv(a: int) -> int:
    return int(lib().orc_gf_inv(a))


def gf_pow2(e: int) -> int:
    return int(lib().orc_gf_pow2(e))


def gf_tables():
    exp = np.zeros(512, np.uint8)
    log = np.zeros(256, np.uint8)
    lib().orc_gf_tables(_p(exp), _p(log))
    return exp, log


def cauchy(k: int, m: int) -> np.ndarray:
    P = np.zeros((m, k), np.uint8)
    if lib().orc_cauchy(k, m, _p(P)) != 0:
        raise ValueError("bad (k, m)")
    return P


def cauchy_min(k: int, m: int) -> np.ndarray:
    """Cauchy rows and columns scaled to few bitmatrix ones (Sec. 7.6)."""
    P = np.zeros((m, k), np.uint8)
    if lib().orc_cauchy_min(k, m, _p(P)) != 0:
        raise ValueError("bad (k, m)")
    return P


def power(k: int, m: int) -> np.ndarray:
    P = np.zeros((m, k), np.uint8)
    if lib().orc_power(k, m, _p(P)) != 0:
        raise ValueError("bad (k, m)")
    return P


def get_elem(block: np.ndarray, e: int) -> int:
    return int(lib().orc_get_elem(_p(block), block.size, e))


def set_elem(block: np.ndarray, e: int, v: int) -> None:
    lib().orc_set_elem(_p(block), block.size, e, v)


def apply(A: np.ndarray, blocks) -> list:
    """out_i = sum_j A[i][j] * blocks[j] over GF(2^8) on bit-sliced blocks."""
    A = np.ascontiguousarray(A, dtype=np.uint8)
    rows, cols = A.shape
    assert len(blocks) == cols
    B = blocks[0].size if cols else 0
    outs = [np.zeros(B, np.uint8) for _ in range(rows)]
    rc = lib().orc_apply(rows, cols, _p(A), _pp(blocks), _pp(outs), B)
    if rc != 0:
        raise ValueError("orc_apply failed")
    return outs


def encode(P: np.ndarray, data) -> list:
    return apply(P, data)


def invert(M: np.ndarray):
    M = np.ascontiguousarray(M, dtype=np.uint8)
    n = M.shape[0]
    out = np.zeros((n, n), np.uint8)
    rc = lib().orc_invert(n, _p(M), _p(out))
    if rc == 1:
        return None
    if rc != 0:
        raise ValueError("orc_invert failed")
    return out


def decode(P: np.ndarray, erasures, blocks) -> list:
    """Recover the blocks at ``erasures`` (oracle self-test path only)."""
    P = np.ascontiguousarray(P, dtype=np.uint8)
    m, k = P.shape
    B = next(b.size for b in blocks if b is not None)
    er = (ctypes.c_int * max(1, len(erasures)))(*erasures)
    outs = [np.zeros(B, np.uint8) for _ in erasures]
    rc = lib().orc_decode(k, m, _p(P), er, len(erasures), _pp(blocks),
                          _pp(outs), B)
    if rc == 1:
        raise ZeroDivisionError("singular survivor submatrix")
    if rc != 0:
        raise ValueError("orc_decode failed")
    return outs


def bitmatrix(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.uint8)
    rows, cols = A.shape
    bits = np.zeros((8 * rows, 8 * cols), np.uint8)
    lib().orc_bitmatrix(rows, cols, _p(A), _p(bits))
    return bits


def apply_bitmatrix(bits: np.ndarray, blocks) -> list:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    rows, cols = bits.shape[0] // 8, bits.shape[1] // 8
    B = blocks[0].size
    outs = [np.zeros(B, np.uint8) for _ in range(rows)]
    rc = lib().orc_apply_bitmatrix(rows, cols, _p(bits), _pp(blocks),
                                   _pp(outs), B)
    if rc != 0:
        raise ValueError("orc_apply_bitmatrix failed")
    return outs


def generator_matrix(P: np.ndarray) -> np.ndarray:
    """The systematic generator [I ; P] (Sec. 1, Sec. 7.1)."""
    m, k = P.shape
    return np.concatenate([np.eye(k, dtype=np.uint8), P], axis=0)


def decode_matrix(P: np.ndarray, erasures) -> np.ndarray:
    """R = G[E] * G[S]^{-1}, S = first k non-erased ids ascending (Sec. 1)."""
    m, k = P.shape
    G = generator_matrix(P)
    er = set(erasures)
    surv = [i for i in range(k + m) if i not in er][:k]
    Minv = invert(G[surv])
    if Minv is None:
        raise ZeroDivisionError("singular survivor submatrix")
    R = np.zeros((len(erasures), k), np.uint8)
    for i, e in enumerate(erasures):
        for c in range(k):
            acc = 0
            for x in range(k):
                acc ^= gf_mul(int(G[e, x]), int(Minv[x, c]))
            R[i, c] = acc
    return R
