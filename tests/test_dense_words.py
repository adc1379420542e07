"""Host check of the dense bitmatrix executor's control words
(ec_plan_dense_words) against the oracle's bitmatrix: output strip r reads
input strip c exactly where bit (r, c) of the bitmatrix of the program's
matrix is set (Sec. 1, property (ii)); the parity matrix for the encoder,
R = G[E] G[S]^{-1} for a decoder (erasures in ascending order, survivors S the
first k non-erased blocks).  Both encodings of the bits (column masks, row
words) are decoded and compared; no GPU needed."""
import numpy as np
import pytest

import oracle
import paper_2108_02692_gb300 as xo


def _decode_words(words, n_in, n_out):
    G = (n_out + 31) // 32
    assert words.size == 2 * G * n_in
    masks, rows = words[:G * n_in], words[G * n_in:]
    from_masks = np.zeros((n_out, n_in), np.uint8)
    from_rows = np.zeros((n_out, n_in), np.uint8)
    for r in range(n_out):
        g, i = divmod(r, 32)
        for c in range(n_in):
            from_masks[r, c] = (int(masks[g * n_in + c]) >> i) & 1
            w, ci = divmod(c, 8)
            j, q = divmod(i, 4)
            from_rows[r, c] = (int(rows[g * n_in + 8 * w + j]) >> (8 * q + ci)) & 1
    # bits of groups' unused rows stay clear
    for g in range(G):
        top = n_out - 32 * g
        if top < 32:
            for c in range(n_in):
                assert int(masks[g * n_in + c]) >> top == 0
    return from_masks, from_rows


@pytest.mark.parametrize("k,m,erasures", [
    (10, 4, None),
    (10, 4, [2, 4, 5, 6]),
    (10, 4, [13, 0]),           # caller order: the program's outputs are sorted
    (6, 3, [7]),
    (3, 5, None),               # 40 output strips: two groups
    (12, 8, [0, 3, 5, 9, 12, 19]),
])
def test_dense_words_are_the_bitmatrix(k, m, erasures):
    _check(k, m, erasures, oracle.cauchy(k, m), None)


@pytest.mark.parametrize("erasures", [None, [2, 4, 5, 6]])
def test_dense_words_of_the_papers_matrix(erasures):
    """The paper's RS(10,4) matrix [2^(r j)] (Sec. 7.5: P_enc, and P_dec with
    blocks 2, 4, 5 and 6 erased)."""
    _check(10, 4, erasures, oracle.power(10, 4), xo.EC_MATRIX_POWER)


def _check(k, m, erasures, P, kind):
    plan = xo.ec_plan_create(k, m) if kind is None else \
        xo.ec_plan_create_ex(k, m, matrix_kind=kind)
    try:
        words = xo.ec_plan_dense_words(plan, erasures)
    finally:
        xo.ec_plan_destroy(plan)
    A = P if erasures is None else oracle.decode_matrix(P, sorted(erasures))
    want = oracle.bitmatrix(A)
    n_out, n_in = want.shape
    from_masks, from_rows = _decode_words(words, n_in, n_out)
    assert np.array_equal(from_masks, want)
    assert np.array_equal(from_rows, want)
