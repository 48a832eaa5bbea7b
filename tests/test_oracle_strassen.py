"""Pins of the oracle's Strassen PC-MM (Section 3.1) and of its count model:
the equivalent-addition model against every Strassen entry of the Appendix
PC-MM table (exact), and the product against the closed form of Eq.
ahe_5_elgamal (which every correct method reaches) on recursion depths that
stop early on odd sizes, with negative block sums and cancelling
ciphertext sums."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_14497_gb300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_counts.json")))


def test_equivalent_counts_match_the_appendix_strassen_column():
    for t in GOLD["t"]:
        for ni, n in enumerate(GOLD["n"]):
            assert O.pcmm_equiv_strassen(n, t) == GOLD["pcmm_equiv"]["strassen"][str(t)][ni], (n, t)


def _problem(seed, m, n, l, w):
    pr = inputs.pcmm_problem(seed, m, n, l, w)
    ct = O.encrypt(O.keygen(pr["sk"]), pr["B"], pr["r"])
    want = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    return pr, ct, want


@pytest.mark.parametrize("m,n,l,w,levels", [(8, 8, 8, 4, 0), (8, 8, 8, 4, 1), (8, 8, 8, 4, 3),
                                            (12, 16, 10, 8, 2), (6, 4, 2, 3, 3), (16, 16, 16, 2, 2)])
def test_strassen_equals_closed_form(m, n, l, w, levels):
    pr, ct, want = _problem(300 + m + n + l + levels, m, n, l, w)
    got, cnt = O.strassen(pr["A"], ct, w, levels)
    assert (got == want).all()
    # Block additions made (two points per ciphertext, 13 block additions per
    # step over (n/2)-sized blocks); with 8-bit entries no block product
    # vanishes, with narrow entries a zero plaintext sum at a 1 x 1 leaf
    # leaves an identity operand, which is not counted.
    adds, mm, nn, ll, nodes = 0, m, n, l, 1
    for _ in range(levels):
        if mm % 2 or nn % 2 or ll % 2:
            break
        adds += nodes * 2 * (5 * (nn // 2) * (ll // 2) + 8 * (mm // 2) * (ll // 2))
        mm, nn, ll, nodes = mm // 2, nn // 2, ll // 2, nodes * 7
    if w >= 8:
        assert cnt["recon_add"] == adds
    else:
        assert 0.8 * adds <= cnt["recon_add"] <= adds


def test_strassen_with_negative_sums_and_cancelling_ciphertexts():
    # A21 = A11 + 1 and A12 = A22 give block differences of both signs and
    # zeros; B12 = B22 makes B12 - B22 the point at infinity; B21 = -B11
    # makes B21 + B11 vanish as well.
    m = n = l = 8
    pr, _, _ = _problem(777, m, n, l, 4)
    A = pr["A"].astype(np.int64)
    A[4:, :4] = np.minimum(A[:4, :4] + 1, 15)
    A[:4, 4:] = A[4:, 4:]
    A = A.astype(np.uint8)
    r = pr["r"].copy()
    B = pr["B"].copy()
    r[:, 4:] = r[:, :4]            # B12 = B22 on rows 0..3 vs 4..7 below
    r[:4, 4:] = r[4:, 4:]
    B[:4, 4:] = B[4:, 4:]
    ct = O.encrypt(O.keygen(pr["sk"]), B, r)
    for k in range(4):                                                          # B21 = -B11
        for j in range(4):
            for c in range(2):
                ct[4 + k, j, c] = O.point_neg(ct[k, j, c])
    want, _ = O.schoolbook(A, ct, 4)
    for levels in (1, 2, 3):
        got, _ = O.strassen(A, ct, 4, levels)
        assert (got == want).all(), levels


def test_strassen_rejects_out_of_range_entries():
    pr, ct, _ = _problem(5, 4, 4, 4, 3)
    A = pr["A"].copy()
    A[1, 2] = 9
    with pytest.raises(O.OracleError):
        O.strassen(A, ct, 3, 1)
