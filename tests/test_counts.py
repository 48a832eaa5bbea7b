"""The host-side operation accounting used for rates and roofline figures
agrees with the operations the CPU oracle counts while executing the same
algorithm (additions of two finite points)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import counts, inputs


@pytest.mark.parametrize("w,k", [(4, 1), (4, 2), (2, 3), (8, 1), (1, 5)])
def test_counts_match_oracle_execution(w, k):
    m, n, l = 40, 11, 3
    pr = inputs.pcmm_problem(77 + w * 10 + k, m, n, l, w)
    H = oracle.keygen(pr["sk"])
    ct = oracle.encrypt(H, pr["B"], pr["r"])
    _, oc = oracle.cussen(pr["A"], ct, w, k)
    c = counts.cussen_counts(pr["A"], w, k, l)
    assert c["gather_madd"] == oc["accum_add"]
    # Reconstruction and tuple additions: levels >= 2 as full additions,
    # level 1 and the tuples as mixed additions; same total as the oracle.
    assert c["table_add"] + c["table_madd"] + c["table_affine"] == oc["recon_add"]
    # Level-N multiplications: one per non-zero compressed value per chain.
    assert oc["ecsm"] == 2 * l * sum(len(counts._levels(pr["A"][:, j])[1]) for j in range(n))


def test_schoolbook_counts():
    A = np.array([[0, 1, 3], [4, 0, 0]], dtype=np.uint8)
    c = counts.schoolbook_counts(A, 2)
    # 1: 0 dbl; 3: 1 dbl + 1 madd; 4: 2 dbl; adds: row 0 has 2 terms -> 1.
    assert c == {"dbl": 4 * 3, "madd": 4 * 1, "add": 4 * 1}


def test_naf4_recoding():
    # The width-4 NAF: digits odd in [-7, 7] or zero, at most one non-zero
    # digit in any four consecutive ones, top digit non-zero, value exact.
    rng = np.random.default_rng(3)
    xs = [1, 2, 7, 8, 9, 15, 16, 17, 255, 2**255, 2**256 - 1]
    xs += [int.from_bytes(rng.bytes(32), "little") for _ in range(50)]
    for x in xs:
        d = counts.naf4(x)
        assert sum(v << i for i, v in enumerate(d)) == x
        assert all(v == 0 or (v % 2 == 1 and -7 <= v <= 7) for v in d)
        assert all(sum(1 for v in d[i:i + 4] if v) <= 1 for i in range(len(d)))
        assert d[-1] != 0 and len(d) <= x.bit_length() + 1
    assert counts.naf4(0) == []
    # About one non-zero digit in five for random 256-bit scalars.
    nz = np.mean([sum(1 for v in counts.naf4(x) if v) for x in xs[11:]])
    assert 45 < nz < 58


def test_strassen_counts():
    import json
    import os

    import numpy as np

    from paper_2504_14497_gb300 import counts
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_counts.json")))
    for t in gold["t"]:
        for ni, n in enumerate(gold["n"]):
            assert counts.strassen_equiv(n, t) == gold["pcmm_equiv"]["strassen"][str(t)][ni]
    rng = np.random.default_rng(4)
    A = rng.integers(0, 16, size=(16, 16), dtype=np.uint8)
    # Depth 0 is the schoolbook product.
    c0, sb = counts.strassen_counts(A, 4, 0, 16), counts.schoolbook_counts(A, 16)
    assert (c0["leaf_dbl"], c0["leaf_madd"], c0["leaf_add"]) == (sb["dbl"], sb["madd"], sb["add"])
    assert c0["block_madd"] == c0["block_add"] == 0
    # One step: 5 ciphertext sums over 8 x 8 quadrants, 8 output additions
    # over 8 x 8 quadrants, both components.
    c1 = counts.strassen_counts(A, 4, 1, 16)
    assert c1["block_madd"] == 2 * 5 * 64 and c1["block_add"] == 2 * 8 * 64
