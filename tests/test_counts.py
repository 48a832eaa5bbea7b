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
