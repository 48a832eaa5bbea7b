"""Pins of the operation-count model (used for roofline accounting)
against the paper's printed Appendix tables (tests/golden)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "appendix_counts.json")))
NS = GOLD["n"]
TS = GOLD["t"]


def _strassen_plain(n):
    # M(n) = 7 M(n/2), A(n) = 7 A(n/2) + 18 (n/2)^2, M(1) = 1, A(1) = 0.
    if n == 1:
        return 1, 0
    m, a = _strassen_plain(n // 2)
    return 7 * m, 7 * a + 18 * (n // 2) ** 2


def _strassen_ct_equiv(n, t):
    # 7^L plaintext-ciphertext products (2 ECSMs of 2t additions each) and
    # 13 ciphertext block additions per level (Section 3.1).
    def rec(k):
        if k == 1:
            return 1, 0
        m, a = rec(k // 2)
        return 7 * m, 7 * a + 13 * (k // 2) ** 2
    mults, adds = rec(n)
    return mults * 2 * 2 * t + 2 * adds


def test_printed_tables_are_mutually_consistent():
    for ti, t in enumerate(TS):
        ts = str(t)
        for ni, n in enumerate(NS):
            vm, va = GOLD["vector_mults"][ts][ni], GOLD["vector_adds"][ts][ni]
            v = O.ct_vector_equiv(vm, va, t)
            assert v == GOLD["ct_vector_equiv"]["proposed"][ts][ni]
            assert GOLD["ct_vector_equiv"]["schoolbook"][ts][ni] == 2 * n * 2 * t
            assert O.pcmm_equiv_cussen(n, v) == GOLD["pcmm_equiv"]["proposed"][ts][ni]
            assert O.pcmm_equiv_schoolbook(n, t) == GOLD["pcmm_equiv"]["schoolbook"][ts][ni]
            assert _strassen_ct_equiv(n, t) == GOLD["pcmm_equiv"]["strassen"][ts][ni]
            assert GOLD["matrix_mults"][ts][ni] == n * n * vm
            assert GOLD["matrix_adds"][ts][ni] == n * n * va + n * n * (n - 1)
    for ni, n in enumerate(NS):
        assert GOLD["matrix_mults"]["schoolbook"][ni] == n ** 3
        assert GOLD["matrix_adds"]["schoolbook"][ni] == n * n * (n - 1)
        assert (GOLD["matrix_mults"]["strassen"][ni], GOLD["matrix_adds"]["strassen"][ni]) == _strassen_plain(n)


def test_toy_example_counts_are_consistent():
    toy = GOLD["toy_example"]
    # Encrypted = two components of the plaintext counts.
    assert toy["encrypted_ecsm"] == 2 * toy["plain_mults"]
    assert toy["encrypted_adds"] == 2 * toy["plain_adds"]
    # 8-bit scalars: one ECSM ~ 16 additions; saving = 16 ECSMs*16 - (6*16 + 30).
    assert 16 * 16 - (6 * 16 + 30) == 130


@pytest.mark.parametrize("t", [4, 8, 12, 16])
def test_count_model_reproduces_vector_tables(t):
    rng = np.random.default_rng(2504 + t)
    for ni, n in enumerate(NS):
        res = np.array([O.compress_counts(rng.integers(0, 2**t, n)) for _ in range(1000)]).mean(axis=0)
        tm = GOLD["vector_mults"][str(t)][ni]
        ta = GOLD["vector_adds"][str(t)][ni]
        # Printed values are rounded means of 1000 random trials.
        assert abs(res[0] - tm) <= 0.9, (t, n, res, tm)
        assert abs(res[1] - ta) <= max(1.6, 0.01 * ta), (t, n, res, ta)


def test_count_model_small_cases():
    # Hand-worked vectors: [5, 5, 5] -> [5] at every level: one non-zero
    # entry on each of levels 1..3 and one multiply at level 4.
    assert O.compress_counts([5, 5, 5]) == (1, 3)
    # [0, 0] contributes nothing.
    assert O.compress_counts([0, 0]) == (0, 0)
    # [1, 2, 3, 4]: level 1 diffs [1,1,1,1] -> 4 non-zero; level 2 [1] -> 1;
    # level 3 [1] -> 1; level 4 [1] -> one multiply.
    assert O.compress_counts([1, 2, 3, 4]) == (1, 6)
