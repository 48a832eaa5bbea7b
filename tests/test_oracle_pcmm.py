"""Pins of the oracle's PC-MM algorithms: schoolbook (Section 3.1), Cussen
(Algorithms 2 and 3, plus the strip-width extension) and the closed form
agree with each other, decrypt to the plain product A B, and agree with
brute-force repeated addition; exceptional additions (doubling and
cancellation inside the sums) are forced with crafted inputs."""
import random

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_14497_gb300 import inputs as I

Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551


def _problem(seed, m, n, l, w, msg_bits=8):
    pr = I.pcmm_problem(seed, m, n, l, w, msg_bits)
    H = O.keygen(pr["sk"])
    ct = O.encrypt(H, pr["B"], pr["r"])
    return pr, ct


def test_tiny_config_all_methods_agree_and_decrypt():
    # 16 x 16 by 16 x 16, 4-bit A and B (the tiny workload).
    pr, ct = _problem(I.SEED_BASE + 1, 16, 16, 16, 4, msg_bits=4)
    ref = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    sb, _ = O.schoolbook(pr["A"], ct, 4)
    assert (sb == ref).all()
    for k in (1, 2, 3, 5):
        cu, _ = O.cussen(pr["A"], ct, 4, k)
        assert (cu == ref).all(), k
    AB = pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)
    assert (O.decrypt(pr["sk"], ref, 16 * 15 * 15) == AB).all()


def test_brute_force_repeated_addition():
    pr, ct = _problem(41, 3, 4, 2, 3)
    m, n, l = 3, 4, 2
    want = np.zeros((m, l, 2, 16), dtype=np.uint32)
    for i in range(m):
        for j in range(l):
            for c in range(2):
                acc = np.zeros(16, dtype=np.uint32)
                for k in range(n):
                    for _ in range(int(pr["A"][i, k])):
                        acc = O.point_add(acc, ct[k, j, c])
                want[i, j, c] = acc
    sb, _ = O.schoolbook(pr["A"], ct, 3)
    cu, _ = O.cussen(pr["A"], ct, 3, 1)
    assert (sb == want).all() and (cu == want).all()


@pytest.mark.parametrize("w", [1, 2, 8])
def test_bit_widths_and_ragged_strips(w):
    pr, ct = _problem(50 + w, 9, 7, 3, w)
    ref = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    for k in (1, 2, 3):
        if w * k > 24:
            continue
        cu, _ = O.cussen(pr["A"], ct, w, k)
        assert (cu == ref).all()
    sb, _ = O.schoolbook(pr["A"], ct, w)
    assert (sb == ref).all()


@pytest.mark.parametrize("w", [9, 12, 16])
def test_wide_values_agree_with_closed_form(w):
    # The paper's t = 12 and 16 grid (Section 4): entries of A up to 16 bits.
    pr, ct = _problem(80 + w, 14, 9, 3, w)
    assert pr["A"].dtype == np.uint16 and int(pr["A"].max()) >= 1 << (w - 1)
    ref = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    cu, _ = O.cussen(pr["A"], ct, w, 1)
    assert (cu == ref).all()
    if 2 * w <= 24:
        assert (O.cussen(pr["A"], ct, w, 2)[0] == ref).all()
    sb, _ = O.schoolbook(pr["A"], ct, w)
    assert (sb == ref).all()
    AB = pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)
    assert (O.decrypt(pr["sk"], ref[:2], 9 * ((1 << w) - 1) * 255) == AB[:2]).all()


def test_wide_values_duplicates_and_extremes():
    # Columns mixing zeros, 1, 2^16 - 1 and repeated mid values, next to a
    # column of distinct values: every compression level is exercised.
    rng = np.random.default_rng(90)
    m, n, l, w = 40, 6, 2, 16
    A = rng.choice(np.array([0, 1, 2, 0x8000, 0xFFFE, 0xFFFF], dtype=np.uint16), size=(m, n))
    A[:, 3] = np.arange(m, dtype=np.uint16) * 1637 + 3
    pr = I.pcmm_problem(91, m, n, l, 8)
    H = O.keygen(pr["sk"])
    ct = O.encrypt(H, pr["B"], pr["r"])
    ref = O.closed_form(A, pr["r"], pr["sk"], pr["B"])
    assert (O.cussen(A, ct, w, 1)[0] == ref).all()
    assert (O.schoolbook(A, ct, w)[0] == ref).all()
    with pytest.raises(O.OracleError):
        O.cussen(A, ct, 15, 1)          # 0xFFFF does not fit in 15 bits


def test_degenerate_shapes_and_zero_matrix():
    pr, ct = _problem(61, 1, 1, 1, 4)
    ref = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    assert (O.cussen(pr["A"], ct, 4, 1)[0] == ref).all()
    assert (O.schoolbook(pr["A"], ct, 4)[0] == ref).all()
    pr, ct = _problem(62, 4, 5, 3, 4)
    Z = np.zeros_like(pr["A"])
    assert (O.cussen(Z, ct, 4, 2)[0] == 0).all()
    assert (O.schoolbook(Z, ct, 4)[0] == 0).all()
    # Empty output (m = 0) is valid.
    out, _ = O.cussen(np.zeros((0, 5), np.uint8), ct, 4, 1)
    assert out.shape == (0, 3, 2, 16)


def _crafted(seed, m, n, l, w, mode):
    """Enc(B) replaced by points u_kj G with chosen discrete logs so that the
    expected product is (sum_k a_ik u_kj) G, checked by base multiplication."""
    rng = np.random.default_rng(seed)
    A = rng.integers(0, 2**w, size=(m, n), dtype=np.uint8)
    u = np.zeros((n, l, 2), dtype=object)
    for k in range(n):
        for j in range(l):
            for c in range(2):
                if mode == "equal":
                    u[k, j, c] = 1 + c              # every ciphertext is the same point
                elif mode == "cancel":
                    u[k, j, c] = (5 + j) if k % 2 == 0 else Q - (5 + j)   # P, -P alternate
                else:
                    u[k, j, c] = int(rng.integers(1, 2**20))
    pts = O.base_mul(np.stack([O.int_to_words(int(v)) for v in u.ravel()])).reshape(n, l, 2, 16)
    if mode == "cancel":
        A[:, 1::2] = A[:, 0::2][:, : A[:, 1::2].shape[1]]   # a_i,2t+1 = a_i,2t
    want_s = np.zeros((m, l, 2), dtype=object)
    for i in range(m):
        for j in range(l):
            for c in range(2):
                want_s[i, j, c] = sum(int(A[i, k]) * int(u[k, j, c]) for k in range(n)) % Q
    want = O.base_mul(np.stack([O.int_to_words(int(v)) for v in want_s.ravel()])).reshape(m, l, 2, 16)
    return A, pts, want


@pytest.mark.parametrize("mode", ["equal", "cancel", "small"])
def test_exceptional_additions(mode):
    A, pts, want = _crafted(7, 6, 6, 2, 3, mode)
    for k in (1, 2):
        assert (O.cussen(A, pts, 3, k)[0] == want).all()
    assert (O.schoolbook(A, pts, 3)[0] == want).all()
    if mode == "cancel":
        assert (want == 0).all()   # every row sums to a multiple of P + (-P)


def test_operation_counts():
    pr, ct = _problem(70, 12, 10, 3, 4)
    A, l = pr["A"], 3
    _, sbc = O.schoolbook(A, ct, 4)
    nnz = int(np.count_nonzero(A))
    assert sbc["ecsm"] == 2 * l * nnz
    # Ladder: every bit of a w-bit scalar doubles and adds once, except
    # operations on the identity (leading zero bits) which are free.
    _, cuc = O.cussen(A, ct, 4, 1)
    mults = sum(O.compress_counts(A[:, k])[0] for k in range(A.shape[1]))
    assert cuc["ecsm"] == 2 * l * mults
    # Executed reconstruction additions: one fewer per non-empty level than
    # the paper's count of non-zero entries (the first prefix element is
    # copied, not added).
    recon = 0
    for k in range(A.shape[1]):
        v = A[:, k].astype(np.int64)
        for w in range(1, 4):
            v = np.unique(v)
            d = v.copy()
            d[1:] = v[1:] - v[:-1]
            recon += max(int(np.count_nonzero(d)) - 1, 0)
            v = d
    assert cuc["recon_add"] == 2 * l * recon
    # Accumulation adds are the same for both methods with k = 1.
    assert cuc["accum_add"] == sbc["accum_add"]
