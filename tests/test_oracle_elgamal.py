"""Pins of the oracle's EC-ElGamal (Section 2.4) against OpenSSL and the
decryption identity; and of the closed form of the homomorphic linear
combination (Eq. ahe_5_elgamal) against decryption to A B."""
import random

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_14497_gb300 import inputs as I

Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551


def _openssl_mul(s):
    ec = pytest.importorskip("cryptography.hazmat.primitives.asymmetric.ec")
    nums = ec.derive_private_key(s, ec.SECP256R1()).public_key().public_numbers()
    return O.ints_to_point((nums.x, nums.y))


def test_keygen_encrypt_match_openssl():
    pr = I.pcmm_problem(17, 1, 3, 4, 4)
    sk = O.words_to_int(pr["sk"])
    H = O.keygen(pr["sk"])
    assert (H == _openssl_mul(sk)).all()
    ct = O.encrypt(H, pr["B"], pr["r"])
    for k in range(3):
        for j in range(4):
            r = O.words_to_int(pr["r"][k, j])
            b = int(pr["B"][k, j])
            assert (ct[k, j, 0] == _openssl_mul(r)).all()
            assert (ct[k, j, 1] == _openssl_mul((r * sk + b) % Q)).all()


def test_encrypt_decrypt_roundtrip():
    s = I.streams(3)
    sk = I.uniform_scalars(s["sk"], (1,))[0]
    H = O.keygen(sk)
    msg = np.array([0, 1, 2, 127, 128, 254, 255, 77], dtype=np.uint8)
    r = I.uniform_scalars(s["r"], (msg.size,))
    ct = O.encrypt(H, msg, r)
    assert (O.decrypt(sk, ct, 255) == msg).all()
    # Out-of-range messages are reported as -1, not mis-decoded.
    assert (O.decrypt(sk, ct[6:7], 100) == -1).all()


def test_homomorphic_linear_combination():
    s = I.streams(4)
    sk = I.uniform_scalars(s["sk"], (1,))[0]
    H = O.keygen(sk)
    msg = s["B"].integers(0, 256, size=5, dtype=np.uint8)
    coef = [3, 0, 15, 1, 9]
    ct = O.encrypt(H, msg, I.uniform_scalars(s["r"], (5,)))
    acc = np.zeros((2, 16), dtype=np.uint32)
    for c, e in zip(coef, ct):
        for comp in range(2):
            acc[comp] = O.point_add(acc[comp], O.ladder(c, 4, e[comp]))
    want = sum(int(c) * int(m) for c, m in zip(coef, msg))
    assert O.decrypt(sk, acc[None], 5 * 15 * 255)[0] == want


def test_closed_form_decrypts_to_plain_product():
    pr = I.pcmm_problem(23, 5, 7, 3, 4)
    C = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"])
    AB = pr["A"].astype(np.int64) @ pr["B"].astype(np.int64)
    assert (O.decrypt(pr["sk"], C, 7 * 15 * 255) == AB).all()
    # C1 of the closed form is (sum_k a_ik r_kj mod q) G, checked with OpenSSL.
    i, j = 2, 1
    s1 = sum(int(pr["A"][i, k]) * O.words_to_int(pr["r"][k, j]) for k in range(7)) % Q
    assert (C[i, j, 0] == _openssl_mul(s1)).all()
    # Sampled evaluation equals the full one.
    pairs = np.array([[4, 2], [0, 0], [2, 1]])
    Cs = O.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"], pairs=pairs)
    for p, (a, b) in enumerate(pairs):
        assert (Cs[p] == C[a, b]).all()


def test_all_zero_row_gives_infinity():
    pr = I.pcmm_problem(29, 3, 4, 2, 2)
    A = pr["A"].copy()
    A[1] = 0
    C = O.closed_form(A, pr["r"], pr["sk"], pr["B"])
    assert (C[1] == 0).all()
    assert C[0].any() or (A[0] == 0).all()


def test_input_generator_ranges():
    s = I.streams(5)
    r = I.uniform_scalars(s["r"], (2000,))
    vals = [O.words_to_int(v) for v in r]
    assert all(1 <= v < Q for v in vals)
    # Top word spans its whole range (uniform over [1, q-1], not truncated).
    top = np.array([int(v[7]) for v in r], dtype=np.float64)
    assert top.max() > 0xF0000000 and abs(top.mean() / 2**32 - 0.5) < 0.03
    pr = I.pcmm_problem(1, 8, 9, 10, 3)
    assert pr["A"].max() < 8 and pr["B"].max() < 256
    assert pr["r"].shape == (9, 10, 8)
    # Same seed, same problem.
    pr2 = I.pcmm_problem(1, 8, 9, 10, 3)
    assert (pr["A"] == pr2["A"]).all() and (pr["r"] == pr2["r"]).all()
