"""Pins of the oracle's P-256 group law and scalar multiplication against
OpenSSL (through the ``cryptography`` package) and against group-law
invariants (Section 2.3)."""
import random

import numpy as np
import pytest

from oracle import oracle as O

P = 2**256 - 2**224 + 2**192 + 2**96 - 1
Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551
INF = np.zeros(16, dtype=np.uint32)


def _on_curve_py(pt):
    xy = O.point_to_ints(pt)
    if xy is None:
        return True
    x, y = xy
    b = O.constants()["b"]
    return (y * y - (x * x * x - 3 * x + b)) % P == 0


def _openssl_mul(s):
    ec = pytest.importorskip("cryptography.hazmat.primitives.asymmetric.ec")
    nums = ec.derive_private_key(s, ec.SECP256R1()).public_key().public_numbers()
    return O.ints_to_point((nums.x, nums.y))


def test_generator_on_curve_and_order():
    G = O.generator()
    assert _on_curve_py(G)
    assert O.on_curve(G)
    assert (O.scalar_mul(Q, G) == 0).all()              # q G = infinity
    assert (O.scalar_mul(Q - 1, G) == O.point_neg(G)).all()
    assert (O.scalar_mul(Q + 1, G) == G).all()
    assert (O.scalar_mul(0, G) == 0).all()


def test_generator_matches_openssl():
    assert (O.generator() == _openssl_mul(1)).all()


def test_scalar_mul_matches_openssl():
    rng = random.Random(11)
    scal = [1, 2, 3, 255, 256, Q - 1, Q - 2, 2**128 + 1] + [rng.randrange(1, Q) for _ in range(12)]
    words = np.stack([O.int_to_words(s) for s in scal])
    base = O.base_mul(words)
    for s, pb in zip(scal, base):
        ref = _openssl_mul(s)
        assert (pb == ref).all()
        assert (O.scalar_mul(s, O.generator()) == ref).all()
    # s (u G) = (s u mod q) G for a non-generator base point.
    u = rng.randrange(1, Q)
    U = _openssl_mul(u)
    for s in scal[:6]:
        assert (O.scalar_mul(s, U) == _openssl_mul(s * u % Q)).all()


def _rand_points(k, seed):
    rng = random.Random(seed)
    s = [rng.randrange(1, Q) for _ in range(k)]
    return O.base_mul(np.stack([O.int_to_words(v) for v in s])), s


def test_group_law_invariants():
    pts, s = _rand_points(6, 5)
    Pp, Qp, Rp = pts[0], pts[1], pts[2]
    assert (O.point_add(Pp, Qp) == O.point_add(Qp, Pp)).all()
    lhs = O.point_add(O.point_add(Pp, Qp), Rp)
    rhs = O.point_add(Pp, O.point_add(Qp, Rp))
    assert (lhs == rhs).all()
    assert (O.point_add(Pp, O.point_neg(Pp)) == 0).all()
    assert (O.point_add(Pp, INF) == Pp).all()
    assert (O.point_add(INF, Pp) == Pp).all()
    assert (O.point_add(INF, INF) == 0).all()
    assert (O.point_dbl(Pp) == O.point_add(Pp, Pp)).all()
    assert (O.point_dbl(INF) == 0).all()
    for X in (lhs, O.point_dbl(Pp), O.point_add(Pp, Qp)):
        assert _on_curve_py(X)
    # Sums agree with OpenSSL on the scalar side.
    assert (O.point_add(Pp, Qp) == _openssl_mul((s[0] + s[1]) % Q)).all()
    assert (O.point_dbl(Rp) == _openssl_mul(2 * s[2] % Q)).all()


def test_off_curve_point_is_detected():
    G = O.generator().copy()
    G[8] ^= 1
    assert not O.on_curve(G)
    bad = O.int_to_words(P)  # x = p is not reduced
    with pytest.raises(O.OracleError):
        O.point_add(np.concatenate([bad, bad]), O.generator())


def test_montgomery_ladder_matches_double_and_add():
    pts, _ = _rand_points(2, 9)
    for Pp in pts:
        for t in range(1, 6):
            for k in range(0, 2**t):
                assert (O.ladder(k, t, Pp) == O.scalar_mul(k, Pp)).all()
        rng = random.Random(3)
        for _ in range(8):
            k = rng.randrange(256)
            assert (O.ladder(k, 8, Pp) == O.scalar_mul(k, Pp)).all()
    with pytest.raises(O.OracleError):
        O.ladder(16, 4, pts[0])  # k needs 5 bits


def test_comb_base_mul_matches_bitwise_sum_and_openssl():
    # The closed form's fixed-base comb (8-bit windows, one shared inversion
    # per window) against the bit-by-bit sum of 2^i G and OpenSSL: random
    # scalars, scalars with zero bytes, and scalars >= q (s = q: the last
    # window adds -acc, a vanishing sum).
    rng = random.Random(21)
    scal = [0, 1, 2, 255, 256, 2**248, 2**255, Q - 1, Q, Q + 1, Q - 2**248, 2**256 - 1, Q + 2**200]
    scal += [rng.randrange(0, Q) & ~(0xFF << (8 * rng.randrange(32))) for _ in range(40)]
    scal += [rng.randrange(0, 2**256) for _ in range(300)]
    words = np.stack([O.int_to_words(s) for s in scal])
    comb = O.base_mul_comb(words)
    assert (comb == O.base_mul(words)).all()
    for s, pt in zip(scal[:16], comb[:16]):
        if s % Q:
            assert (pt == _openssl_mul(s % Q)).all()
        else:
            assert (pt == 0).all()
    # Chunks of 256 scalars: a ragged last chunk, and equal scalars in one
    # chunk (identical accumulators share the window's inversion).
    many = np.repeat(words[:7], 60, axis=0)
    assert (O.base_mul_comb(many) == np.repeat(comb[:7], 60, axis=0)).all()
