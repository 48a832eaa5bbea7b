"""Pins of the oracle's field (mod p) and scalar-field (mod q) arithmetic
against Python's independent big-integer arithmetic (brute force)."""
import random

import pytest

from oracle import oracle as O

P = 2**256 - 2**224 + 2**192 + 2**96 - 1  # Section 4.1
Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551


def _miller_rabin(n, rounds=40, seed=7):
    rng = random.Random(seed)
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for _ in range(rounds):
        a = rng.randrange(2, n - 2)
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def test_constants_match_paper_formula_and_are_prime():
    c = O.constants()
    assert c["p"] == P
    assert c["q"] == Q
    assert _miller_rabin(P) and _miller_rabin(Q)
    assert not _miller_rabin(P + 2)  # the test itself can say "composite"
    # Hasse bound: |q - (p + 1)| <= 2 sqrt(p) (cofactor 1 curve).
    assert (Q - (P + 1)) ** 2 <= 4 * P


EDGE = [0, 1, 2, 3, 2**32 - 1, 2**32, 2**64 - 1, 2**128, 2**224, 2**255]


@pytest.mark.parametrize("which,mod", [("p", P), ("q", Q)])
def test_mod_ops_vs_python_ints(which, mod):
    rng = random.Random(2504)
    vals = [v % mod for v in EDGE] + [mod - 1, mod - 2, mod // 2]
    vals += [rng.randrange(mod) for _ in range(60)]
    for a in vals:
        b = rng.choice(vals)
        assert O.mod_op(which, "add", a, b) == (a + b) % mod
        assert O.mod_op(which, "sub", a, b) == (a - b) % mod
        assert O.mod_op(which, "sub", b, a) == (b - a) % mod
        assert O.mod_op(which, "mul", a, b) == (a * b) % mod
        if a:
            inv = O.mod_op(which, "inv", a)
            assert inv == pow(a, -1, mod)
            assert inv * a % mod == 1


def test_mod_ops_reject_unreduced_operands():
    with pytest.raises(O.OracleError):
        O.mod_op("p", "add", P, 1)
    with pytest.raises(O.OracleError):
        O.mod_op("q", "inv", 0)
