"""GPU parity of the device field and group arithmetic (through the C-ABI
test entry points) against Python integers and the CPU oracle, including
weakly reduced inputs and every exceptional case of the addition laws."""
import random

import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import pcmm
from tests.gpu_common import P, Q, device, ints_to_planar_fe, planar_fe_to_ints

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def test_field_ops_vs_python_ints(dev):
    rng = random.Random(1)
    edge = [0, 1, 2, P - 1, P - 2, 2**255, 2**224, 2**96, 2**32 - 1, (P + 1) // 2]
    weak = [P, P + 1, 2**256 - 1, P + 2**200]          # [p, 2^256): weakly reduced inputs
    a = edge + weak + [rng.randrange(P) for _ in range(700)]
    b = list(reversed(a))
    count = len(a)
    A = pcmm.to_device_words(ints_to_planar_fe(a), dev)
    B = pcmm.to_device_words(ints_to_planar_fe(b), dev)
    ops = {0: lambda x, y: (x + y) % P, 1: lambda x, y: (x - y) % P, 2: lambda x, y: x * y % P,
           3: lambda x, y: x * x % P, 5: lambda x, y: x % P}
    for op, ref in ops.items():
        out = pcmm.test_field(op, A, B)
        got = planar_fe_to_ints(pcmm.to_host_words(out), count)
        for x, y, g in zip(a, b, got):
            assert g == ref(x, y), (op, hex(x), hex(y))
    nz = [v for v in a if v % P]
    Z = pcmm.to_device_words(ints_to_planar_fe(nz), dev)
    got = planar_fe_to_ints(pcmm.to_host_words(pcmm.test_field(4, Z)), len(nz))
    for x, g in zip(nz, got):
        assert g == pow(x, -1, P)


def _rand_affine(n, seed):
    rng = random.Random(seed)
    s = [rng.randrange(1, Q) for _ in range(n)]
    pts = oracle.base_mul(np.stack([oracle.int_to_words(v) for v in s]))
    return pts, s


def _to_jac_words(pt, z):
    """Affine oracle point (16 words) -> Jacobian words (24) with Z = z."""
    xy = oracle.point_to_ints(pt)
    if xy is None:
        return np.concatenate([oracle.int_to_words(1), oracle.int_to_words(1), oracle.int_to_words(0)])
    x, y = xy
    return np.concatenate([oracle.int_to_words(x * z * z % P), oracle.int_to_words(y * z**3 % P),
                           oracle.int_to_words(z)])


def test_point_ops_and_exceptional_cases(dev):
    rng = random.Random(7)
    pts, _ = _rand_affine(40, 3)
    inf = np.zeros(16, dtype=np.uint32)
    Ps, Qs = [], []
    for i in range(40):
        Ps.append(pts[i])
        Qs.append(pts[(i * 7 + 3) % 40])
    # Exceptional pairs: P + P, P + (-P), inf + P, P + inf, inf + inf.
    Ps += [pts[0], pts[1], inf, pts[2], inf]
    Qs += [pts[0], oracle.point_neg(pts[1]), pts[3], inf, inf]
    count = len(Ps)
    zs = [rng.randrange(1, P) for _ in range(count)]
    Pj = np.stack([_to_jac_words(p, z) for p, z in zip(Ps, zs)])
    Qj = np.stack([_to_jac_words(q, rng.randrange(1, P)) for q in Qs])
    Pj_d = pcmm.to_device_words(pcmm.points_to_planar(Pj).reshape(-1), dev)
    Qj_d = pcmm.to_device_words(pcmm.points_to_planar(Qj).reshape(-1), dev)
    Qa_d = pcmm.to_device_words(pcmm.points_to_planar(np.stack(Qs)).reshape(-1), dev)

    def host(out):
        return pcmm.planar_to_points(pcmm.to_host_words(out).reshape(4, count, 4))

    dbl = host(pcmm.test_point(0, Pj_d, count=count))
    madd = host(pcmm.test_point(1, Pj_d, Qa_d, count=count))
    add = host(pcmm.test_point(2, Pj_d, Qj_d, count=count))
    for i in range(count):
        assert (dbl[i] == oracle.point_dbl(Ps[i])).all(), i
        want = oracle.point_add(Ps[i], Qs[i])
        assert (madd[i] == want).all(), i
        assert (add[i] == want).all(), i


def test_small_scalar_multiplication(dev):
    pts, _ = _rand_affine(4, 11)
    ks = list(range(0, 300)) + [2**31 - 1, 2**32 - 1]
    count = len(ks)
    base = np.stack([pts[i % 4] for i in range(count)])
    Pd = pcmm.to_device_words(pcmm.points_to_planar(base).reshape(-1), dev)
    Kd = pcmm.to_device_words(np.array(ks, dtype=np.uint32), dev)
    out = pcmm.planar_to_points(pcmm.to_host_words(pcmm.test_point(3, Pd, k=Kd, count=count)).reshape(4, count, 4))
    for i, k in enumerate(ks):
        assert (out[i] == oracle.scalar_mul(k, base[i])).all(), k
