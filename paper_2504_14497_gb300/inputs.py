"""Seeded synthetic inputs for PC-MM (shared by the tests and the benchmark).

This module holds no arithmetic of the method: it only draws random numbers.
Every random quantity the method uses (secret key, encryption nonces r,
plaintext matrices A and B) is drawn here and passed to both the CUDA path
and the CPU oracle as an input.

Recipe: ``numpy.random.Generator(PCG64(SeedSequence(seed)))`` spawned into
the sub-streams [sk, A, B, r, shapes, arrivals]; A uniform over [0, 2^w),
B uniform over [0, 2^8), sk and r uniform over [1, q-1] by rejection
sampling of 256-bit words (Section 2.4 draws both from [1, q-1]).
"""
from __future__ import annotations

import numpy as np

# Order of the P-256 group (SEC 2 / FIPS 186-4), used only as the rejection
# bound of the uniform draws.
Q_ORDER = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551

SEED_BASE = 2504144970
STREAMS = ("sk", "A", "B", "r", "shapes", "arrivals")


def streams(seed: int) -> dict:
    children = np.random.SeedSequence(seed).spawn(len(STREAMS))
    return {nm: np.random.Generator(np.random.PCG64(ss)) for nm, ss in zip(STREAMS, children)}


def _q_words() -> np.ndarray:
    return np.array([(Q_ORDER >> (32 * i)) & 0xFFFFFFFF for i in range(8)], dtype=np.uint64)


def uniform_scalars(rng: np.random.Generator, shape) -> np.ndarray:
    """uint32[*shape, 8], each value uniform over [1, q-1]."""
    shape = tuple(np.atleast_1d(shape)) if not isinstance(shape, tuple) else shape
    count = int(np.prod(shape)) if shape else 1
    qw = _q_words()
    out = np.empty((count, 8), dtype=np.uint32)
    filled = 0
    while filled < count:
        need = count - filled
        cand = rng.integers(0, 1 << 32, size=(need + need // 8 + 8, 8), dtype=np.uint64)
        # Lexicographic compare against q from the most significant word down.
        less = np.zeros(cand.shape[0], dtype=bool)
        equal = np.ones(cand.shape[0], dtype=bool)
        for i in range(7, -1, -1):
            less |= equal & (cand[:, i] < qw[i])
            equal &= cand[:, i] == qw[i]
        nonzero = cand.any(axis=1)
        ok = cand[less & nonzero][:need]
        out[filled:filled + ok.shape[0]] = ok.astype(np.uint32)
        filled += ok.shape[0]
    return out.reshape(shape + (8,))


def _plaintext(gen, m: int, n: int, w: int) -> np.ndarray:
    adt = np.uint8 if w <= 8 else np.uint16
    return gen.integers(0, 1 << w, size=(m, n), dtype=adt) if m * n else np.zeros((m, n), adt)


def sparse_plaintext(seed: int, m: int, n: int, w: int, density: float) -> np.ndarray:
    """A w-bit plaintext matrix whose entries are non-zero with probability
    `density` (each independently), the non-zero values uniform over
    [1, 2^w) (for example pruned weights)."""
    if not 1 <= w <= 16 or not 0.0 <= density <= 1.0:
        raise ValueError("w must be in [1, 16] and density in [0, 1]")
    gen = streams(seed)["A"]
    adt = np.uint8 if w <= 8 else np.uint16
    vals = gen.integers(1, 1 << w, size=(m, n), dtype=adt)
    keep = gen.random(size=(m, n)) < density
    return np.where(keep, vals, 0).astype(adt)


def plaintext_matrix(seed: int, m: int, n: int, w: int) -> np.ndarray:
    """The A of pcmm_problem(seed, m, n, l, w, ...), drawn alone."""
    if not 1 <= w <= 16:
        raise ValueError("w must be in [1, 16]")
    return _plaintext(streams(seed)["A"], m, n, w)


def pcmm_problem(seed: int, m: int, n: int, l: int, w: int, msg_bits: int = 8) -> dict:
    """One PC-MM instance: plaintext A (m x n, w-bit; uint8 for w <= 8,
    uint16 for 8 < w <= 16), message matrix B (n x l, msg_bits-bit), secret
    key sk and nonces r (n x l)."""
    if not 1 <= w <= 16:
        raise ValueError("w must be in [1, 16]")
    s = streams(seed)
    sk = uniform_scalars(s["sk"], (1,))[0]
    A = _plaintext(s["A"], m, n, w)
    B = s["B"].integers(0, 1 << msg_bits, size=(n, l), dtype=np.uint8) if n * l else np.zeros((n, l), np.uint8)
    r = uniform_scalars(s["r"], (n, l))
    return {"sk": sk, "A": A, "B": B, "r": r, "m": m, "n": n, "l": l, "w": w}


def batched_shapes(seed: int, count: int = 64, lo: int = 32, hi: int = 768):
    """Shapes (m, n, l, w) of the batched workload: m, n, l uniform over
    [lo, hi], w uniform over {1..8}."""
    rng = streams(seed)["shapes"]
    dims = rng.integers(lo, hi + 1, size=(count, 3))
    ws = rng.integers(1, 9, size=count)
    return [(int(a), int(b), int(c), int(d)) for (a, b, c), d in zip(dims, ws)]
