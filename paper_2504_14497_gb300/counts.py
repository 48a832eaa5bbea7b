"""Host-side accounting of the point operations a PC-MM launch performs.

Used to turn measured times into rates (point additions per second) and
roofline fractions.  It recomputes, from the plaintext matrix A alone, the
compression plan the plan kernel builds (same definitions), and counts the
group operations of two finite points that the table and gather kernels
execute for the l useful output columns.  It does no curve arithmetic and is
not on the compute path.

Per-operation integer work, in 32x32->64-bit limb products (a field
multiplication is 64 products, a squaring 36; P-256 special-form reduction
needs none), each product costing two IMAD instructions (low and high word):
    mixed addition    (madd-2007-bl, 7M + 4S)   592 products
    mixed addition into an accumulator kept as (X, Y, Z^2, Z^3) (gather,
      level-1 chains; 8M + 2S: Z^2 and Z^3 updated with H^2 and H^3)  584 products
    full addition     (add-2007-bl, 11M + 5S)   884 products
    doubling, a = -3  (dbl-2001-b, 3M + 5S)     372 products
    normalisation of one level-2 entry (3M for simultaneous inversion,
      then 1S + 3M for x = X Z^-2, y = Y Z^-3)  420 products
    normalisation of one level-1 chain entry (the chain kept as (X, Y,
      Z^2, Z^3); Z^-2 and Z^-3 walked backwards along the chain's factors
      H^2, H^3, 2M, then x = X Z^-2, y = Y Z^-3, 2M)  256 products
    affine addition inside a batch (3M for the shared inversion, then
      1M + 1S + 1M for the slope, x3, y3)       356 products
"""
from __future__ import annotations

import numpy as np

N_ITER = 4
L2_CHAIN_MIN = 32   # level-2 lengths from which the table kernel builds level 2 as a chain
PRODUCTS = {"madd": 592, "madd_acc": 584, "add": 884, "dbl": 372, "norm": 420, "norm_chain": 256,
            "affine": 356}
IMAD_PER_PRODUCT = 2


def _levels(col: np.ndarray, N: int = N_ITER):
    """Lengths of levels 1..N and the level-N values of one column."""
    v = np.unique(col[col != 0]).astype(np.int64)
    lens = [len(v)]
    for _ in range(1, N):
        d = np.diff(v, prepend=0) if len(v) else v
        v = np.unique(d)
        lens.append(len(v))
    return lens, v


def cussen_counts(A: np.ndarray, w: int, k: int, l: int, N: int = N_ITER) -> dict:
    """Operations of one Cussen PC-MM for the l useful output columns (both
    ciphertext components), as the table and gather kernels perform them:

    * ``table_dbl``/``table_ecsm_madd``: double-and-add of the level-N values;
    * ``table_add``: prefix sums of levels N-1..2 (Jacobian + Jacobian;
      N-1..3 when level 2 has at least L2_CHAIN_MIN entries);
    * ``table_madd``: level-1 prefix sums (and those of a long level 2)
      over affine addends;
    * ``table_affine``: k-tuple sums, affine additions sharing one inversion
      per round;
    * ``table_norm``: level-2 entries (level-3 entries when level 2 is
      long) normalised to affine by simultaneous inversion;
    * ``table_norm_chain``: chain entries (level 1: the column tables when
      k > 1, the strip tables when k = 1; a long level 2) normalised along
      their chain's ratios;
    * ``gather_madd``: accumulations of table entries into the outputs.
    Additions with an identity operand are copies and are not counted."""
    A = np.asarray(A).astype(np.int64) & ((1 << w) - 1)
    m, n = A.shape
    chains = 2 * l
    tadd = tmadd = tdbl = tecsm = norm = nchain = taff = 0
    nnz_rows = np.zeros(m, dtype=np.int64)
    for s0 in range(0, n, k):
        cols = A[:, s0:s0 + k]
        kw = cols.shape[1]
        codes = np.zeros(m, dtype=np.int64)
        for t in range(kw):
            codes |= cols[:, t] << (w * t)
            lens, vN = _levels(cols[:, t], N)
            for v in vN:
                v = int(v)
                tdbl += chains * (v.bit_length() - 1)
                tecsm += chains * (bin(v).count("1") - 1)
            tmadd += chains * max(lens[0] - 1, 0)
            if N > 2 and lens[1] >= L2_CHAIN_MIN:
                # long level 2: a chain of mixed additions over level 3
                # normalised to affine, itself normalised along its ratios
                tadd += chains * sum(max(x - 1, 0) for x in lens[2:-1])
                tmadd += chains * max(lens[1] - 1, 0)
                norm += chains * lens[2]
                nchain += chains * lens[1]
            else:
                tadd += chains * sum(max(x - 1, 0) for x in lens[1:-1])
                norm += chains * (lens[1] if N > 1 else 0)
            if kw > 1:
                nchain += chains * lens[0]
        distinct = np.unique(codes[codes != 0])
        if kw > 1:
            for code in distinct:
                parts = sum(1 for t in range(kw) if (int(code) >> (w * t)) & ((1 << w) - 1))
                taff += chains * max(parts - 1, 0)
        else:
            nchain += chains * len(distinct)
        nnz_rows += codes != 0
    gather = chains * int(np.maximum(nnz_rows - 1, 0).sum())
    return {"gather_madd": gather, "table_add": tadd, "table_madd": tmadd, "table_dbl": tdbl,
            "table_ecsm_madd": tecsm, "table_norm": norm, "table_norm_chain": nchain,
            "table_affine": taff}


def point_ops(c: dict) -> int:
    """Point additions and doublings of two finite points performed."""
    return (c["gather_madd"] + c["table_add"] + c["table_madd"] + c["table_dbl"]
            + c["table_ecsm_madd"] + c["table_affine"])


def gather_imad(c: dict) -> int:
    return c["gather_madd"] * PRODUCTS["madd_acc"] * IMAD_PER_PRODUCT


def table_imad(c: dict) -> int:
    p = (c["table_add"] * PRODUCTS["add"]
         + c["table_madd"] * PRODUCTS["madd_acc"] + c["table_ecsm_madd"] * PRODUCTS["madd"]
         + c["table_dbl"] * PRODUCTS["dbl"] + c["table_norm"] * PRODUCTS["norm"]
         + c["table_norm_chain"] * PRODUCTS["norm_chain"]
         + c["table_affine"] * PRODUCTS["affine"])
    return p * IMAD_PER_PRODUCT


def schoolbook_counts(A: np.ndarray, l: int) -> dict:
    """Double-and-add per non-zero entry, then one full addition per term
    after the first in each output."""
    A = np.asarray(A).astype(np.int64)
    nz = A[A != 0]
    bl = np.floor(np.log2(nz)).astype(np.int64) if nz.size else np.zeros(0, np.int64)
    pc = np.array([bin(int(v)).count("1") for v in nz], dtype=np.int64) if nz.size else np.zeros(0, np.int64)
    chains = 2 * l
    rows_nnz = (A != 0).sum(axis=1)
    return {"dbl": chains * int(bl.sum()), "madd": chains * int((pc - 1).sum()),
            "add": chains * int(np.maximum(rows_nnz - 1, 0).sum())}


def strassen_counts(A: np.ndarray, w: int, levels: int, l: int) -> dict:
    """Point operations of pcmm_strassen (Section 3.1) for the l output
    columns, both ciphertext components: per recursion step the ciphertext
    block sums (five mixed additions per position of a quadrant of Enc(B))
    and the combination (eight full additions per position of a quadrant of
    C); at the leaves, per non-zero signed block-sum entry a and output
    column, the double-and-add of |a| (bitlen - 1 doublings, popcount - 1
    additions) and one addition into the output after a row's first term.
    The block sums of A are recomputed here exactly as the kernels form
    them."""
    blocks = (np.asarray(A).astype(np.int64) & ((1 << w) - 1))[None]
    csum = comb = 0
    for t in range(levels):
        nodes, mp, np_ = blocks.shape
        mh, nh, lh = mp // 2, np_ // 2, (l >> t) // 2
        a11, a12 = blocks[:, :mh, :nh], blocks[:, :mh, nh:]
        a21, a22 = blocks[:, mh:, :nh], blocks[:, mh:, nh:]
        blocks = np.stack([a11 + a22, a21 + a22, a11, a22, a11 + a12, a21 - a11, a12 - a22],
                          axis=1).reshape(nodes * 7, mh, nh)
        csum += 2 * nodes * 5 * nh * lh
        comb += 2 * nodes * 8 * mh * lh
    ld = l >> levels
    a = np.abs(blocks)
    nz = a[a != 0]
    bl = np.zeros(nz.shape, dtype=np.int64)
    pc = np.zeros(nz.shape, dtype=np.int64)
    for b in range(16):
        bit = (nz >> b) & 1
        pc += bit
        bl = np.where(bit == 1, b, bl)
    rows_nnz = (a != 0).sum(axis=2)
    chains = 2 * ld
    return {"leaf_dbl": chains * int(bl.sum()), "leaf_madd": chains * int((pc - 1).sum()),
            "leaf_add": chains * int(np.maximum(rows_nnz - 1, 0).sum()), "block_madd": csum, "block_add": comb}


def strassen_point_ops(c: dict) -> int:
    return c["leaf_dbl"] + c["leaf_madd"] + c["leaf_add"] + c["block_madd"] + c["block_add"]


def strassen_equiv(n: int, t: int) -> int:
    """The paper's equivalent point additions of Strassen PC-MM of square
    n x n matrices recursed to single entries (Sections 3.1 and 3.3)."""
    mults, adds, k = 1, 0, 1
    while k < n:
        adds = 7 * adds + 13 * k * k
        mults *= 7
        k *= 2
    return 4 * t * mults + 2 * adds


def naf4(x: int) -> list:
    """Width-4 non-adjacent form of x >= 0, least significant digit first
    (digits in {0, +-1, +-3, +-5, +-7}): the recoding the decryption kernel's
    scalar multiplication uses."""
    d = []
    while x > 0:
        if x & 1:
            r = x & 15
            r = r - 16 if r >= 8 else r
            x -= r
        else:
            r = 0
        d.append(r)
        x >>= 1
    return d


def decrypt_products(sk: int, msgs: np.ndarray, baby: int) -> float:
    """Limb products per decryption, averaged over the messages (all in
    range): the odd multiples of C1 (a doubling, three full additions, three
    normalisations), x C1 (a doubling per NAF digit below the top, a mixed
    addition per non-zero digit), M = C2 - x C1 (one mixed addition and a
    normalisation), one giant step (mixed addition and normalisation) per
    multiple of baby below m, and the check of the hit j G (one mixed
    addition per non-zero byte of j; two multiplications and a squaring)."""
    d = naf4(int(sk))
    scalar = (len(d) - 1) * PRODUCTS["dbl"] + sum(1 for x in d if x) * PRODUCTS["madd"]
    pre = PRODUCTS["dbl"] + 3 * PRODUCTS["add"] + 3 * PRODUCTS["norm"]
    m = np.asarray(msgs, dtype=np.int64).reshape(-1)
    steps = (m // baby).astype(np.float64)
    j = m % baby
    jbytes = sum(((j >> (8 * b)) & 255) != 0 for b in range(3)).astype(np.float64)
    per = (pre + scalar + PRODUCTS["madd"] + PRODUCTS["norm"]
           + steps * (PRODUCTS["madd"] + PRODUCTS["norm"]) + jbytes * PRODUCTS["madd"] + 2 * 64 + 36)
    return float(per.mean())
