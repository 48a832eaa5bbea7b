"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm

P = 2**256 - 2**224 + 2**192 + 2**96 - 1
Q = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551


def device():
    import torch
    from paper_2504_14497_gb300 import build

    build.build()
    pcmm.init(0)
    return torch.device("cuda:0")


def ints_to_planar_fe(vals):
    """Python ints -> flat quad-planar words [2][count][4]."""
    words = np.stack([oracle.int_to_words(v) for v in vals])
    return pcmm.points_to_planar(words).reshape(-1)


def planar_fe_to_ints(flat, count):
    words = pcmm.planar_to_points(np.asarray(flat, dtype=np.uint32).reshape(2, count, 4))
    return [oracle.words_to_int(w) for w in words]


def encrypt_gpu(dev, pr, H=None):
    import torch

    if H is None:
        H = oracle.keygen(pr["sk"])
    tab = pcmm.keytable(H, device=dev)
    msg = torch.from_numpy(np.ascontiguousarray(pr["B"]).reshape(-1)).to(dev)
    r = pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev)
    return pcmm.encrypt_table(tab, msg, r)


def ct_from_aos(dev, ct_aos):
    """Oracle-layout ciphertexts [..., 2, 16] -> device planar words."""
    return pcmm.to_device_words(pcmm.ct_to_planar(ct_aos), dev)


def run_affine(fn, count):
    import torch

    jac = fn()
    aff = pcmm.normalize(jac, count)
    torch.cuda.synchronize()
    return pcmm.planar_to_ct(pcmm.to_host_words(aff), count)


def mismatches(got, want):
    got = got.reshape(-1, 2, 16)
    want = want.reshape(-1, 2, 16)
    return int((got != want).any(axis=(1, 2)).sum())
