"""The C-ABI calls in the form the boundary names them, through ctypes,
against the CPU oracle: pcmm_encrypt with the public key H on the host and a
workspace that caches its comb table (Section 2.4), pcmm_workspace_bytes
sizing a pcmm_cussen call, and pcmm_cussen_batched (Algorithm 3 over many
independent problems in one call)."""
import numpy as np
import pytest

from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import device, mismatches, run_affine

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dev():
    return device()


def _ct_host(ct, count):
    torch.cuda.synchronize()
    return pcmm.planar_to_ct(pcmm.to_host_words(ct), count)


def test_encrypt_with_host_key_and_cached_table(dev):
    """Three calls on one workspace: key 1, key 2 (the cached table must be
    rebuilt), key 1 again; each ciphertext equal to the oracle's, and equal
    to the key-table form."""
    s = inputs.streams(2024)
    sks = inputs.uniform_scalars(s["sk"], (2,))
    keys = [oracle.keygen(sk) for sk in sks]
    count = 777
    msg = (np.arange(count) * 7 % 256).astype(np.uint8)
    r = inputs.uniform_scalars(s["r"], (count,))
    dmsg = torch.from_numpy(msg).to(dev)
    dr = pcmm.to_device_words(pcmm.scalars_to_planar(r), dev)
    ws = torch.empty(pcmm.workspace_bytes(pcmm.OP_ENCRYPT, 1, 1, 1, 1), dtype=torch.uint8, device=dev)
    for call, idx in enumerate((0, 1, 0, 0)):
        got = _ct_host(pcmm.encrypt(keys[idx], dmsg, dr, ws=ws), count)
        want = oracle.encrypt(keys[idx], msg, r)
        assert mismatches(got, want) == 0, f"call {call} (key {idx})"
    # count = 0 only builds the table of key 1 (null buffers allowed); the
    # next call with that key encrypts from it.
    import ctypes
    H1 = np.ascontiguousarray(keys[1], dtype=np.uint32)
    rc = pcmm.lib().pcmm_encrypt(H1.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), None, None, 0, None,
                                 ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert mismatches(_ct_host(pcmm.encrypt(keys[1], dmsg, dr, ws=ws), count),
                      oracle.encrypt(keys[1], msg, r)) == 0
    tab = pcmm.keytable(keys[0], device=dev)
    assert mismatches(_ct_host(pcmm.encrypt_table(tab, dmsg, dr), count), want) == 0
    # Clearing the tag forces a rebuild, so a workspace overwritten by other
    # data and re-tagged by nothing still encrypts correctly.
    ws.zero_()
    assert mismatches(_ct_host(pcmm.encrypt(keys[0], dmsg, dr, ws=ws), count), want) == 0


def test_workspace_query_sizes_a_cussen_call(dev):
    m, n, l, w = 45, 30, 40, 4
    pr = inputs.pcmm_problem(6060, m, n, l, w)
    H = oracle.keygen(pr["sk"])
    ctB = pcmm.encrypt(H, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                       pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
    A = torch.from_numpy(pr["A"]).to(dev)
    want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16)
    for k in (1, 2, 0):
        nb = pcmm.workspace_bytes(pcmm.OP_CUSSEN, m, n, l, w, k)
        assert 0 < nb < pcmm.WS_INVALID
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        got = run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k, ws=ws), m * l)
        assert mismatches(got, want) == 0, k
    assert pcmm.workspace_bytes(pcmm.OP_SCHOOLBOOK, m, n, l, w) == 0
    got = run_affine(lambda: pcmm.schoolbook(A, ctB, l, w), m * l)
    assert mismatches(got, want) == 0


def test_cussen_batched_one_call(dev):
    """pcmm_cussen_batched over uneven problems: every output of every
    instance against the oracle's closed form, on two calls in a row."""
    specs = [(37, 70, 20, 3, 1), (64, 40, 45, 8, 1), (9, 33, 5, 1, 6), (50, 21, 33, 4, 2), (1, 17, 3, 2, 0)]
    items, wants = [], []
    for i, (m, n, l, w, k) in enumerate(specs):
        pr = inputs.pcmm_problem(7100 + i, m, n, l, w)
        H = oracle.keygen(pr["sk"])
        ctB = pcmm.encrypt(H, torch.from_numpy(pr["B"].reshape(-1)).to(dev),
                           pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev))
        items.append((torch.from_numpy(pr["A"]).to(dev), ctB, l, w, k))
        wants.append(oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(-1, 2, 16))
    for call in range(2):
        outs = pcmm.cussen_batched(items)
        for (A, _, l, _, _), out, want in zip(items, outs, wants):
            count = A.shape[0] * l
            got = _ct_host(pcmm.normalize(out, count), count)
            assert mismatches(got, want) == 0, call
