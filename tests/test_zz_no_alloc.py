"""The allocation-free entry point pcmm_cussen_static, for callers that may
not allocate device memory (a plug-in handed only its buffers by a framework
that owns the device pool, a loop that cannot take an allocation's implicit
synchronisation), against the workspace entry point pcmm_cussen.

Both compute the same PC-MM; outputs are compared bit for bit after affine
normalisation, on two calls in a row (the shared static scratch keeps the
previous call's contents, which must not leak into the next result).
pcmm_cussen is compared with the oracle in the other GPU tests."""
import ctypes

import numpy as np
import pytest

from paper_2504_14497_gb300 import inputs, pcmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PCMM_EUNSUPPORTED = 5


@pytest.fixture(scope="module")
def dev():
    from paper_2504_14497_gb300 import build

    build.build()
    pcmm.init(0)
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def _static_entry():
    fn = pcmm.lib().pcmm_cussen_static
    vp, ci = ctypes.c_void_p, ctypes.c_int
    fn.argtypes = [vp, ci, ci, ci, vp, ci, vp, ci, vp, vp]
    fn.restype = ci
    return fn


def _problem(dev, seed, m, n, l, w):
    pr = inputs.pcmm_problem(seed, m, n, l, w)
    H = pcmm.public_key(pr["sk"], device=dev)
    tab = pcmm.keytable(H, device=dev)
    msg = torch.from_numpy(pr["B"].reshape(-1)).to(dev)
    r = pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev)
    ctB = pcmm.encrypt_table(tab, msg, r)
    A = torch.from_numpy(pr["A"]).to(dev)
    return A, ctB


def _affine(jac, count):
    aff = pcmm.normalize(jac, count)
    torch.cuda.synchronize()
    return pcmm.to_host_words(aff)


def _call(fn, A, m, n, w, ctB, l, out, k, status):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sp = ctypes.c_void_p(status.data_ptr()) if status is not None else ctypes.c_void_p(0)
    return fn(ctypes.c_void_p(A.data_ptr()), m, n, w, ctypes.c_void_p(ctB.data_ptr()), l,
              ctypes.c_void_p(out.data_ptr()), k, sp, stream)


@pytest.mark.parametrize("m,n,l,w,k", [(16, 16, 16, 4, 2), (70, 37, 45, 8, 1), (64, 96, 40, 2, 0),
                                       (1024, 1024, 256, 8, 1)])
def test_static_entry_matches_workspace_entry(dev, m, n, l, w, k):
    """Two calls in a row through the C ABI, each bit-identical to
    pcmm_cussen with a status word of 0.  The last shape is the largest the
    32 MiB scratch is documented to hold (one strip per pass).  Around the
    second call the device's free memory must not shrink: a library
    allocation would take at least one 2 MiB page of the pool."""
    A, ctB = _problem(dev, 4242 + m + n + l, m, n, l, w)
    want = _affine(pcmm.cussen(A, ctB, l, w, k=k), m * l)
    fn = _static_entry()
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for call in range(2):
        out = torch.full((48 * m * l,), -1, dtype=torch.int32, device=dev)
        status.fill_(-1)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc = _call(fn, A, m, n, w, ctB, l, out, k, status)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert rc == 0, pcmm.status_string(rc)
        assert int(status.item()) == 0
        if call == 1:
            assert free0 - free1 < (1 << 21), f"device free memory fell by {free0 - free1} bytes"
        got = _affine(out, m * l)
        assert np.array_equal(got, want), f"call {call}: outputs differ"


def test_static_entry_reports_out_of_range_plaintext(dev):
    """An entry of A at or above 2^w sets bit 1 of the status word, which
    the call hands back although its scratch is private to the library."""
    m, n, l, w = 24, 20, 9, 4
    A, ctB = _problem(dev, 991, m, n, l, w)
    A[3, 5] = 200
    fn = _static_entry()
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    out = torch.empty(48 * m * l, dtype=torch.int32, device=dev)
    assert _call(fn, A, m, n, w, ctB, l, out, 1, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    A[3, 5] = 7
    assert _call(fn, A, m, n, w, ctB, l, out, 1, status) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_static_entry_rejects_problems_beyond_its_scratch(dev):
    """1024 x 1024 by 1024 x 4096 at w = 8 needs far more than 32 MiB per
    pass.  The buffers have the problem's true sizes (A 1 MiB, Enc(B)
    512 MiB, C 768 MiB), so a regressed size check would compute into valid
    memory rather than past it; C must stay untouched."""
    m, n, l, w = 1024, 1024, 4096, 8
    fn = _static_entry()
    A = torch.zeros((m, n), dtype=torch.uint8, device=dev)
    ctB = torch.zeros(32 * n * l, dtype=torch.int32, device=dev)
    out = torch.full((48 * m * l,), -1, dtype=torch.int32, device=dev)
    status = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    rc = _call(fn, A, m, n, w, ctB, l, out, 1, status)
    assert rc == PCMM_EUNSUPPORTED
    assert "unsupported" in pcmm.status_string(rc)
    torch.cuda.synchronize()
    assert bool((out == -1).all())          # nothing was launched
    assert int(status.item()) == 12345
    with pytest.raises(pcmm.PcmmError) as e:
        pcmm.cussen_static(A, ctB, l, w, k=1, out=out)
    assert e.value.status == PCMM_EUNSUPPORTED
    del A, ctB, out
    torch.cuda.empty_cache()


def test_static_binding_matches_workspace_entry(dev):
    m, n, l, w = 33, 20, 17, 4
    A, ctB = _problem(dev, 777, m, n, l, w)
    want = _affine(pcmm.cussen(A, ctB, l, w, k=2), m * l)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    got = _affine(pcmm.cussen_static(A, ctB, l, w, k=2, status=status), m * l)
    assert np.array_equal(got, want)
    assert int(status.item()) == 0
