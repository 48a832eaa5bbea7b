"""The allocation-free entry point pcmm_cussen_static, for callers that may
not allocate device memory, against the workspace entry point pcmm_cussen.

Both compute the same PC-MM; outputs are compared bit for bit after affine
normalisation, on two calls in a row (the shared static scratch keeps the
previous call's contents, which must not leak into the next result)."""
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
    fn.argtypes = [vp, ci, ci, ci, vp, ci, vp, ci, vp]
    fn.restype = ci
    return fn


def _problem(dev, seed, m, n, l, w):
    pr = inputs.pcmm_problem(seed, m, n, l, w)
    H = pcmm.public_key(pr["sk"], device=dev)
    tab = pcmm.keytable(H, device=dev)
    msg = torch.from_numpy(pr["B"].reshape(-1)).to(dev)
    r = pcmm.to_device_words(pcmm.scalars_to_planar(pr["r"]), dev)
    ctB = pcmm.encrypt(tab, msg, r)
    A = torch.from_numpy(pr["A"]).to(dev)
    return A, ctB


def _affine(jac, count):
    aff = pcmm.normalize(jac, count)
    torch.cuda.synchronize()
    return pcmm.to_host_words(aff)


@pytest.mark.parametrize("m,n,l,w,k", [(16, 16, 16, 4, 2), (70, 37, 45, 8, 1), (64, 96, 40, 2, 0)])
def test_static_entry_matches_workspace_entry(dev, m, n, l, w, k):
    A, ctB = _problem(dev, 4242 + m + n + l, m, n, l, w)
    want = _affine(pcmm.cussen(A, ctB, l, w, k=k), m * l)
    fn = _static_entry()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((48 * m * l,), -1, dtype=torch.int32, device=dev)
        rc = fn(ctypes.c_void_p(A.data_ptr()), m, n, w, ctypes.c_void_p(ctB.data_ptr()), l,
                ctypes.c_void_p(out.data_ptr()), k, stream)
        assert rc == 0, pcmm.status_string(rc)
        got = _affine(out, m * l)
        assert np.array_equal(got, want), f"call {call}: outputs differ"


def test_static_entry_rejects_problems_beyond_its_scratch(dev):
    fn = _static_entry()
    dummy = torch.zeros(64, dtype=torch.int32, device=dev)
    p = ctypes.c_void_p(dummy.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 1024 x 1024 by 1024 x 4096 at w = 8 needs far more than 32 MiB per pass.
    rc = fn(p, 1024, 1024, 8, p, 4096, p, 1, stream)
    assert rc == PCMM_EUNSUPPORTED
    assert "unsupported" in pcmm.status_string(rc)
    torch.cuda.synchronize()
    assert not dummy.any()      # nothing was launched


def test_static_binding_matches_workspace_entry(dev):
    m, n, l, w = 33, 20, 17, 4
    A, ctB = _problem(dev, 777, m, n, l, w)
    want = _affine(pcmm.cussen(A, ctB, l, w, k=2), m * l)
    got = _affine(pcmm.cussen_static(A, ctB, l, w, k=2), m * l)
    assert np.array_equal(got, want)
    with pytest.raises(pcmm.PcmmError) as e:
        pcmm.cussen_static(torch.zeros((1024, 1024), dtype=torch.uint8, device=dev),
                           torch.zeros(64, dtype=torch.int32, device=dev), 4096, 8, k=1,
                           out=torch.zeros(64, dtype=torch.int32, device=dev))
    assert e.value.status == PCMM_EUNSUPPORTED
