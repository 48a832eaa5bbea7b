"""The debug-bounds build (-DPCMM_DEBUG_BOUNDS): on a clean plan its results
equal the product library's and its status word stays 0; on a plan whose
row ranks, tracking pointers or (k = 2) tuple components were overwritten
with indices one past the table they select from, it raises the bounds bit
(8) in the status word and skips the access.  The corrupted indices are chosen so that even an
unchecked access would stay inside the workspace.  Runs in a child process
that loads the debug library through PCMM_LIBRARY."""
import json
import os
import subprocess
import sys

import pytest

from paper_2504_14497_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_LIB = os.path.join(ROOT, "_build", "libpcmm_debug.so")

CHILD = r"""
import json
import numpy as np
import torch
from oracle import oracle
from paper_2504_14497_gb300 import inputs, pcmm
from tests.gpu_common import encrypt_gpu, mismatches, run_affine
from tests.layout_mirror import NLEV, layout

assert pcmm.LIB_PATH.endswith("libpcmm_debug.so"), pcmm.LIB_PATH
pcmm.init(0)
dev = torch.device("cuda:0")
m, n, l, w, k = 40, 6, 40, 8, 1
pr = inputs.pcmm_problem(4242, m, n, l, w)
ctB = encrypt_gpu(dev, pr)
A = torch.from_numpy(pr["A"]).to(dev)
want = oracle.closed_form(pr["A"], pr["r"], pr["sk"], pr["B"]).reshape(m * l, 2, 16)
L = layout(m, n, w, k, l)
out = {}

def run(corrupt):
    plan = pcmm.Plan(A, w, k)
    torch.cuda.synchronize()
    b = plan.buf.cpu().numpy()
    corrupt(b)
    plan.buf.copy_(torch.from_numpy(b))
    got = run_affine(lambda: plan.execute(ctB, l), m * l)
    return pcmm.workspace_status(plan.buf), mismatches(got, want)

out["clean"] = run(lambda b: None)
out["product"] = mismatches(run_affine(lambda: pcmm.cussen(A, ctB, l, w, k=k), m * l), want)

# A row rank one past the strip's last table entry (still below emax, so
# the table slot exists).
s = 2

def bad_rank(b):
    nent = int(b[L["nent"]:L["nent"] + 4 * L["nstrips"]].view(np.int32)[s])
    assert nent < L["emax"], (nent, L["emax"])
    rank = b[L["rank"]:L["rank"] + 2 * L["nstrips"] * m].view(np.uint16).reshape(L["nstrips"], m)
    i = int(np.nonzero(rank[s] != 0xFFFF)[0][0])
    rank[s, i] = nent
out["rank"] = run(bad_rank)

# A level-1 tracking pointer one past level 2 (level 2 has at most l2max
# entries and the level-2 scratch is followed by more scratch).
def bad_ptr(b):
    lens = b[L["len"]:L["len"] + 2 * n * NLEV].view(np.uint16).reshape(n, NLEV)
    ptr = b[L["ptr"]:L["ptr"] + 2 * n * L["ptr_stride"]].view(np.uint16).reshape(n, L["ptr_stride"])
    assert lens[3, 0] > 0 and lens[3, 1] <= L["l2max"]
    ptr[3, 0] = lens[3, 1]
out["ptr"] = run(bad_ptr)

# k = 2: a tuple component mapped one past its column's table (the column
# tables of a strip are followed by more scratch of the same warp).
m2, n2, l2, w2, k2 = 40, 6, 40, 4, 2
pr2 = inputs.pcmm_problem(4343, m2, n2, l2, w2)
ct2 = encrypt_gpu(dev, pr2)
A2 = torch.from_numpy(pr2["A"]).to(dev)
L2 = layout(m2, n2, w2, k2, l2)

def bad_tuple(b):
    lens = b[L2["len"]:L2["len"] + 2 * n2 * NLEV].view(np.uint16).reshape(n2, NLEV)
    r1 = b[L2["rank1"]:L2["rank1"] + n2 * 256].reshape(n2, 256)
    col = 1
    v = int(pr2["A"][0, col])
    v = v if v else int(pr2["A"][:, col].max())
    assert v and lens[col, 0] <= L2["n1max"]
    r1[col, v] = lens[col, 0]

plan2 = pcmm.Plan(A2, w2, k2)
torch.cuda.synchronize()
b2 = plan2.buf.cpu().numpy()
bad_tuple(b2)
plan2.buf.copy_(torch.from_numpy(b2))
run_affine(lambda: plan2.execute(ct2, l2), m2 * l2)
out["tuple"] = [pcmm.workspace_status(plan2.buf), 0]
want2 = oracle.closed_form(pr2["A"], pr2["r"], pr2["sk"], pr2["B"]).reshape(m2 * l2, 2, 16)
ws2 = pcmm.workspace(m2, n2, l2, w2, k2, device=dev)
got2 = run_affine(lambda: pcmm.cussen(A2, ct2, l2, w2, k=k2, ws=ws2), m2 * l2)
out["clean_k2"] = [pcmm.workspace_status(ws2), mismatches(got2, want2)]
print("RESULT " + json.dumps(out))
"""


def test_debug_bounds_flags_bad_plan_indices():
    build.build()
    build.build(extra_flags=["-DPCMM_DEBUG_BOUNDS"], lib_path=DEBUG_LIB)
    env = dict(os.environ, PCMM_LIBRARY=DEBUG_LIB)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    line = [x for x in p.stdout.splitlines() if x.startswith("RESULT ")][-1]
    r = json.loads(line[len("RESULT "):])
    assert r["clean"] == [0, 0]
    assert r["product"] == 0
    assert r["rank"][0] & 8
    assert r["ptr"][0] & 8
    assert r["tuple"][0] & 8
    assert r["clean_k2"] == [0, 0]
