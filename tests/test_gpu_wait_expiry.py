"""A bounded device-side wait that runs out (failure detection without a
GPU fault).

The staged SpMV engines wait on an mbarrier for each tile's bulk copies,
with a cycle limit; a wait that runs out sets the solve's error flag, lets
the block's copies in flight land (a second wait with the full bound) and
returns, and pcg_solve reports AFSAI_ETIMEOUT.  Here a child process pins
the staged-tile engines (AFSAI_SPMV_MODES=101,101,101) and sets the first
wait's limit to zero (AFSAI_WAIT_CYCLES=0: one non-blocking check of the
copies just issued), so a tile gives up before its copies land: the solve
must return ETIMEOUT, and the context must stay usable (an afsai_apply, an
afsai_spmv and a torch operation after it give correct results).  Every
wait of the expiry path is itself bounded, so nothing here can hang."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2010_14175_gb300 import afsai, matgen as mg
afsai.load()
A = mg.poisson7(16)
b, _ = mg.rhs(A, 3)
Ad = afsai.DeviceCSR.from_host(A)
M = afsai.afsai_setup(Ad, afsai.params(5, 2, 1e-3))
bd = torch.from_numpy(b).cuda()
x = torch.zeros_like(bd)
out = {}
try:
    afsai.pcg_solve(Ad, M, bd, x, rtol=1e-8, maxit=1000)
    out["status"] = 0
except afsai.AfsaiError as e:
    out["status"] = e.status
    out["msg"] = str(e)
torch.cuda.synchronize()
# the context still works: products through the library and torch
r = np.random.default_rng(1).standard_normal(A.n)
y = torch.zeros(A.n, dtype=torch.float64, device="cuda")
afsai.afsai_spmv(Ad, torch.from_numpy(r).cuda(), y)
out["spmv_err"] = float(np.max(np.abs(y.cpu().numpy() - A.to_scipy() @ r)))
rp, ci, va = M.export()
import scipy.sparse as sp
G = sp.csr_matrix((va, ci, rp), shape=(A.n, A.n))
z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
afsai.afsai_apply(M, torch.from_numpy(r).cuda(), z)
out["apply_err"] = float(np.max(np.abs(z.cpu().numpy() - G.T @ (G @ r))))
out["torch_sum"] = float(torch.arange(10, device="cuda", dtype=torch.float64).sum().item())
print(json.dumps(out))
"""


def test_wait_expiry_returns_etimeout_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_14175_gb300 import afsai

    env = dict(os.environ, AFSAI_WAIT_CYCLES="0", AFSAI_SPMV_MODES="101,101,101")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["status"] == afsai.ETIMEOUT, out
    assert "wait" in out["msg"]
    assert out["spmv_err"] <= 1e-12 and out["apply_err"] <= 1e-12
    assert out["torch_sum"] == 45.0
