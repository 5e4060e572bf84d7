"""The dense solve with its FP64 products on the tensor cores by error-free
splitting (MPL_GEMM_SPLIT=1: A X at every order and the large Gram /
projection / update products) reaches the same eigenpairs as LAPACK at the
requested tolerance, and so do the solve with every FP64 product on the
DFMA pipe (MPL_GEMM_SPLIT=0 MPL_AX_SPLIT=0) and the solve whose FP32
factor takes its trailing updates from 3xTF32 tensor-core products
(MPL_FACTOR_TF32X3=1).  The switches are read once per
process, so each solve runs in a child process."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import U_H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import workloads as W  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2302_12528_gb300 as M, workloads as W
n, k, m, cx = int(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), sys.argv[5] == "1"
A, _ = (W.dense_hpd if cx else W.dense_spd)(n, seed=91, kappa=1e6)
X0 = W.start_block(n, m, seed=92, complex_=cx)
Om = W.sketch(n, 8, seed=93, complex_=cx)
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
h = M.create_dense(dev(W.colmajor(A)), k, m, tol=1e-12, policy="mp", Omega=dev(Om))
h.factor()
Xo = torch.empty((k, n), dtype=torch.complex128 if cx else torch.float64, device="cuda:0")
lam, _, hist, its, _ = h.solve(dev(X0), maxit=2000, X_out=Xo)
h.close()
X = Xo.cpu().numpy()
np.save(sys.argv[6], X)
print(json.dumps({"lam": [float(x) for x in lam], "its": list(map(int, its))}))
"""


@pytest.mark.parametrize("switches", [{"MPL_GEMM_SPLIT": "1"}, {"MPL_GEMM_SPLIT": "0", "MPL_AX_SPLIT": "0"},
                                      {"MPL_FACTOR_TF32X3": "1"}],
                         ids=["split", "dfma", "tf32x3-factor"])
@pytest.mark.parametrize("cx,n,k,m", [(True, 4096, 16, 96), (False, 3000, 8, 96)])
def test_split_product_solve_matches_eigh(cx, n, k, m, switches, tmp_path):
    env = dict(os.environ, **switches)
    xfile = str(tmp_path / "X.npy")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, str(n), str(k), str(m), "1" if cx else "0", xfile],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    lam = np.array(out["lam"])
    A, _ = (W.dense_hpd if cx else W.dense_spd)(n, seed=91, kappa=1e6)
    X = np.load(xfile).T
    ev = np.linalg.eigvalsh(A)
    rn = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.all(rn <= 1e-12 * (ev[-1] + np.abs(lam)) * np.linalg.norm(X, axis=0))
    gap = ev[k] - ev[k - 1]
    assert np.all(np.abs(lam - ev[:k]) <= np.maximum(1e-10 * ev[:k], 2 * rn ** 2 / gap) + 10 * U_H * ev[-1])
