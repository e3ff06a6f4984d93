"""The truncated QSVD comparator (Example 4.2) on the GPU against the
oracle's qsvd_truncated: FP64 one-sided Jacobi against LAPACK on the complex
adjoint, relative Frobenius 1e-11 (both backward stable; the gap
sigma_k / sigma_{k+1} of these inputs is large, so the truncated part is
well determined), both orientations (the Jacobi runs on X^H when n > m)."""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import dev, host, rel_fro, run_status

pytestmark = pytest.mark.gpu


# columns of up to 512 rows are rotated in registers, longer ones streamed:
# 512 and 513 rows sit on either side, 700 and the wide 40 x 640 stream
@pytest.mark.parametrize("m,n,k", [(120, 90, 5), (70, 130, 6), (500, 500, 10), (512, 40, 4),
                                   (513, 40, 4), (700, 60, 5), (40, 640, 4)])
def test_qsvd_truncated_matches_oracle(m, n, k):
    X, _ = synth.lowrank_gaussian(m, n, k, seed=m + n, noise_rel=1e-3, dtype=np.float64)
    B = torch.empty(4, m, n, dtype=torch.float64, device="cuda")
    rk = torch.zeros(2, dtype=torch.int32, device="cuda")
    sig = torch.empty(min(m, n), dtype=torch.float64, device="cuda")
    st = Q.status_tensor()
    Q.qsvd_truncated(dev(X), B, k, rank_out=rk, sigma_out=sig, status=st)
    assert run_status(st) == 0
    Bo, ko, so = O.qsvd_truncated(X, k)
    assert int(rk[0]) == ko == k
    assert rel_fro(host(B), Bo) < 1e-11
    assert np.max(np.abs(host(sig) - so) / so[0]) < 1e-12
