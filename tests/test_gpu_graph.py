"""A whole decomposition (qmcur_decompose: probabilities, index draws and
gathers, the core, the GEMMs and the residual) captured in a CUDA graph and
replayed: every call is stream-ordered, with no host synchronisation or copy,
so a replay reproduces the eager run bit for bit on the live input buffer."""
import numpy as np
import pytest
import torch

from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth

pytestmark = pytest.mark.gpu


def _outputs(D):
    return [t.clone() for t in (D.J, D.I, D.U, D.rank, D.out3, D.status)]


@pytest.mark.parametrize("method", [Q.PINV_REFINED_FP64, Q.PINV_JACOBI_FP64,
                                    Q.PINV_SUBSPACE_FP32],
                         ids=["refined", "jacobi", "subspace"])
def test_decomposition_replays_from_a_cuda_graph(method):
    m, n, c, r, k = 384, 320, 48, 40, 8
    inputs = [torch.from_numpy(synth.lowrank_gaussian(m, n, k, seed=s, noise_rel=1e-3,
                                                      dtype=np.float32)[0]).cuda()
              for s in (11, 12)]
    A = torch.empty_like(inputs[0])
    D = Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED)
    kw = dict(sampler=Q.SAMPLER_NORM, seed=5, rank_cap=k, pinv_method=method)

    # eager references (this also loads every kernel before the capture)
    want = []
    for X in inputs:
        A.copy_(X)
        D.status.zero_()
        Q.decompose(A, D, **kw)
        torch.cuda.synchronize()
        assert int(D.status.item()) == 0
        want.append(_outputs(D))

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        Q.decompose(A, D, stream=s, **kw)
    torch.cuda.synchronize()

    for X, ref in zip(inputs, want):
        A.copy_(X)
        D.status.zero_()
        g.replay()
        torch.cuda.synchronize()
        for got, exp in zip(_outputs(D), ref):
            assert torch.equal(got, exp)
