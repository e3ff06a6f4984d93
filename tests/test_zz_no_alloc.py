"""qmcur_probs_noalloc: the allocation-free variant of qmcur_probs.

It serves callers that cannot call cudaMalloc or pass a workspace (a host
framework that owns all device memory, or a latency-bound loop where an
allocation, which may synchronise the device, is not allowed).  Its scratch is
a static device array in the library, shared by all calls on a device.  This
test calls it through the C ABI twice in a row (different shapes, so the
second call runs on scratch left over from the first) and checks each result
against the workspace entry point qmcur_probs within the probabilities
tolerance of the parity tests (24 u32 relative, FP32 input).  It must pass
alone in a fresh process as well as after every other test.
"""
import numpy as np
import pytest
import torch

from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL = 24 * 2.0 ** -24


def _outputs(m, n):
    f = dict(dtype=torch.float64, device="cuda")
    return torch.empty(n, **f), torch.empty(m, **f), torch.empty(1, **f)


@pytest.mark.parametrize("sampler", [Q.SAMPLER_NORM, Q.SAMPLER_UNIFORM])
def test_noalloc_matches_workspace_entry_point(sampler):
    assert torch.cuda.is_available()
    for m, n, seed in ((700, 1500, 1), (2048, 333, 2)):
        A = torch.from_numpy(synth.lowrank_gaussian(m, n, 5, seed=seed, noise_rel=0.1)[0]).cuda()
        col_ref, row_ref, fro_ref = _outputs(m, n)
        st_ref = Q.status_tensor()
        Q.probs(A, sampler, col_ref, row_ref, fro_ref, Q.workspace(m, n, 1, 1, Q.PREC_FP32), st_ref)
        col, row, fro = _outputs(m, n)
        st = Q.status_tensor()
        Q.probs_noalloc(A, sampler, col, row, fro, st)
        torch.cuda.synchronize()
        assert int(st_ref.item()) == 0 and int(st.item()) == 0
        for got, ref in ((col, col_ref), (row, row_ref), (fro, fro_ref)):
            assert np.allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=RTOL, atol=0)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    # 8192 x 8192 needs about 17 MiB of scratch: refused before any launch
    A = torch.zeros(4, 8192, 8192, dtype=torch.float32, device="cuda")
    col, row, fro = _outputs(8192, 8192)
    with pytest.raises(Q.QmcurError) as e:
        Q.probs_noalloc(A, Q.SAMPLER_NORM, col, row, fro, Q.status_tensor())
    assert e.value.code == 7        # QMCUR_ERR_UNSUPPORTED
