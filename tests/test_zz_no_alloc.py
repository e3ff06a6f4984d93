"""qmcur_probs_noalloc: the allocation-free variant of qmcur_probs.

It serves callers that cannot call cudaMalloc or pass a workspace (a host
framework that owns all device memory, or a latency-bound loop where an
allocation, which may synchronise the device, is not allowed).  Its scratch is
a static device array in the library, shared by all calls on a device.  This
test calls it through the C ABI twice in a row (different shapes, so the
second call runs on scratch left over from the first) and checks each result
against the workspace entry point qmcur_probs.  Both entry points run the
same kernels with the same fixed reduction order, so the results must agree
bit for bit.  It also checks the entry point's one promise: after a warm-up
call (which may load the kernels' module), a further call changes neither
torch's allocated bytes nor the device's free memory.  It must pass alone in
a fresh process as well as after every other test.
"""
import numpy as np
import pytest
import torch

from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth

pytestmark = pytest.mark.gpu

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
            assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_allocates_nothing():
    m, n = 1024, 768
    A = torch.from_numpy(synth.lowrank_gaussian(m, n, 4, seed=3, noise_rel=0.1)[0]).cuda()
    col, row, fro = _outputs(m, n)
    st = Q.status_tensor()
    Q.probs_noalloc(A, Q.SAMPLER_NORM, col, row, fro, st)   # warm-up: module load
    torch.cuda.synchronize()
    first = col.clone()
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    Q.probs_noalloc(A, Q.SAMPLER_NORM, col, row, fro, st)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    assert int(st.item()) == 0
    assert torch.equal(col, first)


def test_noalloc_uniform_without_norm_takes_any_size():
    # no ||A||_F^2 asked for: nothing is read and no scratch is needed
    m, n = 8192, 8192
    A = torch.zeros(4, m, n, dtype=torch.float32, device="cuda")
    col, row, _ = _outputs(m, n)
    st = Q.status_tensor()
    Q.probs_noalloc(A, Q.SAMPLER_UNIFORM, col, row, None, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert torch.all(col == 1.0 / n) and torch.all(row == 1.0 / m)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    # 8192 x 8192 needs about 17 MiB of scratch: refused before any launch
    A = torch.zeros(4, 8192, 8192, dtype=torch.float32, device="cuda")
    col, row, fro = _outputs(8192, 8192)
    with pytest.raises(Q.QmcurError) as e:
        Q.probs_noalloc(A, Q.SAMPLER_NORM, col, row, fro, Q.status_tensor())
    assert e.value.code == 7        # QMCUR_ERR_UNSUPPORTED
