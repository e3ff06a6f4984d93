"""Host-side checks of the Python binding that need no GPU: arguments that the
binding refuses before it queues any work or touches a CUDA stream."""
import pytest
import torch

from paper_2402_19147_gb300 import qmcur as Q


def test_decompose_many_refuses_a_capped_method_without_a_cap():
    # the subspace pseudo-inverse needs rank_cap >= 1; the check comes before
    # any stream is made, so CPU tensors suffice to see it
    A = torch.zeros(4, 8, 8)
    with pytest.raises(ValueError):
        Q.decompose_many([A], [object()], [0], pinv_method=Q.PINV_SUBSPACE_FP32, rank_cap=0)


def test_decompose_many_refuses_mismatched_lists():
    with pytest.raises(ValueError):
        Q.decompose_many([torch.zeros(4, 2, 2)], [], [0])


def test_decompose_many_empty_is_a_no_op():
    Q.decompose_many([], [], [])
