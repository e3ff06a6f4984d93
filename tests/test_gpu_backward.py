"""Backward of the masked CUR loss on the GPU against the FP64 oracle gradient,
and directional finite differences through the autograd Function.

Tolerances: the library computes at FP32 level (the large GEMMs, K up to n,
in the six-product BF16 split on the tensor cores; the small ones in FP32),
so its gradient is compared with the FP64 oracle gradient at relative
Frobenius 1e-4 (the rank-60 workload: see its bound);
FP32 central differences (h = 1e-4 relative to the entry scale) carry
truncation ~5e-4 and rounding ~u32 L / h, hence 1e-2 on directional
derivatives.
"""
import numpy as np
import pytest
import torch

from oracle import grad as G
from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import dev, host, rel_fro

pytestmark = pytest.mark.gpu


def _case(m, n, c, r, k, smooth, seed):
    if smooth:
        A = synth.smooth_color(m, n, k // 3, seed, offset=0.0, clip=False, max_freq=96,
                               distinct=True, bounded_amp=True, dtype=np.float64)
    else:
        A, _ = synth.lowrank_gaussian(m, n, k, seed, dtype=np.float64)
    J, _ = O.sample(np.full(n, 1.0 / n), c, seed, 0, 0, O.SAMPLER_UNIFORM)
    I, _ = O.sample(np.full(m, 1.0 / m), r, seed, 0, 1, O.SAMPLER_UNIFORM)
    A = synth.perturb_off_intersection(A, I, J, 1e-2, seed + 1).astype(np.float32)
    mask = synth.bernoulli_mask(m, n, seed + 2)
    return A, I, J, mask


def _gpu_grad(A, I, J, mask, k, method=Q.PINV_SUBSPACE_FP32):
    A_t = dev(A).requires_grad_(True)
    J_t = torch.from_numpy(J.astype(np.int32)).cuda()
    I_t = torch.from_numpy(I.astype(np.int32)).cuda()
    m_t = dev(mask)
    loss = Q.MaskedCURLoss.apply(A_t, J_t, I_t, m_t, k, 1e-10, method)
    (g,) = torch.autograd.grad(loss, A_t)
    return float(loss.item()), host(g), (A_t, J_t, I_t, m_t)


@pytest.mark.parametrize("m,n,c,r,k", [(64, 72, 10, 12, 4), (130, 97, 24, 20, 6)])
def test_backward_matches_oracle_small(m, n, c, r, k):
    A, I, J, mask = _case(m, n, c, r, k, False, m + n)
    loss, g, _ = _gpu_grad(A, I, J, mask, k)
    lo, go = G.masked_loss_grad(A.astype(np.float64), I, J, mask, 1e-10, k)
    assert abs(loss - lo) <= 1e-4 * lo
    assert rel_fro(g, go) < 1e-4


@pytest.mark.parametrize("method", [Q.PINV_JACOBI_FP64, Q.PINV_SUBSPACE_FP32])
def test_backward_differentiable_workload(method):
    # 1024 x 1536 pure quaternion field of rank 60, c = r = 120, rank cap 60,
    # 50% Bernoulli mask; the loss is evaluated off the intersection's
    # perturbation so that it is nonzero while W keeps rank 60.  The backward
    # forms (I - W U), (I - U W) and products cubic in U, so its rounding
    # grows like u kappa(W_k)^2, u the error of one real product.  Its six
    # large products run in the six-product BF16 split, which drops the
    # order-3 piece products x1 y2, x2 y1, x2 y2 (pieces of 8 bits each): up
    # to 3 * 2^-24 |x y| per real product against 2^-24 for an FP32 FMA.  The
    # bound is max(1e-4, 48 u32 kappa^2).
    m, n, c, r, k = 1024, 1536, 120, 120, 60
    A, I, J, mask = _case(m, n, c, r, k, True, 4)
    loss, g, (A_t, J_t, I_t, m_t) = _gpu_grad(A, I, J, mask, k, method)
    lo, go = G.masked_loss_grad(A.astype(np.float64), I, J, mask, 1e-10, k)
    sw = O.qsvd_values(A[:, I][:, :, J].astype(np.float64))
    kappa = sw[0] / sw[k - 1]
    tol = max(1e-4, 48 * 2.0 ** -24 * kappa * kappa)
    assert abs(loss - lo) <= 1e-4 * lo
    assert rel_fro(g, go) < tol
    # Directional central differences through the forward (FP32).  At this
    # point FP64 central differences with h = 1e-3 max|A| are themselves 5%
    # off (truncation, converging as h^2: 5e-4 at 1e-4, 5e-6 at 1e-5), so
    # the FP32 check uses h = 1e-4 max|A|: truncation ~5e-4, rounding
    # ~u32 L / h ~ 1e-3, bound 1e-2.
    rng = np.random.default_rng(7)
    h = 1e-4 * float(np.max(np.abs(A)))
    for _ in range(8):
        D = rng.standard_normal(A.shape).astype(np.float32)
        D_t = dev(D)
        with torch.no_grad():
            lp = float(Q.MaskedCURLoss.apply(A_t + h * D_t, J_t, I_t, m_t, k, 1e-10, method).item())
            lm = float(Q.MaskedCURLoss.apply(A_t - h * D_t, J_t, I_t, m_t, k, 1e-10, method).item())
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(g.astype(np.float64) * D))
        assert abs(fd - an) <= 1e-2 * max(abs(an), 1e-3 * lo), (fd, an)
