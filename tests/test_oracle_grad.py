"""Pin of the oracle gradient of the masked CUR loss: central finite
differences in FP64 along random directions, on exactly low-rank inputs with
the rank cap equal to the rank (where the truncated inverse is smooth)."""
import numpy as np
import pytest

from oracle import grad as G
from paper_2402_19147_gb300 import synth


@pytest.mark.parametrize("masked", [False, True])
def test_gradient_matches_central_differences(masked):
    m, n, k, c, r = 30, 26, 3, 7, 6
    A, _ = synth.lowrank_gaussian(m, n, k, seed=31, dtype=np.float64)
    rng = np.random.default_rng(32)
    I = np.sort(rng.choice(m, r, replace=False))
    J = np.sort(rng.choice(n, c, replace=False))
    # perturb A everywhere but the intersection: W = A(I,J) keeps rank k (where
    # the fixed-rank derivative of W^+ is exact) while C and R leave W's row and
    # column spaces, so every term of the derivative of W^+ is active
    out = np.ones((m, n), dtype=bool)
    out[I[:, None], J[None, :]] = False
    A = A + 0.05 * rng.standard_normal(A.shape) * out
    mask = synth.bernoulli_mask(m, n, seed=33) if masked else None
    loss, g = G.masked_loss_grad(A, I, J, mask, rcond=1e-10, rank_cap=k)
    assert loss > 1e-3 and np.isclose(loss, G.masked_loss(A, I, J, mask, 1e-10, k))
    # central differences: truncation O(h^2) ~ 1e-9, rounding ~ eps L / h ~ 1e-9
    h = 1e-6
    for _ in range(6):
        D = rng.standard_normal(A.shape)
        fd = (G.masked_loss(A + h * D, I, J, mask, 1e-10, k) -
              G.masked_loss(A - h * D, I, J, mask, 1e-10, k)) / (2 * h)
        an = float(np.sum(g * D))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (fd, an)


def test_gradient_is_zero_at_exact_recovery_without_mask():
    # L = 0 at an exactly rank-k input whose intersection has rank k: a minimum
    A, _ = synth.lowrank_gaussian(20, 24, 2, seed=34, dtype=np.float64)
    I, J = np.arange(0, 20, 3), np.arange(1, 24, 4)
    loss, g = G.masked_loss_grad(A, I, J, None, 1e-10, 2)
    assert loss < 1e-20 and np.max(np.abs(g)) < 1e-9
