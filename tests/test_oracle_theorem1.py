"""Example 4.1 on the oracle: Theorem 1's perturbation bound for the paper's
core, and the linear growth of the error with the noise.

X = W_k Sigma_k V_k^H (m = 500, k = 50, orthonormal quaternion columns,
singular values in [100, 1000] so that every noise level stays in the
perturbation regime ||E||_2 < sigma_k(X)),
X~ = X + E with Gaussian E of standard deviation sigma = 1e-1 .. 1e-6, c = r =
100 uniformly drawn columns and rows of X~, and the error
||X - C~ C~^+ X~ R~^+ R~||_2.  Theorem 1 bounds it by
||E||_2 (||W_k(I,:)^+||_2 + ||V_k(J,:)^+||_2 + 3); Example 4.1 reports that it
grows linearly with ||E||_2.  Spectral norms are the largest quaternion
singular value (the SVD of the complex adjoint), independent of the CUR code.
"""
import numpy as np

from oracle import qmcur as O
from oracle import quat as Q
from paper_2402_19147_gb300 import synth

M, K, C, R = 500, 50, 100, 100
SIGMAS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6]


def spec(A):
    return float(O.qsvd_values(A)[0])


def sweep():
    X, Wk, Vk, _ = synth.svd_lowrank(M, M, K, seed=51, smin=100.0, smax=1000.0)
    J, _ = O.sample(np.full(M, 1.0 / M), C, 52, 0, 0, O.SAMPLER_UNIFORM)
    I, _ = O.sample(np.full(M, 1.0 / M), R, 52, 0, 1, O.SAMPLER_UNIFORM)
    gW = 1.0 / O.qsvd_values(Wk[:, I, :])[K - 1]     # ||W_k(I,:)^+||_2
    gV = 1.0 / O.qsvd_values(Vk[:, J, :])[K - 1]     # ||V_k(J,:)^+||_2
    rows = []
    for t, s in enumerate(SIGMAS):
        Xt = X + synth.gaussian_noise(M, M, s, seed=60 + t)
        Ct, Rt, _ = O.gather(Xt, I, J)
        Z = O.reconstruct(Ct, O.core_paper(Xt, Ct, Rt), Rt)
        e, nE = spec(X - Z), spec(Xt - X)
        rows.append((s, nE, e, nE * (gW + gV + 3.0)))
    return rows


def test_theorem1_bound_and_linear_growth():
    rows = sweep()
    ratios = []
    for s, nE, e, bound in rows:
        assert e <= bound, (s, e, bound)
        ratios.append(e / nE)
    med = float(np.median(ratios))
    assert all(0.5 * med <= q <= 2.0 * med for q in ratios), ratios
    # and the noise norm itself scales with sigma: the complex adjoint of a
    # square Gaussian quaternion matrix is a 2m x 2m complex Gaussian matrix
    # with entries of variance 2 sigma^2, so ||E||_2 ~ 2 sqrt(2m) sqrt(2) sigma
    for s, nE, _, _ in rows:
        assert 3.6 * np.sqrt(M) * s < nE < 4.4 * np.sqrt(M) * s
