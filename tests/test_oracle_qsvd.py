"""Pins of the oracle's truncated QSVD (Example 4.2's comparator): the
Eckart-Young identity ||X - X_k||_F^2 = sum_{i>k} sigma_i^2 with the
singular values of the real representation, the real special case against
numpy's real SVD, the rank of X_k, and X_k = X at exact rank."""
import numpy as np

from oracle import qmcur as O
from oracle import quat as Q
from paper_2402_19147_gb300 import synth


def _real_rep(X):
    # the real 4m x 4n block representation of the Hamilton product, whose
    # singular values are those of X, each four times
    X0, X1, X2, X3 = X
    return np.block([[X0, -X1, -X2, -X3], [X1, X0, -X3, X2], [X2, X3, X0, -X1], [X3, -X2, X1, X0]])


def test_eckart_young_identity():
    X, _ = synth.lowrank_gaussian(40, 30, 8, seed=71, noise_rel=1e-2, dtype=np.float64)
    s_real = np.linalg.svd(_real_rep(X), compute_uv=False)[0::4]
    for k in (1, 4, 8, 12):
        Xk, kk, _ = O.qsvd_truncated(X, k)
        assert kk == k
        assert abs(Q.fro2(X - Xk) - np.sum(s_real[k:] ** 2)) < 1e-10 * Q.fro2(X)
        assert abs(Q.fro2(Xk) - np.sum(s_real[:k] ** 2)) < 1e-10 * Q.fro2(X)


def test_real_case_equals_numpy():
    rng = np.random.default_rng(72)
    Xr = rng.standard_normal((25, 18))
    X = np.zeros((4, 25, 18))
    X[0] = Xr
    P, s, Vh = np.linalg.svd(Xr, full_matrices=False)
    Xk, _, _ = O.qsvd_truncated(X, 5)
    assert np.max(np.abs(Xk[0] - (P[:, :5] * s[:5]) @ Vh[:5])) < 1e-12
    assert np.max(np.abs(Xk[1:])) < 1e-12


def test_rank_and_exact_recovery():
    X, _ = synth.lowrank_gaussian(36, 44, 6, seed=73, dtype=np.float64)
    Xk, k, sig = O.qsvd_truncated(X, 6)
    assert k == 6 and np.max(np.abs(Xk - X)) < 1e-11 * np.max(np.abs(X))
    X3, _, _ = O.qsvd_truncated(X, 3)
    assert np.count_nonzero(O.qsvd_values(X3) > 1e-10 * sig[0]) == 3
