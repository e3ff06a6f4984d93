"""Pins of the paper's own core U = C^+ X R^+ (Algorithm 1 step 3) in the
oracle, by facts that do not depend on the oracle: it is the least-squares
core (no U gives a smaller ||X - C U R||_F, a property of orthogonal
projectors); C C^+ is an orthogonal projector of the kept rank (Penrose
conditions); the real special case equals the same product formed with
numpy's SVD; and with rank(W) = rank(X) it equals W^+ (Lemma 1).
"""
import numpy as np

from oracle import qmcur as O
from oracle import quat as Q
from paper_2402_19147_gb300 import synth


def _noisy(m, n, k, seed, noise=1e-2):
    return synth.lowrank_gaussian(m, n, k, seed=seed, noise_rel=noise, dtype=np.float64)[0]


def _cur(A, c, r, seed):
    out = O.qmcur(A, c, r, sampler=O.SAMPLER_UNIFORM, seed=seed)
    return out["C"], out["R"], out


def test_least_squares_core():
    A = _noisy(50, 60, 5, seed=31)
    C, R, out = _cur(A, 12, 10, seed=2)
    Up = O.core_paper(A, C, R)
    res = lambda U: Q.fro2(A - O.reconstruct(C, U, R))
    r0 = res(Up)
    assert r0 <= res(out["U"]) * (1 + 1e-12)          # the intersection core W^+
    rng = np.random.default_rng(3)
    for _ in range(5):
        E = rng.standard_normal(Up.shape)
        assert r0 < res(Up + 1e-3 * np.linalg.norm(Up) / np.linalg.norm(E) * E)


def test_truncated_projector_of_kept_rank():
    A = _noisy(64, 48, 4, seed=32)
    C, R, _ = _cur(A, 16, 14, seed=4)
    Cp = O.pinv_truncated(C, 1e-13, 4)[0]
    P = Q.qmatmul(C, Cp)
    assert np.max(np.abs(Q.qmatmul(P, P) - P)) < 1e-10
    assert np.max(np.abs(Q.conj_transpose(P) - P)) < 1e-10
    assert abs(np.trace(P[0]) - 4.0) < 1e-10           # Re tr of a projector = its rank


def test_real_case_equals_numpy():
    m, n, k = 40, 36, 3
    rng = np.random.default_rng(33)
    Xr = rng.standard_normal((m, k)) @ rng.standard_normal((k, n)) + 1e-2 * rng.standard_normal((m, n))
    A = np.zeros((4, m, n))
    A[0] = Xr
    C, R, _ = _cur(A, 10, 9, seed=5)

    def pk(M):
        P, s, Vh = np.linalg.svd(M, full_matrices=False)
        return (Vh[:k].T / s[:k]) @ P[:, :k].T
    Up = O.core_paper(A, C, R, rank_cap=k)
    ref = pk(C[0]) @ Xr @ pk(R[0])
    assert np.max(np.abs(Up[0] - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(Up[1:])) < 1e-12 * np.max(np.abs(ref))


def test_truncated_core_equals_intersection_pinv_at_exact_rank():
    A, _ = synth.lowrank_gaussian(60, 50, 6, seed=34, dtype=np.float64)
    C, R, out = _cur(A, 14, 15, seed=6)
    Up = O.core_paper(A, C, R, rank_cap=6)
    assert np.linalg.norm(Up - out["U"]) <= 1e-8 * np.linalg.norm(out["U"])
