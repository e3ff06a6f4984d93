"""Pins of the Algorithm 2 oracle (quaternion matrix completion, Example 4.4).

Each check is fixed by the algorithm's definition or by a textbook routine,
not by the oracle itself: the observed entries never move; an all-observed
mask is a fixed point; an exactly low-rank iterate with rank(W) = rank(X) is
a fixed point (exact CUR recovery, Lemma 1); in the real and complex special
cases a step equals the same step written with numpy's SVD on real / complex
matrices; on an exactly low-rank matrix with missing entries the iteration
recovers them; and the loop stops by the stated rule.
"""
import numpy as np
import pytest

from oracle import qmcur as O
from paper_2402_19147_gb300 import synth


def _noisy(m, n, k, seed, noise=1e-2):
    X, _ = synth.lowrank_gaussian(m, n, k, seed=seed, noise_rel=noise, dtype=np.float64)
    return X


def _sets(m, n, c, r, seed):
    J, _ = O.sample(np.full(n, 1.0 / n), c, seed, 0, 0, O.SAMPLER_UNIFORM)
    I, _ = O.sample(np.full(m, 1.0 / m), r, seed, 0, 1, O.SAMPLER_UNIFORM)
    return I, J


def _truncated_pinv(W, k):
    """Rank-k pseudo-inverse of a real or complex matrix by numpy's SVD."""
    P, s, Vh = np.linalg.svd(W, full_matrices=False)
    return (Vh[:k].conj().T / s[:k]) @ P[:, :k].conj().T


def test_observed_entries_never_change():
    m, n, k = 70, 90, 4
    Y = _noisy(m, n, k, seed=1)
    mask = synth.bernoulli_mask(m, n, seed=2, p_observed=0.4)
    I, J = _sets(m, n, 20, 18, seed=3)
    X = np.where(mask[None] != 0, Y, 0.0)
    for _ in range(4):
        X, delta, _, _, _ = O.complete_step(X, mask, I, J, rank_cap=k)
        assert np.array_equal(X[:, mask != 0], Y[:, mask != 0])
        assert delta > 0


def test_all_observed_mask_is_a_fixed_point():
    m, n = 40, 50
    Y = _noisy(m, n, 3, seed=4)
    mask = np.ones((m, n), dtype=np.uint8)
    I, J = _sets(m, n, 10, 12, seed=5)
    X, delta, num2, den2, _ = O.complete_step(Y, mask, I, J, rank_cap=3)
    assert np.array_equal(X, Y) and delta == 0.0 and num2 == 0.0
    assert den2 == pytest.approx(np.sum(Y * Y), rel=1e-14)


def test_exact_low_rank_iterate_is_a_fixed_point():
    # rank(W) = rank(X) makes C W^+ R = X (Lemma 1), so nothing changes
    m, n, k = 64, 72, 5
    X, _ = synth.lowrank_gaussian(m, n, k, seed=6, dtype=np.float64)
    mask = synth.bernoulli_mask(m, n, seed=7, p_observed=0.5)
    I, J = _sets(m, n, 16, 15, seed=8)
    Xn, delta, _, _, rank = O.complete_step(X, mask, I, J)
    assert rank == k
    assert delta < 1e-12
    assert np.max(np.abs(Xn - X)) < 1e-11 * np.max(np.abs(X))


def test_real_case_equals_numpy_real_step():
    m, n, k = 50, 60, 4
    rng = np.random.default_rng(9)
    Xr = rng.standard_normal((m, k)) @ rng.standard_normal((k, n)) + 1e-2 * rng.standard_normal((m, n))
    X = np.zeros((4, m, n))
    X[0] = Xr
    mask = synth.bernoulli_mask(m, n, seed=10, p_observed=0.5)
    I, J = _sets(m, n, 14, 13, seed=11)
    Xn, delta, _, _, _ = O.complete_step(X, mask, I, J, rank_cap=k)
    M = Xr[:, J] @ _truncated_pinv(Xr[np.ix_(I, J)], k) @ Xr[I, :]
    ref = np.where(mask != 0, Xr, M)
    assert np.max(np.abs(Xn[0] - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(Xn[1:])) < 1e-12 * np.max(np.abs(ref))   # rounding of the adjoint SVD
    assert delta == pytest.approx(np.linalg.norm(ref - Xr) / np.linalg.norm(Xr), rel=1e-10)


def test_complex_case_equals_numpy_complex_step():
    # planes (real, i) span a copy of the complex numbers inside H
    m, n, k = 48, 56, 3
    rng = np.random.default_rng(12)
    L = rng.standard_normal((m, k)) + 1j * rng.standard_normal((m, k))
    Rt = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    Xc = L @ Rt + 1e-2 * (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n)))
    X = np.zeros((4, m, n))
    X[0], X[1] = Xc.real, Xc.imag
    mask = synth.bernoulli_mask(m, n, seed=13, p_observed=0.6)
    I, J = _sets(m, n, 12, 12, seed=14)
    Xn, _, _, _, _ = O.complete_step(X, mask, I, J, rank_cap=k)
    M = Xc[:, J] @ _truncated_pinv(Xc[np.ix_(I, J)], k) @ Xc[I, :]
    ref = np.where(mask != 0, Xc, M)
    assert np.max(np.abs((Xn[0] + 1j * Xn[1]) - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(Xn[2:])) < 1e-12 * np.max(np.abs(ref))


def test_recovers_missing_entries_of_an_exactly_low_rank_matrix():
    m, n, k = 60, 80, 3
    Xt, _ = synth.lowrank_gaussian(m, n, k, seed=15, dtype=np.float64)
    mask = synth.bernoulli_mask(m, n, seed=16, p_observed=0.6)
    out = O.complete(Xt, mask, 12, 12, sampler=O.SAMPLER_UNIFORM, seed=17, rank_cap=k,
                     tol=1e-12, t_max=400)
    miss = mask == 0
    err = np.linalg.norm((out["X"] - Xt)[:, miss]) / np.linalg.norm(Xt[:, miss])
    assert err < 1e-6
    h = out["history"]
    assert h[-1] < h[0] * 1e-3


def test_stopping_rule():
    m, n, k = 40, 44, 3
    Y = _noisy(m, n, k, seed=18)
    mask = synth.bernoulli_mask(m, n, seed=19, p_observed=0.5)
    # tol 0 is met only by an exact fixed point: the loop runs t = 0 .. t_max
    out = O.complete(Y, mask, 12, 12, rank_cap=k, tol=0.0, t_max=3)
    assert out["iters"] == 4 and all(d > 0 for d in out["history"])
    # an all-observed input stops after its first iteration (delta = 0)
    out = O.complete(Y, np.ones((m, n), dtype=np.uint8), 12, 12, rank_cap=k, tol=1e-4)
    assert out["iters"] == 1 and out["history"] == [0.0]
