"""Pins of the QMCUR oracle (Algorithm 1, Sec. 3.1-3.2) against closed forms,
invariants, special cases reducing to numpy/LAPACK, brute force and statistics."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import quat as Q
from oracle import qmcur as O
from paper_2402_19147_gb300 import synth


def _rand_q(rng, m, n):
    return rng.standard_normal((4, m, n))


def _householder(rng, n):
    """Quaternion unitary I - 2 v v^H / (v^H v) for a random quaternion vector v."""
    v = _rand_q(rng, n, 1)
    vh = Q.conj_transpose(v)
    nrm = Q.fro2(v)
    H = Q.identity(n) - (2.0 / nrm) * Q.qmatmul(v, vh)
    return H


def _unitary(rng, n, reps=4):
    U = Q.identity(n)
    for _ in range(reps):
        U = Q.qmatmul(U, _householder(rng, n))
    return U


# ------------------------------------------------------------ probabilities -
def test_norms_sum_to_frobenius_and_trace():
    rng = np.random.default_rng(0)
    A = _rand_q(rng, 7, 5)
    col2, row2, F = O.squared_norms(A)
    G = Q.qmatmul(Q.conj_transpose(A), A)
    assert np.isclose(col2.sum(), F) and np.isclose(row2.sum(), F)
    assert np.isclose(Q.trace_real(G), F)
    # column squared norms are the diagonal of A^H A, row ones of A A^H
    assert np.allclose(col2, G[0].diagonal())
    assert np.allclose(row2, Q.qmatmul(A, Q.conj_transpose(A))[0].diagonal())


def test_probabilities_real_special_case_and_uniform():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((6, 9))
    A = np.zeros((4, 6, 9)); A[0] = M
    p, q, F = O.probabilities(A, O.SAMPLER_NORM)
    assert np.allclose(p, np.linalg.norm(M, axis=0) ** 2 / np.linalg.norm(M) ** 2)
    assert np.allclose(q, np.linalg.norm(M, axis=1) ** 2 / np.linalg.norm(M) ** 2)
    assert np.isclose(p.sum(), 1.0) and np.isclose(q.sum(), 1.0)
    pu, qu, _ = O.probabilities(A, O.SAMPLER_UNIFORM)
    assert np.all(pu == 1.0 / 9) and np.all(qu == 1.0 / 6)


def test_probabilities_errors():
    A = np.zeros((4, 3, 3))
    with pytest.raises(ZeroDivisionError):
        O.probabilities(A)
    A[2, 1, 1] = np.nan
    with pytest.raises(FloatingPointError):
        O.probabilities(A)


# ------------------------------------------------------------------ sampling -
@pytest.mark.parametrize("n", [1, 5, 256, 257, 1000, 4096])
def test_fixed_point_prefix_properties(n):
    rng = np.random.default_rng(n)
    p = rng.random(n)
    p[rng.random(n) < 0.2] = 0.0
    p[0] = 0.75                        # a maximum with a known exponent (e = -1)
    P, S = O.fixed_point_prefix(p)
    B = 63 - (n - 1).bit_length()
    q = np.diff(P, prepend=np.uint64(0)).astype(object)
    # the largest entry is scaled into [2^(B-1), 2^B): 0.75 -> 0.75 2^B exactly
    assert int(q[0]) == 3 << (B - 2)
    # every entry is the exact truncation p_k 2^E, E = B, checked in rationals
    for k in range(n):
        x = Fraction(p[k]) * (1 << B)
        assert int(q[k]) == x.numerator // x.denominator
    # exact integer sums: S below 2^63, P non-decreasing, zeros never drawn
    assert S == int(sum(q)) < (1 << 63) and P[-1] == S
    assert np.all(np.diff(P.astype(object)) >= 0)
    assert all(int(q[k]) == 0 for k in range(n) if p[k] == 0.0)
    # scale invariance: multiplying p by a power of two gives the same integers
    P2, S2 = O.fixed_point_prefix(p * 2.0 ** -40)
    assert np.array_equal(P2, P) and S2 == S


def test_inverse_cdf_brute_force():
    rng = np.random.default_rng(7)
    p = rng.random(300)
    p[::7] = 0.0
    P, S = O.fixed_point_prefix(p)
    for _ in range(2000):
        target = int(rng.integers(0, S))
        k = int(np.searchsorted(P, np.uint64(target), side="right"))
        lin = next(i for i in range(len(P)) if int(P[i]) > target)
        assert k == lin and p[k] > 0


def test_sample_sets_and_determinism():
    rng = np.random.default_rng(8)
    p = rng.random(500); p[::3] = 0; p /= p.sum()
    J, t = O.sample(p, 40, seed=11, stream_id=2, which=0, sampler=O.SAMPLER_NORM)
    assert len(J) == 40 and len(set(J.tolist())) == 40 and np.all(np.diff(J) > 0)
    assert np.all(p[J] > 0) and t >= 40
    J2, _ = O.sample(p, 40, seed=11, stream_id=2, which=0, sampler=O.SAMPLER_NORM)
    assert np.array_equal(J, J2)
    J3, _ = O.sample(p, 40, seed=11, stream_id=3, which=0, sampler=O.SAMPLER_NORM)
    J4, _ = O.sample(p, 40, seed=11, stream_id=2, which=1, sampler=O.SAMPLER_NORM)
    assert not np.array_equal(J, J3) and not np.array_equal(J, J4)
    Ju, _ = O.sample(np.full(97, 1 / 97), 97, seed=5, stream_id=0, which=0,
                     sampler=O.SAMPLER_UNIFORM)
    assert np.array_equal(Ju, np.arange(97))


def test_first_draw_follows_p_chi_square():
    # frequency of the first draw over many seeds matches p (chi-square, 7 dof)
    p = np.array([0.05, 0.1, 0.15, 0.2, 0.0, 0.25, 0.05, 0.1, 0.1])
    N = 20000
    counts = np.zeros(len(p))
    for s in range(N):
        J, _ = O.sample(p, 1, seed=s, stream_id=0, which=0, sampler=O.SAMPLER_NORM)
        counts[int(J[0])] += 1
    assert counts[4] == 0
    nz = p > 0
    chi2 = np.sum((counts[nz] - N * p[nz]) ** 2 / (N * p[nz]))
    assert chi2 < 24.3        # 99.9% quantile of chi-square with 7 dof


def test_uniform_draw_chi_square():
    n, N = 10, 20000
    counts = np.zeros(n)
    for s in range(N):
        x0, _, _, _ = O._draw_word(s, 1, 1, 0)
        counts[(x0 * n) >> 32] += 1
    chi2 = np.sum((counts - N / n) ** 2 / (N / n))
    assert chi2 < 27.9        # 99.9% quantile, 9 dof


def test_sample_limit_and_support():
    p = np.zeros(50); p[3] = 0.5; p[9] = 0.5 - 1e-13; p[20] = 1e-13
    with pytest.raises(RuntimeError):
        O.sample(p, 3, seed=0, stream_id=0, which=0, sampler=O.SAMPLER_NORM,
                 max_attempts=100)
    with pytest.raises(ValueError):
        O.sample(p, 4, seed=0, stream_id=0, which=0, sampler=O.SAMPLER_NORM)


# ------------------------------------------------------------------- gather -
def test_gather_consistency():
    rng = np.random.default_rng(9)
    A = _rand_q(rng, 9, 11)
    I, J = np.array([0, 4, 8]), np.array([1, 2, 10, 5])
    C, R, W = O.gather(A, I, J)
    assert C.shape == (4, 9, 4) and R.shape == (4, 3, 11) and W.shape == (4, 3, 4)
    assert np.array_equal(W, C[:, I, :]) and np.array_equal(W, R[:, :, J])
    assert C[2, 4, 2] == A[2, 4, 10]


# ------------------------------------------------------------ pseudo-inverse -
@pytest.mark.parametrize("shape", [(6, 4), (4, 6), (5, 5)])
def test_penrose_conditions(shape):
    rng = np.random.default_rng(sum(shape))
    W = _rand_q(rng, *shape)
    U, k, _ = O.pinv_truncated(W, rcond=1e-12)
    assert k == min(shape)
    WU = Q.qmatmul(W, U)
    UW = Q.qmatmul(U, W)
    assert np.allclose(Q.qmatmul(WU, W), W, atol=1e-12)
    assert np.allclose(Q.qmatmul(UW, U), U, atol=1e-12)
    assert np.allclose(WU, Q.conj_transpose(WU), atol=1e-12)
    assert np.allclose(UW, Q.conj_transpose(UW), atol=1e-12)


def test_pinv_reduces_to_numpy_real_and_complex():
    rng = np.random.default_rng(10)
    M = rng.standard_normal((7, 4))
    W = np.zeros((4, 7, 4)); W[0] = M
    U, _, _ = O.pinv_truncated(W)
    assert np.allclose(U[0], np.linalg.pinv(M)) and np.allclose(U[1:], 0)
    Mc = rng.standard_normal((4, 6)) + 1j * rng.standard_normal((4, 6))
    W = np.zeros((4, 4, 6)); W[0], W[1] = Mc.real, Mc.imag
    U, _, _ = O.pinv_truncated(W)
    P = np.linalg.pinv(Mc)
    assert np.allclose(U[0] + 1j * U[1], P) and np.allclose(U[2:], 0)


def test_truncated_pinv_closed_form():
    # W = P diag(s) V^H with known unitary P, V: the rank-k truncation keeps the
    # k largest singular triplets, U = V_k diag(1/s_k) P_k^H.
    rng = np.random.default_rng(11)
    m, n = 9, 7
    P = _unitary(rng, m)
    V = _unitary(rng, n)
    s = np.array([9.0, 5.0, 3.0, 1.0, 0.5, 1e-3, 1e-11])
    S = np.zeros((4, m, n)); S[0, :n, :n] = np.diag(s)
    W = Q.qmatmul(Q.qmatmul(P, S), Q.conj_transpose(V))
    sig = O.qsvd_values(W)
    assert np.allclose(sig, s, rtol=1e-12, atol=1e-13)
    for cap, rcond, kk in [(4, 1e-10, 4), (0, 1e-10, 6), (0, 1e-2, 5), (3, 0.0, 3)]:
        U, k, _ = O.pinv_truncated(W, rcond=rcond, rank_cap=cap)
        assert k == kk
        Dk = np.zeros((4, kk, kk)); Dk[0] = np.diag(1.0 / s[:kk])
        exact = Q.qmatmul(Q.qmatmul(V[:, :, :kk], Dk), Q.conj_transpose(P[:, :, :kk]))
        assert np.linalg.norm(U - exact) <= 1e-10 * np.linalg.norm(exact)


# --------------------------------------------------- exact recovery, Lemma 1 -
def test_exact_recovery_small():
    A, _ = synth.lowrank_gaussian(64, 48, 5, seed=12, dtype=np.float64)
    out = O.qmcur(A, 12, 12, sampler=O.SAMPLER_UNIFORM, seed=3)
    assert out["rank"] == 5
    assert out["rel"] < 1e-12


def test_exact_recovery_gauss256_rank10():
    # the FP64 workload: 256 x 256, rank 10, c = r = 40, uniform sampling
    w = synth.WORKLOADS["gauss256_rank10_fp64"]
    A = synth.make("gauss256_rank10_fp64")
    out = O.qmcur(A, w["c"], w["r"], sampler=O.SAMPLER_UNIFORM, seed=0,
                  rcond=w["rcond"])
    assert out["rank"] == 10
    assert out["rel"] < 1e-12


def test_lemma1_ranks_and_paper_core_equals_intersection_pinv():
    A, _ = synth.lowrank_gaussian(40, 30, 4, seed=13, dtype=np.float64)
    out = O.qmcur(A, 8, 9, sampler=O.SAMPLER_NORM, seed=1)
    tol = 1e-10
    rk = lambda X: int(np.count_nonzero(O.qsvd_values(X) > tol * O.qsvd_values(X)[0]))
    assert rk(A) == rk(out["C"]) == rk(out["R"]) == rk(out["W"]) == 4
    # C^+ X R^+ (Algorithm 1 step 3) equals W^+ when rank(W) = rank(X)
    Up = O.core_paper(A, out["C"], out["R"])
    assert np.linalg.norm(Up - out["U"]) <= 1e-8 * np.linalg.norm(out["U"])


def test_residual_definition():
    rng = np.random.default_rng(14)
    A = _rand_q(rng, 5, 6)
    Z = A + 1e-3 * _rand_q(rng, 5, 6)
    rel, num2, den2 = O.residual(A, Z)
    assert np.isclose(num2, Q.fro2(A - Z)) and np.isclose(den2, Q.fro2(A))
    assert O.residual(A, A)[0] == 0.0
    mask = (rng.random((5, 6)) < 0.5).astype(np.uint8)
    relm, n2, d2 = O.residual(A, Z, mask)
    assert np.isclose(n2, np.sum(((A - Z) ** 2).sum(0) * mask))
    assert np.isclose(d2, np.sum((A ** 2).sum(0) * mask))


def test_smooth_field_with_distinct_modes_has_rank_three_times_modes():
    # the masked-workload recipe at reduced size: 20 distinct modes per channel
    A = synth.smooth_color(256, 384, 20, 4, offset=0.0, clip=False, max_freq=96,
                           distinct=True, bounded_amp=True, dtype=np.float64)
    s = O.qsvd_values(A)
    assert np.all(A[0] == 0)                        # pure quaternion
    assert s[59] > 1e-8 * s[0] and s[60] < 1e-11 * s[0]
