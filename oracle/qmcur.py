"""Plain FP64 CPU oracle of the QMCUR hot path (arXiv 2402.19147).

TEST INFRASTRUCTURE ONLY (see oracle/quat.py).  Nothing here is fast and
nothing here is shared with the CUDA library; both sides only share the seeded
input generators, which hold none of this arithmetic.

Steps, in the order of Algorithm 1 (Sec. 3.1):

* ``probabilities``   - p_j = ||X(:,j)||^2 / ||X||_F^2, q_i = ||X(i,:)||^2 / ||X||_F^2
                        (QMCUR_length) or p_j = 1/n, q_i = 1/m (QMCUR_uniform), Sec. 3.1.
* ``sample``          - draw J subset [n] from {p_j} and I subset [m] from {q_i}
                        (Algorithm 1 steps 1-2).  The paper names no mechanism; the
                        reading used here is listed in ``sample``'s docstring.
* ``gather``          - C = X(:,J), R = X(I,:) (Sec. 3.1) and the intersection
                        W = X(I,J).
* ``pinv_truncated``  - U = W^+ through the QSVD (Sec. 2.2) of W, computed as the
                        SVD of its complex adjoint, truncated at rcond and rank_cap.
* ``reconstruct``     - Z = C (U R) (Eq. 1, Algorithm 1 output).
* ``residual``        - ||X - Z||_F / ||X||_F (Example 4.2's relative error).
* ``core_paper``      - the paper's own core C^+ X R^+ (Algorithm 1 step 3), with
                        C^+ and R^+ truncated by the rule of W^+; it equals W^+
                        when rank(W) = rank(X).
* ``qsvd_truncated``  - the rank-k truncated QSVD X_k = P_k Sigma_k V_k^H (Sec. 2.2),
                        the comparator of Example 4.2.
* ``complete_step``,  - Algorithm 2 (Example 4.4): quaternion matrix completion by
  ``complete``          repeated QMCUR approximation and re-imposition of the
                        observed entries, with its relative-change stopping test.

Parity status: every function is pinned by tests/test_oracle_*.py (Hamilton
table, complex-adjoint homomorphism, Penrose conditions, reduction to
numpy.linalg.pinv in the real and complex cases, exact recovery on exactly
low-rank inputs, Lemma 1, Philox known-answer vectors, brute-force inverse CDF,
chi-square frequencies of the sampler).
"""
import math

import numpy as np

from .quat import (as_q, qmatmul, conj_transpose, complex_adjoint,
                   from_complex_adjoint, fro2)
from .philox import philox4x32_10

SAMPLER_UNIFORM = 0
SAMPLER_NORM = 1



# ----------------------------------------------------------------- Sec. 3.1 -
def squared_norms(A):
    """Column and row squared norms and ||A||_F^2 (Sec. 3.1, Sec. 2.2).

    col2[j] = sum_i |a_ij|^2, row2[i] = sum_j |a_ij|^2, F = sum_j col2[j].
    """
    A = as_q(A)
    sq = np.sum(A * A, axis=0)              # |a_ij|^2, shape (m, n)
    col2 = sq.sum(axis=0)
    row2 = sq.sum(axis=1)
    F = float(col2.sum())
    return col2, row2, F


def probabilities(A, sampler=SAMPLER_NORM):
    """Sampling probabilities (p over columns, q over rows) and ||A||_F^2 (Sec. 3.1).

    QMCUR_length: p_j = ||A(:,j)||^2/||A||_F^2, q_i = ||A(i,:)||^2/||A||_F^2.
    QMCUR_uniform: p_j = 1/n, q_i = 1/m.
    """
    A = as_q(A)
    m, n = A.shape[1], A.shape[2]
    col2, row2, F = squared_norms(A)
    if sampler == SAMPLER_UNIFORM:
        return np.full(n, 1.0 / n), np.full(m, 1.0 / m), F
    if not np.isfinite(F):
        raise FloatingPointError("non-finite entry in A")
    if F == 0.0:
        raise ZeroDivisionError("||A||_F = 0")
    return col2 / F, row2 / F, F


# -------------------------------------------------------- Algorithm 1, 1-2 -
def fixed_point_prefix(p):
    """Probabilities as 64-bit fixed-point integers and their prefix sums.

    With M = max p_k = f 2^e (f in [1, 2)) and B = 63 - ceil(log2 n), every
    p_k becomes q_k = floor(p_k 2^E), E = B - 1 - e: an exact scaling by a
    power of two, then truncation.  So q_k < 2^B, the total S = sum q_k is
    below 2^63, and the largest entry keeps B bits (52 at n = 2048).  The
    prefix sums P_k = q_0 + ... + q_k are exact integers, so they do not
    depend on the order of the additions (a parallel scan gives the same
    bits) and they are non-decreasing.  Returns (P, S) as Python-int-valued
    uint64 arrays / int; an entry with q_k = 0 can never be drawn.
    """
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    M = float(p.max()) if n else 0.0
    if not M > 0.0:
        return np.zeros(n, dtype=np.uint64), 0
    e = math.frexp(M)[1] - 1                       # M = f 2^e, f in [1, 2)
    B = 63 - (n - 1).bit_length()                  # 63 - ceil(log2 n)
    E = B - 1 - e
    q = [int(math.ldexp(float(x), E)) for x in p]  # exact scaling, truncated
    P = np.array(np.cumsum(np.array(q, dtype=object)), dtype=np.uint64)
    return P, int(P[-1])


def _draw_word(seed, stream_id, which, t):
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    ctr = (t & 0xFFFFFFFF, (t >> 32) & 0xFFFFFFFF, stream_id & 0xFFFFFFFF, which)
    return philox4x32_10(ctr, key)


def sample(p, count, seed, stream_id, which, sampler, max_attempts=0):
    """Draw `count` distinct indices of [len(p)] from the distribution p.

    Reading of Algorithm 1 steps 1-2 (the paper fixes no mechanism):
    * J and I are *sets*, so the draw is without replacement: a draw that
      repeats an accepted index is rejected and the next counter is used;
      the accepted set is returned sorted ascending.
    * Draw t uses Philox4x32-10 with key = (seed_lo, seed_hi) and counter =
      (t_lo, t_hi, stream_id, which), which = 0 for columns, 1 for rows.
    * QMCUR_length (norm): w = (x0 << 32 | x1) >> 11, a 53-bit integer;
      target = (w S) >> 53, exact in integers and below S; index = first k
      with P[k] > target, P and S from ``fixed_point_prefix``.  So index k
      is drawn with probability q_k / S up to 2^-53.
    * QMCUR_uniform: index = (x0 * n) >> 32 (integer multiply-shift).
    * At most max_attempts draws (0 selects 64*count + 1024); running out
      raises RuntimeError (the library reports QMCUR_ERR_SAMPLE_LIMIT).
    """
    p = np.asarray(p, dtype=np.float64)
    n = p.shape[0]
    if count < 1 or count > n:
        raise ValueError("count must be in [1, n]")
    if max_attempts <= 0:
        max_attempts = 64 * count + 1024
    if sampler == SAMPLER_NORM:
        P, S = fixed_point_prefix(p)
        support = int(np.count_nonzero(np.diff(P, prepend=np.uint64(0)))) if S else 0
        if support < count:
            raise ValueError("fewer positive probabilities than requested indices")
    chosen = []
    taken = np.zeros(n, dtype=bool)
    t = 0
    while len(chosen) < count:
        if t >= max_attempts:
            raise RuntimeError("sample attempt limit reached")
        x0, x1, _, _ = _draw_word(seed, stream_id, which, t)
        t += 1
        if sampler == SAMPLER_NORM:
            w = ((x0 << 32) | x1) >> 11
            target = (w * S) >> 53
            k = int(np.searchsorted(P, np.uint64(target), side="right"))
        else:
            k = (x0 * n) >> 32
        if not taken[k]:
            taken[k] = True
            chosen.append(k)
    return np.array(sorted(chosen), dtype=np.int64), t


# ----------------------------------------------------------------- Sec. 3.1 -
def gather(A, I, J):
    """C = A(:,J), R = A(I,:), W = A(I,J) (Sec. 3.1; W is the intersection)."""
    A = as_q(A)
    I = np.asarray(I)
    J = np.asarray(J)
    C = A[:, :, J].copy()
    R = A[:, I, :].copy()
    W = A[:, I][:, :, J].copy()
    return C, R, W


# ------------------------------------------------------------ Sec. 2.2, 3.1 -
def qsvd_values(W):
    """Quaternion singular values of W (descending), from its complex adjoint.

    chi(W) has every quaternion singular value twice; one of each pair is kept.
    """
    s = np.linalg.svd(complex_adjoint(W), compute_uv=False)
    return s[0::2].copy()


def qsvd_truncated(X, rank, rcond=0.0):
    """Rank-k truncated QSVD X_k = P_k Sigma_k V_k^H (Sec. 2.2; Example 4.2's
    comparator), keeping the k = rank largest quaternion singular values that
    exceed rcond * sigma_1.  Formed as the truncated SVD of the complex
    adjoint, whose singular values come in equal pairs: the 2k leading
    triplets are chi(X_k).  Returns (X_k, k, sigma)."""
    X = as_q(X)
    Pc, s, Vh = np.linalg.svd(complex_adjoint(X), full_matrices=False)
    sq = s[0::2]
    k = min(int(rank), sq.size)
    if rcond > 0.0 and sq.size:
        k = min(k, int(np.count_nonzero(sq > rcond * sq[0])))
    kk = 2 * k
    return from_complex_adjoint((Pc[:, :kk] * s[:kk]) @ Vh[:kk]), k, sq.copy()


def pinv_truncated(W, rcond=1e-10, rank_cap=0):
    """Truncated Moore-Penrose inverse of a quaternion matrix (Sec. 2.2, Alg. 1).

    The QSVD W = P Sigma V^H is taken as the SVD of chi(W) (LAPACK, FP64).
    Kept: sigma_i > rcond * sigma_1, and at most rank_cap of them when
    rank_cap > 0.  U = V_k Sigma_k^{-1} P_k^H, mapped back from the adjoint.
    Returns (U, rank, sigma) with sigma the quaternion singular values.
    """
    W = as_q(W)
    X = complex_adjoint(W)
    Pc, s, Vh = np.linalg.svd(X, full_matrices=False)
    sq = s[0::2]
    if sq.size == 0 or sq[0] == 0.0:
        k = 0
    else:
        k = int(np.count_nonzero(sq > rcond * sq[0]))
    if rank_cap > 0:
        k = min(k, rank_cap)
    kk = 2 * k
    Xp = (Vh[:kk].conj().T / s[:kk]) @ Pc[:, :kk].conj().T
    return from_complex_adjoint(Xp), k, sq.copy()


# ----------------------------------------------------------------- Eq. (1) -
def reconstruct(C, U, R):
    """Z = C (U R) (Eq. 1), right product first as the library does."""
    return qmatmul(C, qmatmul(U, R))


def residual(A, Z, mask=None):
    """Relative Frobenius residual ||A - Z||_F / ||A||_F (Example 4.2).

    With a mask (m x n, nonzero = observed, the set Omega of Example 4.4) both
    norms run over the observed entries only.  Returns (rel, num2, den2).
    """
    A = as_q(A)
    Z = as_q(Z)
    D = A - Z
    if mask is not None:
        w = (np.asarray(mask) != 0).astype(np.float64)
        D = D * w
        A = A * w
    num2 = fro2(D)
    den2 = fro2(A)
    return float(np.sqrt(num2 / den2)) if den2 > 0 else float("nan"), num2, den2


def core_paper(A, C, R, rcond=1e-13, rank_cap=0):
    """The paper's core U = C^+ X R^+ (Algorithm 1 step 3).

    C^+ and R^+ are truncated by the same rule as W^+ (pinv_truncated: keep
    sigma_i > rcond * sigma_1, at most rank_cap of them); the defaults keep
    every numerically nonzero singular value, i.e. the plain C^+ X R^+.
    """
    Cp = pinv_truncated(C, rcond, rank_cap)[0]
    Rp = pinv_truncated(R, rcond, rank_cap)[0]
    return qmatmul(qmatmul(Cp, as_q(A)), Rp)


# -------------------------------------------------------------- Algorithm 1 -
def qmcur(A, c, r, sampler=SAMPLER_NORM, seed=0, stream_id=0, rcond=1e-10,
          rank_cap=0, col_p=None, row_p=None):
    """One QMCUR decomposition of A, Algorithm 1 with U = W^+.

    col_p / row_p may be given to sample from externally computed
    probabilities (the tests pass the library's so that index sets can be
    compared bit for bit).
    """
    A = as_q(A)
    p, q, F = probabilities(A, sampler)
    if col_p is not None:
        p = np.asarray(col_p, dtype=np.float64)
    if row_p is not None:
        q = np.asarray(row_p, dtype=np.float64)
    J, _ = sample(p, c, seed, stream_id, 0, sampler)
    I, _ = sample(q, r, seed, stream_id, 1, sampler)
    C, R, W = gather(A, I, J)
    U, rank, sigma = pinv_truncated(W, rcond, rank_cap)
    Z = reconstruct(C, U, R)
    rel, num2, den2 = residual(A, Z)
    return dict(p=p, q=q, F=F, J=J, I=I, C=C, R=R, W=W, U=U, rank=rank,
                sigma=sigma, Z=Z, rel=rel, num2=num2, den2=den2)


# -------------------------------------------------------------- Algorithm 2 -
def complete_step(X, mask, I, J, rcond=1e-10, rank_cap=0):
    """One iteration of Algorithm 2 (Example 4.4) with fixed index sets I, J.

    M = C U R is the QMCUR approximation of the current iterate X^t
    (Algorithm 1 with U = W^+, the truncated inverse of W = X^t(I,J)); then
    X^{t+1} = P_{Omega^c}(M) + P_Omega(X^t), where P_Omega(X^t) = P_Omega(Y)
    because every iterate keeps the observed entries.  The stopping quantity
    is delta = ||X^{t+1} - X^t||_F / ||X^t||_F.
    Returns (X^{t+1}, delta, num2, den2, rank) with num2 = ||X^{t+1} - X^t||_F^2
    and den2 = ||X^t||_F^2.
    """
    X = as_q(X)
    obs = np.asarray(mask) != 0
    C, R, W = gather(X, I, J)
    U, rank, _ = pinv_truncated(W, rcond, rank_cap)
    M = reconstruct(C, U, R)
    Xn = np.where(obs[None], X, M)
    num2 = fro2(Xn - X)
    den2 = fro2(X)
    delta = float(np.sqrt(num2 / den2)) if den2 > 0 else float("nan")
    return Xn, delta, num2, den2, rank


def complete(Y, mask, c, r, sampler=SAMPLER_UNIFORM, seed=0, rcond=1e-10, rank_cap=0,
             tol=1e-4, t_max=200, probs_hook=None):
    """Algorithm 2: recover the unobserved entries of Y (mask 0) from
    X^0 = P_Omega(Y) by iterating Algorithm 1 and complete_step.

    Iteration t runs Algorithm 1 in full on X^t: probabilities of X^t, then
    J and I drawn with Philox key `seed` and stream_id = t (new index sets at
    every iteration), then the masked update.  Iterations t = 0, 1, ... run
    until delta_t <= tol or t >= t_max, so at most t_max + 1 of them.
    probs_hook(t, X^t) may return (p, q) to replace the probabilities (the
    tests pass the library's, so that index sets agree bit for bit).
    """
    Y = as_q(Y)
    obs = np.asarray(mask) != 0
    X = np.where(obs[None], Y, 0.0)
    history = []
    t = 0
    while True:
        p, q, _ = probabilities(X, sampler)
        if probs_hook is not None:
            p, q = probs_hook(t, X)
        J, _ = sample(p, c, seed, t, 0, sampler)
        I, _ = sample(q, r, seed, t, 1, sampler)
        X, delta, _, _, rank = complete_step(X, mask, I, J, rcond, rank_cap)
        history.append(delta)
        if delta <= tol or t >= t_max:
            break
        t += 1
    return dict(X=X, I=I, J=J, iters=len(history), history=history, rank=rank)
