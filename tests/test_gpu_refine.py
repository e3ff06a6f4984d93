"""The FP64-accurate pseudo-inverse cores against the FP64 oracle's truncated
W^+ (Sec. 2.2, Algorithm 1's core), at the intersections the decomposition
workloads produce and on spectra built to a recipe.

* QMCUR_PINV_REFINED_FP64 (subspace iteration with float-float products on
  the FP32 pipe, about 2^-46 relative, and FP32 Cholesky preconditioners): U
  within max(1e-12, 64 u64 kappa sigma_1 / gap)
  relative Frobenius of the oracle, kappa = sigma_1 / sigma_k and gap =
  sigma_k - sigma_{k+1} (the first-order sensitivity of the truncated inverse
  to an FP64 backward error); 1e-12 on the 2048 x 2048 rank-50 workload's
  200 x 200 intersection.  A spectrum without a gap at k is reported as
  QMCUR_ERR_NO_CONVERGENCE.
* QMCUR_PINV_JACOBI_FP64 at the full intersection sizes: 1e-12 at 200 x 200
  (rank 50), and at the 4096 x 4096 colour field's 500 x 500 intersection
  (rank cap 100, sigma_101 / sigma_100 = 0.98) the gap-scaled bound
  64 c u64 sigma_1 / gap.
"""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from oracle import quat as QT
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import U64, dev, host, rel_fro

pytestmark = pytest.mark.gpu


def _intersection(name, sampler, seed):
    """W = A(I, J) of a workload, with I, J drawn by the oracle from the
    oracle's probabilities (the index draw is tested bit-exact elsewhere)."""
    w = synth.WORKLOADS[name]
    A = synth.make(name).astype(np.float64)
    p, q, _ = O.probabilities(A, sampler)
    J, _ = O.sample(p, w["c"], seed, 0, 0, sampler)
    I, _ = O.sample(q, w["r"], seed, 0, 1, sampler)
    return O.gather(A, I, J)[2], w


def _run(W, k, method, rcond=1e-10, max_sweeps=0, u_dtype=torch.float64, w_dtype=torch.float64):
    r, c = W.shape[1], W.shape[2]
    U = torch.empty(4, c, r, dtype=u_dtype, device="cuda")
    rank = torch.zeros(2, dtype=torch.int32, device="cuda")
    ws = Q.workspace(max(r, 1), max(c, 1), c, r, Q.PREC_FP32)
    st = Q.status_tensor()
    Q.pinv_core(dev(W, w_dtype), U, rcond, k, max_sweeps, rank, None, ws, st, method=method)
    torch.cuda.synchronize()
    return host(U).astype(np.float64), host(rank), int(st.item())


def _tol(sv, k):
    gap = sv[k - 1] - sv[k] if k < sv.size else sv[k - 1]
    return max(1e-12, 64 * U64 * (sv[0] / sv[k - 1]) * sv[0] / gap)


def _spectrum_matrix(r, c, sv, seed):
    """W = P diag(sv) V^H with orthonormal quaternion P (r x n), V (c x n)."""
    n = sv.size
    g = np.random.default_rng(seed)
    P = synth._orthonormal_columns(g, r, n)
    V = synth._orthonormal_columns(g, c, n)
    S = np.zeros((4, n, n))
    S[0] = np.diag(sv)
    return QT.qmatmul(QT.qmatmul(P, S), QT.conj_transpose(V))


def test_refined_bench_intersection():
    W, w = _intersection("gauss2048_rank50_noisy", O.SAMPLER_NORM, 1234)
    k = w["rank_cap"]
    Uo, ko, sv = O.pinv_truncated(W, w["rcond"], k)
    U, rank, st = _run(W, k, Q.PINV_REFINED_FP64)
    assert st == 0 and rank[0] == ko == k
    assert 2 <= rank[1] <= 6, rank
    assert rel_fro(U, Uo) < 1e-12, rel_fro(U, Uo)


def test_jacobi_bench_intersection():
    W, w = _intersection("gauss2048_rank50_noisy", O.SAMPLER_NORM, 1234)
    k = w["rank_cap"]
    Uo, ko, _ = O.pinv_truncated(W, w["rcond"], k)
    U, rank, st = _run(W, k, Q.PINV_JACOBI_FP64)
    assert st == 0 and rank[0] == ko == k
    assert rel_fro(U, Uo) < 1e-12, rel_fro(U, Uo)


def test_jacobi_color_field_intersection():
    W, w = _intersection("color4096_smooth100", O.SAMPLER_UNIFORM, 99)
    k = w["rank_cap"]
    Uo, ko, sv = O.pinv_truncated(W, w["rcond"], k)
    gap = sv[k - 1] - sv[k]
    U, rank, st = _run(W, k, Q.PINV_JACOBI_FP64)
    assert st == 0 and rank[0] == ko == k
    tol = 64 * W.shape[2] * U64 * sv[0] / gap
    assert tol < 1e-5   # the bound says something at this gap
    assert rel_fro(U, Uo) < tol, (rel_fro(U, Uo), tol)


def test_refined_reports_the_color_field_gap():
    # sigma_101 / sigma_100 = 0.98: subspace iteration cannot separate the
    # two within the limit, and says so
    W, w = _intersection("color4096_smooth100", O.SAMPLER_UNIFORM, 99)
    _, rank, st = _run(W, w["rank_cap"], Q.PINV_REFINED_FP64, max_sweeps=12)
    assert st == 6 and rank[1] == 12   # QMCUR_ERR_NO_CONVERGENCE


CASES = {
    # r, c, k, spectrum: (geometric top-k from 1 to smin, then tail ratio * smin ...)
    "ragged37x29_k5": (37, 29, 5, 1e-1, 0.2),
    "tall150x120_k50_kappa1e3": (150, 120, 50, 1e-3, 0.3),
    "wide120x150_k30_flat": (120, 150, 30, 1.0, 0.05),
    "k_is_min_40x24": (40, 24, 24, 1e-2, None),
    "slow_gap_96x80_k20": (96, 80, 20, 1e-1, 0.4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_refined_spectra(name):
    r, c, k, smin, ratio = CASES[name]
    n = min(r, c)
    top = np.geomspace(1.0, smin, k)
    tail = ratio * smin * np.geomspace(1.0, 1e-3, n - k) if ratio is not None else np.zeros(0)
    sv_in = np.concatenate([top, tail])
    W = _spectrum_matrix(r, c, sv_in, seed=31 + r + c)
    Uo, ko, sv = O.pinv_truncated(W, 1e-10, k)
    U, rank, st = _run(W, k, Q.PINV_REFINED_FP64)
    assert st == 0 and rank[0] == ko == k
    assert rel_fro(U, Uo) < _tol(sv, k), (rel_fro(U, Uo), _tol(sv, k), rank)


def test_refined_exact_low_rank():
    # the 256 x 256 rank-10 FP64 workload's intersection shape (c = r = 40)
    X = synth.lowrank_gaussian(256, 256, 10, seed=0, dtype=np.float64)[0]
    J = np.arange(0, 256, 256 // 40)[:40]
    I = np.arange(3, 256, 256 // 40)[:40]
    W = O.gather(X, I, J)[2]
    Uo, ko, sv = O.pinv_truncated(W, 1e-10, 10)
    U, rank, st = _run(W, 10, Q.PINV_REFINED_FP64)
    assert st == 0 and rank[0] == ko == 10
    assert rel_fro(U, Uo) < _tol(sv, 10)


def test_refined_f32_in_and_out():
    sv_in = np.concatenate([np.geomspace(1.0, 0.05, 12), 0.01 * np.geomspace(1, 1e-2, 52)])
    W = _spectrum_matrix(70, 64, sv_in, seed=5).astype(np.float32).astype(np.float64)
    Uo, _, _ = O.pinv_truncated(W, 1e-10, 12)
    U, rank, st = _run(W, 12, Q.PINV_REFINED_FP64, u_dtype=torch.float32, w_dtype=torch.float32)
    assert st == 0 and rank[0] == 12
    assert rel_fro(U, Uo) < 4 * 2.0 ** -24   # FP64 result rounded to FP32


def test_refined_is_deterministic():
    W, w = _intersection("gauss2048_rank50_noisy", O.SAMPLER_NORM, 77)
    U1, r1, s1 = _run(W, w["rank_cap"], Q.PINV_REFINED_FP64)
    U2, r2, s2 = _run(W, w["rank_cap"], Q.PINV_REFINED_FP64)
    assert s1 == s2 == 0 and np.array_equal(r1, r2) and np.array_equal(U1, U2)


def test_refined_flat_spectrum_reports_no_convergence():
    # sigma_21 / sigma_20 = 0.9989: the subspace converges far too slowly
    sv_in = np.concatenate([np.geomspace(1.0, 0.9, 20), 0.899 * np.geomspace(1.0, 0.5, 10),
                            0.1 * np.geomspace(1.0, 0.1, 30)])
    W = _spectrum_matrix(64, 60, sv_in, seed=9)
    _, rank, st = _run(W, 20, Q.PINV_REFINED_FP64, max_sweeps=5)
    assert st == 6 and rank[1] == 5


def test_refined_host_refusals():
    W = torch.zeros(4, 30, 20, dtype=torch.float64, device="cuda")
    U = torch.empty(4, 20, 30, dtype=torch.float64, device="cuda")
    ws = Q.workspace(30, 20, 20, 30, Q.PREC_FP32)
    for kwargs in (dict(rank_cap=0), dict(rank_cap=5, rcond=1e-3)):
        with pytest.raises(Q.QmcurError) as e:
            Q.pinv_core(W, U, kwargs.get("rcond", 1e-10), kwargs["rank_cap"], 0, None, None, ws,
                        None, method=Q.PINV_REFINED_FP64)
        assert e.value.code == 7   # QMCUR_ERR_UNSUPPORTED
    W2 = torch.zeros(4, 120, 110, dtype=torch.float64, device="cuda")
    U2 = torch.empty(4, 110, 120, dtype=torch.float64, device="cuda")
    with pytest.raises(Q.QmcurError) as e:
        Q.pinv_core(W2, U2, 1e-10, 105, 0, None, None, Q.workspace(120, 110, 110, 120, Q.PREC_FP32),
                    None, method=Q.PINV_REFINED_FP64)
    assert e.value.code == 7
