"""Algorithm 2 (quaternion matrix completion, Example 4.4) on the GPU against
the FP64 oracle, through qmcur_complete_step.

Each iteration runs Algorithm 1 on the current iterate (uniform sampler: the
probabilities are exactly 1/n and 1/m, so both sides draw the same index sets
bit for bit; the norm sampler is fed the library's probabilities), then the
masked update.  Tolerances:
* observed entries: bit-exact (they are never written);
* index sets: bit-exact;
* unobserved entries after one iteration, relative Frobenius against the
  oracle: FP64 1e-11; FP32 and the mixed BF16 split with the FP64 Jacobi core
  2e-5 (the reconstruction tolerance of the split paths, twice); with the
  FP32 subspace core max(2e-5, 64 u32 kappa^2), kappa = sigma_1 / sigma_k of
  the intersection (the subspace core's own bound), on an iterate whose
  intersection has a clear gap sigma_k >> sigma_{k+1}, which that core
  requires.  (The zero-filled first iterate has no such gap; there the
  benchmarked loop is checked by what it recovers.)
* the relative change delta: the same bounds, relative.
"""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import U32, dev, host, rel_fro, run_status

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    Q.lib()


def _case(m, n, k, seed, p_observed, dtype=np.float32):
    Y, _ = synth.lowrank_gaussian(m, n, k, seed=seed, noise_rel=1e-3, dtype=dtype)
    mask = synth.bernoulli_mask(m, n, seed=seed + 1, p_observed=p_observed)
    X0 = np.where(mask[None] != 0, Y, 0).astype(dtype)
    return X0, mask


def _one_step(X0, mask, c, r, k, prec, pinv, sampler=Q.SAMPLER_UNIFORM, t=0, seed=4):
    m, n = X0.shape[1], X0.shape[2]
    tdt = torch.float64 if X0.dtype == np.float64 else torch.float32
    X = dev(X0)
    S = Q.Completion(m, n, c, r, prec, tdt)
    Q.complete_step(X, dev(mask), S, t, sampler, seed, 1e-10, k, 0, pinv)
    assert run_status(S.status) == 0
    return X, S


def _oracle_step(X0, mask, S, k, sampler, t=0, seed=4):
    Xo = X0.astype(np.float64)
    if sampler == Q.SAMPLER_UNIFORM:
        p, q, _ = O.probabilities(Xo, O.SAMPLER_UNIFORM)
    else:
        p, q = host(S.col_p), host(S.row_p)
    J, _ = O.sample(p, S.c, seed, t, 0, sampler)
    I, _ = O.sample(q, S.r, seed, t, 1, sampler)
    Xn, delta, num2, den2, rank = O.complete_step(Xo, mask, I, J, rank_cap=k)
    return I, J, Xn, delta, rank


def _check(X0, mask, X, S, I, J, Xn, delta, tol):
    obs = mask != 0
    Xg = host(X)
    assert np.array_equal(host(S.J), J) and np.array_equal(host(S.I), I)
    assert np.array_equal(Xg[:, obs], X0[:, obs])
    assert rel_fro(Xg[:, ~obs], Xn[:, ~obs]) < tol
    d = host(S.out3)
    assert abs(d[0] - delta) < tol * delta
    assert abs(d[2] - np.sum(X0.astype(np.float64) ** 2)) < 1e-6 * d[2]


@pytest.mark.parametrize("prec", [Q.PREC_FP32, Q.PREC_BF16_MIXED])
@pytest.mark.parametrize("m,n", [(333, 515), (1100, 1500)])
def test_step_matches_oracle_jacobi(prec, m, n):
    # the split path's update runs 32-column tiles at 333 x 515 and
    # 112-column tiles (ragged rows, 44-column last tile) at 1100 x 1500
    X0, mask = _case(m, n, 6, seed=21, p_observed=0.5)
    X, S = _one_step(X0, mask, 24, 20, 6, prec, Q.PINV_JACOBI_FP64)
    I, J, Xn, delta, _ = _oracle_step(X0, mask, S, 6, Q.SAMPLER_UNIFORM)
    _check(X0, mask, X, S, I, J, Xn, delta, 2e-5)


def test_step_matches_oracle_fp64():
    X0, mask = _case(200, 300, 5, seed=22, p_observed=0.4, dtype=np.float64)
    X, S = _one_step(X0, mask, 20, 24, 5, Q.PREC_FP64, Q.PINV_JACOBI_FP64)
    I, J, Xn, delta, _ = _oracle_step(X0, mask, S, 5, Q.SAMPLER_UNIFORM)
    _check(X0, mask, X, S, I, J, Xn, delta, 1e-11)


@pytest.mark.parametrize("sampler", [Q.SAMPLER_UNIFORM, Q.SAMPLER_NORM])
def test_step_matches_oracle_subspace(sampler):
    # a late iterate: the unobserved entries hold the low-rank values up to a
    # 1e-3 relative perturbation, so the intersection has a clear rank-8 gap
    m, n, k = 384, 640, 8
    Y, Y0 = synth.lowrank_gaussian(m, n, k, seed=23, noise_rel=1e-3)
    mask = synth.bernoulli_mask(m, n, seed=24, p_observed=0.5)
    rng = np.random.default_rng(25)
    late = Y0 + 1e-3 * np.std(Y0) * rng.standard_normal(Y0.shape)
    X0 = np.where(mask[None] != 0, Y, late).astype(np.float32)
    X, S = _one_step(X0, mask, 32, 32, k, Q.PREC_BF16_MIXED, Q.PINV_SUBSPACE_FP32, sampler, t=3)
    I, J, Xn, delta, _ = _oracle_step(X0, mask, S, 8, sampler, t=3)
    _, W = None, O.gather(X0.astype(np.float64), I, J)[2]
    s = O.qsvd_values(W)
    tol = max(2e-5, 64 * U32 * (s[0] / s[7]) ** 2)
    _check(X0, mask, X, S, I, J, Xn, delta, tol)


def test_all_observed_leaves_x_unchanged():
    X0, _ = _case(130, 70, 3, seed=24, p_observed=1.0)
    X = dev(X0)
    S = Q.Completion(130, 70, 12, 12, Q.PREC_BF16_MIXED)
    Q.complete_step(X, None, S, 0, rank_cap=3, pinv_method=Q.PINV_JACOBI_FP64)
    assert run_status(S.status) == 0
    assert np.array_equal(host(X), X0)
    d = host(S.out3)
    assert d[0] == 0.0 and d[1] == 0.0


def test_loop_matches_oracle():
    # five iterations (tol 0 never stops early), FP32 GEMMs, FP64 Jacobi core
    X0, mask = _case(160, 224, 4, seed=25, p_observed=0.5)
    X, S, hist = Q.complete(dev(X0), dev(mask), 16, 16, 4, prec=Q.PREC_FP32, tol=0.0, t_max=4,
                            pinv_method=Q.PINV_JACOBI_FP64, seed=6)
    out = O.complete(X0.astype(np.float64), mask, 16, 16, seed=6, rank_cap=4, tol=0.0, t_max=4)
    assert len(hist) == out["iters"] == 5
    assert np.max(np.abs(np.array(hist) / np.array(out["history"]) - 1)) < 1e-4
    miss = mask == 0
    assert rel_fro(host(X)[:, miss], out["X"][:, miss]) < 1e-4


def test_color512x768_workload():
    # the benchmarked workload: one iteration against the oracle, then the
    # whole loop on the GPU against the ground truth
    w = synth.WORKLOADS["color512x768_rank31_mr70"]
    m, n, c, r, k = w["m"], w["n"], w["c"], w["r"], w["rank_cap"]
    Y = synth.make("color512x768_rank31_mr70")
    mask = synth.bernoulli_mask(m, n, seed=w["mask_seed"], p_observed=w["p_observed"])
    X0 = np.where(mask[None] != 0, Y, 0).astype(np.float32)
    X, S = _one_step(X0, mask, c, r, k, Q.PREC_BF16_MIXED, Q.PINV_JACOBI_FP64, seed=9)
    I, J, Xn, delta, rank = _oracle_step(X0, mask, S, k, Q.SAMPLER_UNIFORM, seed=9)
    _check(X0, mask, X, S, I, J, Xn, delta, 2e-5)
    Xc, S, hist = Q.complete(dev(Y), dev(mask), c, r, k, seed=9, tol=w["tol"], t_max=w["t_max"])
    miss = mask == 0
    err = rel_fro(host(Xc)[:, miss], Y[:, miss])
    assert hist[-1] <= w["tol"] and len(hist) <= w["t_max"] + 1
    assert err < 2e-3, err
