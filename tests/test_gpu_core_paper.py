"""The paper's core U = C^+ X R^+ (Algorithm 1 step 3) on the GPU against the
FP64 oracle, through qmcur_core_paper.

Tolerance: U = C^+ (X R^+) is formed from the truncated inverses; each
product's relative rounding (FP64 ~1e-15, FP32 and the split paths <= 1.5e-5,
FP32 subspace inverses 64 u32 kappa^2) is amplified by at most
kappa(C_k) kappa(R_k), the conditions of the kept parts, which the test
computes from the oracle's singular values.
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


def _kappa(M, k):
    s = O.qsvd_values(M)
    return s[0] / s[k - 1]


def _run(X, C, R, k, prec, method, dtype=torch.float32):
    m, n, c, r = X.shape[1], X.shape[2], C.shape[2], R.shape[1]
    f = dict(dtype=dtype, device="cuda")
    Cp, Rp, U = torch.empty(4, c, m, **f), torch.empty(4, n, r, **f), torch.empty(4, c, r, **f)
    st = Q.status_tensor()
    Q.core_paper(dev(X), dev(C), dev(R), Cp, Rp, U, prec=prec, rank_cap=k, method=method,
                 status=st)
    assert run_status(st) == 0
    return host(U), host(Cp), host(Rp)


def _inputs(m, n, k, c, r, seed, noise, dtype=np.float32):
    X, _ = synth.lowrank_gaussian(m, n, k, seed=seed, noise_rel=noise, dtype=dtype)
    out = O.qmcur(X.astype(np.float64), c, r, sampler=O.SAMPLER_UNIFORM, seed=seed)
    return X, out["C"].astype(dtype), out["R"].astype(dtype)


@pytest.mark.parametrize("prec", [Q.PREC_FP32, Q.PREC_BF16_MIXED])
def test_exact_rank_jacobi(prec):
    m, n, k, c, r = 300, 260, 6, 24, 20
    X, C, R = _inputs(m, n, k, c, r, seed=41, noise=0.0)
    U, Cp, Rp = _run(X, C, R, k, prec, Q.PINV_JACOBI_FP64)
    X64, C64, R64 = (a.astype(np.float64) for a in (X, C, R))
    Uo = O.core_paper(X64, C64, R64, rcond=1e-10, rank_cap=k)
    kap = _kappa(C64, k) * _kappa(R64, k)
    assert rel_fro(Cp, O.pinv_truncated(C64, 1e-10, k)[0]) < 1e-5 * _kappa(C64, k)
    assert rel_fro(U, Uo) < 3e-5 * kap
    # Lemma 1: at exact rank the paper's core is the intersection's W^+
    W = O.gather(X64, *(O.sample(np.full(m, 1.0 / m), r, 41, 0, 1, O.SAMPLER_UNIFORM)[0],
                        O.sample(np.full(n, 1.0 / n), c, 41, 0, 0, O.SAMPLER_UNIFORM)[0]))[2]
    assert rel_fro(U, O.pinv_truncated(W, 1e-10, k)[0]) < 3e-5 * kap


def test_fp64():
    m, n, k, c, r = 200, 180, 5, 20, 18
    X, C, R = _inputs(m, n, k, c, r, seed=42, noise=1e-3, dtype=np.float64)
    U, _, _ = _run(X, C, R, k, Q.PREC_FP64, Q.PINV_JACOBI_FP64, dtype=torch.float64)
    Uo = O.core_paper(X, C, R, rcond=1e-10, rank_cap=k)
    assert rel_fro(U, Uo) < 1e-10 * _kappa(C, k) * _kappa(R, k)


def test_noisy_subspace():
    m, n, k, c, r = 640, 512, 8, 40, 36
    X, C, R = _inputs(m, n, k, c, r, seed=43, noise=1e-3)
    U, _, _ = _run(X, C, R, k, Q.PREC_BF16_MIXED, Q.PINV_SUBSPACE_FP32)
    X64, C64, R64 = (a.astype(np.float64) for a in (X, C, R))
    Uo = O.core_paper(X64, C64, R64, rcond=1e-10, rank_cap=k)
    kc, kr = _kappa(C64, k), _kappa(R64, k)
    tol = max(3e-5, 64 * U32 * max(kc, kr) ** 2) * kc * kr
    assert rel_fro(U, Uo) < tol


def test_gauss2048_workload():
    # the benchmarked shape: 2048 x 2048, rank 50 plus noise, c = r = 200
    w = synth.WORKLOADS["gauss2048_rank50_noisy"]
    X = synth.make("gauss2048_rank50_noisy")
    out = O.qmcur(X.astype(np.float64), w["c"], w["r"], sampler=O.SAMPLER_UNIFORM, seed=7)
    C, R = out["C"].astype(np.float32), out["R"].astype(np.float32)
    k = w["rank_cap"]
    U, _, _ = _run(X, C, R, k, Q.PREC_BF16_MIXED, Q.PINV_SUBSPACE_FP32)
    X64, C64, R64 = (a.astype(np.float64) for a in (X, C, R))
    Uo = O.core_paper(X64, C64, R64, rcond=1e-10, rank_cap=k)
    kc, kr = _kappa(C64, k), _kappa(R64, k)
    assert rel_fro(U, Uo) < max(3e-5, 64 * U32 * max(kc, kr) ** 2) * kc * kr
