"""Example 4.1 through the library: the same sweep as the oracle's Theorem 1
pin (tests/test_oracle_theorem1.py), with the gathers, the paper's core
C~^+ X~ R~^+ (FP64 Jacobi inverses) and the reconstruction on the GPU in
FP64.  Both sides form the projections C~ C~^+ and R~^+ R~ backward-stably
with different algorithms (one-sided Jacobi here, LAPACK there), so their
spectral errors differ by at most about u64 (kappa(C~) + kappa(R~)) ||X||_2;
C~ and R~ carry the noise, so kappa grows to ~1e7 at the smallest sigma.
Theorem 1's bound and the linear growth are checked on the GPU's errors.
"""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import dev, host, run_status
import test_oracle_theorem1 as T

pytestmark = pytest.mark.gpu


def gpu_sweep(prec=Q.PREC_FP64, method=Q.PINV_JACOBI_FP64, sigmas=T.SIGMAS, rank_cap=0):
    M, K, C, R = T.M, T.K, T.C, T.R
    X, Wk, Vk, _ = synth.svd_lowrank(M, M, K, seed=51, smin=100.0, smax=1000.0)
    J, _ = O.sample(np.full(M, 1.0 / M), C, 52, 0, 0, O.SAMPLER_UNIFORM)
    I, _ = O.sample(np.full(M, 1.0 / M), R, 52, 0, 1, O.SAMPLER_UNIFORM)
    dt = torch.float64 if prec == Q.PREC_FP64 else torch.float32
    f = dict(dtype=dt, device="cuda")
    Jd, Id = dev(J.astype(np.int32)), dev(I.astype(np.int32))
    out = []
    for t, s in enumerate(sigmas):
        Xt = X + synth.gaussian_noise(M, M, s, seed=60 + t)
        Xd = dev(Xt, dt)
        Cd, Rd = torch.empty(4, M, C, **f), torch.empty(4, R, M, **f)
        Q.gather(Xd, Jd, Id, Cd, Rd)
        Cp, Rp, U = torch.empty(4, C, M, **f), torch.empty(4, M, R, **f), torch.empty(4, C, R, **f)
        st = Q.status_tensor()
        Q.core_paper(Xd, Cd, Rd, Cp, Rp, U, prec=prec, rcond=1e-13, rank_cap=rank_cap,
                     method=method, status=st)
        Z = torch.empty(4, M, M, **f)
        ws = Q.workspace(M, M, C, R, prec)
        Q.reconstruct(Cd, U, Rd, prec, Z, ws, st)
        assert run_status(st) == 0
        Ct, Rt, _ = O.gather(Xt, I, J)
        kap = O.qsvd_values(Ct)[0] / O.qsvd_values(Ct)[-1] + O.qsvd_values(Rt)[0] / O.qsvd_values(Rt)[-1]
        out.append((s, T.spec(Xt - X), T.spec(X - host(Z).astype(np.float64)), kap))
    return out


def test_gpu_matches_oracle_sweep():
    ref = {s: (nE, e, bound) for s, nE, e, bound in T.sweep()}
    xnorm = 1000.0   # ||X||_2: the largest singular value is at most smax
    ratios = []
    for s, nE, e, kap in gpu_sweep():
        assert abs(e - ref[s][1]) <= 2.0 ** -53 * kap * xnorm + 1e-9 * ref[s][1], (s, e, ref[s][1], kap)
        assert e <= ref[s][2]
        ratios.append(e / nE)
    med = float(np.median(ratios))
    assert all(0.5 * med <= q <= 2.0 * med for q in ratios), ratios


def test_mixed_precision_tracks_fp64_until_its_floor():
    # the rank-capped core (k = 50) in the benchmarked arithmetic: mixed BF16
    # products, FP32 subspace inverses.  Its error follows the FP64 one while
    # that is above the arithmetic's floor (BF16X3: ~2^-16 relative per
    # product, so ~1e-5 ||X||_2), and never exceeds the floor elsewhere.
    ref = gpu_sweep(Q.PREC_FP64, Q.PINV_JACOBI_FP64, rank_cap=T.K)
    got = gpu_sweep(Q.PREC_BF16_MIXED, Q.PINV_SUBSPACE_FP32, rank_cap=T.K)
    floor = 1e-5 * 1000.0
    for (s, _, e64, _), (_, _, e, _) in zip(ref, got):
        assert e <= e64 + floor, (s, e, e64)
        if e64 > 10 * floor:
            assert abs(e - e64) < 0.05 * e64, (s, e, e64)
