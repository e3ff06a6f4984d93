"""Batched, grouped QMCUR (one launch per stage, CUDA graph) against the FP64
oracle, problem by problem.

Tolerances: probabilities 40 u32 elementwise (FP32 runs of 32 squares before
FP64); index sets and gathers bit-exact (the oracle sampler is fed the
library's probabilities, stream_id = problem index); U from the FP32
one-sided Jacobi, a backward-stable QSVD, within 8 c u32 kappa(W_k) of the
FP64 oracle, or from the FP32 subspace core (one CTA per problem) within its
own bound 64 u32 kappa^2, or from the FP64-accurate refined core (one CTA per
problem) in FP64 within 1e-12 kappa(W_k) (the FP64 path's 1e-12, scaled by
the condition of the kept part), its FP32 copy being that FP64 U rounded;
ranks equal; the relative residual within 1e-5 of the oracle's evaluated on
the same U.
"""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import U32, dev, host, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module",
                params=[Q.PINV_JACOBI_FP64, Q.PINV_SUBSPACE_FP32, Q.PINV_REFINED_FP64],
                ids=["jacobi", "subspace", "refined"])
def batch(request):
    probs = synth.batch_problems(count=24, seed=3)
    As = [dev(p["X"]) for p in probs]
    B = Q.Batch(As, [p["c"] for p in probs], [p["r"] for p in probs],
                [p["rank"] for p in probs], sampler=Q.SAMPLER_NORM, seed=11,
                pinv_method=request.param)
    B.run()
    torch.cuda.synchronize()
    assert int(B.status.item()) == 0
    return probs, B, request.param


def test_batch_matches_oracle(batch):
    probs, B, method = batch
    for b, p in enumerate(probs):
        A64 = p["X"].astype(np.float64)
        col_p, row_p = host(B.get(b, "col_p")), host(B.get(b, "row_p"))
        po, qo, _ = O.probabilities(A64, O.SAMPLER_NORM)
        assert np.allclose(col_p, po, rtol=40 * U32, atol=0)
        assert np.allclose(row_p, qo, rtol=40 * U32, atol=0)
        J, I = host(B.get(b, "J")), host(B.get(b, "I"))
        Jo, _ = O.sample(col_p, p["c"], 11, b, 0, O.SAMPLER_NORM)
        Io, _ = O.sample(row_p, p["r"], 11, b, 1, O.SAMPLER_NORM)
        assert np.array_equal(J, Jo) and np.array_equal(I, Io), b
        Co, Ro, Wo = O.gather(A64, Io, Jo)
        assert np.array_equal(host(B.get(b, "W")), Wo.astype(np.float32))
        assert np.array_equal(host(B.get(b, "C")), Co.astype(np.float32))
        U = host(B.get(b, "U")).astype(np.float64)
        Uo, ko, so = O.pinv_truncated(Wo, 1e-10, p["rank"])
        info = host(B.get(b, "info"))
        assert info[0] == ko and info[2] == 0
        kap = so[0] / so[ko - 1]
        if method == Q.PINV_REFINED_FP64:
            U64 = host(B.get(b, "U64"))
            assert np.array_equal(host(B.get(b, "U")), U64.astype(np.float32))
            assert 1 <= info[1] <= 30
            assert rel_fro(U64, Uo) < 1e-12 * max(1.0, kap), (b, rel_fro(U64, Uo), kap)
        tol = 8 * p["c"] * U32 * kap if method == Q.PINV_JACOBI_FP64 else 64 * U32 * kap ** 2
        assert rel_fro(U, Uo) < tol, (b, rel_fro(U, Uo), kap)
        rel = host(B.get(b, "out3"))[0]
        rel_o = O.residual(A64, O.reconstruct(Co, U, Ro))[0]
        assert abs(rel - rel_o) < 1e-5, (b, rel, rel_o)


def test_batch_replay_is_deterministic(batch):
    probs, B, _ = batch
    first = [host(B.get(b, "out3")) for b in range(len(probs))]
    B.run()
    torch.cuda.synchronize()
    again = [host(B.get(b, "out3")) for b in range(len(probs))]
    for a, b in zip(first, again):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("prec", [Q.PREC_BF16_MIXED, Q.PREC_BF16X6, Q.PREC_TF32X3],
                         ids=["bf16mixed", "bf16x6", "tf32x3"])
def test_batch_tensor_core_residual(prec):
    # the grouped tcgen05 Z = C T (stacked operand pieces of all problems, one
    # launch) against the oracle's residual of the same U, and against the
    # CUDA-core FP32 plan of the same batch: both within 1e-5; everything
    # before the product (probabilities, draws, gathers, core, T = U R) is
    # shared, so U and the index sets agree bit for bit
    probs = synth.batch_problems(count=24, seed=3)
    As = [dev(p["X"]) for p in probs]
    args = ([p["c"] for p in probs], [p["r"] for p in probs], [p["rank"] for p in probs])
    kw = dict(sampler=Q.SAMPLER_NORM, seed=11, pinv_method=Q.PINV_SUBSPACE_FP32)
    F = Q.Batch(As, *args, prec=Q.PREC_FP32, **kw)
    T = Q.Batch(As, *args, prec=prec, **kw)
    F.run()
    T.run()
    torch.cuda.synchronize()
    assert int(F.status.item()) == 0 and int(T.status.item()) == 0
    for b, p in enumerate(probs):
        U = host(T.get(b, "U"))
        assert np.array_equal(U, host(F.get(b, "U")))
        assert np.array_equal(host(T.get(b, "J")), host(F.get(b, "J")))
        A64 = p["X"].astype(np.float64)
        Co = host(T.get(b, "C")).astype(np.float64)
        I = host(T.get(b, "I"))
        Ro = A64[:, I, :]
        rel_o = O.residual(A64, O.reconstruct(Co, U.astype(np.float64), Ro))[0]
        rel, rel_f = host(T.get(b, "out3"))[0], host(F.get(b, "out3"))[0]
        assert abs(rel - rel_o) < 1e-5, (b, rel, rel_o)
        assert abs(rel - rel_f) < 1e-5, (b, rel, rel_f)
    again = [host(T.get(b, "out3")) for b in range(len(probs))]
    T.run()
    torch.cuda.synchronize()
    for b in range(len(probs)):
        assert np.array_equal(again[b], host(T.get(b, "out3")))   # fixed-order folds
    F.close()
    T.close()


def test_batch_stage_times():
    # the graph records its stage boundaries: seven non-negative durations
    # whose sum is the replay, timed around it on the stream
    probs = synth.batch_problems(count=16, seed=5)
    As = [dev(p["X"]) for p in probs]
    B = Q.Batch(As, [p["c"] for p in probs], [p["r"] for p in probs], [p["rank"] for p in probs],
                sampler=Q.SAMPLER_NORM, seed=2, pinv_method=Q.PINV_SUBSPACE_FP32,
                prec=Q.PREC_BF16_MIXED)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    B.run()
    e1.record()
    st = B.stage_ms()
    total = e0.elapsed_time(e1)
    assert list(st) == list(Q.Batch.STAGES)
    assert all(v >= 0.0 for v in st.values()), st
    assert sum(st.values()) <= total * 1.05 + 0.01, (st, total)
    assert st["core"] > 0.0 and st["z_gemm_residual"] > 0.0
    B.close()


def test_batch_refined_reports_a_problem_without_gap():
    # one Gaussian 64 x 64 problem (no gap at its rank cap 20: c = r = 64
    # takes the whole matrix as W) among low-rank ones: the refined core
    # runs out of its 5 iterations on it alone, reports NO_CONVERGENCE in
    # that problem's info[2] and in the batch status, and still gives every
    # other problem its FP64-accurate U
    probs = synth.batch_problems(count=5, seed=7)
    flat = np.random.default_rng(8).standard_normal((4, 64, 64)).astype(np.float32)
    probs.insert(2, dict(X=flat, m=64, n=64, rank=20, c=64, r=64))
    As = [dev(p["X"]) for p in probs]
    B = Q.Batch(As, [p["c"] for p in probs], [p["r"] for p in probs],
                [p["rank"] for p in probs], sampler=Q.SAMPLER_NORM, seed=3, max_sweeps=5,
                pinv_method=Q.PINV_REFINED_FP64, prec=Q.PREC_BF16_MIXED)
    B.run()
    torch.cuda.synchronize()
    assert int(B.status.item()) == 6   # QMCUR_ERR_NO_CONVERGENCE
    for b, p in enumerate(probs):
        info = host(B.get(b, "info"))
        if b == 2:
            assert info[2] == 6 and info[1] == 5, info
            continue
        assert info[2] == 0 and info[0] == p["rank"] and info[1] <= 5, (b, info)
        A64 = p["X"].astype(np.float64)
        J, I = host(B.get(b, "J")), host(B.get(b, "I"))
        Wo = O.gather(A64, I, J)[2]
        Uo, ko, so = O.pinv_truncated(Wo, 1e-10, p["rank"])
        kap = so[0] / so[ko - 1]
        assert rel_fro(host(B.get(b, "U64")), Uo) < 1e-12 * max(1.0, kap), b
    B.close()


def test_batch_tensor_core_ragged_shapes():
    # shapes that fill no tile exactly (n and m off the 64- and 128-wide
    # tiles, c and r odd): the grouped T = U R stores and the grouped
    # Z = C T residuals mask every edge; against the oracle's residual of the
    # same U and the FP32 plan's, within 1e-5, for both cores
    shapes = [(70, 100, 7), (131, 250, 13), (64, 65, 5), (257, 63, 20), (90, 333, 31), (45, 77, 9)]
    probs = []
    for s_, (m, n, k) in enumerate(shapes):
        X, _ = synth.lowrank_gaussian(m, n, k, seed=40 + s_, noise_rel=1e-4)
        probs.append(dict(X=X, m=m, n=n, rank=k, c=min(2 * k + 1, n), r=min(2 * k + 1, m)))
    As = [dev(p["X"]) for p in probs]
    args = ([p["c"] for p in probs], [p["r"] for p in probs], [p["rank"] for p in probs])
    for method in (Q.PINV_REFINED_FP64, Q.PINV_SUBSPACE_FP32):
        kw = dict(sampler=Q.SAMPLER_NORM, seed=21, pinv_method=method)
        F = Q.Batch(As, *args, prec=Q.PREC_FP32, **kw)
        T = Q.Batch(As, *args, prec=Q.PREC_BF16_MIXED, **kw)
        F.run()
        T.run()
        torch.cuda.synchronize()
        assert int(F.status.item()) == 0 and int(T.status.item()) == 0
        for b, p in enumerate(probs):
            U = host(T.get(b, "U"))
            assert np.array_equal(U, host(F.get(b, "U")))
            A64 = p["X"].astype(np.float64)
            Co = host(T.get(b, "C")).astype(np.float64)
            Ro = A64[:, host(T.get(b, "I")), :]
            rel_o = O.residual(A64, O.reconstruct(Co, U.astype(np.float64), Ro))[0]
            rel, rel_f = host(T.get(b, "out3"))[0], host(F.get(b, "out3"))[0]
            assert abs(rel - rel_o) < 1e-5, (method, b, rel, rel_o)
            assert abs(rel - rel_f) < 1e-5, (method, b, rel, rel_f)
        F.close()
        T.close()


def test_batch_refined_host_refusals():
    # the refined core needs rank caps and rcond <= 1e-6 (it keeps exactly k
    # values): the plan refuses otherwise, before any launch
    probs = synth.batch_problems(count=3, seed=9)
    As = [dev(p["X"]) for p in probs]
    cs, rs = [p["c"] for p in probs], [p["r"] for p in probs]
    for kw in (dict(rank_caps=None), dict(rank_caps=[p["rank"] for p in probs], rcond=1e-3)):
        with pytest.raises(Q.QmcurError) as e:
            Q.Batch(As, cs, rs, pinv_method=Q.PINV_REFINED_FP64, **kw)
        assert e.value.code == 7   # QMCUR_ERR_UNSUPPORTED
