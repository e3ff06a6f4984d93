"""Decompositions on two or four streams at once, each held to SMs / streams
CTAs (qmcur_opts.max_ctas / qmcur_set_max_ctas), against the same
decompositions run alone with one CTA per SM.

* index sets: bit-exact (the sampler does not depend on the CTA budget);
* FP64 Jacobi pseudo-inverse: bit-exact (each column pair's arithmetic is the
  same whichever CTA takes it);
* FP32 subspace pseudo-inverse: its K splits follow the number of CTAs, so the
  sums round differently: U within 1e-4 relative Frobenius, the relative
  residual within 1e-5 relative (this gap-rich workload's bound).
"""
import numpy as np
import pytest
import torch

from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    Q.lib()
    yield
    Q.set_max_ctas(0)


def _run(A, Ds, streams, seeds, method, k, budget):
    # the buffers were zeroed on the current stream; the streams below are others
    torch.cuda.synchronize()
    for i, (D, sd) in enumerate(zip(Ds, seeds)):
        Q.decompose(A, D, sampler=Q.SAMPLER_NORM, seed=sd, stream_id=0, rcond=1e-10,
                    rank_cap=k, stream=streams[i % len(streams)], pinv_method=method,
                    max_ctas=budget)
    torch.cuda.synchronize()
    for D in Ds:
        Q.check_status(D.status, "decompose")


@pytest.mark.parametrize("nstreams", [2, 4])
@pytest.mark.parametrize("method", [Q.PINV_SUBSPACE_FP32, Q.PINV_JACOBI_FP64])
def test_streams_share_the_sms(method, nstreams):
    m, n, c, r, k = 1024, 1536, 80, 72, 20
    A_np, _ = synth.lowrank_gaussian(m, n, k, seed=41, noise_rel=1e-3)
    A = torch.from_numpy(A_np).cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    seeds = [3, 4, 5, 6]
    ref = [Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED) for _ in seeds]
    got = [Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED) for _ in seeds]
    _run(A, ref, [torch.cuda.current_stream()], seeds, method, k, 0)
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    _run(A, got, streams, seeds, method, k, sms // nstreams)
    for a, b in zip(ref, got):
        assert np.array_equal(host(a.J), host(b.J)) and np.array_equal(host(a.I), host(b.I))
        ua, ub = host(a.U), host(b.U)
        ra, rb = host(a.out3)[0], host(b.out3)[0]
        if method == Q.PINV_JACOBI_FP64:
            assert np.array_equal(ua, ub) and ra == rb
        else:
            assert np.linalg.norm(ua - ub) <= 1e-4 * np.linalg.norm(ua)
            assert abs(ra - rb) <= 1e-5 * ra


def test_thread_budget_applies_to_the_stage_calls():
    # qmcur_set_max_ctas holds the separate stage calls to the budget too
    m, n, c, r, k = 512, 768, 48, 40, 12
    A_np, _ = synth.lowrank_gaussian(m, n, k, seed=43, noise_rel=1e-3)
    A = torch.from_numpy(A_np).cuda()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    outs = []
    for budget in (0, sms // 2, 8):
        Q.set_max_ctas(budget)
        D = Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED)
        Q.probs(A, Q.SAMPLER_NORM, D.col_p, D.row_p, None, D.ws, D.status)
        Q.sample(A, Q.SAMPLER_NORM, D.col_p, D.row_p, c, r, 9, 0, D.J, D.I, D.C, D.R, D.W,
                 ws=D.ws, status=D.status)
        Q.pinv_core(D.W, D.U, 1e-10, k, 0, D.rank, D.sigma, D.ws, D.status,
                    method=Q.PINV_JACOBI_FP64)
        Q.residual(A, D.out3, D.C, D.U, D.R, Q.PREC_BF16_MIXED, None, None, D.ws, D.status)
        torch.cuda.synchronize()
        Q.check_status(D.status, "stages")
        outs.append((host(D.U), host(D.out3)[0]))
    Q.set_max_ctas(0)
    # the Jacobi core and the GEMMs give the same bits at any budget
    for U, rel in outs[1:]:
        assert np.array_equal(U, outs[0][0]) and rel == outs[0][1]


def test_decompose_many_matches_one_at_a_time():
    # the binding's many-matrix helper: eight in flight on eight streams
    m, n, c, r, k = 768, 1024, 64, 56, 16
    A_np, _ = synth.lowrank_gaussian(m, n, k, seed=47, noise_rel=1e-3)
    As = [torch.from_numpy(A_np).cuda()]
    As += [torch.roll(As[0], shifts=31 * q, dims=1).contiguous() for q in range(1, 4)]
    seeds = list(range(10, 18))
    inputs = [As[i % 4] for i in range(len(seeds))]
    ref = [Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED) for _ in seeds]
    got = [Q.Decomposition(m, n, c, r, Q.PREC_BF16_MIXED) for _ in seeds]
    torch.cuda.synchronize()
    for A, D, sd in zip(inputs, ref, seeds):
        Q.decompose(A, D, sampler=Q.SAMPLER_NORM, seed=sd, rank_cap=k,
                    pinv_method=Q.PINV_SUBSPACE_FP32)
    Q.decompose_many(inputs, got, seeds, nstreams=8, sampler=Q.SAMPLER_NORM, rank_cap=k,
                     pinv_method=Q.PINV_SUBSPACE_FP32)
    torch.cuda.current_stream().synchronize()
    for a, b in zip(ref, got):
        Q.check_status(a.status, "one at a time")
        Q.check_status(b.status, "many")
        assert np.array_equal(host(a.J), host(b.J)) and np.array_equal(host(a.I), host(b.I))
        ua, ub = host(a.U), host(b.U)
        assert np.linalg.norm(ua - ub) <= 1e-4 * np.linalg.norm(ua)
        ra, rb = host(a.out3)[0], host(b.out3)[0]
        assert abs(ra - rb) <= 1e-5 * ra


def test_decompose_many_defaults():
    # with its defaults (FP64 Jacobi core, no rank cap) the helper runs and
    # matches one decomposition at a time bit for bit
    m, n, c, r = 256, 320, 24, 20
    A = torch.from_numpy(synth.lowrank_gaussian(m, n, 6, seed=51, noise_rel=0.0)[0]).cuda()
    seeds = [1, 2, 3]
    ref = [Q.Decomposition(m, n, c, r, Q.PREC_FP32) for _ in seeds]
    got = [Q.Decomposition(m, n, c, r, Q.PREC_FP32) for _ in seeds]
    torch.cuda.synchronize()
    for D, sd in zip(ref, seeds):
        Q.decompose(A, D, seed=sd)
    Q.decompose_many([A] * 3, got, seeds, nstreams=2)
    torch.cuda.current_stream().synchronize()
    for a, b in zip(ref, got):
        Q.check_status(a.status, "one at a time")
        Q.check_status(b.status, "many")
        assert np.array_equal(host(a.J), host(b.J)) and np.array_equal(host(a.U), host(b.U))
        assert host(a.out3)[0] == host(b.out3)[0]


def test_decompose_many_failure_keeps_the_join():
    # the third entry's C has one row too few, so its qmcur_decompose fails
    # on the host (the gather's shape check, before the gather is queued;
    # its probabilities fit their buffers) after two decompositions were
    # queued on side streams; the current stream must still wait for those two
    m, n, c, r, k = 512, 640, 40, 36, 8
    A = torch.from_numpy(synth.lowrank_gaussian(m, n, k, seed=53, noise_rel=1e-3)[0]).cuda()
    Ds = [Q.Decomposition(m, n, c, r, Q.PREC_FP32) for _ in range(3)]
    Ds[2].C = torch.empty(4, m - 1, c, dtype=torch.float32, device="cuda")
    for D in Ds:
        D.out3.fill_(float("nan"))
    with pytest.raises(Q.QmcurError):
        Q.decompose_many([A, A, A], Ds, [5, 6, 7], nstreams=3, rank_cap=k)
    cur = torch.cuda.current_stream()
    seen = torch.stack([Ds[0].out3[0].clone(), Ds[1].out3[0].clone()])   # queued on cur
    cur.synchronize()
    vals = host(seen)
    assert np.all(np.isfinite(vals)) and np.all(vals > 0)
    torch.cuda.synchronize()
    Q.check_status(Ds[0].status, "first")
    Q.check_status(Ds[1].status, "second")
