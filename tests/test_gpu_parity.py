"""Parity of every step of the CUDA hot path with the FP64 oracle, through the
C ABI, on seeded synthetic inputs (several tiles and ragged tails), plus the
status-code paths.

Tolerances (derived from the arithmetic, u32 = 2^-24, u64 = 2^-53):
* probabilities of FP32 input: each squared norm is an FP32 sum of at most 20
  rounding steps before FP64 takes over (16 terms per thread piece, a 5-level
  warp tree) -> elementwise relative error <= 24 u32; FP64 input: 1e-12.
* index sets and gathers: bit-exact (integer work; the norm sampler is fed the
  library's own probabilities on both sides).
* pseudo-inverse (FP64 Jacobi vs LAPACK SVD of the complex adjoint): relative
  Frobenius 1e-12 on the FP64 workload, scaled by kappa(W_k) elsewhere.
* reconstruction: FP64 1e-12, FP32 and split paths 1e-5 relative Frobenius
  (both sides given the same U rounded to FP32).
"""
import numpy as np
import pytest
import torch

from oracle import qmcur as O
from paper_2402_19147_gb300 import qmcur as Q
from paper_2402_19147_gb300 import synth
from gpu_util import U32, dev, host, probs, rel_fro, run_status

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    Q.lib()


# ----------------------------------------------------------- probabilities -
@pytest.mark.parametrize("m,n", [(300, 700), (1, 5), (64, 1025), (257, 33), (3, 40000),
                                 (333, 516)])
def test_probs_norm_fp32(m, n):
    # ragged tiles: 333 x 516 leaves 13 rows in the last row tile and 4
    # columns in the last column tile; n % 4 != 0 takes scalar loads
    A = synth.lowrank_gaussian(m, n, 3, seed=m + n, noise_rel=0.1)[0]
    col_p, row_p, fro2, st = probs(dev(A), Q.SAMPLER_NORM)
    assert st == 0
    p, q, F = O.probabilities(A.astype(np.float64), O.SAMPLER_NORM)
    assert np.allclose(host(col_p), p, rtol=24 * U32, atol=0)
    assert np.allclose(host(row_p), q, rtol=24 * U32, atol=0)
    assert abs(host(fro2)[0] - F) <= 24 * U32 * F


def test_probs_norm_fp64_and_uniform():
    A = synth.make("gauss256_rank10_fp64")
    col_p, row_p, fro2, st = probs(dev(A), Q.SAMPLER_NORM)
    assert st == 0
    p, q, F = O.probabilities(A, O.SAMPLER_NORM)
    assert rel_fro(host(col_p), p) < 1e-12 and rel_fro(host(row_p), q) < 1e-12
    col_u, row_u, fro2u, st = probs(dev(A), Q.SAMPLER_UNIFORM)
    assert st == 0
    assert np.all(host(col_u) == 1.0 / 256) and np.all(host(row_u) == 1.0 / 256)
    assert abs(host(fro2u)[0] - F) < 1e-12 * F


def test_probs_status_codes():
    Z = np.zeros((4, 20, 30), dtype=np.float32)
    _, _, _, st = probs(dev(Z), Q.SAMPLER_NORM)
    assert st == 3                                  # ZERO_NORM
    Z[2, 5, 7] = np.nan
    _, _, _, st = probs(dev(Z), Q.SAMPLER_NORM)
    assert st == 2                                  # NONFINITE
    with pytest.raises(Q.QmcurError) as e:          # too small a workspace
        Q.probs(dev(Z), 1, torch.empty(30, dtype=torch.float64, device="cuda"),
                torch.empty(20, dtype=torch.float64, device="cuda"), None,
                torch.empty(8, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 1


# ------------------------------------------------------------ sample/gather -
def _sample(A_t, sampler, col_p, row_p, c, r, seed, stream_id, max_attempts=0, gather=True,
            Wdtype=torch.float64):
    m, n = A_t.shape[1], A_t.shape[2]
    J = torch.full((c,), -1, dtype=torch.int32, device="cuda")
    I = torch.full((r,), -1, dtype=torch.int32, device="cuda")
    C = R = W = None
    if gather:
        C = torch.empty(4, m, c, dtype=A_t.dtype, device="cuda")
        R = torch.empty(4, r, n, dtype=A_t.dtype, device="cuda")
        W = torch.empty(4, r, c, dtype=Wdtype, device="cuda")
    ws = Q.workspace(m, n, c, r, Q.PREC_FP32)
    st = Q.status_tensor()
    Q.sample(A_t, sampler, col_p, row_p, c, r, seed, stream_id, J, I, C, R, W,
             max_attempts=max_attempts, ws=ws, status=st)
    return J, I, C, R, W, run_status(st)


@pytest.mark.parametrize("sampler", [Q.SAMPLER_NORM, Q.SAMPLER_UNIFORM])
@pytest.mark.parametrize("m,n,c,r,seed", [(300, 700, 40, 25, 7), (1000, 257, 257, 3, 1),
                                          (5, 4096, 100, 5, 2**40 + 3)])
def test_sample_bit_exact_and_gather(sampler, m, n, c, r, seed):
    A = synth.lowrank_gaussian(m, n, 4, seed=m, noise_rel=0.05)[0]
    A_t = dev(A)
    col_p, row_p, _, st = probs(A_t, sampler)
    assert st == 0
    J, I, C, R, W, st = _sample(A_t, sampler, col_p, row_p, c, r, seed, 9)
    assert st == 0
    Jo, _ = O.sample(host(col_p), c, seed, 9, 0, sampler)
    Io, _ = O.sample(host(row_p), r, seed, 9, 1, sampler)
    assert np.array_equal(host(J), Jo) and np.array_equal(host(I), Io)
    Co, Ro, Wo = O.gather(A.astype(np.float64), Io, Jo)
    assert np.array_equal(host(C), Co.astype(np.float32))
    assert np.array_equal(host(R), Ro.astype(np.float32))
    assert np.array_equal(host(W), Wo)


@pytest.mark.parametrize("case", ["wide_range", "subnormal_max", "unnormalised", "n1",
                                  "one_heavy"])
def test_sample_fixed_point_edges(case):
    # explicit probability vectors: the integer scaling is taken from the
    # largest entry, so entries far below it are never drawn on either side,
    # a subnormal maximum still scales into B bits, and any positive scale
    # of p draws the same indices
    rng = np.random.default_rng(31)
    n, c = 300, 40
    if case == "wide_range":
        c = 10
        p = 10.0 ** rng.uniform(-30, 0, n)
    elif case == "subnormal_max":
        p = rng.random(n) * 2.0 ** -1060
    elif case == "unnormalised":
        p = rng.random(n) * 3.7e5
    elif case == "n1":
        n, c = 1, 1
        p = np.array([0.3])
    else:
        p = np.full(n, 1e-3)
        p[17] = 1.0
    m, r = n, c
    A_t = dev(np.ones((4, m, n), dtype=np.float32))
    col_p = torch.tensor(p, dtype=torch.float64, device="cuda")
    row_p = torch.tensor(p[::-1].copy(), dtype=torch.float64, device="cuda")
    J, I, *_, st = _sample(A_t, Q.SAMPLER_NORM, col_p, row_p, c, r, 5, 3, gather=False)
    assert st == 0
    Jo, _ = O.sample(p, c, 5, 3, 0, Q.SAMPLER_NORM)
    Io, _ = O.sample(p[::-1].copy(), r, 5, 3, 1, Q.SAMPLER_NORM)
    assert np.array_equal(host(J), Jo) and np.array_equal(host(I), Io)
    if case == "unnormalised":
        # the same draws from p scaled by a power of two
        J2, I2, *_, st = _sample(A_t, Q.SAMPLER_NORM, col_p * 2.0 ** -30, row_p * 2.0 ** -30,
                                 c, r, 5, 3, gather=False)
        assert st == 0 and np.array_equal(host(J2), Jo) and np.array_equal(host(I2), Io)


def test_sample_status_codes():
    A = np.zeros((4, 50, 60), dtype=np.float32)
    A[0, :, 3] = 1.0
    A[0, :, 9] = 1.0
    A_t = dev(A)
    col_p, row_p, _, st = probs(A_t, Q.SAMPLER_NORM)
    assert st == 0
    *_, st = _sample(A_t, Q.SAMPLER_NORM, col_p, row_p, 3, 4, 0, 0, gather=False)
    assert st == 4                                  # INSUFFICIENT_SUPPORT
    A[0, 0, 20] = 1e-7
    A_t = dev(A)
    col_p, row_p, _, st = probs(A_t, Q.SAMPLER_NORM)
    *_, st = _sample(A_t, Q.SAMPLER_NORM, col_p, row_p, 3, 4, 0, 0, max_attempts=64,
                     gather=False)
    assert st == 5                                  # SAMPLE_LIMIT
    with pytest.raises(Q.QmcurError):
        _sample(A_t, Q.SAMPLER_UNIFORM, None, None, 61, 4, 0, 0)   # c > n


# ----------------------------------------------------------- pseudo-inverse -
def _pinv(W, rcond=1e-10, rank_cap=0, Udtype=torch.float64):
    r, c = W.shape[1], W.shape[2]
    U = torch.empty(4, c, r, dtype=Udtype, device="cuda")
    rank = torch.zeros(2, dtype=torch.int32, device="cuda")
    sig = torch.empty(min(r, c), dtype=torch.float64, device="cuda")
    ws = Q.workspace(r, c, c, r, Q.PREC_FP64)
    st = Q.status_tensor()
    Q.pinv_core(dev(W), U, rcond, rank_cap, 0, rank, sig, ws, st)
    return U, int(host(rank)[0]), host(sig), run_status(st)


def _kappa_k(sig, k):
    return sig[0] / sig[k - 1] if k > 0 else 1.0


@pytest.mark.parametrize("r,c", [(30, 20), (20, 30), (17, 17), (1, 5), (6, 1)])
def test_pinv_full_rank(r, c):
    W = np.random.default_rng(r * c).standard_normal((4, r, c))
    U, k, sig, st = _pinv(W)
    assert st == 0
    Uo, ko, so = O.pinv_truncated(W)
    assert k == ko == min(r, c)
    assert rel_fro(sig, so[:min(r, c)]) < 1e-13
    assert rel_fro(host(U), Uo) < 1e-13 * _kappa_k(so, ko) * 10


def test_pinv_gauss256_intersection():
    # the FP64 workload's 40 x 40 intersection of exact rank 10
    A = synth.make("gauss256_rank10_fp64")
    out = O.qmcur(A, 40, 40, sampler=O.SAMPLER_UNIFORM, seed=0)
    U, k, sig, st = _pinv(out["W"], rcond=1e-10)
    assert st == 0 and k == out["rank"] == 10
    assert rel_fro(host(U), out["U"]) < 1e-12


def test_pinv_rank_cap_noisy():
    W, _ = synth.lowrank_gaussian(60, 50, 8, seed=21, noise_rel=1e-3, dtype=np.float64)
    U, k, sig, st = _pinv(W, rcond=1e-10, rank_cap=8)
    assert st == 0 and k == 8
    Uo, ko, so = O.pinv_truncated(W, 1e-10, 8)
    assert rel_fro(sig, so) < 1e-13
    assert rel_fro(host(U), Uo) < 1e-13 * _kappa_k(so, 8) ** 2 * (so[0] / (so[7] - so[8]))


def test_pinv_zero_and_f32_output():
    W = np.zeros((4, 5, 7))
    U, k, sig, st = _pinv(W)
    assert st == 0 and k == 0 and np.all(host(U) == 0)
    W = np.random.default_rng(3).standard_normal((4, 9, 6))
    U, k, _, st = _pinv(W, Udtype=torch.float32)
    assert st == 0 and rel_fro(host(U), O.pinv_truncated(W)[0]) < 1e-6


# ----------------------------------------------------------- reconstruction -
@pytest.mark.parametrize("m,n,c,r", [(200, 300, 40, 30), (129, 65, 7, 9), (1, 1, 1, 1)])
def test_reconstruct_fp64_and_fp32(m, n, c, r):
    rng = np.random.default_rng(m + n)
    C = rng.standard_normal((4, m, c))
    U = rng.standard_normal((4, c, r))
    R = rng.standard_normal((4, r, n))
    Zo = O.reconstruct(C, U, R)
    Z = torch.empty(4, m, n, dtype=torch.float64, device="cuda")
    ws = Q.workspace(m, n, c, r, Q.PREC_FP64)
    st = Q.status_tensor()
    Q.reconstruct(dev(C), dev(U), dev(R), Q.PREC_FP64, Z, ws, st)
    assert run_status(st) == 0
    assert rel_fro(host(Z), Zo) < 1e-12
    C32, U32_, R32 = (x.astype(np.float32) for x in (C, U, R))
    Zo32 = O.reconstruct(C32.astype(np.float64), U32_.astype(np.float64), R32.astype(np.float64))
    Z32 = torch.empty(4, m, n, dtype=torch.float32, device="cuda")
    ws = Q.workspace(m, n, c, r, Q.PREC_FP32)
    Q.reconstruct(dev(C32), dev(U32_), dev(R32), Q.PREC_FP32, Z32, ws, st)
    assert run_status(st) == 0
    assert rel_fro(host(Z32), Zo32) < 1e-5


def test_residual_fused_and_standalone():
    m, n, c, r = 333, 515, 24, 20
    A, _ = synth.lowrank_gaussian(m, n, 6, seed=5, noise_rel=1e-2)
    out = O.qmcur(A.astype(np.float64), c, r, sampler=O.SAMPLER_UNIFORM, seed=4, rank_cap=6)
    U32_ = out["U"].astype(np.float32).astype(np.float64)
    Zo = O.reconstruct(out["C"], U32_, out["R"])
    mask = synth.bernoulli_mask(m, n, seed=6)
    for msk in (None, mask):
        rel_o, num_o, den_o = O.residual(A.astype(np.float64), Zo, msk)
        out3 = torch.empty(3, dtype=torch.float64, device="cuda")
        ws = Q.workspace(m, n, c, r, Q.PREC_FP32)
        st = Q.status_tensor()
        mk = None if msk is None else dev(msk)
        Q.residual(dev(A), out3, dev(out["C"].astype(np.float32)), dev(U32_.astype(np.float32)),
                   dev(out["R"].astype(np.float32)), Q.PREC_FP32, mk, None, ws, st)
        assert run_status(st) == 0
        o = host(out3)
        assert abs(o[0] - rel_o) < 1e-5 and abs(o[2] - den_o) < 24 * U32 * den_o
        Q.residual(dev(A), out3, mask=mk, Z=dev(Zo.astype(np.float32)), ws=ws, status=st)
        assert run_status(st) == 0
        o2 = host(out3)
        assert abs(o2[0] - rel_o) < 1e-5 and abs(o2[2] - den_o) < 1e-12 * den_o


def test_residual_standalone_masked_nan_and_fp64():
    # the standalone pass selects masked-out entries away: a NaN in A or Z
    # where the mask is 0 does not reach the sums; FP64 inputs are summed in
    # FP64, FP32 ones in float-float, both to FP64 level (1e-12 on the two sums)
    m, n = 45, 300   # 45 rows: five 8-row tiles and a ragged one
    rng = np.random.default_rng(12)
    A = rng.standard_normal((4, m, n))
    Z = A + 1e-3 * rng.standard_normal((4, m, n))
    mask = synth.bernoulli_mask(m, n, seed=13, p_observed=0.6)
    A[1, 3, 7] = np.nan
    Z[2, 40, 299] = np.nan
    mask[3, 7] = 0
    mask[40, 299] = 0
    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-12)):
        Ad, Zd = A.astype(dt), Z.astype(dt)
        rel_o, num_o, den_o = O.residual(np.nan_to_num(Ad.astype(np.float64)),
                                         np.nan_to_num(Zd.astype(np.float64)), mask)
        out3 = torch.empty(3, dtype=torch.float64, device="cuda")
        ws = Q.workspace(m, n, 4, 4, Q.PREC_FP32)
        st = Q.status_tensor()
        Q.residual(dev(Ad), out3, mask=dev(mask), Z=dev(Zd), ws=ws, status=st)
        assert run_status(st) == 0
        o = host(out3)
        assert np.all(np.isfinite(o)), o
        assert abs(o[1] - num_o) < tol * num_o and abs(o[2] - den_o) < tol * den_o, (dt, o, num_o, den_o)


# ---------------------------------------------------------------- whole path -
def test_decompose_gauss256_fp64():
    w = synth.WORKLOADS["gauss256_rank10_fp64"]
    A = synth.make("gauss256_rank10_fp64")
    D = Q.Decomposition(256, 256, 40, 40, Q.PREC_FP64, dtype=torch.float64)
    Q.decompose(dev(A), D, sampler=Q.SAMPLER_UNIFORM, seed=0, rcond=w["rcond"])
    assert run_status(D.status) == 0
    out = O.qmcur(A, 40, 40, sampler=O.SAMPLER_UNIFORM, seed=0, rcond=w["rcond"])
    assert np.array_equal(host(D.J), out["J"]) and np.array_equal(host(D.I), out["I"])
    assert int(host(D.rank)[0]) == 10
    assert rel_fro(host(D.U), out["U"]) < 1e-12
    o = host(D.out3)
    assert o[0] < 1e-12 and out["rel"] < 1e-12


# ----------------------------------------------- FP32 subspace pseudo-inverse -
def _pinv_fast(W, rank_cap):
    r, c = W.shape[1], W.shape[2]
    U = torch.empty(4, c, r, dtype=torch.float64, device="cuda")
    rank = torch.zeros(2, dtype=torch.int32, device="cuda")
    ws = Q.workspace(r, c, c, r, Q.PREC_FP32)
    st = Q.status_tensor()
    Q.pinv_core(dev(W), U, 1e-10, rank_cap, 0, rank, None, ws, st, method=Q.PINV_SUBSPACE_FP32)
    return U, host(rank), run_status(st)


@pytest.mark.parametrize("r,c,k,noise", [(200, 200, 50, 1e-3), (120, 90, 12, 1e-4),
                                         (64, 80, 30, 0.0), (33, 17, 5, 1e-3),
                                         (150, 131, 100, 1e-3), (9, 11, 1, 1e-3),
                                         (97, 140, 97, 0.0)])
def test_pinv_subspace_fp32(r, c, k, noise):
    W = synth.lowrank_gaussian(r, c, k, seed=r + c + k, noise_rel=noise)[0]
    U, info, st = _pinv_fast(W, k)
    assert st == 0 and info[0] == k
    W64 = W.astype(np.float64)
    Uo, ko, so = O.pinv_truncated(W64, 1e-10, k)
    kap = so[0] / so[k - 1]
    err = rel_fro(host(U), Uo)
    # FP32 subspace iteration: rounding ~ u32 * kappa_k per step, a few steps
    assert err < 64 * U32 * kap * kap, (err, kap)
    # reconstruction through the fast core equals the oracle's to 1e-5
    A = np.zeros((4, r + 7, c + 5))
    A[:, :r, :c] = W64
    C, R = A[:, :, :c], A[:, :r, :]
    Zf = O.reconstruct(C, host(U), R)
    Zo = O.reconstruct(C, Uo, R)
    assert rel_fro(Zf, Zo) < 1e-5


def test_pinv_subspace_needs_cap():
    W = np.random.default_rng(0).standard_normal((4, 10, 10))
    with pytest.raises(Q.QmcurError) as e:
        _pinv_fast(W, 0)
    assert e.value.code == 7


def test_pinv_subspace_cap_limit():
    # k = min(rank_cap, r, c) above 100 is refused before any launch
    W = np.random.default_rng(1).standard_normal((4, 110, 120))
    with pytest.raises(Q.QmcurError) as e:
        _pinv_fast(W, 101)
    assert e.value.code == 7


# ----------------------------------------------- tensor-core (tcgen05) GEMMs -
# Tolerance per split: TF32X3 and BF16X6 carry ~22-24 significant bits per
# operand (relative Frobenius error ~1e-7 expected, bound 1e-5); BF16X3 carries
# ~17 bits per operand (hi + lo), so its products are exact to ~2^-16 and the
# bound is 6e-5; the mixed split (BF16X6 for U R, BF16X3 for C T) meets 1e-5
# on these well-conditioned random factors.
TC_TOL = {Q.PREC_TF32X3: 1e-5, Q.PREC_BF16X6: 1e-5, Q.PREC_BF16X3: 6e-5,
          Q.PREC_BF16_MIXED: 1e-5}


@pytest.mark.parametrize("prec", [Q.PREC_BF16X3, Q.PREC_BF16X6, Q.PREC_TF32X3,
                                  Q.PREC_BF16_MIXED])
@pytest.mark.parametrize("m,n,c,r", [(128, 64, 64, 64), (200, 300, 40, 30), (129, 65, 7, 9),
                                     (300, 700, 200, 120), (1, 1, 1, 1), (2048, 512, 48, 40),
                                     (1100, 1500, 48, 40)])
def test_reconstruct_tensor_cores(prec, m, n, c, r):
    # Z = C T's tile width follows the tile count: 2048 x 512 takes 64 columns,
    # the smaller shapes 32 (and K splits), 1100 x 1500 and 2048 x 2048 take
    # 112 (ragged rows and a 44-column last tile here), 4096 x 4096 128
    rng = np.random.default_rng(m * 7 + n + c)
    C, U, R = (rng.standard_normal(s).astype(np.float32) for s in
               ((4, m, c), (4, c, r), (4, r, n)))
    Zo = O.reconstruct(C.astype(np.float64), U.astype(np.float64), R.astype(np.float64))
    Z = torch.empty(4, m, n, dtype=torch.float32, device="cuda")
    ws = Q.workspace(m, n, c, r, prec)
    st = Q.status_tensor()
    Q.reconstruct(dev(C), dev(U), dev(R), prec, Z, ws, st)
    assert run_status(st) == 0
    assert rel_fro(host(Z), Zo) < TC_TOL[prec]


@pytest.mark.parametrize("prec", [Q.PREC_BF16X3, Q.PREC_BF16X6, Q.PREC_TF32X3,
                                  Q.PREC_BF16_MIXED])
@pytest.mark.parametrize("m,n", [(333, 515), (1100, 1500)])
def test_residual_tensor_cores_fused(prec, m, n):
    # 333 x 515 runs 32-column tiles, 1100 x 1500 112-column tiles
    c, r = 24, 20
    A, _ = synth.lowrank_gaussian(m, n, 6, seed=5, noise_rel=1e-2)
    out = O.qmcur(A.astype(np.float64), c, r, sampler=O.SAMPLER_UNIFORM, seed=4, rank_cap=6)
    U32_ = out["U"].astype(np.float32)
    Zo = O.reconstruct(out["C"], U32_.astype(np.float64), out["R"])
    mask = synth.bernoulli_mask(m, n, seed=6)
    for msk in (None, mask):
        rel_o, num_o, den_o = O.residual(A.astype(np.float64), Zo, msk)
        out3 = torch.empty(3, dtype=torch.float64, device="cuda")
        ws = Q.workspace(m, n, c, r, prec)
        st = Q.status_tensor()
        Q.residual(dev(A), out3, dev(out["C"].astype(np.float32)), dev(U32_),
                   dev(out["R"].astype(np.float32)), prec, None if msk is None else dev(msk),
                   None, ws, st)
        assert run_status(st) == 0
        o = host(out3)
        assert abs(o[0] - rel_o) < 1e-5 and abs(o[2] - den_o) < 24 * U32 * den_o
        # a second call on the same workspace folds the same partials in the
        # same order: bit-identical sums
        Q.residual(dev(A), out3, dev(out["C"].astype(np.float32)), dev(U32_),
                   dev(out["R"].astype(np.float32)), prec, None if msk is None else dev(msk),
                   None, ws, st)
        assert run_status(st) == 0
        assert np.array_equal(host(out3), o)
