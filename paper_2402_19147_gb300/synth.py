"""Seeded synthetic quaternion matrices shaped like the paper's workloads.

This module only *makes inputs*.  It holds none of the QMCUR steps (norms,
sampling, gathers, pseudo-inverse, reconstruction, residual) and imports
neither the CUDA binding nor the oracle; both sides take their inputs from
here.  Every array is returned as split planes of shape (4, m, n).

Workloads (the paper's own data sets are not available, so these stand in):

* ``lowrank_gaussian`` - X = L Rt (+ E), Gaussian quaternion factors, the
  synthetic model of Examples 4.1-4.2 (Sec. 4).  The low-rank product is formed
  in the Cayley-Dickson form X = Xa + Xb j with complex Xa, Xb:
  (Xa + Xb j)(Ya + Yb j) = (Xa Ya - Xb conj(Yb)) + (Xa Yb + Xb conj(Ya)) j.
* ``smooth_color`` - a pure quaternion "colour image" X = R i + G j + B k
  (Example 4.3's encoding) whose channels are sums of separable cosine modes.
* ``batch_problems`` - the uneven batch of small low-rank problems.
* ``bernoulli_mask`` - an observation set Omega (Example 4.4's random missing
  entries), one bit per quaternion entry.
* ``svd_lowrank`` - X = W_k Sigma_k V_k^H with orthonormal quaternion columns
  in W_k, V_k (Example 4.1's model), plus ``gaussian_noise``.
"""
import numpy as np


def _cd_product(X, Y):
    Xa = X[0] + 1j * X[1]
    Xb = X[2] + 1j * X[3]
    Ya = Y[0] + 1j * Y[1]
    Yb = Y[2] + 1j * Y[3]
    Za = Xa @ Ya - Xb @ Yb.conj()
    Zb = Xa @ Yb + Xb @ Ya.conj()
    return np.stack([Za.real, Za.imag, Zb.real, Zb.imag])


def lowrank_gaussian(m, n, rank, seed, noise_rel=0.0, dtype=np.float32):
    """X = L Rt + E.

    Draw order from numpy.random.default_rng(seed): L (4 x m x rank, N(0,1)),
    then Rt (4 x rank x n, N(0,1)), then (only if noise_rel > 0) E (4 x m x n,
    N(0,1)) scaled so that each quaternion entry has standard deviation
    sigma = noise_rel * ||L Rt||_F / sqrt(m n), i.e. each of its four
    components has standard deviation sigma / 2.
    Returns (X, X_clean), both of `dtype`.
    """
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((4, m, rank))
    Rt = rng.standard_normal((4, rank, n))
    X0 = _cd_product(L, Rt)
    X = X0
    if noise_rel > 0.0:
        sigma = noise_rel * np.sqrt(np.sum(X0 * X0)) / np.sqrt(m * n)
        X = X0 + rng.standard_normal((4, m, n)) * (0.5 * sigma)
    return np.ascontiguousarray(X.astype(dtype)), np.ascontiguousarray(X0.astype(dtype))


def smooth_color(m, n, modes, seed, offset=0.5, clip=True, max_freq=16,
                 dtype=np.float32, distinct=False, bounded_amp=False):
    """Pure quaternion field X = R i + G j + B k (real plane zero).

    For each channel in the order R, G, B the generator draws f (modes ints in
    [0, max_freq]), g (same), phi (U[0, 2pi)), psi (U[0, 2pi)) and
    a (N(0,1) * 0.5 / sqrt(modes)), then sets
    F[y, x] = offset + sum_t a_t cos(2 pi f_t x / n + phi_t) cos(2 pi g_t y / m + psi_t)
    for row y and column x, clipped to [0, 1] when `clip`.
    With `distinct`, all 3*modes column frequencies and all 3*modes row
    frequencies are instead drawn up front without replacement from
    [1, max_freq] (first f, then g; channel ch takes entries ch*modes ..), so
    that with max_freq < min(m, n)/2, no offset and no clipping the Fourier
    vectors are linearly independent: every channel has rank modes and X has
    quaternion rank exactly 3*modes.  With `bounded_amp` the amplitudes are
    a = s * (0.5 + 0.5 v) * 0.5 / sqrt(modes) with v ~ U[0, 1) and s a random
    sign (both drawn in place of the Gaussian a), so no mode is negligible.
    """
    rng = np.random.default_rng(seed)
    X = np.zeros((4, m, n), dtype=np.float64)
    x = np.arange(n, dtype=np.float64)
    y = np.arange(m, dtype=np.float64)
    if distinct:
        fall = rng.choice(np.arange(1, max_freq + 1), size=3 * modes, replace=False)
        gall = rng.choice(np.arange(1, max_freq + 1), size=3 * modes, replace=False)
    for ch in range(3):
        if distinct:
            f = fall[ch * modes:(ch + 1) * modes]
            g = gall[ch * modes:(ch + 1) * modes]
        else:
            f = rng.integers(0, max_freq + 1, size=modes)
            g = rng.integers(0, max_freq + 1, size=modes)
        phi = rng.uniform(0.0, 2 * np.pi, size=modes)
        psi = rng.uniform(0.0, 2 * np.pi, size=modes)
        if bounded_amp:
            v = rng.random(modes)
            sgn = np.where(rng.random(modes) < 0.5, -1.0, 1.0)
            a = sgn * (0.5 + 0.5 * v) * (0.5 / np.sqrt(modes))
        else:
            a = rng.standard_normal(modes) * (0.5 / np.sqrt(modes))
        colf = np.cos(2 * np.pi * np.outer(x, f) / n + phi)     # n x modes
        rowf = np.cos(2 * np.pi * np.outer(y, g) / m + psi)     # m x modes
        F = offset + (rowf * a) @ colf.T
        if clip:
            F = np.clip(F, 0.0, 1.0)
        X[ch + 1] = F
    return np.ascontiguousarray(X.astype(dtype))


def _orthonormal_columns(rng, m, k):
    """A quaternion m x k matrix Q with Q^H Q = I: the polar factor of a
    Gaussian quaternion matrix G, G (G^H G)^{-1/2}.  It is formed on the
    complex adjoint chi(G) = [[Ga, Gb], [-conj(Gb), conj(Ga)]] (G = Ga + Gb j),
    whose polar factor U V^H (numpy's SVD) is chi(Q), and read back from the
    first block row."""
    G = rng.standard_normal((4, m, k))
    Ga, Gb = G[0] + 1j * G[1], G[2] + 1j * G[3]
    chi = np.block([[Ga, Gb], [-Gb.conj(), Ga.conj()]])
    Us, _, Vh = np.linalg.svd(chi, full_matrices=False)
    P = Us @ Vh
    Qa, Qb = P[:m, :k], P[:m, k:]
    return np.stack([Qa.real, Qa.imag, Qb.real, Qb.imag])


def svd_lowrank(m, n, k, seed, smin=1.0, smax=10.0, dtype=np.float64):
    """X = W_k Sigma_k V_k^H (Example 4.1): W_k (m x k) and V_k (n x k) with
    orthonormal quaternion columns, Sigma_k = diag of k values drawn
    uniformly from [smin, smax], sorted descending.  Draw order from
    default_rng(seed): W_k's Gaussian, V_k's Gaussian, the k values.
    Returns (X, W_k, V_k, sigma)."""
    rng = np.random.default_rng(seed)
    Wk = _orthonormal_columns(rng, m, k)
    Vk = _orthonormal_columns(rng, n, k)
    sig = np.sort(rng.uniform(smin, smax, size=k))[::-1].copy()
    WS = Wk * sig[None, None, :]
    VkH = np.stack([Vk[0].T, -Vk[1].T, -Vk[2].T, -Vk[3].T])   # conjugate transpose
    X = _cd_product(WS, VkH)
    return X.astype(dtype), Wk, Vk, sig


def gaussian_noise(m, n, sigma, seed, dtype=np.float64):
    """E = E0 + E1 i + E2 j + E3 k with i.i.d. N(0, sigma^2) components
    (Example 4.1; its "variance sigma" is read as the standard deviation)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((4, m, n)) * sigma).astype(dtype)


def bernoulli_mask(m, n, seed, p_observed=0.5):
    """Omega: uint8 m x n, 1 = observed, i.i.d. Bernoulli(p_observed)."""
    rng = np.random.default_rng(seed)
    return (rng.random((m, n)) < p_observed).astype(np.uint8)


def batch_problems(count=512, seed=3, ms=(64, 128, 256, 512),
                   ns=(64, 192, 384, 768), rank_lo=5, rank_hi=40,
                   noise_rel=1e-4, dtype=np.float32):
    """Uneven batch of low-rank problems.

    Draw order from default_rng(seed): m indices, n indices, ranks (count
    each); then per problem b a child seed = seed * 1_000_003 + b feeds
    ``lowrank_gaussian``.  c = min(2 rank, n), r = min(2 rank, m).
    Returns a list of dicts with keys X, m, n, rank, c, r.
    """
    rng = np.random.default_rng(seed)
    mi = rng.integers(0, len(ms), size=count)
    ni = rng.integers(0, len(ns), size=count)
    rk = rng.integers(rank_lo, rank_hi + 1, size=count)
    out = []
    for b in range(count):
        m, n, k = ms[mi[b]], ns[ni[b]], int(rk[b])
        X, _ = lowrank_gaussian(m, n, k, seed * 1_000_003 + b, noise_rel, dtype)
        out.append(dict(X=X, m=m, n=n, rank=k, c=min(2 * k, n), r=min(2 * k, m)))
    return out


def perturb_off_intersection(X, I, J, rel, seed):
    """X plus Gaussian noise of standard deviation rel * std(X) on every entry
    outside the intersection I x J (draw: default_rng(seed), shape of X).
    The intersection, and with it its rank, is left unchanged."""
    rng = np.random.default_rng(seed)
    keep = np.ones(X.shape[1:], dtype=bool)
    keep[np.asarray(I)[:, None], np.asarray(J)[None, :]] = False
    noise = rng.standard_normal(X.shape) * (rel * float(np.std(X)))
    return np.ascontiguousarray((X + noise * keep).astype(X.dtype))


# The workloads, by what they are.  `scale` shrinks a workload for tests.
WORKLOADS = {
    "gauss256_rank10_fp64": dict(kind="lowrank", m=256, n=256, rank=10, seed=0,
                                 noise_rel=0.0, dtype="f64", c=40, r=40,
                                 sampler="uniform", rank_cap=0, rcond=1e-10),
    "gauss2048_rank50_noisy": dict(kind="lowrank", m=2048, n=2048, rank=50, seed=1,
                                   noise_rel=1e-3, dtype="f32", c=200, r=200,
                                   sampler="norm", rank_cap=50, rcond=1e-10),
    "color4096_smooth100": dict(kind="smooth", m=4096, n=4096, modes=100, seed=2,
                                dtype="f32", c=500, r=500, sampler="uniform",
                                rank_cap=100, rcond=1e-10),
    "batch512_uneven": dict(kind="batch", count=512, seed=3, dtype="f32"),
    "color1024x1536_rank60_masked": dict(kind="smooth", m=1024, n=1536, modes=20,
                                         seed=4, offset=0.0, clip=False, dtype="f32",
                                         distinct=True, max_freq=96, bounded_amp=True,
                                         c=120, r=120, sampler="uniform", rank_cap=60,
                                         rcond=1e-10, mask_seed=5, perturb_rel=1e-2,
                                         perturb_seed=6),
    # Algorithm 2 (Example 4.4) on a Kodak-sized (512 x 768) colour field:
    # 10 distinct modes per channel plus the 0.5 offset, no clipping, so the
    # quaternion rank is exactly 31; 70% of the pixels missing (MR = 70%).
    "color512x768_rank31_mr70": dict(kind="smooth", m=512, n=768, modes=10, seed=7,
                                     offset=0.5, clip=False, dtype="f32", distinct=True,
                                     max_freq=64, bounded_amp=True, c=124, r=124,
                                     sampler="uniform", rank_cap=31, rcond=1e-10, mask_seed=8,
                                     p_observed=0.3, tol=1e-4, t_max=200),
}


def make(name, m=None, n=None):
    """Build the input of a named workload (optionally at another m x n)."""
    w = dict(WORKLOADS[name])
    dt = np.float64 if w.get("dtype") == "f64" else np.float32
    if w["kind"] == "lowrank":
        X, _ = lowrank_gaussian(m or w["m"], n or w["n"], w["rank"], w["seed"],
                                w["noise_rel"], dt)
        return X
    if w["kind"] == "smooth":
        return smooth_color(m or w["m"], n or w["n"], w["modes"], w["seed"],
                            offset=w.get("offset", 0.5), clip=w.get("clip", True),
                            max_freq=w.get("max_freq", 16), distinct=w.get("distinct", False),
                            bounded_amp=w.get("bounded_amp", False), dtype=dt)
    raise ValueError("batch workloads are built with batch_problems()")
