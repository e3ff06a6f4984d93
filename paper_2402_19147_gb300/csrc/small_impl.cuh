// Device code of the small dense quaternion kernels, shared by the
// standalone kernels (small.cu) and the fused subspace pseudo-inverse
// (pinv_fast.cu).  A GEMM tile is computed by a worker of 256 threads; the
// Cholesky inverse by one CTA of 512.
#pragma once

#include "small.cuh"

namespace qmcur {

constexpr int kSmTS = 16;    // 16 x 16 quaternion outputs per tile, one per thread
constexpr int kSmBK = 32;    // k-slice per stage; the next is prefetched into registers
constexpr int kSmTileThreads = 256;
// Shared memory of one tile worker, in float4 (one quaternion each): the
// op(X) slice [16][32 + 1] and the op(Y)^T slice [32][16 + 1]; the padding
// keeps the transposed stores free of bank conflicts.
constexpr int kSmGemmQuats = kSmTS * (kSmBK + 1) + kSmBK * (kSmTS + 1);

struct SmallGemmArgs {
  QPtr X, Y, Z;
  int M, N, K;
  float alpha, beta;
  int xh, yh;
};

// Named barrier over the 256 threads of one tile worker.
__device__ __forceinline__ void worker_sync(int bar_id) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(kSmTileThreads) : "memory");
}

// Loads of one k-slice of one operand, viewed as a (rows x k) matrix: 16 x 32
// entries, two per thread.  KMAJOR: entry (r, k) lives at P[r][k] (read
// coalesced along k); otherwise at P[k][r] (coalesced along r).  CONJ
// negates the imaginary planes.  Slots (r, k) are returned for the store.
template <bool KMAJOR, bool CONJ>
__device__ __forceinline__ void sm_load(const QPtr& P, int rows_lim, int k_lim, int r0, int k0,
                                        int tid, float4 v[2], int sr[2], int sk[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * kSmTileThreads;
    int rr, kk;
    if (KMAJOR) { rr = e / kSmBK; kk = e % kSmBK; }
    else { kk = e / kSmTS; rr = e % kSmTS; }
    const int gr = r0 + rr, gk = k0 + kk;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr < rows_lim && gk < k_lim) {
      const int64_t off = KMAJOR ? (int64_t)gr * P.ld + gk : (int64_t)gk * P.ld + gr;
      a.x = reinterpret_cast<const float*>(P.p[0])[off];
      a.y = reinterpret_cast<const float*>(P.p[1])[off];
      a.z = reinterpret_cast<const float*>(P.p[2])[off];
      a.w = reinterpret_cast<const float*>(P.p[3])[off];
      if (CONJ) { a.y = -a.y; a.z = -a.z; a.w = -a.w; }
    }
    v[h] = a;
    sr[h] = rr;
    sk[h] = kk;
  }
}

// Accumulates one 16 x 16 output tile (tm, tn) of op(X) op(Y) over the
// k-range [kb, ke) with the 256 threads of worker `bar_id` (thread index tid
// in 0..255); thread (ty, tx) = (tid / 16, tid % 16) holds entry (ty, tx).
template <bool XH, bool YH>
__device__ __forceinline__ float4 sm_tile_acc_t(const SmallGemmArgs& a, int tm, int tn, int kb,
                                                int ke, float4* sm, int tid, int bar_id) {
  float4 (*xs)[kSmBK + 1] = reinterpret_cast<float4 (*)[kSmBK + 1]>(sm);
  float4 (*ys)[kSmTS + 1] = reinterpret_cast<float4 (*)[kSmTS + 1]>(sm + kSmTS * (kSmBK + 1));
  const int tx = tid % kSmTS, ty = tid / kSmTS;
  const int m0 = tm * kSmTS, n0 = tn * kSmTS;
  float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
  float4 xv[2], yv[2];
  int xr[2], xk[2], yr[2], yk[2];
  // op(X) as (m x k): identity -> X[m][k]; X^H -> conj(X[k][m]).
  // op(Y)^T as (n x k): identity -> Y[k][n]; Y^H -> conj(Y[n][k]).
  sm_load<!XH, XH>(a.X, a.M, ke, m0, kb, tid, xv, xr, xk);
  sm_load<YH, YH>(a.Y, a.N, ke, n0, kb, tid, yv, yr, yk);
  for (int k0 = kb; k0 < ke; k0 += kSmBK) {
    worker_sync(bar_id);   // the previous tile or slice is no longer read
    xs[xr[0]][xk[0]] = xv[0]; xs[xr[1]][xk[1]] = xv[1];
    ys[yk[0]][yr[0]] = yv[0]; ys[yk[1]][yr[1]] = yv[1];
    worker_sync(bar_id);
    if (k0 + kSmBK < ke) {
      sm_load<!XH, XH>(a.X, a.M, ke, m0, k0 + kSmBK, tid, xv, xr, xk);
      sm_load<YH, YH>(a.Y, a.N, ke, n0, k0 + kSmBK, tid, yv, yr, yk);
    }
#pragma unroll 8
    for (int l = 0; l < kSmBK; ++l) {
      const float4 p = xs[ty][l], q = ys[l][tx];
      z0 = fmaf(p.x, q.x, z0); z0 = fmaf(-p.y, q.y, z0); z0 = fmaf(-p.z, q.z, z0); z0 = fmaf(-p.w, q.w, z0);
      z1 = fmaf(p.x, q.y, z1); z1 = fmaf(p.y, q.x, z1); z1 = fmaf(p.z, q.w, z1); z1 = fmaf(-p.w, q.z, z1);
      z2 = fmaf(p.x, q.z, z2); z2 = fmaf(-p.y, q.w, z2); z2 = fmaf(p.z, q.x, z2); z2 = fmaf(p.w, q.y, z2);
      z3 = fmaf(p.x, q.w, z3); z3 = fmaf(p.y, q.z, z3); z3 = fmaf(-p.z, q.y, z3); z3 = fmaf(p.w, q.x, z3);
    }
  }
  return make_float4(z0, z1, z2, z3);
}

__device__ __forceinline__ float4 sm_tile_acc(const SmallGemmArgs& a, int tm, int tn, int kb, int ke,
                                              float4* sm, int tid, int bar_id) {
  if (!a.xh && !a.yh) return sm_tile_acc_t<false, false>(a, tm, tn, kb, ke, sm, tid, bar_id);
  if (a.xh && !a.yh) return sm_tile_acc_t<true, false>(a, tm, tn, kb, ke, sm, tid, bar_id);
  if (!a.xh && a.yh) return sm_tile_acc_t<false, true>(a, tm, tn, kb, ke, sm, tid, bar_id);
  return sm_tile_acc_t<true, true>(a, tm, tn, kb, ke, sm, tid, bar_id);
}

// Epilogue of entry (ty, tx) of tile (tm, tn): Z = alpha acc + beta Z.
__device__ __forceinline__ void sm_tile_store(const SmallGemmArgs& a, int tm, int tn, int tid,
                                              float4 acc) {
  const int i = tm * kSmTS + tid / kSmTS, j = tn * kSmTS + tid % kSmTS;
  if (i >= a.M || j >= a.N) return;
  const int64_t off = (int64_t)i * a.Z.ld + j;
  const float zz[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (a.Z.dtype == QMCUR_F64) {
      double* p = reinterpret_cast<double*>(a.Z.p[t]) + off;
      double v = (double)(a.alpha * zz[t]);
      if (a.beta != 0.f) v += (double)a.beta * *p;
      *p = v;
    } else {
      float* p = reinterpret_cast<float*>(a.Z.p[t]) + off;
      float v = a.alpha * zz[t];
      if (a.beta != 0.f) v = fmaf(a.beta, *p, v);
      *p = v;
    }
  }
}

// One whole tile: Z(tile) = alpha op(X) op(Y) + beta Z(tile).
__device__ __forceinline__ void sm_gemm_tile(const SmallGemmArgs& a, int tm, int tn, float4* sm,
                                             int tid, int bar_id) {
  sm_tile_store(a, tm, tn, tid, sm_tile_acc(a, tm, tn, 0, a.K, sm, tid, bar_id));
}

// ---------------------------------------------------------------------------
// Cholesky factor inverse of a small Hermitian positive definite matrix.
//
// Gaussian elimination of the augmented [G | I] with the pivots in order:
// after step i every row j > i has had (G_ji / G_ii) times row i subtracted
// (multipliers on the left, as quaternion row operations must be), so at the
// end the left block is U' = D L^H and the right block is B = L^-1, where
// G = L D L^H with L unit lower triangular and D real positive.  With
// R = D^(1/2) L^H (so G = R^H R, R upper triangular with a real positive
// diagonal) the inverse needed downstream is R^-1 = B^H D^(-1/2).
//
// Storage: the k x k matrix whose row j holds B_jc for c < j and U'_jc for
// c >= j.  Entry e = s * kCholThreads + tid of this row-major matrix lives in
// register slot s of thread tid (S = ceil(k^2 / kCholThreads) slots, a
// template parameter so that no slot is spent on nothing); its row is
// j = floor(e / k), formed as umulhi(e, floor((2^32 - 1) / k) + 1), which is
// exact for e, k < 2^16 (the multiplier's excess over 2^32 / k is below 1 and
// e < 2^16 keeps the product's error under 2^-16 < 1 / k).  Step i reads row
// i of both blocks from a shared-memory broadcast buffer (B_ii = 1 stored
// there); the owners of row i + 1 publish it into the other buffer as they
// update it, so one barrier per step suffices.  Rows grow with the slot
// index, so the finished rows j <= i occupy a prefix of every warp's slots:
// the slots are walked downwards and left at the first one whose 32 entries
// are all finished (a warp-uniform exit).

constexpr int kCholThreads = 512;
constexpr int kCholSlots = (kSmallCholMax * kSmallCholMax + kCholThreads - 1) / kCholThreads;

// Shared-memory bytes of sm_chol_inv: two row buffers of each block and the pivots.
__host__ __device__ constexpr size_t sm_chol_bytes() {
  return (size_t)4 * kSmallCholMax * 16 + (size_t)kSmallCholMax * 4;
}

// conj(a) b (quaternion product).
__device__ __forceinline__ float4 q_conj_mul(const float4 a, const float4 b) {
  return make_float4(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w,
                     a.x * b.y - a.y * b.x - a.z * b.w + a.w * b.z,
                     a.x * b.z + a.y * b.w - a.z * b.x - a.w * b.y,
                     a.x * b.w - a.y * b.z + a.z * b.y - a.w * b.x);
}

template <int S>
__device__ __forceinline__ void sm_chol_inv_s(const QPtr& G, int k, const QPtr& Rinv,
                                              int32_t* status, unsigned char* smraw) {
  float4* rowA = reinterpret_cast<float4*>(smraw);          // [2][kSmallCholMax]
  float4* rowB = rowA + 2 * kSmallCholMax;                  // [2][kSmallCholMax]
  float* piv = reinterpret_cast<float*>(rowB + 2 * kSmallCholMax);
  const int tid = threadIdx.x;
  const int kk = k * k;
  const unsigned kmag = 0xffffffffu / (unsigned)k + 1u;
  const float4 one = make_float4(1.f, 0.f, 0.f, 0.f);
  float4 v[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = s * kCholThreads + tid;
    v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < kk) {
      const int j = (int)__umulhi((unsigned)e, kmag), c = e - j * k;
      if (c >= j) {
        const int64_t off = (int64_t)j * G.ld + c;
        v[s] = make_float4(reinterpret_cast<const float*>(G.p[0])[off],
                           reinterpret_cast<const float*>(G.p[1])[off],
                           reinterpret_cast<const float*>(G.p[2])[off],
                           reinterpret_cast<const float*>(G.p[3])[off]);
      }
      if (j == 0) rowA[c] = v[s];
    }
  }
  if (tid == 0) rowB[0] = one;
  __syncthreads();
  const float g00 = fabsf(rowA[0].x);
  const float floor_v = (g00 > 0.f && isfinite(g00) ? g00 : 1.f) * 1e-30f;
  const int wlast = tid | 31;   // the warp's highest thread index
  for (int i = 0; i < k; ++i) {
    const float4* rA = rowA + (i & 1) * kSmallCholMax;
    const float4* rB = rowB + (i & 1) * kSmallCholMax;
    float4* nA = rowA + ((i + 1) & 1) * kSmallCholMax;
    float4* nB = rowB + ((i + 1) & 1) * kSmallCholMax;
    float d = rA[i].x;
    const bool bad = !(d > 0.f) || !isfinite(d);
    if (bad) d = floor_v;
    if (tid == 0) {
      piv[i] = d;
      if (bad) set_status(status, QMCUR_ERR_ILL_CONDITIONED);
      if (i + 1 < k) nB[i + 1] = one;
    }
    const float inv_d = 1.0f / d;
    // Re-derive each slot's (j, c) every step rather than keep 2 S
    // loop-invariant registers live beside the entries.
    unsigned kmag_i = kmag;
    asm volatile("" : "+r"(kmag_i));
    const int first_live = (i + 1) * k;   // entries below this index are finished
#pragma unroll
    for (int s = S - 1; s >= 0; --s) {
      if (s * kCholThreads + wlast < first_live) break;
      const int e = s * kCholThreads + tid;
      const int j = (int)__umulhi((unsigned)e, kmag_i), c = e - j * k;
      const bool in = (s < S - 1) || (e < kk);
      const bool left = c <= i;                       // B block, else U' block when c >= j
      const bool ok = in && j > i && (left || c >= j);
      const float4 a = rA[in ? j : 0];
      const float4 b = left ? rB[c] : rA[c];
      const float4 m = q_conj_mul(a, b);
      const float sc = ok ? inv_d : 0.f;
      v[s].x = fmaf(-m.x, sc, v[s].x);
      v[s].y = fmaf(-m.y, sc, v[s].y);
      v[s].z = fmaf(-m.z, sc, v[s].z);
      v[s].w = fmaf(-m.w, sc, v[s].w);
      if (ok && j == i + 1) {
        if (left) nB[c] = v[s];
        else nA[c] = v[s];
      }
    }
    __syncthreads();
  }
  float* O0 = reinterpret_cast<float*>(Rinv.p[0]);
  float* O1 = reinterpret_cast<float*>(Rinv.p[1]);
  float* O2 = reinterpret_cast<float*>(Rinv.p[2]);
  float* O3 = reinterpret_cast<float*>(Rinv.p[3]);
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = s * kCholThreads + tid;
    if (e < kk) {
      const int j = (int)__umulhi((unsigned)e, kmag), c = e - j * k;
      const float sc = 1.0f / sqrtf(piv[j]);
      // Rinv[c][j] = conj(B_jc) D_j^(-1/2) (c < j), D_j^(-1/2) (c == j), 0 (c > j)
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (c < j) q = make_float4(v[s].x * sc, -v[s].y * sc, -v[s].z * sc, -v[s].w * sc);
      else if (c == j) q.x = sc;
      const int64_t off = (int64_t)c * Rinv.ld + j;
      O0[off] = q.x; O1[off] = q.y; O2[off] = q.z; O3[off] = q.w;
    }
  }
  __syncthreads();
}

template <int S>
__device__ __forceinline__ void sm_chol_inv_from(int need, const QPtr& G, int k, const QPtr& Rinv,
                                                 int32_t* status, unsigned char* smraw) {
  if (need <= S) sm_chol_inv_s<S>(G, k, Rinv, status, smraw);
  else if constexpr (S < kCholSlots) sm_chol_inv_from<S + 1>(need, G, k, Rinv, status, smraw);
}

// One CTA of kCholThreads threads: Rinv = R^-1 where G = R^H R (k x k, FP32,
// 1 <= k <= kSmallCholMax; only the upper triangle of G is read).  Rinv is
// written in full (zeros below the diagonal).  A non-positive or non-finite
// pivot sets ILL_CONDITIONED and continues with a tiny pivot.
__device__ __forceinline__ void sm_chol_inv(const QPtr& G, int k, const QPtr& Rinv,
                                            int32_t* status, unsigned char* smraw) {
  sm_chol_inv_from<1>((k * k + kCholThreads - 1) / kCholThreads, G, k, Rinv, status, smraw);
}

}  // namespace qmcur
