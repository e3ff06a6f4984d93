// Rank-capped pseudo-inverse U = W_k^+ by subspace iteration in FP32.
//
// The truncated inverse of Sec. 2.2 / Algorithm 1 depends only on the top-k
// singular subspaces of W.  With k = rank_cap:
//   Y0 = W Omega (Omega a Philox Gaussian c x k), Q0 = orth(Y0)
//   P1 = orth(W^H Q0), Q1 = orth(W P1), P = orth(W^H Q1)      (two iterations)
//   W P = Q R  (CholeskyQR2),  U = P R^-1 Q^H.
// Because P has orthonormal columns, P (W P)^+ is the Moore-Penrose inverse of
// W P P^H, i.e. of W restricted to span(P); when span(P) is the top-k right
// singular subspace this is W_k^+.  The subspace error after the two
// iterations is of order (sigma_{k+1}/sigma_k)^4 plus FP32 rounding.
// orth() is CholeskyQR (G = Y^H Y = R^H R, Q = Y R^-1), applied twice
// (CholeskyQR2) where orthonormality to working accuracy matters.
//
// Every step is a small batched quaternion GEMM (op(X) op(Y), op in {N, H})
// or a one-CTA Cholesky-and-triangular-inverse, so the same kernels also
// serve many problems at once (one table entry per problem).
#include "common.cuh"
#include "small.cuh"

namespace qmcur {
namespace {

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Gaussian quaternion entries (Box-Muller on two Philox words per pair of
// components), rows x cols, row stride ld; counter (entry, 0, stream, 7).
__global__ void k_randn_q(QPtr out, int rows, int cols, uint64_t seed, uint32_t stream) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 x = philox(make_uint4((unsigned)e, (unsigned)(e >> 32), stream, 7u),
                           make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float u0 = ((float)x.x + 1.0f) * 0x1.0p-32f, v0 = (float)x.y * 0x1.0p-32f;
    const float u1 = ((float)x.z + 1.0f) * 0x1.0p-32f, v1 = (float)x.w * 0x1.0p-32f;
    const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u1));
    float s0, c0, s1, c1;
    sincospif(2.0f * v0, &s0, &c0);
    sincospif(2.0f * v1, &s1, &c1);
    const int64_t i = e / cols, j = e % cols;
    float* p0 = reinterpret_cast<float*>(out.p[0]);
    float* p1 = reinterpret_cast<float*>(out.p[1]);
    float* p2 = reinterpret_cast<float*>(out.p[2]);
    float* p3 = reinterpret_cast<float*>(out.p[3]);
    p0[i * out.ld + j] = r0 * c0;
    p1[i * out.ld + j] = r0 * s0;
    p2[i * out.ld + j] = r1 * c1;
    p3[i * out.ld + j] = r1 * s1;
  }
}

__global__ void k_to_f32(QView in, QPtr out) {
  const int64_t total = in.rows * in.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / in.cols, j = e % in.cols;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      reinterpret_cast<float*>(out.p[t])[i * out.ld + j] = (float)ld_as_double(in, t, i, j);
  }
}

}  // namespace

// Workspace of the subspace method for an r x c intersection with cap k.
struct FastWs {
  QPtr W32, Om, Y, Q, Z, P, G, R, Ri, T;
  int32_t* info;
};

static QPtr carve_q(Carve& cv, int64_t rows, int64_t cols) {
  QPtr q;
  const int64_t ld = (cols + 3) / 4 * 4;
  float* base = cv.take<float>((size_t)(4 * rows * ld));
  for (int t = 0; t < 4; ++t) q.p[t] = base ? base + (size_t)t * rows * ld : nullptr;
  q.ld = ld;
  q.dtype = QMCUR_F32;
  return q;
}

static FastWs carve_fast(Carve& cv, int64_t r, int64_t c, int64_t k) {
  FastWs w;
  const int64_t mx = r > c ? r : c;
  w.W32 = carve_q(cv, r, c);
  w.Om = carve_q(cv, c, k);
  w.Y = carve_q(cv, mx, k);
  w.Q = carve_q(cv, mx, k);
  w.Z = carve_q(cv, mx, k);
  w.P = carve_q(cv, mx, k);
  w.G = carve_q(cv, k, k);
  w.R = carve_q(cv, k, k);
  w.Ri = carve_q(cv, k, k);
  w.T = carve_q(cv, mx, k);
  w.info = cv.take<int32_t>(4);
  return w;
}

size_t pinv_fast_ws_bytes(int64_t r, int64_t c, int64_t k) {
  Carve cv(nullptr, 0);
  carve_fast(cv, r, c, k);
  return cv.off;
}

// Y (rows x k) -> Q = Y R^-1 by CholeskyQR with `passes` passes (2 =
// CholeskyQR2).  The inverse triangular factors of the passes are left in
// Rinv1 (first) and Rinv2 (second), so that Y = Q R2 R1.
static qmcur_status cholqr(const QPtr& Y, int rows, int k, const QPtr& Q, FastWs& w, int passes,
                           QPtr Rinv1, QPtr Rinv2, int32_t* status, cudaStream_t st) {
  qmcur_status s;
  const QPtr& Qa = passes == 2 ? w.T : Q;
  if ((s = small_qgemm(true, false, k, k, rows, 1.0f, Y, Y, 0.0f, w.G, st)) != QMCUR_OK) return s;
  if ((s = small_chol_inv(w.G, k, Rinv1, status, st)) != QMCUR_OK) return s;
  if ((s = small_qgemm(false, false, rows, k, k, 1.0f, Y, Rinv1, 0.0f, Qa, st)) != QMCUR_OK) return s;
  if (passes == 1) return QMCUR_OK;
  if ((s = small_qgemm(true, false, k, k, rows, 1.0f, w.T, w.T, 0.0f, w.G, st)) != QMCUR_OK) return s;
  if ((s = small_chol_inv(w.G, k, Rinv2, status, st)) != QMCUR_OK) return s;
  return small_qgemm(false, false, rows, k, k, 1.0f, w.T, Rinv2, 0.0f, Q, st);
}

qmcur_status launch_pinv_fast(const qmcur_qmat* W, int32_t rank_cap, qmcur_qmat* U,
                              int32_t* rank_out, uint64_t seed, void* ws, size_t ws_bytes,
                              int32_t* dev_status, cudaStream_t st) {
  const int64_t r = W->rows, c = W->cols;
  const int64_t nmin = r < c ? r : c;
  if (rank_cap < 1) return QMCUR_ERR_UNSUPPORTED;   // the method needs the cap
  const int k = (int)(rank_cap < nmin ? rank_cap : nmin);
  if (k > kSmallCholMax) return QMCUR_ERR_UNSUPPORTED;
  Carve cv(ws, ws_bytes);
  FastWs w = carve_fast(cv, r, c, k);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  QPtr Rinv1 = w.R, Rinv2 = w.Ri;
  {
    int blocks = (int)((r * c + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    k_to_f32<<<blocks, 256, 0, st>>>(view(W), w.W32);
    blocks = (int)((c * k + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    k_randn_q<<<blocks, 256, 0, st>>>(w.Om, (int)c, k, seed, 0x51u);
  }
  const int ri = (int)r, ci = (int)c;
  qmcur_status s;
  // Y0 = W Omega -> Q
  if ((s = small_qgemm(false, false, ri, k, ci, 1.0f, w.W32, w.Om, 0.0f, w.Y, st)) != QMCUR_OK) return s;
  // Intermediate bases only have to span the subspaces: one CholeskyQR pass.
  // The last P must be orthonormal to working accuracy and W P = Q R2 R1
  // exact to it: CholeskyQR2 for both.
  if ((s = cholqr(w.Y, ri, k, w.Q, w, 1, Rinv1, Rinv2, dev_status, st)) != QMCUR_OK) return s;
  for (int it = 0; it < 2; ++it) {
    const int passes = it == 1 ? 2 : 1;
    // P = orth(W^H Q)
    if ((s = small_qgemm(true, false, ci, k, ri, 1.0f, w.W32, w.Q, 0.0f, w.Z, st)) != QMCUR_OK) return s;
    if ((s = cholqr(w.Z, ci, k, w.P, w, passes, Rinv1, Rinv2, dev_status, st)) != QMCUR_OK) return s;
    // Q = orth(W P)
    if ((s = small_qgemm(false, false, ri, k, ci, 1.0f, w.W32, w.P, 0.0f, w.Y, st)) != QMCUR_OK) return s;
    if ((s = cholqr(w.Y, ri, k, w.Q, w, passes, Rinv1, Rinv2, dev_status, st)) != QMCUR_OK) return s;
  }
  // U = P R1^-1 R2^-1 Q^H
  if ((s = small_qgemm(false, false, ci, k, k, 1.0f, w.P, Rinv1, 0.0f, w.Z, st)) != QMCUR_OK) return s;
  if ((s = small_qgemm(false, false, ci, k, k, 1.0f, w.Z, Rinv2, 0.0f, w.T, st)) != QMCUR_OK) return s;
  QPtr Uo;
  for (int t = 0; t < 4; ++t) Uo.p[t] = U->plane[t];
  Uo.ld = U->ld;
  Uo.dtype = U->dtype;
  if ((s = small_qgemm(false, true, ci, ri, k, 1.0f, w.T, w.Q, 0.0f, Uo, st)) != QMCUR_OK) return s;
  if (rank_out != nullptr) small_set_rank(rank_out, k, 2, st);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
