// Gradient of the masked CUR reconstruction loss (FP32-level accuracy: the six
// large products on the tensor cores in the six-product BF16 split, the
// small pseudo-inverse adjoint products in FP32 on the CUDA cores).
//
//   L(A) = || P_Omega(A - C U R) ||_F^2,  C = A(:,J), R = A(I,:), W = A(I,J), U = W^+.
// With E = P_Omega(A - Z), Z = C T, T = U R and <X, Y> = Re tr(X^H Y):
//   G_C = -2 E T^H,  G_T = -2 C^H E,  G_U = G_T R^H,  G_R = U^H G_T,
//   G_W = -U^H G_U U^H + (I - W U) G_U^H U U^H + U^H U G_U^H (I - U W)
// (the derivative of the Moore-Penrose inverse at fixed rank, Golub-Pereyra,
// in quaternion form), and dL/dA = 2 E + G_C scattered to the columns J,
// + G_R to the rows I, + G_W to (I, J).  The incoming gradient `scale`
// multiplies everything.  J and I are sets, so every scatter touches each
// destination once; the three scatters run one after the other.
#include "common.cuh"
#include "small.cuh"

namespace qmcur {

__global__ void k_residual_fold(const double* partial, int64_t count, double* out3);
size_t tc_gemm_ws_bytes(int64_t M, int64_t N, int64_t K, int32_t prec);
qmcur_status tc_gemm(const QView& X, bool xh, const QView& Y, bool yh, int64_t M, int64_t N,
                     int64_t K, float alpha, const QView& Z, int32_t prec, void* ws,
                     size_t ws_bytes, int32_t* dev_status, cudaStream_t st);

// The six large products (T = U R, Z = C T and the four GEMM adjoints) run on
// the tensor cores in the six-product BF16 split, which carries FP32-level
// accuracy (each operand as three BF16 pieces, the products of order <= 2).
constexpr int32_t kBwdTcPrec = QMCUR_PREC_BF16X6;

namespace {

__global__ void k_to_qptr_f32(QView in, QPtr out) {
  const int64_t total = in.rows * in.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / in.cols, j = e % in.cols;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      reinterpret_cast<float*>(out.p[t])[i * out.ld + j] = (float)ld_as_double(in, t, i, j);
  }
}

// E = mask * (A - Z), in place over Z; dA = 2 s E; and the loss's sums.
// One CTA per kLossRows x 256 tile (the standalone residual's tiling, so
// that its partial count and k_residual_fold apply), one column per thread:
// partial[2 cta] = sum |e|^2, partial[2 cta + 1] = sum over Omega of |a|^2,
// FP32 over the thread's at most 4 kLossRows terms, FP64 from there on.
constexpr int kLossRows = 8;

__global__ void __launch_bounds__(256)
k_residual_matrix(QView A, const uint8_t* __restrict__ mask, QPtr Z, QView dA, float two_s,
                  double* __restrict__ partial) {
  const int64_t m = A.rows, n = A.cols;
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * kLossRows;
  float num = 0.f, den = 0.f;
  if (j < n) {
    // every load of the tile's column first, then the sums and stores
    float av[kLossRows][4], zv[kLossRows][4];
    bool on[kLossRows];
#pragma unroll
    for (int rr = 0; rr < kLossRows; ++rr) {
      const int64_t i = i0 + rr;
      const bool in = i < m;
      on[rr] = in && (mask == nullptr || mask[i * n + j] != 0);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        av[rr][t] = in ? (float)ld_as_double(A, t, i, j) : 0.f;
        zv[rr][t] = in ? reinterpret_cast<const float*>(Z.p[t])[i * Z.ld + j] : 0.f;
      }
    }
#pragma unroll
    for (int rr = 0; rr < kLossRows; ++rr) {
      const int64_t i = i0 + rr;
      if (i >= m) break;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float ev = on[rr] ? av[rr][t] - zv[rr][t] : 0.f;
        reinterpret_cast<float*>(Z.p[t])[i * Z.ld + j] = ev;
        st_from_double(dA, t, i, j, (double)(two_s * ev));
        num = fmaf(ev, ev, num);
        den = on[rr] ? fmaf(av[rr][t], av[rr][t], den) : den;
      }
    }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = (double)num;
  red[1][threadIdx.x] = (double)den;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
    partial[2 * cta] = red[0][0];
    partial[2 * cta + 1] = red[1][0];
  }
}

// which 0: dA(:, J[b]) += G(:, b); 1: dA(I[a], :) += G(a, :); 2: dA(I[a], J[b]) += G(a, b)
__global__ void k_scatter_add(QView dA, QPtr G, int64_t rows, int64_t cols, const int32_t* I,
                              const int32_t* J, int which) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = e / cols, b = e % cols;
    const int64_t di = (which == 0) ? a : (int64_t)I[a];
    const int64_t dj = (which == 1) ? b : (int64_t)J[b];
    if (di < 0 || di >= dA.rows || dj < 0 || dj >= dA.cols) continue;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float g = reinterpret_cast<const float*>(G.p[t])[a * G.ld + b];
      st_from_double(dA, t, di, dj, ld_as_double(dA, t, di, dj) + (double)g);
    }
  }
}

// X = I (r x r) and Y = I (c x c), the starting values of I - W U and I - U W
__global__ void k_two_eyes(QPtr X, int64_t r, QPtr Y, int64_t c) {
  const int64_t total = r * r + c * c;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool first = e < r * r;
    const int64_t f = first ? e : e - r * r, n = first ? r : c;
    const int64_t i = f / n, j = f % n;
    const QPtr& Q = first ? X : Y;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      reinterpret_cast<float*>(Q.p[t])[i * Q.ld + j] = (t == 0 && i == j) ? 1.f : 0.f;
  }
}

// Rows r0.. and columns c0.. of q, as a matrix of its own
QPtr sub_q(const QPtr& q, int64_t r0, int64_t c0) {
  QPtr v = q;
  for (int t = 0; t < 4; ++t) v.p[t] = reinterpret_cast<float*>(q.p[t]) + r0 * q.ld + c0;
  return v;
}

int64_t loss_partials(int64_t m, int64_t n) {
  return ((m + kLossRows - 1) / kLossRows) * ((n + 255) / 256);
}

QPtr take_q(Carve& cv, int64_t rows, int64_t cols) {
  QPtr q;
  const int64_t ld = (cols + 3) / 4 * 4;
  float* base = cv.take<float>((size_t)(4 * rows * ld));
  for (int t = 0; t < 4; ++t) q.p[t] = base ? base + (size_t)t * rows * ld : nullptr;
  q.ld = ld;
  q.dtype = QMCUR_F32;
  return q;
}

struct BwdWs {
  // XL = [I - W U | M3] (r x (r + c)) and YL = [M2; I - U W] ((r + c) x c), so
  // that (I - W U) M2 + M3 (I - U W) is one product XL YL
  QPtr U32, W32, T, E, GC, GT, GU, GR, X1, UUh, UhU, XL, YL, GW;
  double* partial;
  double* out3;
  void* tc;          // operand pieces and K-split partials of the tensor-core products
  size_t tc_bytes;
};

// Workspace of the largest of the six tensor-core products.
size_t bwd_tc_bytes(int64_t m, int64_t n, int64_t c, int64_t r) {
  const int32_t p = kBwdTcPrec;
  size_t b = tc_gemm_ws_bytes(c, n, r, p);                     // T = U R
  const size_t s[5] = {tc_gemm_ws_bytes(m, n, c, p),            // Z = C T
                       tc_gemm_ws_bytes(m, c, n, p),            // G_C = E T^H
                       tc_gemm_ws_bytes(c, n, m, p),            // G_T = C^H E
                       tc_gemm_ws_bytes(c, r, n, p),            // G_U = G_T R^H
                       tc_gemm_ws_bytes(r, n, c, p)};           // G_R = U^H G_T
  for (size_t x : s) b = x > b ? x : b;
  return b;
}

QView qv(const QPtr& q, int64_t rows, int64_t cols) {
  QView v;
  for (int t = 0; t < 4; ++t) v.p[t] = q.p[t];
  v.rows = rows;
  v.cols = cols;
  v.ld = q.ld;
  v.dtype = q.dtype;
  return v;
}

BwdWs carve_bwd(Carve& cv, int64_t m, int64_t n, int64_t c, int64_t r) {
  BwdWs w;
  w.U32 = take_q(cv, c, r);
  w.W32 = take_q(cv, r, c);
  w.T = take_q(cv, c, n);
  w.E = take_q(cv, m, n);
  w.GC = take_q(cv, m, c);
  w.GT = take_q(cv, c, n);
  w.GU = take_q(cv, c, r);
  w.GR = take_q(cv, r, n);
  w.X1 = take_q(cv, r, r);
  w.UUh = take_q(cv, c, c);
  w.UhU = take_q(cv, r, r);
  w.XL = take_q(cv, r, r + c);
  w.YL = take_q(cv, r + c, c);
  w.GW = take_q(cv, r, c);
  w.partial = cv.take<double>(2 * loss_partials(m, n));
  w.out3 = cv.take<double>(4);
  w.tc_bytes = bwd_tc_bytes(m, n, c, r);
  w.tc = cv.take<char>(w.tc_bytes);
  return w;
}

int blocks_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

size_t backward_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r) {
  Carve cv(nullptr, 0);
  carve_bwd(cv, m, n, c, r);
  return cv.off;
}

qmcur_status launch_backward(const qmcur_qmat* A, const uint8_t* mask, const int32_t* J,
                             const int32_t* I, const qmcur_qmat* C, const qmcur_qmat* U,
                             const qmcur_qmat* R, const qmcur_qmat* W, double scale, qmcur_qmat* dA,
                             double* loss_out, void* ws, size_t ws_bytes, int32_t* dev_status,
                             cudaStream_t st) {
  if (!valid_qmat(A) || !valid_qmat(C) || !valid_qmat(U) || !valid_qmat(R) || !valid_qmat(W) ||
      !valid_qmat(dA) || J == nullptr || I == nullptr)
    return QMCUR_ERR_INVALID_ARG;
  const int64_t m = A->rows, n = A->cols, c = C->cols, r = R->rows;
  if (C->rows != m || R->cols != n || U->rows != c || U->cols != r || W->rows != r ||
      W->cols != c || dA->rows != m || dA->cols != n || m < 1 || n < 1 || c < 1 || r < 1)
    return QMCUR_ERR_INVALID_ARG;
  if (C->dtype != QMCUR_F32 || R->dtype != QMCUR_F32) return QMCUR_ERR_INVALID_ARG;
  if (m > INT32_MAX || n > INT32_MAX) return QMCUR_ERR_UNSUPPORTED;
  Carve cv(ws, ws_bytes);
  BwdWs w = carve_bwd(cv, m, n, c, r);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  const int ci = (int)c, ri = (int)r;
  QPtr Cq, Rq;
  for (int t = 0; t < 4; ++t) { Cq.p[t] = C->plane[t]; Rq.p[t] = R->plane[t]; }
  Cq.ld = C->ld; Rq.ld = R->ld;
  Cq.dtype = Rq.dtype = QMCUR_F32;
  const float s = (float)scale;
  qmcur_status e;
  k_to_qptr_f32<<<blocks_for(c * r), 256, 0, st>>>(view(U), w.U32);
  k_to_qptr_f32<<<blocks_for(r * c), 256, 0, st>>>(view(W), w.W32);
  const QView vU = qv(w.U32, c, r), vR = qv(Rq, r, n), vC = qv(Cq, m, c), vT = qv(w.T, c, n),
              vE = qv(w.E, m, n), vGT = qv(w.GT, c, n);
  auto tc = [&](const QView& X, bool xh, const QView& Y, bool yh, int64_t M, int64_t N,
                int64_t K, float alpha, const QPtr& Z) {
    return tc_gemm(X, xh, Y, yh, M, N, K, alpha, qv(Z, M, N), kBwdTcPrec, w.tc, w.tc_bytes,
                   dev_status, st);
  };
  // forward pieces: T = U R, Z = C T (into E); then in one pass
  // E = P_Omega(A - Z), dA = 2 s E and the loss's sums, folded in order
  if ((e = tc(vU, false, vR, false, c, n, r, 1.f, w.T)) != QMCUR_OK) return e;
  if ((e = tc(vC, false, vT, false, m, n, c, 1.f, w.E)) != QMCUR_OK) return e;
  {
    const dim3 lgrid((unsigned)((n + 255) / 256), (unsigned)((m + kLossRows - 1) / kLossRows));
    if (lgrid.y > 65535) return QMCUR_ERR_UNSUPPORTED;
    k_residual_matrix<<<lgrid, 256, 0, st>>>(view(A), mask, w.E, view(dA), 2.f * s, w.partial);
    k_residual_fold<<<1, 1024, 0, st>>>(w.partial, loss_partials(m, n), w.out3);
    if (loss_out != nullptr)
      cudaMemcpyAsync(loss_out, w.out3 + 1, sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  // adjoints of the two GEMMs (the conjugate transposes of Sec. 2.2: X^H Y
  // and X Y^H, never plain transposes, which do not reverse quaternion products)
  if ((e = tc(vE, false, vT, true, m, c, n, -2.f * s, w.GC)) != QMCUR_OK) return e;
  if ((e = tc(vC, true, vE, false, c, n, m, -2.f * s, w.GT)) != QMCUR_OK) return e;
  if ((e = tc(vGT, false, vR, true, c, r, n, 1.f, w.GU)) != QMCUR_OK) return e;
  if ((e = tc(vU, true, vGT, false, r, n, c, 1.f, w.GR)) != QMCUR_OK) return e;
  // G_W = -U^H G_U U^H + (I - W U) G_U^H U U^H + U^H U G_U^H (I - U W),
  // by dependency level, one launch each:
  //   X1 = U^H G_U, U U^H, U^H U, I - W U, I - U W;
  //   G_W = -X1 U^H, M2 = G_U^H (U U^H), M3 = (U^H U) G_U^H;
  //   G_W += [I - W U | M3] [M2; I - U W]
  const QPtr IWU = sub_q(w.XL, 0, 0), M3 = sub_q(w.XL, 0, r);
  const QPtr M2 = sub_q(w.YL, 0, 0), IUW = sub_q(w.YL, r, 0);
  k_two_eyes<<<blocks_for(r * r + c * c), 256, 0, st>>>(IWU, r, IUW, c);
  {
    const SmallGemmArgs l1[5] = {{w.U32, w.GU, w.X1, ri, ri, ci, 1.f, 0.f, 1, 0},
                                 {w.U32, w.U32, w.UUh, ci, ci, ri, 1.f, 0.f, 0, 1},
                                 {w.U32, w.U32, w.UhU, ri, ri, ci, 1.f, 0.f, 1, 0},
                                 {w.W32, w.U32, IWU, ri, ri, ci, -1.f, 1.f, 0, 0},
                                 {w.U32, w.W32, IUW, ci, ci, ri, -1.f, 1.f, 0, 0}};
    if ((e = small_qgemm_batch(l1, 5, st)) != QMCUR_OK) return e;
    const SmallGemmArgs l2[3] = {{w.X1, w.U32, w.GW, ri, ci, ri, -1.f, 0.f, 0, 1},
                                 {w.GU, w.UUh, M2, ri, ci, ci, 1.f, 0.f, 1, 0},
                                 {w.UhU, w.GU, M3, ri, ci, ri, 1.f, 0.f, 0, 1}};
    if ((e = small_qgemm_batch(l2, 3, st)) != QMCUR_OK) return e;
    if ((e = small_qgemm(false, false, ri, ci, ri + ci, 1.f, w.XL, w.YL, 1.f, w.GW, st)) != QMCUR_OK)
      return e;
  }
  // scatters
  QView vdA = view(dA);
  k_scatter_add<<<blocks_for(m * c), 256, 0, st>>>(vdA, w.GC, m, c, I, J, 0);
  k_scatter_add<<<blocks_for(r * n), 256, 0, st>>>(vdA, w.GR, r, n, I, J, 1);
  k_scatter_add<<<blocks_for(r * c), 256, 0, st>>>(vdA, w.GW, r, c, I, J, 2);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
