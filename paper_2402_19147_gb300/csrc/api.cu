// C ABI of libqmcur (declared and documented in include/qmcur.h): argument
// checks, workspace sizing and the composition of the stages.
#include "common.cuh"
#include "small.cuh"

namespace qmcur {

size_t simt_partials(int64_t m, int64_t n);
size_t residual_partials(int64_t m, int64_t n);
qmcur_status launch_qgemm_simt(const QView& X, const QView& Y, const QView* Z, const QView* A,
                               const uint8_t* mask, double* partial, bool fp64, cudaStream_t st,
                               bool complete);
__global__ void k_residual_fold(const double* partial, int64_t count, double* out3);

// Subspace pseudo-inverse (pinv_fast.cu).
size_t pinv_fast_ws_bytes(int64_t r, int64_t c, int64_t k);
qmcur_status launch_pinv_fast(const qmcur_qmat* W, int32_t rank_cap, qmcur_qmat* U,
                              int32_t* rank_out, uint64_t seed, void* ws, size_t ws_bytes,
                              int32_t* dev_status, cudaStream_t st);

// FP64-accurate refined subspace pseudo-inverse (pinv_refine.cu).
size_t pinv_refine_ws_bytes(int64_t r, int64_t c, int64_t k);
qmcur_status launch_pinv_refine(const qmcur_qmat* W, double rcond, int32_t rank_cap,
                                int32_t max_iter, qmcur_qmat* U, int32_t* rank_out, uint64_t seed,
                                void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t st);

// Backward of the masked reconstruction loss (backward.cu).
size_t backward_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r);
qmcur_status launch_backward(const qmcur_qmat* A, const uint8_t* mask, const int32_t* J,
                             const int32_t* I, const qmcur_qmat* C, const qmcur_qmat* U,
                             const qmcur_qmat* R, const qmcur_qmat* W, double scale, qmcur_qmat* dA,
                             double* loss_out, void* ws, size_t ws_bytes, int32_t* dev_status,
                             cudaStream_t st);
qmcur_status launch_gather(const qmcur_qmat* A, const int32_t* J, const int32_t* I, int64_t c,
                           int64_t r, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, cudaStream_t st);

// Tensor-core path (qgemm_tc.cu).
size_t tc_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec);
qmcur_status launch_reconstruct_tc(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                                   int32_t prec, qmcur_qmat* Z, const qmcur_qmat* A,
                                   const uint8_t* mask, double* out3, void* ws, size_t ws_bytes,
                                   int32_t* dev_status, cudaStream_t st, bool complete);

size_t gemm_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec) {
  if (prec == QMCUR_PREC_FP64 || prec == QMCUR_PREC_FP32) {
    Carve cv(nullptr, 0);
    cv.take<double>((size_t)(4 * c * n));   // T = U R (FP64 worst case)
    const size_t p1 = simt_partials(m, n), p2 = residual_partials(m, n);
    cv.take<double>(2 * (p1 > p2 ? p1 : p2));
    return cv.off;
  }
  return tc_ws_bytes(m, n, c, r, prec);
}

qmcur_status launch_reconstruct(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                                int32_t prec, qmcur_qmat* Z, const qmcur_qmat* A,
                                const uint8_t* mask, double* out3, void* ws, size_t ws_bytes,
                                int32_t* dev_status, cudaStream_t st, bool complete) {
  if (!valid_qmat(C) || !valid_qmat(U) || !valid_qmat(R)) return QMCUR_ERR_INVALID_ARG;
  if (complete && (Z != nullptr || A == nullptr || out3 == nullptr)) return QMCUR_ERR_INVALID_ARG;
  const int64_t m = C->rows, c = C->cols, r = R->rows, n = R->cols;
  if (U->rows != c || U->cols != r || m < 1 || n < 1 || c < 1 || r < 1) return QMCUR_ERR_INVALID_ARG;
  if (Z != nullptr && (!valid_qmat(Z) || Z->rows != m || Z->cols != n)) return QMCUR_ERR_INVALID_ARG;
  if (Z == nullptr && (A == nullptr || out3 == nullptr)) return QMCUR_ERR_INVALID_ARG;
  if (A != nullptr && (!valid_qmat(A) || A->rows != m || A->cols != n)) return QMCUR_ERR_INVALID_ARG;
  if (prec == QMCUR_PREC_FP64 || prec == QMCUR_PREC_FP32) {
    const bool fp64 = prec == QMCUR_PREC_FP64;
    if (fp64 && (C->dtype != QMCUR_F64 || U->dtype != QMCUR_F64 || R->dtype != QMCUR_F64))
      return QMCUR_ERR_INVALID_ARG;
    if (!fp64 && (C->dtype != QMCUR_F32 || R->dtype != QMCUR_F32)) return QMCUR_ERR_INVALID_ARG;
    if (Z != nullptr && fp64 && Z->dtype != QMCUR_F64) return QMCUR_ERR_INVALID_ARG;
    Carve cv(ws, ws_bytes);
    const size_t es = fp64 ? 8 : 4;
    char* tbuf = cv.take<char>((size_t)(4 * c * n) * es);
    const size_t p1 = simt_partials(m, n), p2 = residual_partials(m, n);
    double* partial = cv.take<double>(2 * (p1 > p2 ? p1 : p2));
    if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
    QView T;
    for (int t = 0; t < 4; ++t) T.p[t] = tbuf + (size_t)t * c * n * es;
    T.rows = c; T.cols = n; T.ld = n; T.dtype = fp64 ? QMCUR_F64 : QMCUR_F32;
    QView vU = view(U), vR = view(R), vC = view(C);
    qmcur_status s = launch_qgemm_simt(vU, vR, &T, nullptr, nullptr, nullptr, fp64, st, false);
    if (s != QMCUR_OK) return s;
    if (Z != nullptr) {
      QView vZ = view(Z);
      return launch_qgemm_simt(vC, T, &vZ, nullptr, nullptr, nullptr, fp64, st, false);
    }
    QView vA = view(A);
    if (complete && fp64 && A->dtype != QMCUR_F64) return QMCUR_ERR_INVALID_ARG;
    s = launch_qgemm_simt(vC, T, complete ? &vA : nullptr, &vA, mask, partial, fp64, st, complete);
    if (s != QMCUR_OK) return s;
    k_residual_fold<<<1, 1024, 0, st>>>(partial, (int64_t)p1, out3);
    return cuda_ok(cudaGetLastError());
  }
  if (prec == QMCUR_PREC_TF32X3 || prec == QMCUR_PREC_BF16X3 || prec == QMCUR_PREC_BF16X6 ||
      prec == QMCUR_PREC_BF16_MIXED)
    return launch_reconstruct_tc(C, U, R, prec, Z, A, mask, out3, ws, ws_bytes, dev_status, st,
                                 complete);
  return QMCUR_ERR_INVALID_ARG;
}

}  // namespace qmcur

using namespace qmcur;

extern "C" {

const char* qmcur_status_str(int32_t s) {
  switch (s) {
    case QMCUR_OK: return "QMCUR_OK";
    case QMCUR_ERR_INVALID_ARG: return "QMCUR_ERR_INVALID_ARG";
    case QMCUR_ERR_NONFINITE: return "QMCUR_ERR_NONFINITE";
    case QMCUR_ERR_ZERO_NORM: return "QMCUR_ERR_ZERO_NORM";
    case QMCUR_ERR_INSUFFICIENT_SUPPORT: return "QMCUR_ERR_INSUFFICIENT_SUPPORT";
    case QMCUR_ERR_SAMPLE_LIMIT: return "QMCUR_ERR_SAMPLE_LIMIT";
    case QMCUR_ERR_NO_CONVERGENCE: return "QMCUR_ERR_NO_CONVERGENCE";
    case QMCUR_ERR_UNSUPPORTED: return "QMCUR_ERR_UNSUPPORTED";
    case QMCUR_ERR_CUDA: return "QMCUR_ERR_CUDA";
    case QMCUR_ERR_TIMEOUT: return "QMCUR_ERR_TIMEOUT";
    case QMCUR_ERR_ILL_CONDITIONED: return "QMCUR_ERR_ILL_CONDITIONED";
    default: return "QMCUR_ERR_UNKNOWN";
  }
}

qmcur_status qmcur_set_max_ctas(int32_t max_ctas) {
  if (max_ctas < 0) return QMCUR_ERR_INVALID_ARG;
  cta_budget_ref() = max_ctas;
  return QMCUR_OK;
}

size_t qmcur_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec) {
  if (m < 1 || n < 1 || c < 1 || r < 1) return 0;
  size_t s = probs_ws_bytes(m, n);
  const size_t s2 = sample_ws_bytes(m, n), s3 = pinv_ws_bytes(r, c), s4 = gemm_ws_bytes(m, n, c, r, prec);
  const int64_t kmax = (r < c ? r : c) < kSmallCholMax ? (r < c ? r : c) : kSmallCholMax;
  const size_t s5 = pinv_fast_ws_bytes(r, c, kmax);
  const size_t s6 = pinv_refine_ws_bytes(r, c, kmax);
  if (s5 > s) s = s5;
  if (s6 > s) s = s6;
  if (s2 > s) s = s2;
  if (s3 > s) s = s3;
  if (s4 > s) s = s4;
  return s + 256;
}

qmcur_status qmcur_probs(const qmcur_qmat* A, int32_t sampler, double* col_p, double* row_p,
                         double* fro2, void* workspace, size_t ws_bytes, int32_t* dev_status,
                         cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_probs");
  return launch_probs(A, sampler, col_p, row_p, fro2, workspace, ws_bytes, dev_status, stream);
}

qmcur_status qmcur_sample(const qmcur_qmat* A, int32_t sampler, const double* col_p,
                          const double* row_p, int64_t c, int64_t r, uint64_t seed,
                          uint32_t stream_id, int32_t max_attempts, int32_t* J, int32_t* I,
                          qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, void* workspace,
                          size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_sample");
  return launch_sample(A, sampler, col_p, row_p, c, r, seed, stream_id, max_attempts, J, I, C, R, W,
                       workspace, ws_bytes, dev_status, stream);
}

static qmcur_status pinv_dispatch(const qmcur_qmat* W, int32_t method, double rcond,
                                  int32_t rank_cap, int32_t max_sweeps, qmcur_qmat* U,
                                  int32_t* rank_out, double* sigma_out, void* workspace,
                                  size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  if (method == QMCUR_PINV_JACOBI_FP64)
    return launch_pinv(W, rcond, rank_cap, max_sweeps, U, rank_out, sigma_out, workspace,
                       ws_bytes, dev_status, stream);
  if (method == QMCUR_PINV_REFINED_FP64)
    return launch_pinv_refine(W, rcond, rank_cap, max_sweeps, U, rank_out, 0x9e3779b97f4a7c15ull,
                              workspace, ws_bytes, dev_status, stream);
  if (method != QMCUR_PINV_SUBSPACE_FP32) return QMCUR_ERR_INVALID_ARG;
  if (!valid_qmat(W) || !valid_qmat(U)) return QMCUR_ERR_INVALID_ARG;
  if (W->rows < 1 || W->cols < 1 || U->rows != W->cols || U->cols != W->rows)
    return QMCUR_ERR_INVALID_ARG;
  return launch_pinv_fast(W, rank_cap, U, rank_out, 0x9e3779b97f4a7c15ull, workspace, ws_bytes,
                          dev_status, stream);
}

qmcur_status qmcur_pinv_core(const qmcur_qmat* W, int32_t method, double rcond, int32_t rank_cap,
                             int32_t max_sweeps, qmcur_qmat* U, int32_t* rank_out,
                             double* sigma_out, void* workspace, size_t ws_bytes,
                             int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_pinv_core");
  return pinv_dispatch(W, method, rcond, rank_cap, max_sweeps, U, rank_out, sigma_out, workspace,
                       ws_bytes, dev_status, stream);
}

qmcur_status qmcur_reconstruct(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                               int32_t prec, qmcur_qmat* Z, void* workspace, size_t ws_bytes,
                               int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_reconstruct");
  if (Z == nullptr) return QMCUR_ERR_INVALID_ARG;
  return launch_reconstruct(C, U, R, prec, Z, nullptr, nullptr, nullptr, workspace, ws_bytes,
                            dev_status, stream);
}

qmcur_status qmcur_residual(const qmcur_qmat* A, const qmcur_qmat* C, const qmcur_qmat* U,
                            const qmcur_qmat* R, int32_t prec, const uint8_t* mask,
                            const qmcur_qmat* Z, double* out3, void* workspace,
                            size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_residual");
  if (A == nullptr || out3 == nullptr) return QMCUR_ERR_INVALID_ARG;
  if (Z != nullptr)
    return launch_residual_standalone(A, Z, mask, out3, workspace, ws_bytes, dev_status, stream);
  return launch_reconstruct(C, U, R, prec, nullptr, A, mask, out3, workspace, ws_bytes, dev_status,
                            stream);
}

qmcur_status qmcur_gather(const qmcur_qmat* A, const int32_t* J, const int32_t* I, int64_t c,
                          int64_t r, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W,
                          cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_gather");
  return launch_gather(A, J, I, c, r, C, R, W, stream);
}

size_t qmcur_backward_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r) {
  if (m < 1 || n < 1 || c < 1 || r < 1) return 0;
  return backward_ws_bytes(m, n, c, r) + 256;
}

qmcur_status qmcur_reconstruct_backward(const qmcur_qmat* A, const uint8_t* mask, const int32_t* J,
                                        const int32_t* I, const qmcur_qmat* C, const qmcur_qmat* U,
                                        const qmcur_qmat* R, const qmcur_qmat* W, double scale,
                                        qmcur_qmat* dA, double* loss_out, void* workspace,
                                        size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_reconstruct_backward");
  return launch_backward(A, mask, J, I, C, U, R, W, scale, dA, loss_out, workspace, ws_bytes,
                         dev_status, stream);
}

qmcur_status qmcur_decompose(const qmcur_qmat* A, int64_t c, int64_t r, const qmcur_opts* o,
                             double* col_p, double* row_p, int32_t* J, int32_t* I,
                             qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, qmcur_qmat* U,
                             int32_t* rank_out, double* sigma_out, double* out3,
                             void* workspace, size_t ws_bytes, int32_t* dev_status,
                             cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_decompose");
  if (A == nullptr || o == nullptr || C == nullptr || R == nullptr || W == nullptr || U == nullptr)
    return QMCUR_ERR_INVALID_ARG;
  if (o->max_ctas < 0) return QMCUR_ERR_INVALID_ARG;
  CtaBudgetScope budget(o->max_ctas > 0 ? o->max_ctas : cta_budget_ref());
  qmcur_status s = launch_probs(A, o->sampler, col_p, row_p, nullptr, workspace, ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  s = launch_sample(A, o->sampler, col_p, row_p, c, r, o->seed, o->stream_id, o->max_attempts, J, I,
                    C, R, W, workspace, ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  s = pinv_dispatch(W, o->pinv_method, o->rcond, o->rank_cap, o->max_sweeps, U, rank_out,
                    sigma_out, workspace, ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  return launch_reconstruct(C, U, R, o->prec, nullptr, A, nullptr, out3, workspace, ws_bytes,
                            dev_status, stream);
}

size_t qmcur_core_paper_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r,
                                       int32_t prec) {
  if (m < 1 || n < 1 || c < 1 || r < 1) return 0;
  // C^+ of the m x c C and R^+ of the r x n R by either method, then the
  // product C^+ (X R^+): a reconstruction with m' = c, n' = r, c' = m, r' = n
  const int64_t kc = (m < c ? m : c) < kSmallCholMax ? (m < c ? m : c) : kSmallCholMax;
  const int64_t kr = (r < n ? r : n) < kSmallCholMax ? (r < n ? r : n) : kSmallCholMax;
  size_t s = pinv_ws_bytes(m, c);
  const size_t s2 = pinv_ws_bytes(r, n), s3 = pinv_fast_ws_bytes(m, c, kc),
               s4 = pinv_fast_ws_bytes(r, n, kr), s5 = gemm_ws_bytes(c, r, m, n, prec);
  const size_t s6 = pinv_refine_ws_bytes(m, c, kc), s7 = pinv_refine_ws_bytes(r, n, kr);
  if (s6 > s) s = s6;
  if (s7 > s) s = s7;
  if (s2 > s) s = s2;
  if (s3 > s) s = s3;
  if (s4 > s) s = s4;
  if (s5 > s) s = s5;
  return s + 256;
}

qmcur_status qmcur_core_paper(const qmcur_qmat* X, const qmcur_qmat* C, const qmcur_qmat* R,
                              int32_t method, double rcond, int32_t rank_cap, int32_t prec,
                              qmcur_qmat* Cp, qmcur_qmat* Rp, qmcur_qmat* U, void* workspace,
                              size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_core_paper");
  if (!valid_qmat(X) || !valid_qmat(C) || !valid_qmat(R) || !valid_qmat(Cp) || !valid_qmat(Rp) ||
      !valid_qmat(U))
    return QMCUR_ERR_INVALID_ARG;
  const int64_t m = X->rows, n = X->cols, c = C->cols, r = R->rows;
  if (C->rows != m || R->cols != n || Cp->rows != c || Cp->cols != m || Rp->rows != n ||
      Rp->cols != r || U->rows != c || U->cols != r)
    return QMCUR_ERR_INVALID_ARG;
  if (Cp->dtype != QMCUR_F32 || Rp->dtype != QMCUR_F32 || U->dtype != QMCUR_F32) {
    if (prec != QMCUR_PREC_FP64) return QMCUR_ERR_INVALID_ARG;
  }
  qmcur_status s = pinv_dispatch(C, method, rcond, rank_cap, 0, Cp, nullptr, nullptr, workspace,
                                 ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  s = pinv_dispatch(R, method, rcond, rank_cap, 0, Rp, nullptr, nullptr, workspace, ws_bytes,
                    dev_status, stream);
  if (s != QMCUR_OK) return s;
  return launch_reconstruct(Cp, X, Rp, prec, U, nullptr, nullptr, nullptr, workspace, ws_bytes,
                            dev_status, stream);
}

size_t qmcur_qsvd_workspace_size(int64_t m, int64_t n) {
  if (m < 1 || n < 1) return 0;
  return pinv_ws_bytes(m, n) + 256;
}

qmcur_status qmcur_qsvd_truncated(const qmcur_qmat* X, int32_t rank, double rcond,
                                  int32_t max_sweeps, qmcur_qmat* B, int32_t* rank_out,
                                  double* sigma_out, void* workspace, size_t ws_bytes,
                                  int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_qsvd_truncated");
  return launch_qsvd_truncated(X, rcond, rank, max_sweeps, B, rank_out, sigma_out, workspace,
                               ws_bytes, dev_status, stream);
}

qmcur_status qmcur_complete_step(qmcur_qmat* X, const uint8_t* mask, int64_t c, int64_t r,
                                 const qmcur_opts* o, double* col_p, double* row_p, int32_t* J,
                                 int32_t* I, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W,
                                 qmcur_qmat* U, int32_t* rank_out, double* out3, void* workspace,
                                 size_t ws_bytes, int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_complete_step");
  if (X == nullptr || o == nullptr || C == nullptr || R == nullptr || W == nullptr ||
      U == nullptr || out3 == nullptr || !valid_qmat(X))
    return QMCUR_ERR_INVALID_ARG;
  if (C->plane[0] == X->plane[0] || R->plane[0] == X->plane[0]) return QMCUR_ERR_INVALID_ARG;
  qmcur_status s = launch_probs(X, o->sampler, col_p, row_p, nullptr, workspace, ws_bytes,
                                dev_status, stream);
  if (s != QMCUR_OK) return s;
  s = launch_sample(X, o->sampler, col_p, row_p, c, r, o->seed, o->stream_id, o->max_attempts, J,
                    I, C, R, W, workspace, ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  s = pinv_dispatch(W, o->pinv_method, o->rcond, o->rank_cap, o->max_sweeps, U, rank_out, nullptr,
                    workspace, ws_bytes, dev_status, stream);
  if (s != QMCUR_OK) return s;
  return launch_reconstruct(C, U, R, o->prec, nullptr, X, mask, out3, workspace, ws_bytes,
                            dev_status, stream, true);
}

}  // extern "C"
