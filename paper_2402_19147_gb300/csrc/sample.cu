// Algorithm 1 steps 1-2: draw J subset [n] from {p_j} and I subset [m] from
// {q_i}, then gather C = X(:,J), R = X(I,:) and the intersection W = X(I,J).
//
// k_sample runs one CTA per index set (CTA 0 -> J, CTA 1 -> I).
//  * Norm sampler: the prefix sums of p are taken in 256 contiguous blocks
//    (thread b sums block b left to right, thread 0 chains the 256 block
//    totals left to right, then every entry adds its block offset); every
//    operation is an explicit round-to-nearest double add/multiply, so the
//    bits match any other implementation of the same order.
//  * Draw t: Philox4x32-10 (Salmon et al., SC'11), key (seed_lo, seed_hi),
//    counter (t_lo, t_hi, stream_id, which).  256 draws are generated in
//    parallel per round; thread 0 then accepts them in counter order,
//    rejecting repeats (a bitmap), which reproduces sequential sampling
//    without replacement exactly.
//  * The accepted set is emitted in ascending order from the bitmap.
#include "sample_impl.cuh"

namespace qmcur {
namespace {

__global__ void __launch_bounds__(kSampleThreads) k_sample(SampleArgs a, int P_in_smem) {
  extern __shared__ __align__(16) unsigned char dyn[];
  sample_one_set(a, blockIdx.x, P_in_smem, dyn);
}

// which: 0 -> C (m x c), 1 -> R (r x n), 2 -> W (r x c)
__global__ void k_gather(QView A, const int32_t* __restrict__ J, const int32_t* __restrict__ I,
                         QView C, QView R, QView W, int hasC, int hasR, int hasW) {
  const int which = blockIdx.y;
  QView out = which == 0 ? C : (which == 1 ? R : W);
  if ((which == 0 && !hasC) || (which == 1 && !hasR) || (which == 2 && !hasW)) return;
  const int64_t rows = out.rows, cols = out.cols;
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    const int64_t si = (which == 0) ? i : (int64_t)I[i];
    const int64_t sj = (which == 1) ? j : (int64_t)J[j];
    // After a sampling error the index sets are unspecified: never read
    // outside A (the status word already carries the error).
    const bool in = si >= 0 && si < A.rows && sj >= 0 && sj < A.cols;
#pragma unroll
    for (int t = 0; t < 4; ++t) st_from_double(out, t, i, j, in ? ld_as_double(A, t, si, sj) : 0.0);
  }
}

}  // namespace

qmcur_status launch_gather(const qmcur_qmat* A, const int32_t* J, const int32_t* I, int64_t c,
                           int64_t r, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, cudaStream_t st) {
  if (!valid_qmat(A) || J == nullptr || I == nullptr || c < 1 || r < 1) return QMCUR_ERR_INVALID_ARG;
  const int64_t m = A->rows, n = A->cols;
  if (C && (!valid_qmat(C) || C->rows != m || C->cols != c)) return QMCUR_ERR_INVALID_ARG;
  if (R && (!valid_qmat(R) || R->rows != r || R->cols != n)) return QMCUR_ERR_INVALID_ARG;
  if (W && (!valid_qmat(W) || W->rows != r || W->cols != c)) return QMCUR_ERR_INVALID_ARG;
  if (!C && !R && !W) return QMCUR_OK;
  QView vA = view(A);
  QView vC = C ? view(C) : vA, vR = R ? view(R) : vA, vW = W ? view(W) : vA;
  const int64_t biggest = m * c > r * n ? m * c : r * n;
  int blocks = (int)((biggest + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_gather<<<dim3(blocks, 3), 256, 0, st>>>(vA, J, I, vC, vR, vW, C != nullptr, R != nullptr,
                                           W != nullptr);
  return cuda_ok(cudaGetLastError());
}

size_t sample_ws_bytes(int64_t m, int64_t n) {
  Carve c(nullptr, 0);
  c.take<double>((size_t)n);
  c.take<double>((size_t)m);
  c.take<uint32_t>((size_t)((n + 31) / 32));
  c.take<uint32_t>((size_t)((m + 31) / 32));
  c.take<int32_t>(2);
  return c.off;
}

qmcur_status launch_sample(const qmcur_qmat* A, int32_t sampler, const double* col_p,
                           const double* row_p, int64_t c, int64_t r, uint64_t seed,
                           uint32_t stream_id, int32_t max_attempts, int32_t* J, int32_t* I,
                           qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, void* ws,
                           size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!valid_qmat(A) || J == nullptr || I == nullptr) return QMCUR_ERR_INVALID_ARG;
  const int64_t m = A->rows, n = A->cols;
  if (c < 1 || c > n || r < 1 || r > m || n > INT32_MAX || m > INT32_MAX) return QMCUR_ERR_INVALID_ARG;
  if (sampler == QMCUR_SAMPLER_NORM && (col_p == nullptr || row_p == nullptr)) return QMCUR_ERR_INVALID_ARG;
  if (sampler != QMCUR_SAMPLER_NORM && sampler != QMCUR_SAMPLER_UNIFORM) return QMCUR_ERR_INVALID_ARG;
  if (C && (!valid_qmat(C) || C->rows != m || C->cols != c)) return QMCUR_ERR_INVALID_ARG;
  if (R && (!valid_qmat(R) || R->rows != r || R->cols != n)) return QMCUR_ERR_INVALID_ARG;
  if (W && (!valid_qmat(W) || W->rows != r || W->cols != c)) return QMCUR_ERR_INVALID_ARG;
  Carve cv(ws, ws_bytes);
  SampleArgs a;
  a.P[0] = cv.take<double>((size_t)n);
  a.P[1] = cv.take<double>((size_t)m);
  a.bits[0] = cv.take<uint32_t>((size_t)((n + 31) / 32));
  a.bits[1] = cv.take<uint32_t>((size_t)((m + 31) / 32));
  a.attempts_out = cv.take<int32_t>(2);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  a.prob[0] = col_p;
  a.prob[1] = row_p;
  a.N[0] = n;
  a.N[1] = m;
  a.count[0] = c;
  a.count[1] = r;
  a.out[0] = J;
  a.out[1] = I;
  a.seed = seed;
  a.stream_id = stream_id;
  a.max_attempts[0] = max_attempts > 0 ? max_attempts : 64 * c + 1024;
  a.max_attempts[1] = max_attempts > 0 ? max_attempts : 64 * r + 1024;
  a.norm = sampler == QMCUR_SAMPLER_NORM;
  a.status = dev_status;
  const int64_t nmax = n > m ? n : m;
  const size_t bits_bytes = (size_t)((nmax + 31) / 32 * 4 + 15) / 16 * 16;
  const size_t p_bytes = (size_t)nmax * 8;
  const size_t kSmemCap = 200 * 1024;
  if (bits_bytes > kSmemCap) return QMCUR_ERR_UNSUPPORTED;
  const int P_in_smem = bits_bytes + p_bytes <= kSmemCap;
  const size_t smem = bits_bytes + (P_in_smem ? p_bytes : 0);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap) !=
          cudaSuccess)
    return QMCUR_ERR_CUDA;
  k_sample<<<2, kSampleThreads, smem, st>>>(a, P_in_smem);
  if (C || R || W) {
    QView vA = view(A);
    QView vC = C ? view(C) : vA, vR = R ? view(R) : vA, vW = W ? view(W) : vA;
    int64_t biggest = m * c > r * n ? m * c : r * n;
    int blocks = (int)((biggest + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_gather<<<dim3(blocks, 3), 256, 0, st>>>(vA, J, I, vC, vR, vW, C != nullptr, R != nullptr,
                                             W != nullptr);
  }
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
