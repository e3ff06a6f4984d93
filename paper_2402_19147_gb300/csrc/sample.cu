// Algorithm 1 steps 1-2: draw J subset [n] from {p_j} and I subset [m] from
// {q_i}, then gather C = X(:,J), R = X(I,:) and the intersection W = X(I,J).
//
// k_sample runs one CTA per index set (CTA 0 -> J, CTA 1 -> I).
//  * Norm sampler, in exact integers: with M = max p_k = f 2^e and
//    B = 63 - ceil(log2 N), q_k = floor(p_k 2^(B - 1 - e)) (an exact
//    power-of-two scaling, then truncation), so the sum S of the q_k is
//    below 2^63.  Their prefix sums are exact, so the CTA takes them in any
//    order: thread b sums block b, a shuffle scan gives the block offsets.
//    A draw's 53-bit word w gives target = (w S) >> 53 < S, and the index
//    is the first k with P[k] > target (binary search).
//  * Draw t: Philox4x32-10 (Salmon et al., SC'11), key (seed_lo, seed_hi),
//    counter (t_lo, t_hi, stream_id, which).  256 draws are generated in
//    parallel per round and accepted in counter order, repeats rejected (a
//    bitmap), 32 at a time by one warp; this reproduces sequential sampling
//    without replacement exactly (see sample_one_set).
//  * The accepted set is emitted in ascending order from the bitmap.
// The gathers are 2-D kernels per output (k_gather_t, k_gather_rows_f4).
#include "sample_impl.cuh"

namespace qmcur {
namespace {

__global__ void __launch_bounds__(kSampleThreads) k_sample(SampleArgs a, int P_in_smem) {
  extern __shared__ __align__(16) unsigned char dyn[];
  sample_one_set(a, blockIdx.x, P_in_smem, dyn);
}

// out[i][j] = A[ROWS ? I[i] : i][COLS ? J[j] : j] for the four planes (C:
// COLS, R: ROWS, W: both).  blockIdx.y strides over output rows; a thread
// takes consecutive output columns (the sampled column index is read once
// for the four planes).  Indices outside A (possible only after a sampling
// error, already in the status word) read as zero.
template <typename TS, typename TD, bool ROWS, bool COLS>
__global__ void __launch_bounds__(256)
k_gather_t(QView A, const int32_t* __restrict__ I, const int32_t* __restrict__ J, QView out) {
  const int64_t rows = out.rows, cols = out.cols;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    const int64_t si = ROWS ? (int64_t)I[i] : i;
    const bool rin = si >= 0 && si < A.rows;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cols;
         j += (int64_t)gridDim.x * blockDim.x) {
      const int64_t sj = COLS ? (int64_t)J[j] : j;
      const bool in = rin && sj >= 0 && sj < A.cols;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const TS v = in ? reinterpret_cast<const TS*>(A.p[t])[si * A.ld + sj] : TS(0);
        reinterpret_cast<TD*>(out.p[t])[i * out.ld + j] = (TD)v;
      }
    }
  }
}

// R = A(I, :) as whole rows, float4 copies when every row start is 16-byte
// aligned (F32 to F32).
__global__ void __launch_bounds__(256)
k_gather_rows_f4(QView A, const int32_t* __restrict__ I, QView out) {
  const int64_t rows = out.rows, n4 = out.cols / 4;
  for (int64_t i = blockIdx.y; i < rows; i += gridDim.y) {
    const int64_t si = (int64_t)I[i];
    const bool rin = si >= 0 && si < A.rows;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n4;
         j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float4 v = rin ? reinterpret_cast<const float4*>(
                                   reinterpret_cast<const float*>(A.p[t]) + si * A.ld)[j]
                             : make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4*>(reinterpret_cast<float*>(out.p[t]) + i * out.ld)[j] = v;
      }
    }
  }
}

// One streaming pass over the rows of A (FP32 planes) giving C = A(:, J),
// R = A(I, :) and W = A(I, J) at once.  Sampling 10% of the columns touches
// most 64-byte granules of every row anyway, so reading whole rows in order
// beats gathering the columns in random order.  A CTA stages J and I in
// shared memory, then takes a row at a time: chunks of kGatherChunk columns
// (four planes, float4, two per plane per thread in flight) go through
// shared memory, to R when the row is in I, and C (and W) are picked from
// them.  The pass serves calls that want C.  J and I are sorted, so a chunk's columns of J are contiguous in J and
// the row's position in I is found by binary search.
constexpr int kGatherThreads = 256;
constexpr int kGatherChunk = 2048;
constexpr int kGatherMaxIdx = 4096;   // c, r held in shared memory

__device__ __forceinline__ int first_at_least(const int32_t* v, int len, int64_t x) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)v[mid] < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

inline size_t gather_stream_smem(int64_t c, int64_t r) {
  return (size_t)4 * kGatherChunk * 4 + (size_t)4 * (c + r);
}

template <typename TW>
__global__ void __launch_bounds__(kGatherThreads)
k_gather_stream(QView A, const int32_t* __restrict__ I, const int32_t* __restrict__ J, int r, int c,
                QView C, QView R, QView W, int hasR, int hasW) {
  extern __shared__ __align__(16) unsigned char gsm[];
  float* rowbuf = reinterpret_cast<float*>(gsm);                   // [4][kGatherChunk]
  int32_t* Js = reinterpret_cast<int32_t*>(rowbuf + 4 * kGatherChunk);
  int32_t* Is = Js + c;
  for (int q = threadIdx.x; q < c; q += kGatherThreads) Js[q] = J[q];
  for (int q = threadIdx.x; q < r; q += kGatherThreads) Is[q] = I[q];
  __syncthreads();
  const int64_t m = A.rows, n = A.cols;
  constexpr int kPer = kGatherChunk / 4 / kGatherThreads;   // float4 per plane per thread
  // The CTA's work is a flat list of (row, chunk) items: rows blockIdx.x,
  // blockIdx.x + gridDim.x, ...; the loads of item k + 1 are issued before
  // item k's columns are picked, so the pass keeps reading while it writes.
  const int64_t nchunks = (n + kGatherChunk - 1) / kGatherChunk;
  const int64_t my_rows = blockIdx.x < m ? (m - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t items = my_rows * nchunks;
  float4 v[4][kPer];
  auto load_item = [&](int64_t k) {
    const int64_t i = blockIdx.x + (k / nchunks) * gridDim.x;
    const int64_t c0 = (k % nchunks) * kGatherChunk;
    const int cw = (int)(n - c0 < kGatherChunk ? n - c0 : kGatherChunk);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float* arow = reinterpret_cast<const float*>(A.p[t]) + i * A.ld + c0;
#pragma unroll
      for (int h = 0; h < kPer; ++h) {
        const int q = threadIdx.x + h * kGatherThreads;
        v[t][h] = q < cw / 4 ? reinterpret_cast<const float4*>(arow)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  if (items > 0) load_item(0);
  for (int64_t k = 0; k < items; ++k) {
    const int64_t i = blockIdx.x + (k / nchunks) * gridDim.x;
    const int64_t c0 = (k % nchunks) * kGatherChunk;
    const int cw = (int)(n - c0 < kGatherChunk ? n - c0 : kGatherChunk);
    const int ri = first_at_least(Is, r, i);
    const int rpos = (ri < r && (int64_t)Is[ri] == i) ? ri : -1;   // row of R / W, or -1
    __syncthreads();   // the previous item's chunk is no longer read
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int h = 0; h < kPer; ++h) {
        const int q = threadIdx.x + h * kGatherThreads;
        if (q < cw / 4) {
          reinterpret_cast<float4*>(rowbuf + t * kGatherChunk)[q] = v[t][h];
          if (hasR && rpos >= 0)
            reinterpret_cast<float4*>(reinterpret_cast<float*>(R.p[t]) + (int64_t)rpos * R.ld + c0)[q] =
                v[t][h];
        }
      }
    if (k + 1 < items) load_item(k + 1);
    __syncthreads();
    const int b0 = first_at_least(Js, c, c0), b1 = first_at_least(Js, c, c0 + cw);
    for (int b = b0 + threadIdx.x; b < b1; b += kGatherThreads) {
      const int64_t jj = (int64_t)Js[b] - c0;
      // a valid sorted J puts jj in [0, cw); after a sampling error J is
      // unspecified, and nothing outside the chunk may be read
      if (jj < 0 || jj >= cw) continue;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float x = rowbuf[t * kGatherChunk + jj];
        reinterpret_cast<float*>(C.p[t])[i * C.ld + b] = x;
        if (hasW && rpos >= 0) reinterpret_cast<TW*>(W.p[t])[(int64_t)rpos * W.ld + b] = (TW)x;
      }
    }
  }
}

template <bool ROWS, bool COLS>
qmcur_status gather_one(const QView& A, const int32_t* I, const int32_t* J, const QView& out,
                        cudaStream_t st) {
  const int64_t work_cols = out.cols;
  const unsigned gx = (unsigned)((work_cols + 255) / 256 < 64 ? (work_cols + 255) / 256 : 64);
  const unsigned gy = (unsigned)(out.rows < 65535 ? out.rows : 65535);
  const dim3 grid(gx, gy);
  const bool f32in = A.dtype == QMCUR_F32, f32out = out.dtype == QMCUR_F32;
  if (f32in && f32out) k_gather_t<float, float, ROWS, COLS><<<grid, 256, 0, st>>>(A, I, J, out);
  else if (f32in) k_gather_t<float, double, ROWS, COLS><<<grid, 256, 0, st>>>(A, I, J, out);
  else if (f32out) k_gather_t<double, float, ROWS, COLS><<<grid, 256, 0, st>>>(A, I, J, out);
  else k_gather_t<double, double, ROWS, COLS><<<grid, 256, 0, st>>>(A, I, J, out);
  return cuda_ok(cudaGetLastError());
}

// The streaming pass needs FP32 A and outputs (W may be F32 or F64), float4
// alignment of A and R, n a multiple of 4, and J, I that are valid sorted
// sets (the sampler's output; qmcur_gather's callers may pass any index
// arrays, so that entry point takes the per-output kernels).
bool stream_ok(const QView& A, int64_t c, int64_t r, const qmcur_qmat* C, const qmcur_qmat* R,
               const qmcur_qmat* W) {
  if (A.dtype != QMCUR_F32 || A.cols % 4 != 0 || A.ld % 4 != 0) return false;
  if (c > kGatherMaxIdx || r > kGatherMaxIdx || C == nullptr) return false;   // C drives the pass
  if (C && C->dtype != QMCUR_F32) return false;
  if (R && (R->dtype != QMCUR_F32 || R->ld % 4 != 0)) return false;
  for (int t = 0; t < 4; ++t) {
    if (reinterpret_cast<uintptr_t>(A.p[t]) % 16 != 0) return false;
    if (R && reinterpret_cast<uintptr_t>(R->plane[t]) % 16 != 0) return false;
  }
  return true;
}

qmcur_status gather_stream(const QView& A, const int32_t* J, const int32_t* I, int64_t c, int64_t r,
                           const qmcur_qmat* C, const qmcur_qmat* R, const qmcur_qmat* W,
                           cudaStream_t st) {
  const QView vC = C ? view(C) : A, vR = R ? view(R) : A, vW = W ? view(W) : A;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  static bool attr_set[64] = {};
  if (dev < 0 || dev >= 64) return QMCUR_ERR_CUDA;
  if (!attr_set[dev]) {
    const int mx = (int)gather_stream_smem(kGatherMaxIdx, kGatherMaxIdx);
    if (cudaFuncSetAttribute(k_gather_stream<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_gather_stream<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             mx) != cudaSuccess)
      return QMCUR_ERR_CUDA;
    attr_set[dev] = true;
  }
  const size_t smem = gather_stream_smem(c, r);
  const int64_t want = (int64_t)sms * 4;
  const unsigned grid = (unsigned)(A.rows < want ? A.rows : want);
  if (W != nullptr && W->dtype == QMCUR_F64)
    k_gather_stream<double><<<grid, kGatherThreads, smem, st>>>(
        A, I, J, (int)r, (int)c, vC, vR, vW, R != nullptr, W != nullptr);
  else
    k_gather_stream<float><<<grid, kGatherThreads, smem, st>>>(
        A, I, J, (int)r, (int)c, vC, vR, vW, R != nullptr, W != nullptr);
  return cuda_ok(cudaGetLastError());
}

qmcur_status gather_all(const QView& A, const int32_t* J, const int32_t* I, const qmcur_qmat* C,
                        const qmcur_qmat* R, const qmcur_qmat* W, cudaStream_t st) {
  qmcur_status s = QMCUR_OK;
  if (C != nullptr && (s = gather_one<false, true>(A, I, J, view(C), st)) != QMCUR_OK) return s;
  if (R != nullptr) {
    const QView vR = view(R);
    bool vec = A.dtype == QMCUR_F32 && vR.dtype == QMCUR_F32 && vR.cols % 4 == 0 &&
               A.ld % 4 == 0 && vR.ld % 4 == 0;
    for (int t = 0; t < 4; ++t)
      vec = vec && reinterpret_cast<uintptr_t>(A.p[t]) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(vR.p[t]) % 16 == 0;
    if (vec) {
      const int64_t n4 = vR.cols / 4;
      const dim3 grid((unsigned)((n4 + 255) / 256 < 64 ? (n4 + 255) / 256 : 64),
                      (unsigned)(vR.rows < 65535 ? vR.rows : 65535));
      k_gather_rows_f4<<<grid, 256, 0, st>>>(A, I, vR);
      if ((s = cuda_ok(cudaGetLastError())) != QMCUR_OK) return s;
    } else if ((s = gather_one<true, false>(A, I, J, vR, st)) != QMCUR_OK) {
      return s;
    }
  }
  if (W != nullptr && (s = gather_one<true, true>(A, I, J, view(W), st)) != QMCUR_OK) return s;
  return QMCUR_OK;
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
  return gather_all(view(A), J, I, C, R, W, st);
}

size_t sample_ws_bytes(int64_t m, int64_t n) {
  Carve c(nullptr, 0);
  c.take<unsigned long long>((size_t)n);
  c.take<unsigned long long>((size_t)m);
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
  a.P[0] = cv.take<unsigned long long>((size_t)n);
  a.P[1] = cv.take<unsigned long long>((size_t)m);
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
  if (cudaGetLastError() != cudaSuccess) return QMCUR_ERR_CUDA;
  if (!(C || R || W)) return QMCUR_OK;
  // the sampler's J, I are sorted sets: one streaming pass when the layout allows
  if (stream_ok(view(A), c, r, C, R, W)) return gather_stream(view(A), J, I, c, r, C, R, W, st);
  return gather_all(view(A), J, I, C, R, W, st);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
