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
#include "common.cuh"

namespace qmcur {
namespace {

constexpr int kSampleThreads = 256;
constexpr int kPrefixBlocks = 256;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const unsigned W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) { k.x += W0; k.y += W1; }
    const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// First k in [0, N) with P[k] > target, N if none.
__device__ __forceinline__ int64_t upper_bound(const double* P, int64_t N, double target) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (P[mid] > target) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

struct SampleArgs {
  const double* prob[2];
  int64_t N[2];
  int64_t count[2];
  int32_t* out[2];
  double* P[2];
  uint32_t* bits[2];
  uint64_t seed;
  uint32_t stream_id;
  int64_t max_attempts[2];
  int norm;
  int32_t* status;
  int32_t* attempts_out;  // optional: draws consumed per set (2 ints)
};

__global__ void __launch_bounds__(kSampleThreads) k_sample(SampleArgs a, int P_in_smem) {
  const int set = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t N = a.N[set];
  const int64_t count = a.count[set];
  const double* p = a.prob[set];
  const int64_t words = (N + 31) / 32;
  // Dynamic shared memory: the acceptance bitmap (and the prefix sums when
  // they fit), so that the sequential acceptance and the binary searches stay
  // on chip.
  extern __shared__ __align__(16) unsigned char dyn[];
  uint32_t* bits = reinterpret_cast<uint32_t*>(dyn);
  double* P = P_in_smem ? reinterpret_cast<double*>(dyn + ((words * 4 + 15) / 16) * 16) : a.P[set];

  __shared__ double blk_total[kPrefixBlocks];
  __shared__ double blk_off[kPrefixBlocks];
  __shared__ int64_t blk_support[kPrefixBlocks];
  __shared__ int64_t blk_last[kPrefixBlocks];
  __shared__ double S_sh;
  __shared__ int64_t last_pos_sh;
  __shared__ int abort_sh;
  __shared__ int64_t cand[kSampleThreads];
  __shared__ int64_t accepted_sh;
  __shared__ int64_t used_sh;
  __shared__ int64_t scan[kSampleThreads];

  for (int64_t w = tid; w < words; w += kSampleThreads) bits[w] = 0u;
  if (tid == 0) { abort_sh = 0; accepted_sh = 0; used_sh = 0; S_sh = 0.0; last_pos_sh = -1; }

  if (a.norm) {
    const int64_t L = (N + kPrefixBlocks - 1) / kPrefixBlocks;
    const int64_t lo = (int64_t)tid * L;
    const int64_t hi = lo + L < N ? lo + L : N;
    double s = 0.0;
    int64_t sup = 0, last = -1;
    for (int64_t k = lo; k < hi; ++k) {
      const double pk = p[k];
      s = (k == lo) ? pk : __dadd_rn(s, pk);
      P[k] = s;
      if (pk > 0.0) { ++sup; last = k; }
    }
    blk_total[tid] = (lo < hi) ? s : 0.0;
    blk_support[tid] = sup;
    blk_last[tid] = last;
    __syncthreads();
    if (tid == 0) {
      double o = 0.0;
      int64_t support = 0, lastp = -1;
      for (int b = 0; b < kPrefixBlocks; ++b) {
        blk_off[b] = o;
        o = __dadd_rn(o, blk_total[b]);
        support += blk_support[b];
        if (blk_last[b] > lastp) lastp = blk_last[b];
      }
      S_sh = o;
      last_pos_sh = lastp;
      if (support < count) { abort_sh = 1; set_status(a.status, QMCUR_ERR_INSUFFICIENT_SUPPORT); }
    }
    __syncthreads();
    const double off = blk_off[tid];
    for (int64_t k = lo; k < hi; ++k) P[k] = __dadd_rn(off, P[k]);
  }
  __syncthreads();
  if (abort_sh) return;

  const uint2 key = make_uint2((unsigned)(a.seed & 0xffffffffu), (unsigned)(a.seed >> 32));
  const double S = S_sh;
  const int64_t last_pos = last_pos_sh;
  const int64_t max_att = a.max_attempts[set];
  for (int64_t base = 0; base < max_att; base += kSampleThreads) {
    const int64_t t = base + tid;
    int64_t k = -1;
    if (t < max_att) {
      const uint4 x = philox4x32_10(
          make_uint4((unsigned)(t & 0xffffffff), (unsigned)(t >> 32), a.stream_id, (unsigned)set), key);
      if (a.norm) {
        const uint64_t w = (((uint64_t)x.x << 32) | (uint64_t)x.y) >> 11;
        const double u = __dmul_rn((double)w, 0x1.0p-53);
        const double target = __dmul_rn(u, S);
        k = upper_bound(P, N, target);
        if (k >= N) k = last_pos;
      } else {
        k = (int64_t)(((uint64_t)x.x * (uint64_t)N) >> 32);
      }
    }
    cand[tid] = k;
    __syncthreads();
    if (tid == 0) {
      int64_t acc = accepted_sh;
      for (int j = 0; j < kSampleThreads && acc < count; ++j) {
        const int64_t kk = cand[j];
        if (kk < 0) break;
        used_sh = base + j + 1;
        const uint32_t bit = 1u << (kk & 31);
        if (!(bits[kk >> 5] & bit)) { bits[kk >> 5] |= bit; ++acc; }
      }
      accepted_sh = acc;
    }
    __syncthreads();
    if (accepted_sh >= count) break;
  }
  if (tid == 0) {
    if (accepted_sh < count) set_status(a.status, QMCUR_ERR_SAMPLE_LIMIT);
    if (a.attempts_out != nullptr) a.attempts_out[set] = (int32_t)used_sh;
  }
  __syncthreads();

  // Ascending output: each thread owns a contiguous range of bitmap words.
  const int64_t w0 = words * tid / kSampleThreads;
  const int64_t w1 = words * (tid + 1) / kSampleThreads;
  int64_t mine = 0;
  for (int64_t w = w0; w < w1; ++w) mine += __popc(bits[w]);
  scan[tid] = mine;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (int j = 0; j < kSampleThreads; ++j) { const int64_t v = scan[j]; scan[j] = run; run += v; }
  }
  __syncthreads();
  int64_t pos = scan[tid];
  int32_t* out = a.out[set];
  for (int64_t w = w0; w < w1; ++w) {
    uint32_t b = bits[w];
    while (b) {
      const int bit = __ffs(b) - 1;
      b &= b - 1;
      if (pos < count) out[pos] = (int32_t)(w * 32 + bit);
      ++pos;
    }
  }
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
