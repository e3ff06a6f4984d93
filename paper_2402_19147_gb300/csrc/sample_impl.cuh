// Index draws of Algorithm 1 steps 1-2, shared by the single-problem and the
// batched sampler kernels (see sample.cu for the definition of the draws).
#pragma once

#include "common.cuh"

namespace qmcur {

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

// One index set (set 0: J over columns, 1: I over rows) by one CTA of
// kSampleThreads threads; `dyn` is the CTA's dynamic shared memory.
__device__ __forceinline__ void sample_one_set(const SampleArgs& a, int set, int P_in_smem,
                                               unsigned char* dyn) {
  const int tid = threadIdx.x;
  const int64_t N = a.N[set];
  const int64_t count = a.count[set];
  const double* p = a.prob[set];
  const int64_t words = (N + 31) / 32;
  // Dynamic shared memory: the acceptance bitmap (and the prefix sums when
  // they fit), so that the sequential acceptance and the binary searches stay
  // on chip.
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


}  // namespace qmcur
