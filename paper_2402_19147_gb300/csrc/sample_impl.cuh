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
__device__ __forceinline__ int64_t upper_bound(const unsigned long long* P, int64_t N,
                                               unsigned long long target) {
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
  unsigned long long* P[2];   // scratch: the prefix sums when they do not fit shared memory
  uint32_t* bits[2];
  uint64_t seed;
  uint32_t stream_id;
  int64_t max_attempts[2];
  int norm;
  int32_t* status;
  int32_t* attempts_out;  // optional: draws consumed per set (2 ints)
};

// Exclusive prefix sum of one int per thread over the CTA (kSampleThreads).
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int own = lane < kSampleThreads / 32 ? warp_tot[lane] : 0;
    int t = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kSampleThreads / 32) warp_tot[lane] = t - own;   // exclusive
  }
  __syncthreads();
  const int r = warp_tot[warp] + x - v;
  __syncthreads();
  return r;
}

// Exclusive prefix sum of one uint64 per thread over the CTA (kSampleThreads);
// integer sums, so the order of the additions does not matter.
__device__ __forceinline__ unsigned long long block_exclusive_scan_u64(unsigned long long v,
                                                                       unsigned long long* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long own = lane < kSampleThreads / 32 ? warp_tot[lane] : 0ull;
    unsigned long long t = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kSampleThreads / 32) warp_tot[lane] = t - own;   // exclusive
  }
  __syncthreads();
  const unsigned long long r = warp_tot[warp] + x - v;
  __syncthreads();
  return r;
}

// One index set (set 0: J over columns, 1: I over rows) by one CTA of
// kSampleThreads threads; `dyn` is the CTA's dynamic shared memory.
//
// The draws and their acceptance are defined sequentially (draw t in counter
// order; a draw that repeats an accepted index is rejected; stop when the
// set is full).  Here warp 0 takes a round's candidates 32 at a time: a
// candidate is new when its index is not in the bitmap and no earlier
// candidate of its 32 carries the same index (__match_any_sync); the new
// ones are taken in lane order until the set is full.  This accepts exactly
// the indices, and consumes exactly the draws, of the sequential definition.
__device__ __forceinline__ void sample_one_set(const SampleArgs& a, int set, int P_in_smem,
                                               unsigned char* dyn) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t N = a.N[set];
  const int64_t count = a.count[set];
  const double* p = a.prob[set];
  const int64_t words = (N + 31) / 32;
  // Dynamic shared memory: the acceptance bitmap (and the prefix sums when
  // they fit), so that the acceptance and the binary searches stay on chip.
  uint32_t* bits = reinterpret_cast<uint32_t*>(dyn);
  unsigned long long* P =
      P_in_smem ? reinterpret_cast<unsigned long long*>(dyn + ((words * 4 + 15) / 16) * 16)
                : a.P[set];

  __shared__ unsigned long long warp_tot64[kSampleThreads / 32];
  __shared__ double red_max[kSampleThreads / 32];
  __shared__ long long red_sup[kSampleThreads / 32];
  __shared__ unsigned long long S_sh;
  __shared__ int E_sh;
  __shared__ int abort_sh;
  __shared__ int64_t cand[kSampleThreads];
  __shared__ int64_t accepted_sh;
  __shared__ int64_t used_sh;
  __shared__ int warp_tot[kSampleThreads / 32];

  for (int64_t w = tid; w < words; w += kSampleThreads) bits[w] = 0u;
  if (tid == 0) { abort_sh = 0; accepted_sh = 0; used_sh = 0; S_sh = 0ull; E_sh = 0; }

  static_assert(kPrefixBlocks == kSampleThreads, "one prefix block per thread");
  if (a.norm) {
    // stage p as doubles (coalesced, eight loads in flight per thread) and
    // take its maximum (exact in any order)
    double pmax = 0.0;
    for (int64_t k0 = tid; k0 < N; k0 += 8 * kSampleThreads) {
      double v[8];
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int64_t k = k0 + (int64_t)h * kSampleThreads;
        v[h] = k < N ? p[k] : 0.0;
      }
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const int64_t k = k0 + (int64_t)h * kSampleThreads;
        if (k < N) {
          reinterpret_cast<double*>(P)[k] = v[h];
          pmax = fmax(pmax, v[h]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pmax = fmax(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
    if (lane == 0) red_max[warp] = pmax;
    __syncthreads();
    if (tid == 0) {
      double M = red_max[0];
      for (int w = 1; w < kSampleThreads / 32; ++w) M = fmax(M, red_max[w]);
      if (!isfinite(M)) {
        abort_sh = 1;
        set_status(a.status, QMCUR_ERR_NONFINITE);
      } else if (!(M > 0.0)) {
        abort_sh = 1;
        set_status(a.status, QMCUR_ERR_INSUFFICIENT_SUPPORT);
      } else {
        // q_k = floor(p_k 2^E), E = B - 1 - e with M = f 2^e, B = 63 - ceil(log2 N)
        const int clog = N > 1 ? 64 - __clzll((unsigned long long)(N - 1)) : 0;
        E_sh = (63 - clog) - 1 - ilogb(M);
      }
    }
    __syncthreads();
    if (abort_sh) return;
    const int E = E_sh;
    // block b = tid: q_k and their running sum left to right, in place
    const int64_t L = (N + kPrefixBlocks - 1) / kPrefixBlocks;
    const int64_t lo = (int64_t)tid * L;
    const int64_t hi = lo + L < N ? lo + L : N;
    unsigned long long run = 0ull;
    long long sup = 0;
    for (int64_t k = lo; k < hi; ++k) {
      const double pk = reinterpret_cast<const double*>(P)[k];
      const unsigned long long q = pk > 0.0 ? __double2ull_rz(ldexp(pk, E)) : 0ull;
      run += q;
      P[k] = run;
      sup += q != 0ull;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sup += __shfl_xor_sync(0xffffffffu, sup, o);
    if (lane == 0) red_sup[warp] = sup;
    const unsigned long long off = block_exclusive_scan_u64(run, warp_tot64);   // syncs
    for (int64_t k = lo; k < hi; ++k) P[k] += off;
    if (tid == 0) {
      long long support = 0;
      for (int w = 0; w < kSampleThreads / 32; ++w) support += red_sup[w];
      if (support < count) { abort_sh = 1; set_status(a.status, QMCUR_ERR_INSUFFICIENT_SUPPORT); }
    }
    __syncthreads();
    if (tid == 0) S_sh = P[N - 1];
  }
  __syncthreads();
  if (abort_sh) return;

  const uint2 key = make_uint2((unsigned)(a.seed & 0xffffffffu), (unsigned)(a.seed >> 32));
  const unsigned long long S = S_sh;
  const int64_t max_att = a.max_attempts[set];
  for (int64_t base = 0; base < max_att; base += kSampleThreads) {
    const int64_t t = base + tid;
    int64_t k = -1;
    if (t < max_att) {
      const uint4 x = philox4x32_10(
          make_uint4((unsigned)(t & 0xffffffff), (unsigned)(t >> 32), a.stream_id, (unsigned)set), key);
      if (a.norm) {
        // target = (w S) >> 53 for the 53-bit word w: below S, so some P[k] exceeds it
        const unsigned long long w = (((unsigned long long)x.x << 32) | (unsigned long long)x.y) >> 11;
        const unsigned long long lo64 = w * S, hi64 = __umul64hi(w, S);
        const unsigned long long target = (hi64 << 11) | (lo64 >> 53);
        k = upper_bound(P, N, target);
        if (k >= N) k = N - 1;   // unreachable: P[N - 1] = S > target
      } else {
        k = (int64_t)(((uint64_t)x.x * (uint64_t)N) >> 32);
      }
    }
    cand[tid] = k;
    __syncthreads();
    if (warp == 0) {
      int64_t acc = accepted_sh;
      int64_t used = used_sh;
      for (int q = 0; q < kSampleThreads / 32; ++q) {
        const int j = q * 32 + lane;
        const int64_t kk = cand[j];
        const unsigned vmask = __ballot_sync(0xffffffffu, kk >= 0);
        const int firstinv = vmask == 0xffffffffu ? 32 : __ffs(~vmask) - 1;   // draws end there
        const bool live = lane < firstinv;
        const bool seen = live && ((bits[kk >> 5] >> (kk & 31)) & 1u);
        const unsigned same = __match_any_sync(0xffffffffu, live ? (unsigned long long)kk
                                                                  : ~(unsigned long long)lane);
        const bool isnew = live && !seen && (__ffs(same) - 1) == lane;
        const unsigned newmask = __ballot_sync(0xffffffffu, isnew);
        const int64_t need = count - acc;
        const int rank = __popc(newmask & ((1u << lane) - 1u));
        if (isnew && rank < need) atomicOr(&bits[kk >> 5], 1u << (kk & 31));
        const int nnew = __popc(newmask);
        if (nnew >= need) {
          // the candidate that fills the set: the need-th new lane
          const unsigned fin = __ballot_sync(0xffffffffu, isnew && rank == need - 1);
          used = base + q * 32 + (__ffs(fin) - 1) + 1;
          acc = count;
          break;
        }
        acc += nnew;
        used = base + q * 32 + firstinv;
        __syncwarp();
        if (firstinv < 32) break;
      }
      if (lane == 0) { accepted_sh = acc; used_sh = used; }
    }
    __syncthreads();
    if (accepted_sh >= count || cand[kSampleThreads - 1] < 0) break;
  }
  if (tid == 0) {
    if (accepted_sh < count) set_status(a.status, QMCUR_ERR_SAMPLE_LIMIT);
    if (a.attempts_out != nullptr) a.attempts_out[set] = (int32_t)used_sh;
  }
  __syncthreads();

  // Ascending output: each thread owns a contiguous range of bitmap words.
  const int64_t w0 = words * tid / kSampleThreads;
  const int64_t w1 = words * (tid + 1) / kSampleThreads;
  int mine = 0;
  for (int64_t w = w0; w < w1; ++w) mine += __popc(bits[w]);
  int64_t pos = block_exclusive_scan(mine, warp_tot);
  int32_t* out = a.out[set];
  for (int64_t w = w0; w < w1; ++w) {
    uint32_t bb = bits[w];
    while (bb) {
      const int bit = __ffs(bb) - 1;
      bb &= bb - 1;
      if (pos < count) out[pos] = (int32_t)(w * 32 + bit);
      ++pos;
    }
  }
}


}  // namespace qmcur
