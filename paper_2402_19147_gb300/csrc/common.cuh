// Shared device/host helpers of libqmcur (status words, bounded waits,
// workspace carving).  Quaternion planes are row-major real arrays; see
// include/qmcur.h for the storage and error conventions.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/qmcur.h"

namespace qmcur {

constexpr int kNumPlanes = 4;

// Iteration limit of every device-side spin wait (mbarrier, grid barrier).
// At ~100 ns per poll with back-off this is several seconds: far beyond any
// legitimate wait, short enough that a broken pipeline returns an error
// instead of hanging the GPU.
constexpr unsigned long long kSpinLimit = 1ull << 26;

// First error wins: the word goes from 0 to `code` once.
__device__ __forceinline__ void set_status(int32_t* st, int32_t code) {
  if (st != nullptr) atomicCAS(reinterpret_cast<int*>(st), 0, code);
}

// Grid-wide barrier of a cooperative launch.  bar[0] counts arrivals over
// the whole launch (never reset: the n-th barrier completes when it reaches
// n * gridDim.x, kept by the caller in `target`), bar[2] is the abort flag;
// both are zero before the launch.  One atomic per CTA, then a bounded poll.
// On timeout the abort flag is raised, QMCUR_ERR_TIMEOUT is reported and
// false is returned (also to every later caller).
__device__ __forceinline__ bool grid_sync(unsigned* bar, int32_t* status, unsigned& target) {
  __shared__ int ok_sh;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    volatile unsigned* vcount = bar;
    volatile unsigned* vabort = bar + 2;
    int ok = (*vabort == 0u);
    if (ok) {
      __threadfence();   // this CTA's writes before its arrival
      atomicAdd(bar, 1u);
      const long long t0 = clock64();
      while (*vcount < target) {
        if (*vabort != 0u) { ok = 0; break; }
        if (clock64() - t0 > 4000000000ll) {
          atomicExch(bar + 2, 1u);
          set_status(status, QMCUR_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
      __threadfence();   // the other CTAs' writes after their arrivals
    }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

struct QView {          // plain-old-data view of a qmcur_qmat for kernels
  void* p[4];
  int64_t rows, cols, ld;
  int32_t dtype;
};

inline QView view(const qmcur_qmat* q) {
  QView v;
  for (int t = 0; t < 4; ++t) v.p[t] = q->plane[t];
  v.rows = q->rows;
  v.cols = q->cols;
  v.ld = q->ld;
  v.dtype = q->dtype;
  return v;
}

template <typename T>
__device__ __forceinline__ T* plane(const QView& v, int t) {
  return reinterpret_cast<T*>(v.p[t]);
}

__device__ __forceinline__ double ld_as_double(const QView& v, int t, int64_t i, int64_t j) {
  if (v.dtype == QMCUR_F64) return reinterpret_cast<const double*>(v.p[t])[i * v.ld + j];
  return (double)reinterpret_cast<const float*>(v.p[t])[i * v.ld + j];
}

__device__ __forceinline__ void st_from_double(const QView& v, int t, int64_t i, int64_t j, double x) {
  if (v.dtype == QMCUR_F64) reinterpret_cast<double*>(v.p[t])[i * v.ld + j] = x;
  else reinterpret_cast<float*>(v.p[t])[i * v.ld + j] = (float)x;
}

// Host-side argument checks.
inline bool valid_qmat(const qmcur_qmat* q, bool allow_f32 = true, bool allow_f64 = true) {
  if (q == nullptr) return false;
  if (q->rows < 0 || q->cols < 0 || q->ld < q->cols || q->ld < 1) return false;
  if (q->dtype == QMCUR_F32 && !allow_f32) return false;
  if (q->dtype == QMCUR_F64 && !allow_f64) return false;
  if (q->dtype != QMCUR_F32 && q->dtype != QMCUR_F64) return false;
  if (q->rows > 0 && q->cols > 0)
    for (int t = 0; t < 4; ++t)
      if (q->plane[t] == nullptr) return false;
  return true;
}

inline size_t esize(int32_t dtype) { return dtype == QMCUR_F64 ? 8 : 4; }

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bump allocator over the caller's workspace (256-byte aligned slices).
struct Carve {
  char* base;
  size_t cap;
  size_t off;
  bool ok;
  Carve(void* b, size_t c) : base(static_cast<char*>(b)), cap(c), off(0), ok(true) {}
  template <typename T>
  T* take(size_t count) {
    size_t o = align_up(off, 256);
    size_t bytes = align_up(count * sizeof(T), 256);
    if (base == nullptr || o + bytes > cap) {
      ok = false;
      off = o + bytes;
      return nullptr;
    }
    off = o + bytes;
    return reinterpret_cast<T*>(base + o);
  }
};

// Workspace bytes of each stage (host, exact counterparts of the carving).
size_t probs_ws_bytes(int64_t m, int64_t n);
size_t sample_ws_bytes(int64_t m, int64_t n);
size_t pinv_ws_bytes(int64_t r, int64_t c);
size_t gemm_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec);

// Stage launchers (defined in the .cu files; all return synchronously on
// argument errors and enqueue on `st` otherwise).
qmcur_status launch_probs(const qmcur_qmat* A, int32_t sampler, double* col_p, double* row_p,
                          double* fro2, void* ws, size_t ws_bytes, int32_t* dev_status,
                          cudaStream_t st);
qmcur_status launch_sample(const qmcur_qmat* A, int32_t sampler, const double* col_p,
                           const double* row_p, int64_t c, int64_t r, uint64_t seed,
                           uint32_t stream_id, int32_t max_attempts, int32_t* J, int32_t* I,
                           qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, void* ws,
                           size_t ws_bytes, int32_t* dev_status, cudaStream_t st);
qmcur_status launch_pinv(const qmcur_qmat* W, double rcond, int32_t rank_cap, int32_t max_sweeps,
                         qmcur_qmat* U, int32_t* rank_out, double* sigma_out, void* ws,
                         size_t ws_bytes, int32_t* dev_status, cudaStream_t st);
qmcur_status launch_qsvd_truncated(const qmcur_qmat* W, double rcond, int32_t rank,
                                   int32_t max_sweeps, qmcur_qmat* B, int32_t* rank_out,
                                   double* sigma_out, void* ws, size_t ws_bytes,
                                   int32_t* dev_status, cudaStream_t st);
// Z = C (U R); if Z == nullptr the product is not written and, with A != nullptr,
// the residual sums are formed instead (fused epilogue).  With `complete`, A is
// the iterate of a masked completion step (Algorithm 2) and is updated in place.
qmcur_status launch_reconstruct(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                                int32_t prec, qmcur_qmat* Z, const qmcur_qmat* A,
                                const uint8_t* mask, double* out3, void* ws, size_t ws_bytes,
                                int32_t* dev_status, cudaStream_t st, bool complete = false);
qmcur_status launch_residual_standalone(const qmcur_qmat* A, const qmcur_qmat* Z,
                                        const uint8_t* mask, double* out3, void* ws,
                                        size_t ws_bytes, int32_t* dev_status, cudaStream_t st);

inline qmcur_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? QMCUR_OK : QMCUR_ERR_CUDA; }

// A named NVTX range around one C-ABI call, so that a profiler's timeline
// groups each call's kernels under the entry point's name; without a
// profiler attached the push and pop do nothing.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// CTA budget of the persistent kernels (the pseudo-inverse's cooperative
// launches and the tensor-core GEMMs) launched by this host thread: 0 = one
// CTA per SM.  qmcur_decompose sets it from its options for the duration of
// the call, so that two decompositions on two streams can each hold part of
// the SMs at once.
inline int& cta_budget_ref() {
  static thread_local int budget = 0;
  return budget;
}
inline int cta_cap(int sms) {
  const int b = cta_budget_ref();
  return b > 0 && b < sms ? b : sms;
}
struct CtaBudgetScope {
  int saved;
  explicit CtaBudgetScope(int b) : saved(cta_budget_ref()) { cta_budget_ref() = b > 0 ? b : 0; }
  ~CtaBudgetScope() { cta_budget_ref() = saved; }
};

}  // namespace qmcur
