// Sampling probabilities of QMCUR (Sec. 3.1):
//   QMCUR_length  p_j = ||X(:,j)||^2 / ||X||_F^2,  q_i = ||X(i,:)||^2 / ||X||_F^2
//   QMCUR_uniform p_j = 1/n, q_i = 1/m.
// One streaming pass over the four planes (HBM bound): a CTA owns a tile of
// kRows rows x kCols columns; each thread owns 4 adjacent columns, so a warp
// reads 512 contiguous bytes of a row per plane (float4), and keeps the loads
// of kUnroll rows in flight at once (the pass is latency-bound otherwise).
// Squares are summed in FP32 over short runs (16 terms for a row piece, 32
// for a column piece) and carried in FP64 from there on.  Every reduction has
// a fixed order, so the result is bit-reproducible and no atomics touch
// values.  Three launches: the pass, the fold of the tile partials, and the
// scaling, in which every CTA forms ||X||_F^2 itself in the same order (GB300's
// FP64 divide is slow enough that the scaling wants many SMs).
#include <mutex>

#include "common.cuh"

namespace qmcur {
namespace {

constexpr int kThreads = 64;
constexpr int kRows = 32;              // rows per CTA tile
constexpr int kFlush = 8;              // FP32 column run length (rows)
constexpr int kCols = kThreads * 4;    // columns per CTA tile

template <typename T>
struct Acc { using type = float; };
template <>
struct Acc<double> { using type = double; };

template <typename T>
__device__ __forceinline__ void load4(const T* row, int64_t j0, int64_t n, bool vec, T out[4]) {
  if (vec && j0 + 3 < n) {
    if constexpr (sizeof(T) == 4) {
      float4 v = __ldcs(reinterpret_cast<const float4*>(row + j0));
      out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else {
      double2 a = __ldcs(reinterpret_cast<const double2*>(row + j0));
      double2 b = __ldcs(reinterpret_cast<const double2*>(row + j0 + 2));
      out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = (j0 + u < n) ? row[j0 + u] : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_norm_partial(QView A, bool vec, double* __restrict__ col_part, double* __restrict__ row_part) {
  using acc_t = typename Acc<T>::type;
  const int64_t m = A.rows, n = A.cols;
  const int ctile = blockIdx.x, rtile = blockIdx.y;
  const int64_t j0 = (int64_t)ctile * kCols + threadIdx.x * 4;
  const int64_t i0 = (int64_t)rtile * kRows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ acc_t row_warp[kRows][kThreads / 32];

  double col64[4] = {0.0, 0.0, 0.0, 0.0};
  acc_t col32[4] = {0, 0, 0, 0};
  const T* P0 = plane<T>(A, 0);
  const T* P1 = plane<T>(A, 1);
  const T* P2 = plane<T>(A, 2);
  const T* P3 = plane<T>(A, 3);
  // rows in flight per thread: four planes x four values each
  constexpr int kUnroll = sizeof(T) == 4 ? 8 : 4;
  static_assert(kFlush % kUnroll == 0 && kRows % kFlush == 0, "whole runs");
  for (int r0 = 0; r0 < kRows; r0 += kUnroll) {
    T x[kUnroll][4][4];
#pragma unroll
    for (int h = 0; h < kUnroll; ++h) {
      const int64_t i = i0 + r0 + h;
      if (i < m) {
        load4<T>(P0 + i * A.ld, j0, n, vec, x[h][0]);
        load4<T>(P1 + i * A.ld, j0, n, vec, x[h][1]);
        load4<T>(P2 + i * A.ld, j0, n, vec, x[h][2]);
        load4<T>(P3 + i * A.ld, j0, n, vec, x[h][3]);
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int u = 0; u < 4; ++u) x[h][t][u] = T(0);
      }
    }
#pragma unroll
    for (int h = 0; h < kUnroll; ++h) {
      const int rr = r0 + h;
      acc_t rs = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc_t s = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) s = fma((acc_t)x[h][t][u], (acc_t)x[h][t][u], s);
        col32[u] += s;
        rs += s;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
      if (lane == 0) row_warp[rr][warp] = rs;
      if ((rr + 1) % kFlush == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) { col64[u] += (double)col32[u]; col32[u] = 0; }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (j0 + u < n) col_part[(int64_t)rtile * n + j0 + u] = col64[u];
  __syncthreads();
  if (threadIdx.x < kRows) {
    const int64_t i = i0 + threadIdx.x;
    if (i < m) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) s += (double)row_warp[threadIdx.x][w];
      row_part[(int64_t)ctile * m + i] = s;
    }
  }
}

// col2[j] = sum over row tiles, row2[i] = sum over column tiles.  A CTA
// folds 32 consecutive outputs (columns first, then rows): its kFoldGroups
// thread groups each sum a contiguous run of tiles left to right (loads
// issued together), then group 0 adds the group sums in group order; a
// column CTA also writes the sum of its 32 col2 values (a fixed shuffle
// tree) to blocktot.  The orders are fixed, so the result is reproducible.
constexpr int kFoldGroups = 8;

__global__ void __launch_bounds__(32 * kFoldGroups)
k_norm_fold(const double* __restrict__ col_part, const double* __restrict__ row_part, int64_t m,
            int64_t n, int rtiles, int ctiles, double* __restrict__ col2,
            double* __restrict__ row2, double* __restrict__ blocktot) {
  __shared__ double part[kFoldGroups][32];
  const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t col_blocks = (n + 31) / 32;
  const bool cols = blockIdx.x < col_blocks;
  const int64_t base = cols ? (int64_t)blockIdx.x * 32 : ((int64_t)blockIdx.x - col_blocks) * 32;
  const int64_t len = cols ? n : m, idx = base + lane;
  const int tiles = cols ? rtiles : ctiles;
  const double* src = cols ? col_part : row_part;
  const int per = (tiles + kFoldGroups - 1) / kFoldGroups;
  const int t0 = grp * per, t1 = t0 + per < tiles ? t0 + per : tiles;
  double s = 0.0;
  if (idx < len) {
    constexpr int kBatch = 8;
    for (int tb = t0; tb < t1; tb += kBatch) {
      double v[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) v[u] = tb + u < t1 ? src[(int64_t)(tb + u) * len + idx] : 0.0;
#pragma unroll
      for (int u = 0; u < kBatch; ++u) s += v[u];
    }
  }
  part[grp][lane] = s;
  __syncthreads();
  if (grp == 0) {
    double tot = 0.0;
    if (idx < len) {
      tot = part[0][lane];
#pragma unroll
      for (int g = 1; g < kFoldGroups; ++g) tot += part[g][lane];
      (cols ? col2 : row2)[idx] = tot;
    }
    if (cols) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
      if (lane == 0) blocktot[blockIdx.x] = tot;
    }
  }
}

// F = the sum of the fold's column-block totals in a fixed order, formed by
// every CTA (bit-identical copies); CTA 0 reports NONFINITE / ZERO_NORM and
// writes fro2.  With `scale`
// the CTAs then write their grid-strided share of col_p = col2 (1 / F) and
// row_p = row2 (1 / F) (separate buffers: no CTA rewrites what another reads;
// one FP64 division per CTA, the rest multiplies, within an ulp of col2 / F).
constexpr int kScaleThreads = 256;

__global__ void __launch_bounds__(kScaleThreads)
k_norm_total_scale(const double* __restrict__ col2, const double* __restrict__ row2,
                   const double* __restrict__ blocktot, int64_t m, int64_t n,
                   double* __restrict__ col_p, double* __restrict__ row_p,
                   double* __restrict__ fro2, int scale, int32_t* status) {
  __shared__ double red[kScaleThreads];
  double s = 0.0;
  const int64_t nb = (n + 31) / 32;
  for (int64_t j = threadIdx.x; j < nb; j += kScaleThreads) s += blocktot[j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kScaleThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double F = red[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (fro2 != nullptr) *fro2 = F;
    if (!isfinite(F)) set_status(status, QMCUR_ERR_NONFINITE);
    else if (scale && F == 0.0) set_status(status, QMCUR_ERR_ZERO_NORM);
  }
  if (!scale) return;
  const double rF = 1.0 / F;
  const int64_t stride = (int64_t)gridDim.x * kScaleThreads;
  for (int64_t g = (int64_t)blockIdx.x * kScaleThreads + threadIdx.x; g < n + m; g += stride) {
    if (g < n) col_p[g] = col2[g] * rF;
    else row_p[g - n] = row2[g - n] * rF;
  }
}

__global__ void k_uniform(double* __restrict__ col_p, double* __restrict__ row_p, int64_t m, int64_t n) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) col_p[g] = 1.0 / (double)n;
  else if (g < n + m) row_p[g - n] = 1.0 / (double)m;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t probs_ws_bytes(int64_t m, int64_t n) {
  Carve c(nullptr, 0);
  const int64_t rt = cdiv(m, kRows), ct = cdiv(n, kCols);
  c.take<double>((size_t)(rt * n));
  c.take<double>((size_t)(ct * m));
  c.take<double>((size_t)(n + m));
  c.take<double>((size_t)cdiv(n, 32) + 4);
  return c.off;
}

qmcur_status launch_probs(const qmcur_qmat* A, int32_t sampler, double* col_p, double* row_p,
                          double* fro2, void* ws, size_t ws_bytes, int32_t* dev_status,
                          cudaStream_t st) {
  if (!valid_qmat(A) || col_p == nullptr || row_p == nullptr) return QMCUR_ERR_INVALID_ARG;
  if (sampler != QMCUR_SAMPLER_UNIFORM && sampler != QMCUR_SAMPLER_NORM) return QMCUR_ERR_INVALID_ARG;
  const int64_t m = A->rows, n = A->cols;
  if (m < 1 || n < 1) return QMCUR_ERR_INVALID_ARG;
  const int64_t total = m + n;
  const int fold_blocks = (int)cdiv(total, 256);
  if (sampler == QMCUR_SAMPLER_UNIFORM) {
    k_uniform<<<fold_blocks, 256, 0, st>>>(col_p, row_p, m, n);
    if (fro2 == nullptr) return cuda_ok(cudaGetLastError());
  }
  const int64_t rt = cdiv(m, kRows), ct = cdiv(n, kCols);
  if (rt > 65535) return QMCUR_ERR_UNSUPPORTED;
  Carve cv(ws, ws_bytes);
  double* col_part = cv.take<double>((size_t)(rt * n));
  double* row_part = cv.take<double>((size_t)(ct * m));
  double* sums = cv.take<double>((size_t)(n + m));
  double* blocktot = cv.take<double>((size_t)cdiv(n, 32) + 4);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  // The squared norms go to scratch; norm mode then writes the outputs from
  // them, uniform mode (which only wants ||A||_F^2) keeps 1/n, 1/m.
  double* col2 = sums;
  double* row2 = sums + n;
  QView v = view(A);
  const size_t es = esize(A->dtype);
  bool vec = (A->ld * es) % 16 == 0;
  for (int t = 0; t < 4; ++t) vec = vec && (reinterpret_cast<uintptr_t>(A->plane[t]) % 16 == 0);
  dim3 grid((unsigned)ct, (unsigned)rt);
  if (A->dtype == QMCUR_F32) k_norm_partial<float><<<grid, kThreads, 0, st>>>(v, vec, col_part, row_part);
  else k_norm_partial<double><<<grid, kThreads, 0, st>>>(v, vec, col_part, row_part);
  const int fold_ctas = (int)(cdiv(n, 32) + cdiv(m, 32));
  k_norm_fold<<<fold_ctas, 32 * kFoldGroups, 0, st>>>(col_part, row_part, m, n, (int)rt, (int)ct,
                                                      col2, row2, blocktot);
  const int64_t scale_ctas = cdiv(n + m, kScaleThreads) < 64 ? cdiv(n + m, kScaleThreads) : 64;
  k_norm_total_scale<<<(unsigned)scale_ctas, kScaleThreads, 0, st>>>(
      col2, row2, blocktot, m, n, col_p, row_p, fro2, sampler == QMCUR_SAMPLER_NORM, dev_status);
  return cuda_ok(cudaGetLastError());
}

// ------------------------------------------------------------------------
// Allocation-free variant of qmcur_probs.
//
// For callers that cannot call cudaMalloc or hand the library a workspace:
// code inside a host framework whose allocator owns all device memory, or a
// latency-bound loop where an allocation (which can synchronise the device)
// is not acceptable, and whose interface has no place to thread a scratch
// buffer through.  Its scratch is this file-scope array: every GPU that loads
// the library holds it until the process exits, all calls on a device share
// it and it keeps the last call's contents.  Every scratch entry the kernels
// read is written earlier in the same call, so nothing needs clearing; calls
// that overlap on the GPU (e.g. on two streams at once) race on it.
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;   // 8 MiB per device
static __device__ __align__(256) unsigned char g_probs_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_scratch_mu;
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_probs_scratch on the current device, looked up once per
// device (in host code the array's name is only a host-side stand-in).
qmcur_status scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QMCUR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_probs_scratch) != cudaSuccess || p == nullptr) return QMCUR_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return QMCUR_OK;
}
}  // namespace

}  // namespace qmcur

extern "C" qmcur_status qmcur_probs_noalloc(const qmcur_qmat* A, int32_t sampler, double* col_p,
                                            double* row_p, double* fro2, int32_t* dev_status,
                                            cudaStream_t stream) {
  qmcur::NvtxRange nvtx_range("qmcur_probs_noalloc");
  using namespace qmcur;
  if (!valid_qmat(A)) return QMCUR_ERR_INVALID_ARG;
  // the uniform sampler without ||A||_F^2 reads neither A nor scratch
  const bool needs_scratch = !(sampler == QMCUR_SAMPLER_UNIFORM && fro2 == nullptr);
  if (needs_scratch && probs_ws_bytes(A->rows, A->cols) > kNoAllocScratchBytes)
    return QMCUR_ERR_UNSUPPORTED;
  void* scratch = nullptr;
  const qmcur_status s = scratch_address(&scratch);
  if (s != QMCUR_OK) return s;
  return launch_probs(A, sampler, col_p, row_p, fro2, scratch, kNoAllocScratchBytes, dev_status,
                      stream);
}
