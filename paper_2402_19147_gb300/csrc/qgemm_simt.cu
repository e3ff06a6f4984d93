// Quaternion GEMM on CUDA cores: the plain FP32 path (and FP64 for FP64
// inputs), plus the relative Frobenius residual (Example 4.2's measure).
//
// Z = X Y with the Hamilton product (Sec. 2.2), planes split:
//   Z0 = X0Y0 - X1Y1 - X2Y2 - X3Y3      Z1 = X0Y1 + X1Y0 + X2Y3 - X3Y2
//   Z2 = X0Y2 - X1Y3 + X2Y0 + X3Y1      Z3 = X0Y3 + X1Y2 - X2Y1 + X3Y0
// A CTA computes a 64 x 64 tile of quaternion outputs; each of its 256
// threads a 4 x 4 block (64 accumulators), so every pair of quaternions read
// from shared memory feeds 16 FMAs.  The k-loop stages 4 planes x 64 x 8 of X
// (transposed to k-major) and 4 x 8 x 64 of Y per step, double buffered.
//
// MODE_STORE writes Z.  MODE_RESIDUAL never writes Z: the epilogue reads the
// matching tile of A and accumulates sum |a - z|^2 and sum |a|^2 (optionally
// over the observed set Omega of a mask) into one FP64 pair per CTA, folded
// afterwards in a fixed order.  MODE_COMPLETE is one step of masked
// completion (Algorithm 2): A is the iterate, its unobserved entries (mask 0)
// are overwritten in place by Z (the Z view aliases A), and the pair is
// {sum over unobserved of |z - a|^2, sum over all of |a|^2}.
#include "common.cuh"

namespace qmcur {
namespace {

constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4, kGemmThreads = 256;

enum { MODE_STORE = 0, MODE_RESIDUAL = 1, MODE_COMPLETE = 2 };

template <typename T>
struct QAcc { T v[4]; };

template <typename TX, typename TY, typename T, int MODE>
__global__ void __launch_bounds__(kGemmThreads)
k_qgemm_simt(QView X, QView Y, QView Z, QView A, const uint8_t* __restrict__ mask,
             double* __restrict__ partial) {
  const int64_t M = X.rows, K = X.cols, N = Y.cols;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  __shared__ __align__(16) T xs[2][4][BK][BM];
  __shared__ __align__(16) T ys[2][4][BK][BN];

  T acc[TM][TN][4];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[i][j][t] = T(0);

  // global -> shared mapping: X tile 64 rows x 8 k: thread loads rows
  // (tid / 8) and (tid / 8) + 32, k = tid % 8, all 4 planes.
  auto load_tile = [&](int buf, int64_t k0) {
    const int kx = tid % BK;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int mm = tid / BK + 32 * h;
      const int64_t gi = m0 + mm, gk = k0 + kx;
      const bool in = gi < M && gk < K;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        xs[buf][t][kx][mm] = in ? (T)reinterpret_cast<const TX*>(X.p[t])[gi * X.ld + gk] : T(0);
    }
    // Y tile 8 k x 64 columns: thread loads k = tid / 32, columns tid % 32 (+32)
    const int ky = tid / 32;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nn = tid % 32 + 32 * h;
      const int64_t gk = k0 + ky, gj = n0 + nn;
      const bool in = gk < K && gj < N;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        ys[buf][t][ky][nn] = in ? (T)reinterpret_cast<const TY*>(Y.p[t])[gk * Y.ld + gj] : T(0);
    }
  };

  const int64_t nk = (K + BK - 1) / BK;
  load_tile(0, 0);
  __syncthreads();
  for (int64_t kt = 0; kt < nk; ++kt) {
    const int buf = (int)(kt & 1);
    if (kt + 1 < nk) load_tile(buf ^ 1, (kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T x[TM][4], y[TN][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
#pragma unroll
        for (int i = 0; i < TM; ++i) x[i][t] = xs[buf][t][kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) y[j][t] = ys[buf][t][kk][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const T* a = x[i];
          const T* b = y[j];
          T* z = acc[i][j];
          z[0] = fma(a[0], b[0], z[0]); z[0] = fma(-a[1], b[1], z[0]);
          z[0] = fma(-a[2], b[2], z[0]); z[0] = fma(-a[3], b[3], z[0]);
          z[1] = fma(a[0], b[1], z[1]); z[1] = fma(a[1], b[0], z[1]);
          z[1] = fma(a[2], b[3], z[1]); z[1] = fma(-a[3], b[2], z[1]);
          z[2] = fma(a[0], b[2], z[2]); z[2] = fma(-a[1], b[3], z[2]);
          z[2] = fma(a[2], b[0], z[2]); z[2] = fma(a[3], b[1], z[2]);
          z[3] = fma(a[0], b[3], z[3]); z[3] = fma(a[1], b[2], z[3]);
          z[3] = fma(-a[2], b[1], z[3]); z[3] = fma(a[3], b[0], z[3]);
        }
    }
    __syncthreads();
  }

  if constexpr (MODE == MODE_STORE) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gi = m0 + ty * TM + i, gj = n0 + tx * TN + j;
        if (gi < M && gj < N)
#pragma unroll
          for (int t = 0; t < 4; ++t) st_from_double(Z, t, gi, gj, (double)acc[i][j][t]);
      }
  } else if constexpr (MODE == MODE_COMPLETE) {
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      T rn = T(0), rd = T(0);
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gi = m0 + ty * TM + i, gj = n0 + tx * TN + j;
        if (gi < M && gj < N) {
          const bool observed = mask == nullptr || mask[gi * N + gj] != 0;
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const T av = (T)ld_as_double(A, t, gi, gj);
            rd = fma(av, av, rd);
            if (!observed) {
              const T d = acc[i][j][t] - av;
              rn = fma(d, d, rn);
            }
          }
          if (!observed)
#pragma unroll
            for (int t = 0; t < 4; ++t) st_from_double(Z, t, gi, gj, (double)acc[i][j][t]);
        }
      }
      num += (double)rn;
      den += (double)rd;
    }
    __shared__ double redc[2][kGemmThreads];
    redc[0][tid] = num;
    redc[1][tid] = den;
    __syncthreads();
    for (int w = kGemmThreads / 2; w > 0; w >>= 1) {
      if (tid < w) { redc[0][tid] += redc[0][tid + w]; redc[1][tid] += redc[1][tid + w]; }
      __syncthreads();
    }
    if (tid == 0) {
      const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      partial[2 * cta] = redc[0][0];
      partial[2 * cta + 1] = redc[1][0];
    }
  } else {
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      T rn = T(0), rd = T(0);
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t gi = m0 + ty * TM + i, gj = n0 + tx * TN + j;
        if (gi < M && gj < N && (mask == nullptr || mask[gi * N + gj] != 0)) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const T av = (T)ld_as_double(A, t, gi, gj);
            const T d = av - acc[i][j][t];
            rn = fma(d, d, rn);
            rd = fma(av, av, rd);
          }
        }
      }
      num += (double)rn;
      den += (double)rd;
    }
    __shared__ double red[2][kGemmThreads];
    red[0][tid] = num;
    red[1][tid] = den;
    __syncthreads();
    for (int w = kGemmThreads / 2; w > 0; w >>= 1) {
      if (tid < w) { red[0][tid] += red[0][tid + w]; red[1][tid] += red[1][tid + w]; }
      __syncthreads();
    }
    if (tid == 0) {
      const int64_t cta = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      partial[2 * cta] = red[0][0];
      partial[2 * cta + 1] = red[1][0];
    }
  }
}

// Standalone residual over materialised A and Z: one CTA per kResRows x 256
// tile, one column per thread.  FP32 inputs are summed in float-float on the
// FP32 pipe (a - z split exactly by TwoSum, squares by TwoProd, Knuth's
// TwoSum into the pair), about 2^-44 of the sum over the tile's rows, and the
// tile's partials are carried in FP64: FP64-level sums without FP64 work per
// entry.  FP64 inputs are summed in FP64.
constexpr int kResRows = 8;

__device__ __forceinline__ void res_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (S, C) += x^2 (x = xh + xl exactly), in float-float
__device__ __forceinline__ void res_add_sq(float& S, float& C, float xh, float xl) {
  const float p = __fmul_rn(xh, xh);
  const float e = __fmaf_rn(xh, xh, -p);
  float s, t;
  res_two_sum(S, p, s, t);
  S = s;
  C = __fadd_rn(C, __fadd_rn(t, __fmaf_rn(__fmul_rn(2.f, xh), xl, e)));
}

template <typename TA, typename TZ>
__global__ void __launch_bounds__(256)
k_residual(QView A, QView Z, const uint8_t* __restrict__ mask, double* __restrict__ partial) {
  const int64_t m = A.rows, n = A.cols;
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.y * kResRows;
  constexpr bool ff = sizeof(TA) == 4 && sizeof(TZ) == 4;
  double num = 0.0, den = 0.0;
  if (j < n) {
    // every load of the tile's column first (rows past m read as zero), then
    // the sums; masked entries are selected away, so that whatever they hold
    // (even a NaN) does not count
    TA av[kResRows][4];
    TZ zv[kResRows][4];
    bool on[kResRows];
#pragma unroll
    for (int rr = 0; rr < kResRows; ++rr) {
      const int64_t i = i0 + rr;
      const bool in = i < m;
      on[rr] = in && (mask == nullptr || mask[i * n + j] != 0);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        av[rr][t] = in ? reinterpret_cast<const TA*>(A.p[t])[i * A.ld + j] : TA(0);
        zv[rr][t] = in ? reinterpret_cast<const TZ*>(Z.p[t])[i * Z.ld + j] : TZ(0);
      }
    }
    float Sn = 0.f, Cn = 0.f, Sd = 0.f, Cd = 0.f;
#pragma unroll
    for (int rr = 0; rr < kResRows; ++rr) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if constexpr (ff) {
          float dh, dl;
          res_two_sum((float)av[rr][t], -(float)zv[rr][t], dh, dl);
          res_add_sq(Sn, Cn, on[rr] ? dh : 0.f, on[rr] ? dl : 0.f);
          res_add_sq(Sd, Cd, on[rr] ? (float)av[rr][t] : 0.f, 0.f);
        } else {
          const double d = on[rr] ? (double)av[rr][t] - (double)zv[rr][t] : 0.0;
          const double a = on[rr] ? (double)av[rr][t] : 0.0;
          num = fma(d, d, num);
          den = fma(a, a, den);
        }
      }
    }
    if constexpr (ff) {
      num = (double)Sn + (double)Cn;
      den = (double)Sd + (double)Cd;
    }
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = num;
  red[1][threadIdx.x] = den;
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

}  // namespace

// Fold per-CTA (num, den) pairs in a fixed order: out3 = {rel, num, den}.
__global__ void __launch_bounds__(1024) k_residual_fold(const double* __restrict__ partial, int64_t count,
                                                        double* __restrict__ out3) {
  // strided sums, then a fixed shuffle tree per warp and across the warps
  __shared__ double red[2][32];
  double num = 0.0, den = 0.0;
  for (int64_t k = threadIdx.x; k < count; k += 1024) { num += partial[2 * k]; den += partial[2 * k + 1]; }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if (lane == 0) { red[0][warp] = num; red[1][warp] = den; }
  __syncthreads();
  if (warp == 0) {
    num = red[0][lane];
    den = red[1][lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_xor_sync(0xffffffffu, num, o);
      den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
      out3[1] = num;
      out3[2] = den;
      out3[0] = den > 0.0 ? sqrt(num / den) : __longlong_as_double(0x7ff8000000000000ll);
    }
  }
}

size_t simt_partials(int64_t m, int64_t n) {
  return (size_t)(((m + BM - 1) / BM) * ((n + BN - 1) / BN));
}

size_t residual_partials(int64_t m, int64_t n) {
  return (size_t)(((m + kResRows - 1) / kResRows) * ((n + 255) / 256));
}

// X (M x K) times Y (K x N) -> Z, or the fused residual against A, or (complete)
// one masked completion step of A in place (Z must then view A's planes).
qmcur_status launch_qgemm_simt(const QView& X, const QView& Y, const QView* Z, const QView* A,
                               const uint8_t* mask, double* partial, bool fp64, cudaStream_t st,
                               bool complete) {
  if (complete && (Z == nullptr || A == nullptr)) return QMCUR_ERR_INVALID_ARG;
  const int64_t M = X.rows, N = Y.cols;
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  if (grid.y > 65535) return QMCUR_ERR_UNSUPPORTED;
  QView dummy = X;
  const QView& z = Z ? *Z : dummy;
  const QView& a = A ? *A : dummy;
  const bool xd = X.dtype == QMCUR_F64, yd = Y.dtype == QMCUR_F64;
  if (complete) {
    if (fp64) {
      if (!xd || !yd) return QMCUR_ERR_INVALID_ARG;
      k_qgemm_simt<double, double, double, MODE_COMPLETE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
    } else {
      if (yd) return QMCUR_ERR_INVALID_ARG;
      if (xd) k_qgemm_simt<double, float, float, MODE_COMPLETE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
      else k_qgemm_simt<float, float, float, MODE_COMPLETE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
    }
    return cuda_ok(cudaGetLastError());
  }
  if (fp64) {
    if (!xd || !yd) return QMCUR_ERR_INVALID_ARG;
    if (Z) k_qgemm_simt<double, double, double, MODE_STORE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
    else k_qgemm_simt<double, double, double, MODE_RESIDUAL><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
  } else {
    if (yd) return QMCUR_ERR_INVALID_ARG;
    if (Z) {
      if (xd) k_qgemm_simt<double, float, float, MODE_STORE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
      else k_qgemm_simt<float, float, float, MODE_STORE><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
    } else {
      if (xd) k_qgemm_simt<double, float, float, MODE_RESIDUAL><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
      else k_qgemm_simt<float, float, float, MODE_RESIDUAL><<<grid, kGemmThreads, 0, st>>>(X, Y, z, a, mask, partial);
    }
  }
  return cuda_ok(cudaGetLastError());
}

qmcur_status launch_residual_standalone(const qmcur_qmat* A, const qmcur_qmat* Z,
                                        const uint8_t* mask, double* out3, void* ws,
                                        size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  (void)dev_status;
  if (!valid_qmat(A) || !valid_qmat(Z) || out3 == nullptr) return QMCUR_ERR_INVALID_ARG;
  if (A->rows != Z->rows || A->cols != Z->cols || A->rows < 1 || A->cols < 1) return QMCUR_ERR_INVALID_ARG;
  const int64_t m = A->rows, n = A->cols;
  const int64_t cnt = (int64_t)residual_partials(m, n);
  Carve cv(ws, ws_bytes);
  double* partial = cv.take<double>((size_t)(2 * cnt));
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)((m + kResRows - 1) / kResRows));
  if (grid.y > 65535) return QMCUR_ERR_UNSUPPORTED;
  QView a = view(A), z = view(Z);
  const bool ad = A->dtype == QMCUR_F64, zd = Z->dtype == QMCUR_F64;
  if (ad && zd) k_residual<double, double><<<grid, 256, 0, st>>>(a, z, mask, partial);
  else if (ad) k_residual<double, float><<<grid, 256, 0, st>>>(a, z, mask, partial);
  else if (zd) k_residual<float, double><<<grid, 256, 0, st>>>(a, z, mask, partial);
  else k_residual<float, float><<<grid, 256, 0, st>>>(a, z, mask, partial);
  k_residual_fold<<<1, 1024, 0, st>>>(partial, cnt, out3);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
