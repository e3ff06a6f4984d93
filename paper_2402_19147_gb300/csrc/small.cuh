// Small dense quaternion kernels (FP32 compute) used by the subspace
// pseudo-inverse and the backward pass: op(X) op(Y) GEMMs with op in
// {identity, conjugate transpose}; the device code (also a one-CTA Cholesky
// factorisation and a warp-per-row triangular solve) is in small_impl.cuh.
#pragma once

#include "common.cuh"

namespace qmcur {

// Element type of workspace planes that hold float-float pairs: each plane
// entry is a float2 (h, l) standing for h + l (internal to the library,
// beside QMCUR_F32 and QMCUR_F64).
constexpr int32_t kDtypeFF = 2;

// Four plane pointers with a common row stride (elements) and element type.
struct QPtr {
  void* p[4];
  int64_t ld;
  int32_t dtype;
};

// Largest k of the small Cholesky factorisation: the k (k + 1) / 2 entries
// of the upper triangle are held in registers of a 512-thread CTA, and a
// triangular-solve row in 4 registers per lane.
constexpr int kSmallCholMax = 100;

// One small product Z = alpha op(X) op(Y) + beta Z, op(X) M x K, op(Y) K x N.
// With xh, X is stored K x M and op(X) = X^H (conjugate transpose, Sec. 2.2);
// likewise yh.  X, Y are FP32; Z may be FP32 or FP64.  beta == 0 never reads Z.
struct SmallGemmArgs {
  QPtr X, Y, Z;
  int M, N, K;
  float alpha, beta;
  int xh, yh;
};

qmcur_status small_qgemm(bool xh, bool yh, int M, int N, int K, float alpha, const QPtr& X,
                         const QPtr& Y, float beta, const QPtr& Z, cudaStream_t st);

// Up to kSmallBatchMax independent small products in one launch (their tiles
// side by side in the grid).  No product may read another's output.
constexpr int kSmallBatchMax = 6;
qmcur_status small_qgemm_batch(const SmallGemmArgs* jobs, int count, cudaStream_t st);

}  // namespace qmcur
