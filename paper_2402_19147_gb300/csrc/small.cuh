// Small dense quaternion kernels (FP32 compute) used by the subspace
// pseudo-inverse: op(X) op(Y) GEMMs with op in {identity, conjugate
// transpose}, and a one-CTA Cholesky factorisation with triangular inverse.
#pragma once

#include "common.cuh"

namespace qmcur {

// Four plane pointers with a common row stride (elements) and element type.
struct QPtr {
  void* p[4];
  int64_t ld;
  int32_t dtype;
};

// Largest k of small_chol_inv (R and R^-1 packed in shared memory).
constexpr int kSmallCholMax = 112;

// Z = alpha op(X) op(Y) + beta Z, op(X) M x K, op(Y) K x N.  With xh, X is
// stored K x M and op(X) = X^H (conjugate transpose, Sec. 2.2); likewise yh.
// X, Y are FP32; Z may be FP32 or FP64.  beta == 0 never reads Z.
qmcur_status small_qgemm(bool xh, bool yh, int M, int N, int K, float alpha, const QPtr& X,
                         const QPtr& Y, float beta, const QPtr& Z, cudaStream_t st);

// G (k x k Hermitian positive definite) = R^H R with R upper triangular with
// a real positive diagonal; writes Rinv = R^-1 (k x k, zeros below the
// diagonal).  A non-positive or non-finite pivot sets ILL_CONDITIONED.
qmcur_status small_chol_inv(const QPtr& G, int k, const QPtr& Rinv, int32_t* status,
                            cudaStream_t st);

void small_set_rank(int32_t* rank_out, int k, int iters, cudaStream_t st);

}  // namespace qmcur
