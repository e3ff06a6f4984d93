// Small dense quaternion GEMM kernel (see small.cuh); the device code lives
// in small_impl.cuh so that the fused pseudo-inverse can reuse it.
#include "small_impl.cuh"

namespace qmcur {
namespace {

__global__ void __launch_bounds__(kSmTileThreads) k_qgemm_small(SmallGemmArgs a, int tiles_n) {
  __shared__ float4 sm[kSmGemmQuats];
  sm_gemm_tile(a, blockIdx.x / tiles_n, blockIdx.x % tiles_n, sm, threadIdx.x, 1);
}

}  // namespace

qmcur_status small_qgemm(bool xh, bool yh, int M, int N, int K, float alpha, const QPtr& X,
                         const QPtr& Y, float beta, const QPtr& Z, cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1) return QMCUR_ERR_INVALID_ARG;
  SmallGemmArgs a{X, Y, Z, M, N, K, alpha, beta, xh ? 1 : 0, yh ? 1 : 0};
  const int tm = (M + kSmTS - 1) / kSmTS, tn = (N + kSmTS - 1) / kSmTS;
  const int64_t tiles = (int64_t)tm * tn;
  if (tiles > INT32_MAX) return QMCUR_ERR_UNSUPPORTED;
  k_qgemm_small<<<(unsigned)tiles, kSmTileThreads, 0, st>>>(a, tn);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
