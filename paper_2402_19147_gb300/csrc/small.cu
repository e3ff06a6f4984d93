// Small dense quaternion GEMM kernel (see small.cuh); the device code lives
// in small_impl.cuh so that the fused pseudo-inverse can reuse it.
#include "small_impl.cuh"

namespace qmcur {
namespace {

__global__ void __launch_bounds__(kSmTileThreads) k_qgemm_small(SmallGemmArgs a, int tiles_n) {
  __shared__ float4 sm[kSmGemmQuats];
  sm_gemm_tile(a, blockIdx.x / tiles_n, blockIdx.x % tiles_n, sm, threadIdx.x, 1);
}

struct SmallGemmBatch {
  SmallGemmArgs job[kSmallBatchMax];
  int tile0[kSmallBatchMax + 1];   // first tile of each job, then the total
  int tn[kSmallBatchMax];          // tile columns of each job
  int count;
};

__global__ void __launch_bounds__(kSmTileThreads)
k_qgemm_small_batch(const __grid_constant__ SmallGemmBatch b) {
  __shared__ float4 sm[kSmGemmQuats];
  int q = 0;
  while (q + 1 < b.count && (int)blockIdx.x >= b.tile0[q + 1]) ++q;
  const int t = (int)blockIdx.x - b.tile0[q];
  sm_gemm_tile(b.job[q], t / b.tn[q], t % b.tn[q], sm, threadIdx.x, 1);
}

}  // namespace

qmcur_status small_qgemm_batch(const SmallGemmArgs* jobs, int count, cudaStream_t st) {
  if (jobs == nullptr || count < 1 || count > kSmallBatchMax) return QMCUR_ERR_INVALID_ARG;
  SmallGemmBatch b{};
  int64_t total = 0;
  for (int q = 0; q < count; ++q) {
    const SmallGemmArgs& a = jobs[q];
    if (a.M < 1 || a.N < 1 || a.K < 1) return QMCUR_ERR_INVALID_ARG;
    b.job[q] = a;
    b.tn[q] = (a.N + kSmTS - 1) / kSmTS;
    b.tile0[q] = (int)total;
    total += (int64_t)((a.M + kSmTS - 1) / kSmTS) * b.tn[q];
    if (total > INT32_MAX) return QMCUR_ERR_UNSUPPORTED;
  }
  b.tile0[count] = (int)total;
  b.count = count;
  k_qgemm_small_batch<<<(unsigned)total, kSmTileThreads, 0, st>>>(b);
  return cuda_ok(cudaGetLastError());
}

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
