// Tensor-core (tcgen05) quaternion GEMM: placeholder until the kernel lands.
#include "common.cuh"

namespace qmcur {

size_t tc_ws_bytes(int64_t, int64_t, int64_t, int64_t, int32_t) { return 0; }

qmcur_status launch_reconstruct_tc(const qmcur_qmat*, const qmcur_qmat*, const qmcur_qmat*, int32_t,
                                   qmcur_qmat*, const qmcur_qmat*, const uint8_t*, double*, void*,
                                   size_t, int32_t*, cudaStream_t) {
  return QMCUR_ERR_UNSUPPORTED;
}

}  // namespace qmcur
