// Grouped tensor-core products of the batched path: one launch of the
// tcgen05 GEMM over the tiles of many problems whose operand pieces are
// stacked along rows in two shared buffers (every problem's A = C pieces
// under one TMA map, its B = T^T pieces under another), with the relative
// residual against each problem's A fused into the epilogue.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace qmcur {

// An FP32 value rounded to TF32 (nearest, ties away from zero).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Pieces of one value for the split products: BF16 (npieces 2 or 3) or
// TF32 (npieces 2).
template <bool BF16, typename T>
__device__ __forceinline__ void split_value(T x, int npieces, float out[3]) {
  // The pieces carry at most ~24 significant bits, so the split runs in FP32
  // (GB300's FP64 rate is 1/64 of FP32); each residual below is exact in FP32.
  const float xf = (float)x;
  if constexpr (BF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    out[0] = __bfloat162float(h);
    out[1] = __bfloat162float(m);
    out[2] = npieces > 2 ? __bfloat162float(__float2bfloat16_rn(r2)) : 0.f;
  } else {
    const float b = tf32_rna(xf);
    out[0] = b;
    out[1] = xf - b;
    out[2] = 0.f;
  }
}

// One 128-row output tile of problem `prob` at (m0, n0) of its Z = C T.
struct TcGroupTile {
  int prob, m0, n0;
};

// What the grouped kernel needs of one problem: its input A (residual),
// shape, inner dimension K and its pieces' k-blocks, the first rows of its
// operands in the stacked buffers, and (pieces' store) its first row in the
// output piece buffer.
struct TcGroupProb {
  const float* a[4];
  int64_t lda;
  int m, n, K, kblocks, arow, brow, a_vec;
  int64_t zrow;
};

// Tile width (columns of T^T, i.e. rows of T) of the grouped T^T = R^T U.
constexpr int kGroupTBn = 64;

// One operand of one problem for the batched split: S (rows x K as stored,
// or K x rows when trans) into rows row0 .. row0 + rows of a stacked piece
// buffer dst[(q * 4 + t)][row][k] (plane stride = rows_total * kpad), k below
// kp_job = K rounded up to the pieces' row width (zeros beyond K).
struct TcSplitJob {
  QView S;
  void* dst;
  int64_t rows, K, kp_job, kpad, row0, plane_stride;
  int trans;
  int tiles_k, first_tile;
};

// product selects the split of the precision: 1 for Z = C T, 0 for T = U R
// (the mixed split: BF16X3 and BF16X6).
// Elements per 64-byte piece row of a precision (32 BF16, 16 TF32).
int tc_group_epr(int32_t prec, int product = 1);
// Pieces per operand value of a precision (2 or 3).
int tc_group_npieces(int32_t prec, int product = 1);
// Bytes of one stacked piece buffer of `rows` rows.
size_t tc_group_piece_bytes(int32_t prec, int64_t rows, int64_t kpad, int product = 1);
// The batched split of the jobs (device table, tiles in all) into pieces.
qmcur_status tc_group_split(int32_t prec, const TcSplitJob* jobs, int njobs, int tiles,
                            cudaStream_t st, int product = 1);
// The grouped T^T = R^T U (the split of product 0; R_all holds every
// problem's R^T pieces, rows n, U_all its U pieces, rows c, K = r), each
// tile cut into the pieces of product 1's split and stored K-major at rows
// zrow + (0 .. n) of `pieces` (pieces_rows rows of pieces_kpad elements per
// plane and piece): Z = C T's B operand, with T never stored.
qmcur_status tc_group_t_pieces(int32_t prec, const void* R_all, int64_t rows_r, const void* U_all,
                               int64_t rows_u, int64_t kpad, const TcGroupTile* tiles, int ntiles,
                               const TcGroupProb* probs, void* pieces, int64_t pieces_kpad,
                               int64_t pieces_rows, int32_t* dev_status, cudaStream_t st);

// The grouped Z = C T with the residual: partial[2 t], partial[2 t + 1] =
// sum |a - z|^2, sum |a|^2 over tile t of the device tile list.
qmcur_status tc_group_residual(int32_t prec, int bn, const void* A_all, int64_t rows_a,
                               const void* B_all, int64_t rows_b, int64_t kpad,
                               const TcGroupTile* tiles, int ntiles, const TcGroupProb* probs,
                               double* partial, int32_t* dev_status, cudaStream_t st);

}  // namespace qmcur
