// Grouped tensor-core products of the batched path: one launch of the
// tcgen05 GEMM over the tiles of many problems whose operand pieces are
// stacked along rows in two shared buffers (every problem's A = C pieces
// under one TMA map, its B = T^T pieces under another), with the relative
// residual against each problem's A fused into the epilogue.
#pragma once

#include "common.cuh"

namespace qmcur {

// One 128-row output tile of problem `prob` at (m0, n0) of its Z = C T.
struct TcGroupTile {
  int prob, m0, n0;
};

// What the grouped kernel needs of one problem: its input A (residual) or
// its output Z (store), shape, inner dimension K and its pieces' k-blocks,
// and the first rows of its operands in the stacked buffers.
struct TcGroupProb {
  const float* a[4];
  int64_t lda;
  int m, n, K, kblocks, arow, brow, a_vec;
  float* z[4];          // the store's output planes (row stride ldz)
  int64_t ldz;
  int z_vec;            // planes 16-byte aligned and ldz % 4 == 0
};

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
// The grouped T = U R (T = A_all B_all^T per problem, the split of product
// 0), each tile stored into its problem's z planes, masked by its m and n.
qmcur_status tc_group_store(int32_t prec, int bn, const void* A_all, int64_t rows_a,
                            const void* B_all, int64_t rows_b, int64_t kpad,
                            const TcGroupTile* tiles, int ntiles, const TcGroupProb* probs,
                            int32_t* dev_status, cudaStream_t st);
// The grouped Z = C T with the residual: partial[2 t], partial[2 t + 1] =
// sum |a - z|^2, sum |a|^2 over tile t of the device tile list.
qmcur_status tc_group_residual(int32_t prec, int bn, const void* A_all, int64_t rows_a,
                               const void* B_all, int64_t rows_b, int64_t kpad,
                               const TcGroupTile* tiles, int ntiles, const TcGroupProb* probs,
                               double* partial, int32_t* dev_status, cudaStream_t st);

}  // namespace qmcur
