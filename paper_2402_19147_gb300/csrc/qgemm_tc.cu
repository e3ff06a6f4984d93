// Quaternion GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Z = X Y with the Hamilton product (Sec. 2.2) in split planes:
//   Z_p = sum_t s(p,t) X_t Y_{y(p,t)},
//   Z0 = X0Y0 - X1Y1 - X2Y2 - X3Y3      Z1 = X0Y1 + X1Y0 + X2Y3 - X3Y2
//   Z2 = X0Y2 - X1Y3 + X2Y0 + X3Y1      Z3 = X0Y3 + X1Y2 - X2Y1 + X3Y0,
// i.e. the real 4x4 block representation, issued as 16 real MMAs per K step
// whose minus signs come from the instruction descriptor's negate-A bit.
//
// Precision: every FP32 operand is split into pieces (BF16 hi/lo or
// hi/mid/lo, or TF32 big/small); a "term" multiplies one piece of X by one of
// Y, and the terms (3 or 6) accumulate into the same FP32 TMEM accumulator.
// The two GEMMs may use different splits (QMCUR_PREC_BF16_MIXED: six terms
// for T = U R, three for Z = C T).
//
// Layout: pieces are stored K-major, [piece][plane][rows][Kpad] (Kpad a
// multiple of 64 bytes, zero padded), one 3-D tensor map per operand, so a
// single TMA copy brings the four planes of one piece for one 64-byte K
// slice into shared memory (64-byte swizzle).  K steps that lie entirely in
// the padding are not issued.
//
// Kernel: persistent, warp-specialised (10 warps).  Warp 0 lane 0 issues TMA
// loads into a ring of 3-5 stages; warp 1 owns the TMEM allocation and its
// lane 0 issues the MMAs (M = 128, N = BN per MMA: 112 for T^T = R^T U, 128
// or 112 for Z = C T, narrower for small outputs; the four output planes
// side by side in TMEM, with two
// accumulator buffers where 2 x 4 x BN columns fit in 512, so that the
// epilogue of one tile overlaps the MMAs of the next); warps 2-9 are the
// epilogue, two per 32-lane TMEM sub-partition (one output row per thread),
// taking alternate 16-column chunks.  Epilogue modes:
//   STORE_Z   write Z (FP32 planes);
//   RESIDUAL  never write Z: read the matching tile of A and accumulate
//             sum |a - z|^2, sum |a|^2 (optionally over a mask) into one FP64
//             pair per tile; the last CTA to finish folds the pairs in a
//             fixed order into {rel, num, den};
//   STORE_ZT  write the tile transposed (T^T's split-K partials, summed and
//             cut into the pieces of Z = C T's B operand by k_t_reduce).
// Every wait is bounded: on timeout the kernel raises an abort flag, the
// roles drain, TMEM is freed and QMCUR_ERR_TIMEOUT is reported.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc_group.cuh"

namespace qmcur {

namespace {

constexpr int BM = 128;
constexpr int ROWB = 64;                      // bytes of K per shared row (one swizzle row)
constexpr int A_PLANE = BM * ROWB;            // 8 KiB
constexpr int A_STAGE = 4 * A_PLANE;
constexpr int kEpiWarps = 8;                  // two per TMEM sub-partition
constexpr int kTcThreads = 64 + 32 * kEpiWarps;

// Shape of one instantiation: output tiles of BM x BNT (per plane).  The
// reversed product T^T = R^T U always takes BNT = kBn1 = 112 columns of U's c;
// Z = C T takes 128 or 112 (whichever fills whole waves over the SMs better),
// halved to 64 or 32 when the output has too few tiles (z_bn).
constexpr int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p *= 2;
  return p;
}

template <int BNT>
struct TcShape {
  static constexpr int BN = BNT;
  static constexpr int B_PLANE = BN * ROWB;            // 4 KiB at BN 64
  static constexpr int B_STAGE = 4 * B_PLANE;
  static constexpr int STAGE = A_STAGE + B_STAGE;      // 48 KiB at BN 64
  static constexpr int STAGES = BN >= 112 ? 3 : BN == 64 ? 4 : 5;
  static constexpr int ACC_COLS = 4 * BN;              // FP32 TMEM columns per accumulator
  // two accumulators where they fit the 512 columns, so that the epilogue of
  // one tile overlaps the MMAs of the next; one at BN 128
  static constexpr int NACC = 2 * ACC_COLS <= 512 ? 2 : 1;
  static constexpr int TMEM_COLS = pow2_at_least(NACC * ACC_COLS);   // the allocation unit
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;   // barriers, TMEM slot, reductions
};
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz

// MODE_STORE_ZT stores the tile transposed, z[t][col][row] with ldz between
// columns: the lanes of a warp hold consecutive rows, so each store of one
// column is one contiguous 128-byte line.
// MODE_COMPLETE is one step of masked completion (Algorithm 2): A is the
// iterate X^t, and each unobserved entry (mask 0) is overwritten in place by
// z, while the sums are sum over unobserved entries of |z - a|^2 and sum over
// all entries of |a|^2 (the stopping test's ||X^{t+1} - X^t||^2 and ||X^t||^2).
// MODE_GROUPED is MODE_RESIDUAL over the tiles of many problems (tc_group.cuh):
// each tile's coordinates, inner dimension and A come from the group tables,
// and its partials go to partial[2 tile], with no fold in the kernel.
// MODE_GROUPED_PIECES (with REV: the tiles of T^T = R^T U of many problems)
// cuts each output value into the pieces of the next product's split and
// stores them K-major at the problem's rows of that product's stacked B
// operand: row = the tile row (a column of T), k = the tile column.
enum { MODE_STORE_Z = 0, MODE_RESIDUAL = 1, MODE_STORE_ZT = 2, MODE_COMPLETE = 3, MODE_GROUPED = 4,
       MODE_GROUPED_PIECES = 5 };

struct TcParams {
  int M, N;
  int K;                  // true inner dimension (the rest of Kpad is zero)
  int kblocks;            // Kpad / (elements per 64 bytes)
  int nterms;
  int ta[6], tb[6];       // piece of X and of Y of each term
  int mode;
  int nsplit;             // K-range splits per tile; split s of a tile stores to z + s * zsplit
  // MODE_STORE_Z
  float* z[4];
  int64_t ldz, zsplit;
  int z_vec;              // planes (and split offsets) 16-byte aligned and ldz % 4 == 0
  // MODE_RESIDUAL
  const float* a[4];
  int64_t lda;
  int a_vec;              // planes 16-byte aligned and lda % 4 == 0
  const uint8_t* mask;
  double* partial;        // two doubles per tile
  double* out3;           // the last CTA folds the partials into out3
  unsigned* done;         // arrival count of that fold, zero at launch
  int32_t* status;
  // MODE_GROUPED
  const TcGroupTile* gtiles;
  const TcGroupProb* gprobs;
  int gcount;
  // MODE_GROUPED_PIECES: the stacked piece buffer, its row width (elements),
  // plane stride (elements) and pieces per value
  void* pieces;
  int64_t pk_kpad, pk_plane;
  int pk_npieces;
};

// ------------------------------------------------------------- PTX helpers -
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of parity `parity`; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 63u) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kWaitCycles) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(saddr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups
// 512 bytes apart (SBO), descriptor version 1 (bits 46-47), swizzle mode 4
// (bits 61-63).  The leading-byte offset is unused for this layout.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8 * ROWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor of kind::f16 (BF16 operands) or kind::tf32: FP32
// accumulator (bits 4-5 = 1), A/B formats (bits 7-9, 10-12), negate A (bit 13),
// both operands K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(bool bf16, bool neg_a, int n) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) |
         ((neg_a ? 1u : 0u) << 13) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                     uint32_t accumulate) {
  if constexpr (BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   saddr(bar))
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// split_value (the pieces of one value) is in tc_group.cuh, shared with the
// batched gather, which writes C's pieces as it gathers C.

// ------------------------------------------------------------------ kernel -
// REV: Z = sum_k Y[n][k] X[m][k] (the B operand on the left of each
// quaternion product) instead of X[m][k] Y[n][k]; the two differ in the sign
// of the cross terms.  Work item w is split w % nsplit of tile w / nsplit.
template <bool BF16, int BNT, bool REV, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
k_qgemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
           TcParams p) {
  using Sh = TcShape<BNT>;
  constexpr int BN = Sh::BN, B_PLANE = Sh::B_PLANE, STAGE = Sh::STAGE, STAGES = Sh::STAGES;
  constexpr int ACC_COLS = Sh::ACC_COLS, TMEM_COLS = Sh::TMEM_COLS, NACC = Sh::NACC;
  static_assert(BN % 16 == 0 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(tmem_slot + 2);   // [2][4]

  constexpr int kY[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
  constexpr int kNegFwd[4][4] = {{0, 1, 1, 1}, {0, 0, 0, 1}, {0, 1, 0, 0}, {0, 0, 1, 0}};
  constexpr int kNegRev[4][4] = {{0, 1, 1, 1}, {0, 0, 1, 0}, {0, 0, 0, 1}, {0, 1, 0, 0}};
  constexpr uint32_t kIdPos = make_idesc(BF16, false, BN), kIdNeg = make_idesc(BF16, true, BN);
  constexpr int kElemsPerRow = ROWB / (BF16 ? 2 : 4);
  constexpr int kStepElems = 32 / (BF16 ? 2 : 4);          // K of one MMA (32 bytes)
  constexpr bool grouped = MODE == MODE_GROUPED || MODE == MODE_GROUPED_PIECES;
  constexpr bool sums_mode = MODE == MODE_RESIDUAL || MODE == MODE_COMPLETE || MODE == MODE_GROUPED;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mtiles = (p.M + BM - 1) / BM, ntiles = (p.N + BN - 1) / BN;
  const int tiles = mtiles * ntiles;
  const int kiters = p.nterms * p.kblocks;
  const int items = grouped ? p.gcount : tiles * p.nsplit;
  const int kper = (kiters + p.nsplit - 1) / p.nsplit;   // every split non-empty (host)

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int a = 0; a < 2; ++a) { mbar_init(&tfull[a], 1); mbar_init(&tempty[a], kEpiWarps); }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------- TMA producer --
    uint32_t it = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int arow, brow, kbl, k0, k1;
      if constexpr (grouped) {
        const TcGroupTile tl = p.gtiles[item];
        const TcGroupProb& gp = p.gprobs[tl.prob];
        arow = gp.arow + tl.m0;
        brow = gp.brow + tl.n0;
        kbl = gp.kblocks;
        k0 = 0;
        k1 = p.nterms * kbl;
      } else {
        const int tile = item / p.nsplit, split = item % p.nsplit;
        const int mt = tile % mtiles, nt = tile / mtiles;
        arow = mt * BM;
        brow = nt * BN;
        kbl = p.kblocks;
        k0 = split * kper;
        k1 = min(k0 + kper, kiters);
      }
      for (int ki = k0; ki < k1; ++ki, ++it) {
          const int term = ki / kbl, kb = ki % kbl;
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) { ok = false; break; }
          mbar_expect_tx(&full[s], STAGE);
          const uint32_t sa = saddr(smem + s * STAGE);
          tma_load_3d(sa, &mapA, &full[s], kb * kElemsPerRow, arow, p.ta[term] * 4);
          tma_load_3d(sa + A_STAGE, &mapB, &full[s], kb * kElemsPerRow, brow, p.tb[term] * 4);
        }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------------ MMA issuer --
    uint32_t it = 0;
    int local = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x, ++local) {
      int kbl, kval, k0, k1;
      if constexpr (grouped) {
        const TcGroupProb& gp = p.gprobs[p.gtiles[item].prob];
        kbl = gp.kblocks;
        kval = gp.K;
        k0 = 0;
        k1 = p.nterms * kbl;
      } else {
        const int split = item % p.nsplit;
        kbl = p.kblocks;
        kval = p.K;
        k0 = split * kper;
        k1 = min(k0 + kper, kiters);
      }
      const int a = local % NACC;
      const uint32_t aph = (local / NACC) & 1;
      if (!mbar_wait(&tempty[a], aph ^ 1u, abort_flag)) break;
      tc_fence_after();
      const uint32_t dbase = tmem_base + (uint32_t)(a * ACC_COLS);
      for (int ki = k0; ki < k1; ++ki, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = saddr(smem + s * STAGE), sb = sa + A_STAGE;
        // Descriptors of the stage's first A and B rows; every other operand
        // of the stage lies a constant number of 16-byte units further on, and
        // stage offsets stay below 2^18 bytes, so adding (offset >> 4) to the
        // 14-bit start-address field never carries out of it.
        const uint64_t ad0 = sdesc(sa), bd0 = sdesc(sb);
        const int kb = ki % kbl;
        const int kleft = kval - kb * kElemsPerRow;         // valid elements in this slice
        const int ksteps = kleft >= kElemsPerRow ? ROWB / 32 : (kleft + kStepElems - 1) / kStepElems;
#pragma unroll
        for (int ks = 0; ks < ROWB / 32; ++ks) {
          if (ks >= ksteps) break;
          // consecutive MMAs write different accumulators (output planes)
          // and share their A operand
#pragma unroll
          for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
              const uint64_t ad = ad0 + (uint64_t)((t * A_PLANE + ks * 32) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((kY[pl][t] * B_PLANE + ks * 32) >> 4);
              const uint32_t acc = (ki > k0 || ks > 0 || t > 0) ? 1u : 0u;
              const int neg = REV ? kNegRev[pl][t] : kNegFwd[pl][t];
              umma<BF16>(dbase + pl * BN, ad, bd, neg ? kIdNeg : kIdPos, acc);
            }
          }
        }
        umma_commit(&empty[s]);   // the stage is free once these MMAs retire
      }
      if (ok) umma_commit(&tfull[a]);
    }
  } else if (warp >= 2) {
    // -------------------------------------------------------- epilogue --
    const int sp = warp % 4;                 // TMEM sub-partition (lanes 32 sp ...)
    const int epi = warp - 2;
    const int half = epi / 4;                // the two warps of a sub-partition take alternate chunks
    int local = 0;
    // the current tile's problem (the group tables, or p itself)
    // (grouped only; otherwise the accessors below read p directly)
    int Mv = 0, Nv = 0, avec = 0;
    int64_t zrowg = 0;   // MODE_GROUPED_PIECES: the problem's first row in the piece buffer
    int64_t ldav = 0;
    const float* ap[4] = {nullptr, nullptr, nullptr, nullptr};
    auto EM = [&]() -> int { if constexpr (grouped) return Mv; else return p.M; };
    auto EN = [&]() -> int { if constexpr (grouped) return Nv; else return p.N; };
    auto EAV = [&]() -> int { if constexpr (grouped) return avec; else return p.a_vec; };
    auto ELD = [&]() -> int64_t { if constexpr (grouped) return ldav; else return p.lda; };
    auto EAP = [&](int pl) -> const float* { if constexpr (grouped) return ap[pl]; else return p.a[pl]; };
    auto EMASK = [&]() -> const uint8_t* { if constexpr (grouped) return nullptr; else return p.mask; };
    // A values of all four planes of one 16-column chunk (row `row`)
    auto load_a = [&](float4 (&av)[4][4], int row, int c0) {
      const bool in_row = row < EM();
      const bool full16 = EAV() && c0 + 16 <= EN();
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) {
        const float* ar = EAP(pl) + (int64_t)row * ELD() + c0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (in_row && full16) {
            av[pl][q] = __ldcs(reinterpret_cast<const float4*>(ar) + q);
          } else {
            float e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) e[u] = (in_row && c0 + 4 * q + u < EN()) ? ar[4 * q + u] : 0.f;
            av[pl][q] = make_float4(e[0], e[1], e[2], e[3]);
          }
        }
      }
    };
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++local) {
      const int tile = grouped ? item : item / p.nsplit, split = grouped ? 0 : item % p.nsplit;
      const int a = local % NACC;
      const uint32_t aph = (local / NACC) & 1;
      int row, n0;
      if constexpr (grouped) {
        const TcGroupTile tl = p.gtiles[item];
        const TcGroupProb& gp = p.gprobs[tl.prob];
        Mv = gp.m;
        Nv = gp.n;
        avec = gp.a_vec;
        ldav = gp.lda;
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) ap[pl] = gp.a[pl];
        if constexpr (MODE == MODE_GROUPED_PIECES) zrowg = gp.zrow;
        row = tl.m0 + sp * 32 + lane;
        n0 = tl.n0;
      } else {
        const int mt = tile % mtiles, nt = tile / mtiles;
        row = mt * BM + sp * 32 + lane;
        n0 = nt * BN;
      }
      // the residual's first A chunk is fetched while the MMAs still run,
      // and this thread's later chunks of the tile are prefetched into L2, so
      // that the epilogue, which holds the only accumulator, reads A from L2
      float4 anext[4][4];
      if constexpr (sums_mode) {
        load_a(anext, row, n0 + 16 * half);
        if (row < EM()) {
#pragma unroll 1
          for (int ch = half + 2; ch < BN / 16 && n0 + ch * 16 < EN(); ch += 2)
#pragma unroll
            for (int pl = 0; pl < 4; ++pl)
              asm volatile("prefetch.global.L2 [%0];" ::"l"(EAP(pl) + (int64_t)row * ELD() + n0 + ch * 16));
        }
      }
      if (!mbar_wait(&tfull[a], aph, abort_flag)) break;
      tc_fence_after();
      const uint32_t tb = tmem_base + (uint32_t)(a * ACC_COLS) + ((uint32_t)(sp * 32) << 16);
      double dsum = 0.0, asum = 0.0;
      if constexpr (sums_mode) {
        constexpr bool cmpl = MODE == MODE_COMPLETE;
#pragma unroll 1
        for (int ch = half; ch < BN / 16; ch += 2) {
          const int c0 = n0 + ch * 16;
          float4 av[4][4];
#pragma unroll
          for (int pl = 0; pl < 4; ++pl)
#pragma unroll
            for (int q = 0; q < 4; ++q) av[pl][q] = anext[pl][q];
          if (ch + 2 < BN / 16) load_a(anext, row, c0 + 32);   // this warp's next chunk in flight
          const bool in_row = row < EM();
          const bool full16 = EAV() && c0 + 16 <= EN();
          float sd = 0.f, sa2 = 0.f;
          if constexpr (!cmpl) {
            unsigned keep = 0xffffu;   // columns of the chunk that count
            if (!full16 || EMASK() != nullptr) {
              keep = 0;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const bool ok = in_row && c0 + j < EN() &&
                                (EMASK() == nullptr || EMASK()[(int64_t)row * EN() + c0 + j] != 0);
                keep |= (ok ? 1u : 0u) << j;
              }
            }
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
              float z[16];
              tmem_ld16(tb + pl * BN + ch * 16, z);
              const float* avf = reinterpret_cast<const float*>(av[pl]);
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const float w = ((keep >> j) & 1u) ? 1.f : 0.f;
                const float d = (avf[j] - z[j]) * w;
                sd = fmaf(d, d, sd);
                sa2 = fmaf(avf[j] * w, avf[j], sa2);
              }
            }
          } else {
            // inb: columns inside Z; obs: observed (mask nonzero, or no
            // mask).  The change sums over inb & ~obs, |a|^2 over inb.
            unsigned inb = 0xffffu, obs = 0xffffu;
            if (!full16 || !in_row) {
              inb = 0;
#pragma unroll
              for (int j = 0; j < 16; ++j) inb |= ((in_row && c0 + j < p.N) ? 1u : 0u) << j;
            }
            if (p.mask != nullptr) {
              obs = 0;
#pragma unroll
              for (int j = 0; j < 16; ++j)
                obs |= (((inb >> j) & 1u) && p.mask[(int64_t)row * p.N + c0 + j] != 0 ? 1u : 0u) << j;
            }
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) {
              float z[16];
              tmem_ld16(tb + pl * BN + ch * 16, z);
              const float* avf = reinterpret_cast<const float*>(av[pl]);
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const bool moved = ((inb & ~obs) >> j) & 1u;
                const float d = moved ? z[j] - avf[j] : 0.f;
                sd = fmaf(d, d, sd);
                const float a2 = ((inb >> j) & 1u) ? avf[j] : 0.f;
                sa2 = fmaf(a2, a2, sa2);
                z[j] = ((obs >> j) & 1u) ? avf[j] : z[j];   // X^{t+1}
              }
              if (in_row) {
                float* xr = p.z[pl] + (int64_t)row * p.ldz + c0;
                if (full16 && p.z_vec) {
#pragma unroll
                  for (int q = 0; q < 4; ++q)
                    reinterpret_cast<float4*>(xr)[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
                } else {
#pragma unroll
                  for (int j = 0; j < 16; ++j)
                    if ((inb >> j) & 1u) xr[j] = z[j];
                }
              }
            }
          }
          if (in_row) { dsum += (double)sd; asum += (double)sa2; }
        }
      } else {
#pragma unroll 1
        for (int pl = 0; pl < 4; ++pl) {
#pragma unroll 1
          for (int ch = half; ch < BN / 16; ch += 2) {
            float z[16];
            tmem_ld16(tb + pl * BN + ch * 16, z);
            const int c0 = n0 + ch * 16;
            if constexpr (MODE == MODE_GROUPED_PIECES) {
              if (row < Mv) {
                const int64_t rowoff = (zrowg + row) * p.pk_kpad + c0;
                const int nv = Nv - c0 < 16 ? Nv - c0 : 16;   // valid columns (k) of the chunk
                float pc[3][16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  float q3[3];
                  split_value<BF16, float>(z[j], p.pk_npieces, q3);
                  pc[0][j] = q3[0];
                  pc[1][j] = q3[1];
                  pc[2][j] = q3[2];
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                  if (q >= p.pk_npieces) break;
                  const int64_t base = (int64_t)(q * 4 + pl) * p.pk_plane + rowoff;
                  if constexpr (BF16) {
                    __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(p.pieces) + base;
                    if (nv == 16) {
                      uint32_t w[8];
#pragma unroll
                      for (int h = 0; h < 8; ++h) {
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(pc[q][2 * h], pc[q][2 * h + 1]);
                        w[h] = *reinterpret_cast<const uint32_t*>(&b2);
                      }
                      reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                      reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
                    } else {
#pragma unroll
                      for (int j = 0; j < 16; ++j)
                        if (j < nv) dst[j] = __float2bfloat16_rn(pc[q][j]);
                    }
                  } else {
                    float* dst = reinterpret_cast<float*>(p.pieces) + base;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                      if (j < nv) dst[j] = pc[q][j];
                  }
                }
              }
            } else if constexpr (MODE == MODE_STORE_ZT) {
              if (row < p.M) {
                float* zc = p.z[pl] + split * p.zsplit + (int64_t)c0 * p.ldz + row;
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  if (c0 + j < p.N) zc[(int64_t)j * p.ldz] = z[j];
              }
            } else if (row < p.M) {   // MODE_STORE_Z
              float* zr = p.z[pl] + split * p.zsplit + (int64_t)row * p.ldz + c0;
              if (c0 + 16 <= p.N && p.z_vec) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                  reinterpret_cast<float4*>(zr)[q] =
                      make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
              } else {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  if (c0 + j < p.N) zr[j] = z[j];
              }
            }
          }
        }
      }
      tc_fence_before();
      if (lane == 0) mbar_arrive(&tempty[a]);
      if constexpr (sums_mode) {
        // fixed-order reduction: warp tree, then the eight warps in order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
          asum += __shfl_xor_sync(0xffffffffu, asum, o);
        }
        double* rb = red + (local & 1) * 2 * kEpiWarps;
        if (lane == 0) { rb[epi] = dsum; rb[kEpiWarps + epi] = asum; }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
        if (epi == 0 && lane == 0) {
          static_assert(kEpiWarps == 8, "fixed-order sum of eight warps");
          p.partial[2 * tile] = ((rb[0] + rb[1]) + (rb[2] + rb[3])) + ((rb[4] + rb[5]) + (rb[6] + rb[7]));
          p.partial[2 * tile + 1] = ((rb[8] + rb[9]) + (rb[10] + rb[11])) + ((rb[12] + rb[13]) + (rb[14] + rb[15]));
          __threadfence();   // visible to the CTA that folds the partials
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag) set_status(p.status, QMCUR_ERR_TIMEOUT);
  if (sums_mode && p.done != nullptr) {
    // The last CTA to finish folds the per-item partials into out3 in a fixed
    // order: strided sums, a shuffle tree per warp, then the warps in order.
    __shared__ int s_last;
    __shared__ double s_red[2][kTcThreads / 32];
    if (threadIdx.x == 0) s_last = atomicAdd(p.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      const int64_t count = tiles;
      double num = 0.0, den = 0.0;
      for (int64_t k = threadIdx.x; k < count; k += kTcThreads) {
        num += __ldcg(p.partial + 2 * k);
        den += __ldcg(p.partial + 2 * k + 1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
      }
      if (lane == 0) { s_red[0][warp] = num; s_red[1][warp] = den; }
      __syncthreads();
      if (threadIdx.x == 0) {
        num = 0.0;
        den = 0.0;
        for (int w = 0; w < kTcThreads / 32; ++w) { num += s_red[0][w]; den += s_red[1][w]; }
        p.out3[1] = num;
        p.out3[2] = den;
        p.out3[0] = den > 0.0 ? sqrt(num / den) : __longlong_as_double(0x7ff8000000000000ll);
      }
    }
  }
}


// Operand pieces of up to three operands in one launch: for job j,
// dst[(q*4 + t)][i][k] for i < rows_out, k < kpad is piece q of plane t of
// S(i, k) (or S(k, i) when trans), zero for k >= K.  A CTA owns a tile of
// 32 rows x 64 k: every load of the tile is issued before the first store
// (the tile passes through shared memory, which also transposes it), then
// each lane splits a pair of k and writes the pieces in pairs.
constexpr int kSplitRows = 32, kSplitK = 64, kSplitPitch = kSplitK + 2;
constexpr int kMaxSplitJobs = 3;
struct SplitJob {
  QView S;
  void* dst;
  int64_t rows_out, K, kpad;
  int npieces, trans, f64, vec2;   // vec2: non-trans rows read as float2
  int tiles_k, first_tile;         // tiles along k; index of the job's first tile
  float scale;                     // every value is multiplied by scale before the split,
  int conj;                        // and planes 1..3 by -1 with conj (conjugate, Sec. 2.2)
};
struct SplitJobs {
  SplitJob j[kMaxSplitJobs];
  int count;
};

template <bool BF16>
__global__ void __launch_bounds__(256) k_split_ops(const __grid_constant__ SplitJobs jobs) {
  __shared__ __align__(16) float tile[4][kSplitRows][kSplitPitch];
  int jb = 0;
#pragma unroll
  for (int q = 1; q < kMaxSplitJobs; ++q)
    if (q < jobs.count && (int)blockIdx.x >= jobs.j[q].first_tile) jb = q;
  const SplitJob J = jobs.j[jb];   // by value: the fields are read once
  const int tl = (int)blockIdx.x - J.first_tile;
  const int64_t i0 = (int64_t)(tl / J.tiles_k) * kSplitRows, k0 = (int64_t)(tl % J.tiles_k) * kSplitK;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  if (!J.trans) {
    // S(i0 + warp + 8u, k0 + 2 lane + {0, 1}): 16 loads per thread
    const int64_t k = k0 + 2 * lane;
    float2 v[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + warp + 8 * u;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float2 x = make_float2(0.f, 0.f);
        if (i < J.rows_out && k < J.K) {
          if (J.f64) {
            const double* src = reinterpret_cast<const double*>(J.S.p[t]) + i * J.S.ld + k;
            x.x = (float)src[0];
            if (k + 1 < J.K) x.y = (float)src[1];
          } else {
            const float* src = reinterpret_cast<const float*>(J.S.p[t]) + i * J.S.ld + k;
            if (J.vec2 && k + 1 < J.K) {
              x = *reinterpret_cast<const float2*>(src);
            } else {
              x.x = src[0];
              if (k + 1 < J.K) x.y = src[1];
            }
          }
        }
        v[u][t] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t)
        *reinterpret_cast<float2*>(&tile[t][warp + 8 * u][2 * lane]) = v[u][t];
  } else {
    // S(k0 + warp + 8u, i0 + lane), coalesced along i: 32 loads per thread
    const int64_t i = i0 + lane;
    float v[8][4];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t k = k0 + warp + 8 * u;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float x = 0.f;
        if (i < J.rows_out && k < J.K)
          x = J.f64 ? (float)reinterpret_cast<const double*>(J.S.p[t])[k * J.S.ld + i]
                    : reinterpret_cast<const float*>(J.S.p[t])[k * J.S.ld + i];
        v[u][t] = x;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) tile[t][lane][warp + 8 * u] = v[u][t];
  }
  __syncthreads();
  const int64_t k = k0 + 2 * lane;   // kpad is even: k < kpad implies k + 1 < kpad
  if (k >= J.kpad) return;
  const int64_t plane_stride = J.rows_out * J.kpad;   // between (piece, plane) blocks
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int il = warp + 8 * u;
    const int64_t i = i0 + il;
    if (i >= J.rows_out) break;
    const int64_t rowoff = i * J.kpad + k;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float2 x = *reinterpret_cast<const float2*>(&tile[t][il][2 * lane]);
      const float sg = (J.conj && t > 0) ? -J.scale : J.scale;
      x.x *= sg;
      x.y *= sg;
      float p0[3], p1[3];
      split_value<BF16, float>(x.x, J.npieces, p0);
      split_value<BF16, float>(x.y, J.npieces, p1);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= J.npieces) break;
        const int64_t idx = (int64_t)(q * 4 + t) * plane_stride + rowoff;
        if constexpr (BF16)
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(J.dst) + idx) =
              __floats2bfloat162_rn(p0[q], p1[q]);
        else
          *reinterpret_cast<float2*>(reinterpret_cast<float*>(J.dst) + idx) = make_float2(p0[q], p1[q]);
      }
    }
  }
}

// Pieces of T^T from the split partials of T^T = R^T (x) U, stored
// transposed: P[split][t][i][j] (column i of T^T, row j; ld = ldp, a multiple of 4).
// For j < rows and i < kpad: v = P[0] + P[1] + ... in split order (zero for
// i >= c), then dst[(q*4 + t)][j][i] = piece q of plane t.  A CTA takes 32
// columns x 64 rows through shared memory: every load of all planes and
// splits is in flight at once, read along j in pairs, written along i in
// pairs.
constexpr int kRedI = 32, kRedJ = 64;
constexpr int kMaxSplits = 4;   // K splits of T^T at most
template <bool BF16>
__global__ void __launch_bounds__(256) k_t_reduce(const float* __restrict__ P, int nsplit,
                                                  int64_t split_stride, int64_t plane_stride,
                                                  int64_t ldp, int64_t rows, int64_t c, int64_t kpad,
                                                  int npieces, void* dst, unsigned* done) {
  __shared__ float tile[4][kRedI][kRedJ + 1];
  const int tid = threadIdx.x;
  // arrival count of the residual fold of the GEMM that follows on the stream
  if (done != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) *done = 0u;
  const int64_t i0 = (int64_t)blockIdx.x * kRedI, j0 = (int64_t)blockIdx.y * kRedJ;
  {
    const int jl = 2 * (tid % 32), r0 = tid / 32;   // rows j0 + jl, j0 + jl + 1; columns r0 + 8 k
    const int64_t j = j0 + jl;
#pragma unroll
    for (int k = 0; k < kRedI / 8; ++k) {
      const int r = r0 + 8 * k;
      const int64_t i = i0 + r;
      float2 v[4] = {};
      if (i < c && j < rows) {   // j + 1 < ldp: the pair stays in the padded column
        const float* src = P + i * ldp + j;
        float2 x[kMaxSplits][4];   // every load of the column pair issued before the sums
#pragma unroll
        for (int sp = 0; sp < kMaxSplits; ++sp)
#pragma unroll
          for (int t = 0; t < 4; ++t)
            x[sp][t] = sp < nsplit
                           ? __ldcs(reinterpret_cast<const float2*>(src + sp * split_stride + t * plane_stride))
                           : make_float2(0.f, 0.f);
#pragma unroll
        for (int sp = 0; sp < kMaxSplits; ++sp)
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            v[t].x += x[sp][t].x;
            v[t].y += x[sp][t].y;
          }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        tile[t][r][jl] = v[t].x;
        tile[t][r][jl + 1] = v[t].y;
      }
    }
  }
  __syncthreads();
  const int il = 2 * (tid % 16), jr0 = tid / 16;   // columns i0 + il, + 1; rows jr0 + 16 k
  const int64_t i = i0 + il;
  const int64_t out_stride = rows * kpad;            // between (piece, plane) blocks
#pragma unroll 1
  for (int k = 0; k < kRedJ / 16; ++k) {
    const int jr = jr0 + 16 * k;
    const int64_t j = j0 + jr;
    if (j >= rows || i >= kpad) continue;   // kpad is even: i + 1 < kpad as well
    const int64_t rowoff = j * kpad + i;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float p0[3], p1[3];
      split_value<BF16, float>(tile[t][il][jr], npieces, p0);
      split_value<BF16, float>(tile[t][il + 1][jr], npieces, p1);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= npieces) break;
        const int64_t idx = (int64_t)(q * 4 + t) * out_stride + rowoff;
        if constexpr (BF16)
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(dst) + idx) =
              __floats2bfloat162_rn(p0[q], p1[q]);
        else
          *reinterpret_cast<float2*>(reinterpret_cast<float*>(dst) + idx) = make_float2(p0[q], p1[q]);
      }
    }
  }
}

// ------------------------------------------------------------ host side ---
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 3-D map over [npieces*4][rows][kpad] with a box of one 64-byte K slice x
// box_rows rows x 4 planes, 64-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* map, void* base, bool bf16, int64_t rows, int64_t kpad, int npieces,
              int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (fn == nullptr) return false;
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)(npieces * 4)};
  cuuint64_t strides[2] = {(cuuint64_t)(kpad * es), (cuuint64_t)(kpad * es * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(ROWB / es), (cuuint32_t)box_rows, 4};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base,
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcPlan {
  bool bf16;
  int npieces, nterms;
  int ta[6], tb[6];
  int64_t epr;   // elements per 64-byte row
};

TcPlan plan_for(int32_t prec) {
  if (prec == QMCUR_PREC_BF16_MIXED) prec = QMCUR_PREC_BF16X6;
  TcPlan pl{};
  pl.bf16 = prec != QMCUR_PREC_TF32X3;
  pl.npieces = prec == QMCUR_PREC_BF16X6 ? 3 : 2;
  pl.epr = pl.bf16 ? 32 : 16;
  // smallest terms first
  if (prec == QMCUR_PREC_BF16X6) {
    const int a[6] = {2, 1, 0, 1, 0, 0}, b[6] = {0, 1, 2, 0, 1, 0};
    pl.nterms = 6;
    for (int i = 0; i < 6; ++i) { pl.ta[i] = a[i]; pl.tb[i] = b[i]; }
  } else {
    const int a[3] = {1, 0, 0}, b[3] = {0, 1, 0};
    pl.nterms = 3;
    for (int i = 0; i < 3; ++i) { pl.ta[i] = a[i]; pl.tb[i] = b[i]; }
  }
  return pl;
}

// Splits of the two GEMMs: T = U R (first) and Z = C T (second).
void plans_for(int32_t prec, TcPlan& first, TcPlan& second) {
  first = plan_for(prec);
  second = plan_for(prec == QMCUR_PREC_BF16_MIXED ? QMCUR_PREC_BF16X3 : prec);
}

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct TcWs {
  void *A1, *B1, *A2, *B2;
  float* P;   // split partials of T^T: [split][plane][n][kpad of Z = C T]
  double* partial;   // residual partials of Z = C T, two per tile
  unsigned* done;    // arrival count of the residual fold
  float* Pz;         // K-split partials of a stored Z with few tiles: [split][plane][m][ldp]
};

// Tile widths: T^T = R^T (x) U (N over c) and Z = C T (N over n).  Both use
// MMAs of N >= 112: an MMA costs about the same issue time up to N = 128, so
// narrower ones waste the tensor pipe.
constexpr int kBn1 = 112, kBn2 = 128;
constexpr int kSplitItems = 128;   // work items T^T aims for (tiles x K splits)

// K splits of T^T, from the shape alone (the workspace depends on it); every
// split non-empty.
int t_splits(int64_t n, int64_t c, const TcPlan& p1, int64_t kp1) {
  const int64_t tiles = ((n + BM - 1) / BM) * ((c + kBn1 - 1) / kBn1);
  const int kiters = p1.nterms * (int)(kp1 / p1.epr);
  int64_t ns = kSplitItems / tiles;
  if (ns > kMaxSplits) ns = kMaxSplits;
  if (ns > kiters) ns = kiters;
  if (ns < 1) ns = 1;
  const int per = (int)((kiters + ns - 1) / ns);
  return (kiters + per - 1) / per;
}

// Tile width of Z = C T: 128, or 64 or 32 when 128-wide tiles would leave
// more than half the SMs idle (a small output: its epilogue may be
// nonlinear, so K cannot always be split; narrower tiles also give two
// accumulators in TMEM, so the epilogue overlaps the next tile).  Otherwise
// 112 when that takes fewer waves x width over the 152 SMs: a tile's time
// grows with its width (the MMAs are bound by shared-memory reads, which
// scale with N), and 2048 columns in 19 tiles of 112 fill two whole waves
// where 16 tiles of 128 leave the second wave a third empty.
constexpr int kZTileFloor = 76;
constexpr int kWaveSms = 152;
int z_bn(int64_t m, int64_t n) {
  int bn = kBn2;
  while (bn > 32 && ((m + BM - 1) / BM) * ((n + bn - 1) / bn) < kZTileFloor) bn /= 2;
  if (bn == kBn2) {
    const int64_t mt = (m + BM - 1) / BM;
    const int64_t w128 = (mt * ((n + 127) / 128) + kWaveSms - 1) / kWaveSms;
    const int64_t w112 = (mt * ((n + 111) / 112) + kWaveSms - 1) / kWaveSms;
    if (w112 * 112 < w128 * 128) bn = 112;
  }
  return bn;
}

// K splits of a stored Z = C T whose tiles are too few to occupy the GPU
// (a small output with a long K, e.g. the paper's core C^+ (X R^+)); 1 when
// the tiles suffice.  From the shape alone; every split at least 4 stages.
constexpr int kZSplitItems = 152, kMaxZSplits = 32;
int z_splits(int64_t m, int64_t n, const TcPlan& p2, int64_t kp2) {
  const int bn = z_bn(m, n);
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + bn - 1) / bn);
  const int kiters = p2.nterms * (int)(kp2 / p2.epr);
  int64_t ns = kZSplitItems / tiles;
  if (ns > kMaxZSplits) ns = kMaxZSplits;
  if (ns > kiters / 4) ns = kiters / 4;
  if (ns < 2) return 1;
  const int per = (int)((kiters + ns - 1) / ns);
  return (kiters + per - 1) / per;
}

// Stored Z from its K-split partials: Z[t](i, j) = sum over s, in split
// order, of P[s][t][i][j] (P row stride ldp).
__global__ void __launch_bounds__(256) k_z_reduce(const float* __restrict__ P, int nsplit,
                                                  int64_t split_stride, int64_t plane_stride,
                                                  int64_t ldp, int64_t m, int64_t n, QView Z) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= n) return;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float* src = P + t * plane_stride + i * ldp + j;
    float v = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) v += __ldcs(src + sp * split_stride);
    reinterpret_cast<float*>(Z.p[t])[i * Z.ld + j] = v;
  }
}

TcWs carve_tc(Carve& cv, const TcPlan& p1, const TcPlan& p2, int64_t m, int64_t n, int64_t c,
              int64_t r) {
  const int64_t es = p1.bf16 ? 2 : 4;   // both plans have the same element type
  const int64_t kp1 = rup(r, p1.epr), kp2 = rup(c, p2.epr);
  TcWs w;
  w.A1 = cv.take<char>((size_t)(p1.npieces * 4 * rup(c, BM) * kp1 * es));
  w.B1 = cv.take<char>((size_t)(p1.npieces * 4 * n * kp1 * es));
  w.A2 = cv.take<char>((size_t)(p2.npieces * 4 * m * kp2 * es));
  w.B2 = cv.take<char>((size_t)(p2.npieces * 4 * n * kp2 * es));
  w.P = cv.take<float>((size_t)(t_splits(n, c, p1, kp1) * 4 * kp2 * rup(n, 4)));
  const int bn2 = z_bn(m, n);
  const int64_t tiles = ((m + BM - 1) / BM) * ((n + bn2 - 1) / bn2);
  w.partial = cv.take<double>((size_t)(2 * tiles));
  w.done = cv.take<unsigned>(1);
  const int nsz = z_splits(m, n, p2, kp2);
  w.Pz = nsz > 1 ? cv.take<float>((size_t)(nsz * 4 * m * rup(n, 4))) : nullptr;
  return w;
}

// Adds the pieces of operand S (rows_out x K as stored, or K x rows_out when
// trans) to a split launch.
bool add_split_view(SplitJobs& js, int& tiles, const QView& S, bool trans, void* dst,
                    int64_t rows_out, int64_t K, int64_t kpad, int npieces, float scale = 1.f,
                    bool conj = false) {
  if (js.count >= kMaxSplitJobs || kpad % 2 != 0) return false;
  SplitJob& j = js.j[js.count++];
  j.S = S;
  j.dst = dst;
  j.rows_out = rows_out;
  j.K = K;
  j.kpad = kpad;
  j.npieces = npieces;
  j.trans = trans ? 1 : 0;
  j.f64 = S.dtype == QMCUR_F64 ? 1 : 0;
  j.scale = scale;
  j.conj = conj ? 1 : 0;
  j.vec2 = S.ld % 2 == 0;
  for (int t = 0; t < 4; ++t) j.vec2 = j.vec2 && reinterpret_cast<uintptr_t>(S.p[t]) % 8 == 0;
  j.tiles_k = (int)((kpad + kSplitK - 1) / kSplitK);
  j.first_tile = tiles;
  const int64_t t = (int64_t)j.tiles_k * ((rows_out + kSplitRows - 1) / kSplitRows);
  if (tiles + t > INT32_MAX) return false;
  tiles += (int)t;
  return true;
}

bool add_split(SplitJobs& js, int& tiles, const qmcur_qmat* S, bool trans, void* dst,
               int64_t rows_out, int64_t K, int64_t kpad, int npieces) {
  return add_split_view(js, tiles, view(S), trans, dst, rows_out, K, kpad, npieces);
}

template <bool BF16>
qmcur_status launch_splits(const SplitJobs& js, int tiles, cudaStream_t st) {
  k_split_ops<BF16><<<(unsigned)tiles, 256, 0, st>>>(js);
  return cuda_ok(cudaGetLastError());
}

template <bool BF16, int BNT, bool REV, int MODE>
qmcur_status launch_gemm_mode(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& p,
                              cudaStream_t st) {
  static bool attr_done[64] = {};
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QMCUR_ERR_CUDA;
  if (!attr_done[dev]) {
    if (cudaFuncSetAttribute(k_qgemm_tc<BF16, BNT, REV, MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             TcShape<BNT>::SMEM) != cudaSuccess)
      return QMCUR_ERR_CUDA;
    attr_done[dev] = true;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  const int items = (MODE == MODE_GROUPED || MODE == MODE_GROUPED_PIECES) ? p.gcount
                                         : ((p.M + BM - 1) / BM) * ((p.N + BNT - 1) / BNT) * p.nsplit;
  const int cap = cta_cap(sms);
  const int grid = items < cap ? items : cap;
  k_qgemm_tc<BF16, BNT, REV, MODE><<<grid, kTcThreads, TcShape<BNT>::SMEM, st>>>(ma, mb, p);
  return cuda_ok(cudaGetLastError());
}

// One instantiation per epilogue mode, so that each carries only its own
// epilogue's registers.  Tᵀ (REV) only stores transposed; Z = C T stores,
// folds the residual or updates the completion iterate.
template <bool BF16, int BNT, bool REV>
qmcur_status launch_gemm(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& p,
                         cudaStream_t st) {
  if constexpr (REV) {
    if (p.mode != MODE_STORE_ZT) return QMCUR_ERR_INVALID_ARG;
    return launch_gemm_mode<BF16, BNT, REV, MODE_STORE_ZT>(ma, mb, p, st);
  } else {
    switch (p.mode) {
      case MODE_STORE_Z: return launch_gemm_mode<BF16, BNT, REV, MODE_STORE_Z>(ma, mb, p, st);
      case MODE_RESIDUAL: return launch_gemm_mode<BF16, BNT, REV, MODE_RESIDUAL>(ma, mb, p, st);
      case MODE_COMPLETE: return launch_gemm_mode<BF16, BNT, REV, MODE_COMPLETE>(ma, mb, p, st);
      default: return QMCUR_ERR_INVALID_ARG;
    }
  }
}

// Z = C T at the tile width z_bn chose.
template <bool BF16>
qmcur_status launch_z(int bn, const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& p,
                      cudaStream_t st) {
  switch (bn) {
    case 128: return launch_gemm<BF16, 128, false>(ma, mb, p, st);
    case 112: return launch_gemm<BF16, 112, false>(ma, mb, p, st);
    case 64: return launch_gemm<BF16, 64, false>(ma, mb, p, st);
    case 32: return launch_gemm<BF16, 32, false>(ma, mb, p, st);
    default: return QMCUR_ERR_INVALID_ARG;
  }
}

}  // namespace

size_t tc_ws_bytes(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec) {
  Carve cv(nullptr, 0);
  TcPlan p1, p2;
  plans_for(prec, p1, p2);
  carve_tc(cv, p1, p2, m, n, c, r);
  return cv.off;
}

qmcur_status launch_reconstruct_tc(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                                   int32_t prec, qmcur_qmat* Z, const qmcur_qmat* A,
                                   const uint8_t* mask, double* out3, void* ws, size_t ws_bytes,
                                   int32_t* dev_status, cudaStream_t st, bool complete) {
  const int64_t m = C->rows, c = C->cols, r = R->rows, n = R->cols;
  if (C->dtype != QMCUR_F32 || R->dtype != QMCUR_F32) return QMCUR_ERR_INVALID_ARG;
  if (Z != nullptr && Z->dtype != QMCUR_F32) return QMCUR_ERR_INVALID_ARG;
  if (A != nullptr && A->dtype != QMCUR_F32) return QMCUR_ERR_INVALID_ARG;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2) return QMCUR_ERR_UNSUPPORTED;
  TcPlan pl, pl2;   // splits of T = U R and of Z = C T
  plans_for(prec, pl, pl2);
  Carve cv(ws, ws_bytes);
  TcWs w = carve_tc(cv, pl, pl2, m, n, c, r);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  const int64_t kp1 = rup(r, pl.epr), kp2 = rup(c, pl2.epr);
  qmcur_status s;
  // operand pieces, one launch: U (c x r) and C (m x c) as they are, R (r x n)
  // transposed
  SplitJobs js{};
  int stiles = 0;
  if (!add_split(js, stiles, U, false, w.A1, c, r, kp1, pl.npieces) ||
      !add_split(js, stiles, R, true, w.B1, n, r, kp1, pl.npieces) ||
      !add_split(js, stiles, C, false, w.A2, m, c, kp2, pl2.npieces))
    return QMCUR_ERR_UNSUPPORTED;
  s = pl.bf16 ? launch_splits<true>(js, stiles, st) : launch_splits<false>(js, stiles, st);
  if (s != QMCUR_OK) return s;
  // T^T = R^T (x) U: M over n (R's pieces, K-major), N over c (U's pieces),
  // the reversed product; its split partials are summed and cut into the
  // pieces of Z = C T's B operand by k_t_reduce.
  CUtensorMap mA1, mB1, mA2, mB2;
  if (!make_map(&mA1, w.B1, pl.bf16, n, kp1, pl.npieces, BM) ||
      !make_map(&mB1, w.A1, pl.bf16, c, kp1, pl.npieces, kBn1) ||
      !make_map(&mA2, w.A2, pl2.bf16, m, kp2, pl2.npieces, BM) ||
      !make_map(&mB2, w.B2, pl2.bf16, n, kp2, pl2.npieces, z_bn(m, n)))
    return QMCUR_ERR_CUDA;
  const int nsplit = t_splits(n, c, pl, kp1);
  TcParams p1{};
  p1.M = (int)n;
  p1.N = (int)c;
  p1.K = (int)r;
  p1.kblocks = (int)(kp1 / pl.epr);
  p1.nterms = pl.nterms;
  for (int i = 0; i < 6; ++i) { p1.ta[i] = pl.tb[i]; p1.tb[i] = pl.ta[i]; }   // R's piece, U's piece
  p1.mode = MODE_STORE_ZT;
  p1.nsplit = nsplit;
  const int64_t ldp = rup(n, 4);   // partial columns padded for paired loads
  for (int t = 0; t < 4; ++t) p1.z[t] = w.P + (int64_t)t * kp2 * ldp;
  p1.ldz = ldp;
  p1.zsplit = 4 * kp2 * ldp;
  p1.status = dev_status;
  TcParams p2 = p1;
  p2.M = (int)m;
  p2.N = (int)n;
  p2.K = (int)c;
  p2.nsplit = 1;
  p2.zsplit = 0;
  p2.kblocks = (int)(kp2 / pl2.epr);
  p2.nterms = pl2.nterms;
  for (int i = 0; i < 6; ++i) { p2.ta[i] = pl2.ta[i]; p2.tb[i] = pl2.tb[i]; }
  const int nsz = Z != nullptr ? z_splits(m, n, pl2, kp2) : 1;
  const int64_t ldpz = rup(n, 4);
  if (nsz > 1 && m > 65535) return QMCUR_ERR_UNSUPPORTED;   // k_z_reduce's grid
  if (Z != nullptr && nsz > 1) {   // partials, summed by k_z_reduce
    p2.mode = MODE_STORE_Z;
    p2.nsplit = nsz;
    for (int t = 0; t < 4; ++t) p2.z[t] = w.Pz + (int64_t)t * m * ldpz;
    p2.ldz = ldpz;
    p2.zsplit = 4 * m * ldpz;
    p2.z_vec = 1;   // 256-byte aligned base, plane and row strides multiples of 4 floats
  } else if (Z != nullptr) {
    p2.mode = MODE_STORE_Z;
    for (int t = 0; t < 4; ++t) p2.z[t] = reinterpret_cast<float*>(Z->plane[t]);
    p2.ldz = Z->ld;
    p2.z_vec = Z->ld % 4 == 0;
    for (int t = 0; t < 4; ++t)
      p2.z_vec = p2.z_vec && reinterpret_cast<uintptr_t>(Z->plane[t]) % 16 == 0;
  } else {
    p2.mode = complete ? MODE_COMPLETE : MODE_RESIDUAL;
    for (int t = 0; t < 4; ++t) p2.a[t] = reinterpret_cast<const float*>(A->plane[t]);
    p2.lda = A->ld;
    p2.a_vec = A->ld % 4 == 0;
    for (int t = 0; t < 4; ++t)
      p2.a_vec = p2.a_vec && reinterpret_cast<uintptr_t>(A->plane[t]) % 16 == 0;
    if (complete) {   // the iterate is updated in place
      for (int t = 0; t < 4; ++t) p2.z[t] = reinterpret_cast<float*>(A->plane[t]);
      p2.ldz = A->ld;
      p2.z_vec = p2.a_vec;
    }
    p2.mask = mask;
    p2.partial = w.partial;
    p2.out3 = out3;
    p2.done = w.done;
  }
  if ((n + kRedJ - 1) / kRedJ > 65535) return QMCUR_ERR_UNSUPPORTED;
  const dim3 rgrid((unsigned)((kp2 + kRedI - 1) / kRedI), (unsigned)((n + kRedJ - 1) / kRedJ));
  // (the residual GEMM folds its own partials: k_t_reduce zeroes the count)
  if (pl.bf16) {
    if ((s = launch_gemm<true, kBn1, true>(mA1, mB1, p1, st)) != QMCUR_OK) return s;
    k_t_reduce<true><<<rgrid, 256, 0, st>>>(w.P, nsplit, p1.zsplit, kp2 * ldp, ldp, n, c, kp2,
                                            pl2.npieces, w.B2, w.done);
    if ((s = launch_z<true>(z_bn(m, n), mA2, mB2, p2, st)) != QMCUR_OK) return s;
  } else {
    if ((s = launch_gemm<false, kBn1, true>(mA1, mB1, p1, st)) != QMCUR_OK) return s;
    k_t_reduce<false><<<rgrid, 256, 0, st>>>(w.P, nsplit, p1.zsplit, kp2 * ldp, ldp, n, c, kp2,
                                             pl2.npieces, w.B2, w.done);
    if ((s = launch_z<false>(z_bn(m, n), mA2, mB2, p2, st)) != QMCUR_OK) return s;
  }
  if (Z != nullptr && nsz > 1) {
    const dim3 zgrid((unsigned)((n + 255) / 256), (unsigned)m);
    k_z_reduce<<<zgrid, 256, 0, st>>>(w.Pz, nsz, p2.zsplit, m * ldpz, ldpz, m, n, view(Z));
  }
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// One general product on the tensor cores: Z = alpha op(X) op(Y), op(X)
// M x K, op(Y) K x N, op = identity or the conjugate transpose (X^H: X
// stored K x M, xh), Z (M x N, F32) stored.  The kernel multiplies operand
// pieces laid out K-major (A[i][k] = op(X)[i][k], B[j][k] = op(Y)[k][j]), so
// each operand is split straight or transposed, conjugated for an ^H, and
// alpha is folded into X's pieces.  K splits with partials summed by
// k_z_reduce when the output has too few tiles to occupy the GPU.

namespace {

// Tile width and K splits of a general product.  An output whose 128- or
// 112-wide tiles fill the SMs keeps the stored product's rule (z_bn,
// z_splits).  A smaller one takes, among the widths 128, 64 and 32 and the K
// splits (each at least 4 k-iterations) that keep the items within one wave
// over the SMs, the pair with the least modelled time: the tile's work per
// split / the width's efficiency.  The efficiencies (1, 0.6, 0.35) are the
// shared-memory bound of M = 128 MMAs at N = 128, 64 and 32: a narrow tile
// reads A's slice for fewer outputs.  So a small output with a long K (the
// backward's G_C = -2 E T^H, 1024 x 120 x 1536) keeps its wide tiles and
// splits K instead of halving the width.
struct GemmShape {
  int bn, nsplit;
};

GemmShape gemm_shape(int64_t M, int64_t N, const TcPlan& pl, int64_t kp) {
  const int bz = z_bn(M, N);
  if (bz >= 112) return GemmShape{bz, z_splits(M, N, pl, kp)};
  const int kiters = pl.nterms * (int)(kp / pl.epr);
  const int64_t mt = (M + BM - 1) / BM;
  const int widths[3] = {kBn2, 64, 32};
  const double eff[3] = {1.0, 0.6, 0.35};
  int max_ns = kiters / 4;
  if (max_ns > kMaxZSplits) max_ns = kMaxZSplits;
  if (max_ns < 1) max_ns = 1;
  GemmShape best{bz, 1};
  double best_cost = -1.0;
  for (int w = 0; w < 3; ++w) {
    const int64_t tiles = mt * ((N + widths[w] - 1) / widths[w]);
    for (int ns = 1; ns <= max_ns; ++ns) {
      const int per = (kiters + ns - 1) / ns;
      const int nsz = (kiters + per - 1) / per;   // every split non-empty
      if (nsz != ns || (ns > 1 && tiles * nsz > kWaveSms)) continue;
      const double cost = (double)((tiles + kWaveSms - 1) / kWaveSms) * widths[w] * per / eff[w];
      if (best_cost < 0.0 || cost < best_cost) {
        best_cost = cost;
        best = GemmShape{widths[w], nsz};
      }
    }
  }
  return best;
}

struct TcGemmWs {
  void *A, *B;
  float* Pz;
};

TcGemmWs carve_tc_gemm(Carve& cv, const TcPlan& pl, int64_t M, int64_t N, int64_t K) {
  const int64_t es = pl.bf16 ? 2 : 4;
  const int64_t kp = rup(K, pl.epr);
  TcGemmWs w;
  w.A = cv.take<char>((size_t)(pl.npieces * 4 * M * kp * es));
  w.B = cv.take<char>((size_t)(pl.npieces * 4 * N * kp * es));
  const int nsz = gemm_shape(M, N, pl, kp).nsplit;
  w.Pz = nsz > 1 ? cv.take<float>((size_t)(nsz * 4 * M * rup(N, 4))) : nullptr;
  return w;
}

}  // namespace

size_t tc_gemm_ws_bytes(int64_t M, int64_t N, int64_t K, int32_t prec) {
  Carve cv(nullptr, 0);
  carve_tc_gemm(cv, plan_for(prec), M, N, K);
  return cv.off;
}

qmcur_status tc_gemm(const QView& X, bool xh, const QView& Y, bool yh, int64_t M, int64_t N,
                     int64_t K, float alpha, const QView& Z, int32_t prec, void* ws,
                     size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (prec != QMCUR_PREC_TF32X3 && prec != QMCUR_PREC_BF16X3 && prec != QMCUR_PREC_BF16X6)
    return QMCUR_ERR_INVALID_ARG;
  if (M < 1 || N < 1 || K < 1 || M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
    return QMCUR_ERR_UNSUPPORTED;
  if (Z.dtype != QMCUR_F32 || Z.rows != M || Z.cols != N) return QMCUR_ERR_INVALID_ARG;
  const TcPlan pl = plan_for(prec);
  const int64_t kp = rup(K, pl.epr);
  Carve cv(ws, ws_bytes);
  TcGemmWs w = carve_tc_gemm(cv, pl, M, N, K);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  SplitJobs js{};
  int tiles = 0;
  // A[i][k] = op(X)[i][k]: X (M x K) as stored, or X^H from X (K x M) read transposed
  // B[j][k] = op(Y)[k][j]: Y (K x N) read transposed, or Y^H from Y (N x K) as stored
  if (!add_split_view(js, tiles, X, xh, w.A, M, K, kp, pl.npieces, alpha, xh) ||
      !add_split_view(js, tiles, Y, !yh, w.B, N, K, kp, pl.npieces, 1.f, yh))
    return QMCUR_ERR_UNSUPPORTED;
  qmcur_status s = pl.bf16 ? launch_splits<true>(js, tiles, st) : launch_splits<false>(js, tiles, st);
  if (s != QMCUR_OK) return s;
  const GemmShape shape = gemm_shape(M, N, pl, kp);
  const int bn = shape.bn;
  CUtensorMap mA, mB;
  if (!make_map(&mA, w.A, pl.bf16, M, kp, pl.npieces, BM) ||
      !make_map(&mB, w.B, pl.bf16, N, kp, pl.npieces, bn))
    return QMCUR_ERR_CUDA;
  TcParams p{};
  p.M = (int)M;
  p.N = (int)N;
  p.K = (int)K;
  p.kblocks = (int)(kp / pl.epr);
  p.nterms = pl.nterms;
  for (int i = 0; i < 6; ++i) { p.ta[i] = pl.ta[i]; p.tb[i] = pl.tb[i]; }
  p.mode = MODE_STORE_Z;
  p.status = dev_status;
  const int nsz = shape.nsplit;
  const int64_t ldpz = rup(N, 4);
  if (nsz > 1 && M > 65535) return QMCUR_ERR_UNSUPPORTED;   // k_z_reduce's grid
  if (nsz > 1) {
    p.nsplit = nsz;
    for (int t = 0; t < 4; ++t) p.z[t] = w.Pz + (int64_t)t * M * ldpz;
    p.ldz = ldpz;
    p.zsplit = 4 * M * ldpz;
    p.z_vec = 1;
  } else {
    p.nsplit = 1;
    for (int t = 0; t < 4; ++t) p.z[t] = reinterpret_cast<float*>(Z.p[t]);
    p.ldz = Z.ld;
    p.z_vec = Z.ld % 4 == 0;
    for (int t = 0; t < 4; ++t) p.z_vec = p.z_vec && reinterpret_cast<uintptr_t>(Z.p[t]) % 16 == 0;
  }
  s = pl.bf16 ? launch_z<true>(bn, mA, mB, p, st) : launch_z<false>(bn, mA, mB, p, st);
  if (s != QMCUR_OK) return s;
  if (nsz > 1) {
    const dim3 zgrid((unsigned)((N + 255) / 256), (unsigned)M);
    k_z_reduce<<<zgrid, 256, 0, st>>>(w.Pz, nsz, p.zsplit, M * ldpz, ldpz, M, N, Z);
  }
  return cuda_ok(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Grouped products of the batched path (tc_group.cuh).

namespace {

// Pieces of many operands from a device job table: CTA b takes tile
// b - first_tile of the job whose tiles hold b (binary search over the
// table's first tiles), 32 rows x 64 k through shared memory as in
// k_split_ops, and writes the pieces into the job's rows of its stacked
// buffer.
template <bool BF16>
__global__ void __launch_bounds__(256) k_split_table(const TcSplitJob* __restrict__ jobs, int njobs,
                                                     int npieces) {
  __shared__ __align__(16) float tile[4][kSplitRows][kSplitPitch];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {   // the last job whose first tile is <= blockIdx.x
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].first_tile <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const TcSplitJob& J = jobs[lo];
  const int tl = (int)blockIdx.x - J.first_tile;
  const int64_t i0 = (int64_t)(tl / J.tiles_k) * kSplitRows, k0 = (int64_t)(tl % J.tiles_k) * kSplitK;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const float* planes[4] = {reinterpret_cast<const float*>(J.S.p[0]), reinterpret_cast<const float*>(J.S.p[1]),
                            reinterpret_cast<const float*>(J.S.p[2]), reinterpret_cast<const float*>(J.S.p[3])};
  if (!J.trans) {
    const int64_t k = k0 + 2 * lane;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t i = i0 + warp + 8 * u;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float2 x = make_float2(0.f, 0.f);
        if (i < J.rows && k < J.K) {
          const float* src = planes[t] + i * J.S.ld + k;
          x.x = src[0];
          if (k + 1 < J.K) x.y = src[1];
        }
        *reinterpret_cast<float2*>(&tile[t][warp + 8 * u][2 * lane]) = x;
      }
    }
  } else {
    const int64_t i = i0 + lane;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t k = k0 + warp + 8 * u;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        tile[t][lane][warp + 8 * u] = (i < J.rows && k < J.K) ? planes[t][k * J.S.ld + i] : 0.f;
    }
  }
  __syncthreads();
  const int64_t k = k0 + 2 * lane;   // kp_job is even
  if (k >= J.kp_job) return;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int il = warp + 8 * u;
    const int64_t i = i0 + il;
    if (i >= J.rows) break;
    const int64_t rowoff = (J.row0 + i) * J.kpad + k;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float2 x = *reinterpret_cast<const float2*>(&tile[t][il][2 * lane]);
      float p0[3], p1[3];
      split_value<BF16, float>(x.x, npieces, p0);
      split_value<BF16, float>(x.y, npieces, p1);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (q >= npieces) break;
        const int64_t idx = (int64_t)(q * 4 + t) * J.plane_stride + rowoff;
        if constexpr (BF16)
          *reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(J.dst) + idx) =
              __floats2bfloat162_rn(p0[q], p1[q]);
        else
          *reinterpret_cast<float2*>(reinterpret_cast<float*>(J.dst) + idx) = make_float2(p0[q], p1[q]);
      }
    }
  }
}

// The plan of Z = C T for a batch precision (the second product's split).
// The split of a precision for Z = C T (product 1) or for T = U R (product 0).
TcPlan group_plan(int32_t prec, int product = 1) {
  TcPlan a, b;
  plans_for(prec, a, b);
  return product == 0 ? a : b;
}

}  // namespace

int tc_group_epr(int32_t prec, int product) { return (int)group_plan(prec, product).epr; }
int tc_group_npieces(int32_t prec, int product) { return group_plan(prec, product).npieces; }

size_t tc_group_piece_bytes(int32_t prec, int64_t rows, int64_t kpad, int product) {
  const TcPlan pl = group_plan(prec, product);
  return (size_t)pl.npieces * 4 * rows * kpad * (pl.bf16 ? 2 : 4);
}

qmcur_status tc_group_split(int32_t prec, const TcSplitJob* jobs, int njobs, int tiles,
                            cudaStream_t st, int product) {
  if (njobs < 1 || tiles < 1) return QMCUR_ERR_INVALID_ARG;
  const TcPlan pl = group_plan(prec, product);
  if (pl.bf16) k_split_table<true><<<tiles, 256, 0, st>>>(jobs, njobs, pl.npieces);
  else k_split_table<false><<<tiles, 256, 0, st>>>(jobs, njobs, pl.npieces);
  return cuda_ok(cudaGetLastError());
}

qmcur_status tc_group_residual(int32_t prec, int bn, const void* A_all, int64_t rows_a,
                               const void* B_all, int64_t rows_b, int64_t kpad,
                               const TcGroupTile* tiles, int ntiles, const TcGroupProb* probs,
                               double* partial, int32_t* dev_status, cudaStream_t st) {
  if (ntiles < 1 || (bn != 64 && bn != 128)) return QMCUR_ERR_INVALID_ARG;
  const TcPlan pl = group_plan(prec);
  CUtensorMap mA, mB;
  if (!make_map(&mA, const_cast<void*>(A_all), pl.bf16, rows_a, kpad, pl.npieces, BM) ||
      !make_map(&mB, const_cast<void*>(B_all), pl.bf16, rows_b, kpad, pl.npieces, bn))
    return QMCUR_ERR_CUDA;
  TcParams p{};
  p.M = 1;
  p.N = 1;
  p.nterms = pl.nterms;
  for (int i = 0; i < 6; ++i) { p.ta[i] = pl.ta[i]; p.tb[i] = pl.tb[i]; }
  p.mode = MODE_GROUPED;
  p.nsplit = 1;
  p.partial = partial;
  p.done = nullptr;   // k_batch_fold folds per problem
  p.status = dev_status;
  p.gtiles = tiles;
  p.gprobs = probs;
  p.gcount = ntiles;
  if (pl.bf16)
    return bn == 64 ? launch_gemm_mode<true, 64, false, MODE_GROUPED>(mA, mB, p, st)
                    : launch_gemm_mode<true, 128, false, MODE_GROUPED>(mA, mB, p, st);
  return bn == 64 ? launch_gemm_mode<false, 64, false, MODE_GROUPED>(mA, mB, p, st)
                  : launch_gemm_mode<false, 128, false, MODE_GROUPED>(mA, mB, p, st);
}

qmcur_status tc_group_t_pieces(int32_t prec, const void* R_all, int64_t rows_r, const void* U_all,
                               int64_t rows_u, int64_t kpad, const TcGroupTile* tiles, int ntiles,
                               const TcGroupProb* probs, void* pieces, int64_t pieces_kpad,
                               int64_t pieces_rows, int32_t* dev_status, cudaStream_t st) {
  if (ntiles < 1 || pieces == nullptr) return QMCUR_ERR_INVALID_ARG;
  const TcPlan pl = group_plan(prec, 0), pz = group_plan(prec, 1);
  if (pl.bf16 != pz.bf16) return QMCUR_ERR_UNSUPPORTED;   // the pieces take the MMA's type
  CUtensorMap mA, mB;
  if (!make_map(&mA, const_cast<void*>(R_all), pl.bf16, rows_r, kpad, pl.npieces, BM) ||
      !make_map(&mB, const_cast<void*>(U_all), pl.bf16, rows_u, kpad, pl.npieces, kGroupTBn))
    return QMCUR_ERR_CUDA;
  TcParams p{};
  p.M = 1;
  p.N = 1;
  p.nterms = pl.nterms;
  for (int i = 0; i < 6; ++i) { p.ta[i] = pl.tb[i]; p.tb[i] = pl.ta[i]; }   // R's piece, U's piece
  p.mode = MODE_GROUPED_PIECES;
  p.nsplit = 1;
  p.status = dev_status;
  p.gtiles = tiles;
  p.gprobs = probs;
  p.gcount = ntiles;
  p.pieces = pieces;
  p.pk_kpad = pieces_kpad;
  p.pk_plane = pieces_rows * pieces_kpad;
  p.pk_npieces = pz.npieces;
  if (pl.bf16) return launch_gemm_mode<true, kGroupTBn, true, MODE_GROUPED_PIECES>(mA, mB, p, st);
  return launch_gemm_mode<false, kGroupTBn, true, MODE_GROUPED_PIECES>(mA, mB, p, st);
}

}  // namespace qmcur
