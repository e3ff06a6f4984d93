// Rank-capped pseudo-inverse U = W_k^+ to FP64 accuracy on GB300, whose FP64
// units run at 1/64 of its FP32 rate (about 2 FP64 FMA per clock per SM).
//
// The truncated inverse of Sec. 2.2 / Algorithm 1 keeps the k = rank_cap
// largest singular triplets of W (r x c): U = V_k Sigma_k^-1 P_k^H.  It only
// depends on the top-k right singular subspace S = span(V_k): for ANY basis
// P of S (full column rank, not necessarily orthonormal),
//   U = P (W P)^+,
// because W P = P_k Sigma_k (V_k^H P) and (V_k^H P) is invertible.  So the
// method finds S to FP64 accuracy by subspace iteration with FP64 products
// (all SMs), and never factors anything in FP64: every k x k Cholesky factor
// is taken in FP32 (one CTA, shared memory) and used only as a right
// preconditioner, Z R^-1 with the FP32 R applied in FP64 arithmetic.  Such a
// solve changes the basis but not its span, so the FP32 rounding of R never
// reaches the result; it only leaves the bases orthonormal to FP32 accuracy,
// and the one place where orthonormality matters (the final Q^+ = Q^H) is
// corrected to first order with the FP64 Gram matrix E = Q^H Q - I.
//
// Iteration s, from P (c x k, near-orthonormal) and Y = W P:
//   Z  = W^H Y                         FP64 product (c x k, K = r)
//   M  = P^H Z,  E = P^H P - I          FP64 Gram products (k x k)
//   R_Y = chol32(M);  Z' = Z R_Y^-1     (= W^H Q with Q = Y R_Y^-1, the
//                                        left basis normalised)
//   M' = M - E M                        (P (I - E) P^H: the projector on span P
//                                        to first order in E)
//   G' = Z'^H Z';  rho_s = ||Z - P M'||_F / ||Z||_F
//   R' = chol32(G');  P <- Z' R'^-1;  Y <- W P
// rho_s measures how far W^H W moves span(P); times kappa^2 (kappa^2 taken
// from the diagonal of R_Y, whose Gram M ~ Sigma_k^2) it bounds the angle of
// span(P) to S, and the angle shrinks by (sigma_{k+1} / sigma_k)^2 per
// iteration.  The iteration stops when the predicted angle of the new P is
// below kAngleTol (extrapolated at the observed contraction once rho_s
// reaches its rounding floor), or after max_iter iterations
// (QMCUR_ERR_NO_CONVERGENCE: the spectrum has no usable gap at k).
//
// Then U = P (W P)^+ by CholeskyQR2 with FP32 factors:
//   Y = W P;  R1 = chol32(Y^H Y);  Q1 = Y R1^-1, T1 = P R1^-1
//   R2 = chol32(Q1^H Q1);  Q2 = Q1 R2^-1, T2 = T1 R2^-1      (Y = Q2 R2 R1,
//                                                            P = T2 R2 R1)
//   E2 = Q2^H Q2 - I;  V = T2 - T2 E2 ~ T2 (I + E2)^-1;  U = V Q2^H,
// i.e. U = T2 Q2^+ = P (R2 R1)^-1 Q2^+ = P Y^+, with ||E2|| ~ u32 ||E1||, so
// that the first-order correction leaves O(||E2||^2) behind.
//
// Everything runs in ONE cooperative persistent kernel of one 512-thread CTA
// per SM, with a bounded grid barrier between steps.  A product step is a
// list of (16 x 16 output tile, k-range) items dealt to the 2 x SMs tile
// workers; items of one tile sum their partials in k order (the last to
// arrive does it), so results do not depend on timing.  In a solve step every
// CTA that holds rows factors the Gram matrix itself (identical arithmetic,
// identical factors, no barrier) and solves its rows, one warp per row.
// Every CTA evaluates the stopping rule itself from the same global values,
// so all take the same branch.
#include <type_traits>

#include "small_impl.cuh"

namespace qmcur {
namespace {

constexpr int kRfThreads = kCholThreads;             // 512
constexpr int kRfTileThreads = 256;
constexpr int kRfWorkers = kRfThreads / kRfTileThreads;
constexpr int kRfTS = 16;                            // output tile edge (quaternions)
constexpr int kRfBK = 16;                            // k-slice
constexpr int kRfMaxSplits = 8;
constexpr int kRfMaxParts = 1024;                    // split partial tiles per step
constexpr int kRfMaxTiles = 8192;                    // tiles of a norm product, split-tile counters
constexpr int kRfMaxDim = 16384;                     // r, c at most (tiles of the norm product)
constexpr int kRfMaxIter = 64;
constexpr double kAngleTol = 1e-14;                  // target angle of span(P) to S
constexpr float kCholShift = 1e-5f;                  // relative diagonal shift of a retried factor

static_assert(kRfWorkers * kRfTileThreads == kRfThreads, "whole tile workers");

struct __align__(16) Q64 { double x, y, z, w; };

__device__ __forceinline__ Q64 q64_zero() { return Q64{0.0, 0.0, 0.0, 0.0}; }

// acc += a b (Hamilton product, Sec. 2.2), FP64
__device__ __forceinline__ void q64_fma(Q64& acc, const Q64& a, const Q64& b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x); acc.x = fma(-a.z, b.z, acc.x); acc.x = fma(-a.w, b.w, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y); acc.y = fma(a.z, b.w, acc.y); acc.y = fma(-a.w, b.z, acc.y);
  acc.z = fma(a.x, b.z, acc.z); acc.z = fma(-a.y, b.w, acc.z); acc.z = fma(a.z, b.x, acc.z); acc.z = fma(a.w, b.y, acc.z);
  acc.w = fma(a.x, b.w, acc.w); acc.w = fma(a.y, b.z, acc.w); acc.w = fma(-a.z, b.y, acc.w); acc.w = fma(a.w, b.x, acc.w);
}

// acc -= a b with b given in FP32 (a factor entry)
__device__ __forceinline__ void q64_fms_f(Q64& acc, const Q64& a, const float4 bf) {
  const double bx = bf.x, by = bf.y, bz = bf.z, bw = bf.w;
  acc.x -= a.x * bx - a.y * by - a.z * bz - a.w * bw;
  acc.y -= a.x * by + a.y * bx + a.z * bw - a.w * bz;
  acc.z -= a.x * bz - a.y * bw + a.z * bx + a.w * by;
  acc.w -= a.x * bw + a.y * bz - a.z * by + a.w * bx;
}

__device__ __forceinline__ double ldp(const QPtr& q, int t, int64_t off) {
  if (q.dtype == QMCUR_F64) return reinterpret_cast<const double*>(q.p[t])[off];
  return (double)reinterpret_cast<const float*>(q.p[t])[off];
}

__device__ __forceinline__ Q64 ldq64(const QPtr& q, int64_t off) {
  return Q64{ldp(q, 0, off), ldp(q, 1, off), ldp(q, 2, off), ldp(q, 3, off)};
}

__device__ __forceinline__ void stq64(const QPtr& q, int64_t off, const Q64& v) {
  if (q.dtype == QMCUR_F64) {
    reinterpret_cast<double*>(q.p[0])[off] = v.x;
    reinterpret_cast<double*>(q.p[1])[off] = v.y;
    reinterpret_cast<double*>(q.p[2])[off] = v.z;
    reinterpret_cast<double*>(q.p[3])[off] = v.w;
  } else {
    reinterpret_cast<float*>(q.p[0])[off] = (float)v.x;
    reinterpret_cast<float*>(q.p[1])[off] = (float)v.y;
    reinterpret_cast<float*>(q.p[2])[off] = (float)v.z;
    reinterpret_cast<float*>(q.p[3])[off] = (float)v.w;
  }
}

// One product of a step: Zout = alpha op(X) op(Y) + beta Zin - [minus_eye] I,
// op(X) M x K (X stored K x M when xh: op(X) = X^H), op(Y) K x N likewise.
// With norm, nothing is stored: the step folds ||Zin - op(X) op(Y)||_F^2 and
// ||Zin||_F^2 into norm_out[0..1] (fixed order).
struct RfJob {
  QPtr X, Y, Zin, Zout;
  int M, N, K;
  int xh, yh;
  double alpha, beta;
  int minus_eye;
  int norm;
  int fp64;             // native FP64 tiles (else float-float on the FP32 pipe)
  int splits, kchunk;   // filled by plan_jobs
  int tiles, tn;        // output tiles, tiles along N
};

struct RfArgs {
  QPtr W;              // r x c input (F32 or F64 planes)
  int r, c, k;
  int max_iter;
  uint64_t seed;
  // FP64 workspaces
  QPtr P[2], Y, Z, Zp, M, E, Mp, Gp, G1, G2, E2, Q1, Q2, T1, T2, V;
  QPtr U;              // c x r output
  Q64* part;           // kRfMaxParts x kRfTileThreads split partials
  unsigned* cnt;       // kRfMaxTiles split-tile arrival counts, then the norm fold's
  double* normpart;    // kRfMaxTiles x 2 tile norm partials
  double* norms;       // (kRfMaxIter + 1) x 2
  double* kap2;        // kRfMaxIter + 1
  unsigned* bar;       // grid barrier words
  int32_t* status;
  int32_t* rank_out;
  int workers;         // gridDim.x * kRfWorkers (for the split plans)
};

// smem: two tile workers' operand slices, or the packed factor + Cholesky buffers
constexpr int kRfWorkerQ64 = 2 * kRfTS * (kRfBK + 1);
constexpr size_t rf_chol_off(int k) { return (sm_trsm_bytes(k) + 15) / 16 * 16; }
constexpr size_t rf_smem(int k) {
  const size_t g = (size_t)kRfWorkers * kRfWorkerQ64 * sizeof(Q64);
  const size_t s = rf_chol_off(k) + sm_chol_bytes();
  return g > s ? g : s;
}

// ---------------------------------------------------------------------------
// Products.

// Entry (row i, k-index l) of op(X) for an M x K operand view (X stored K x M
// and conjugated when xh); zero outside.
__device__ __forceinline__ Q64 ld_opx(const QPtr& X, int xh, int M, int K, int i, int l) {
  if (i >= M || l >= K) return q64_zero();
  if (!xh) return ldq64(X, (int64_t)i * X.ld + l);
  Q64 v = ldq64(X, (int64_t)l * X.ld + i);
  v.y = -v.y; v.z = -v.z; v.w = -v.w;
  return v;
}

// Entry (k-index l, column j) of op(Y) for a K x N operand view.
__device__ __forceinline__ Q64 ld_opy(const QPtr& Y, int yh, int K, int N, int l, int j) {
  if (l >= K || j >= N) return q64_zero();
  if (!yh) return ldq64(Y, (int64_t)l * Y.ld + j);
  Q64 v = ldq64(Y, (int64_t)j * Y.ld + l);
  v.y = -v.y; v.z = -v.z; v.w = -v.w;
  return v;
}

__device__ __forceinline__ void worker_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kRfTileThreads) : "memory");
}

// Float-float arithmetic on the FP32 pipe (GB300 runs FP32 at 64x its FP64
// rate).  An FP64 operand v is carried as the pair (h, l) = (fl32(v),
// fl32(v - h)), 48 significant bits.  A real product (a_h + a_l)(b_h + b_l)
// adds into the running pair (S, C) as
//   p = a_h b_h, e = fma(a_h, b_h, -p)         (exact product: p + e)
//   S, err = TwoSum(S, p)                     (exact sum: S + err)
//   C += err + e + a_h b_l + a_l b_h          (the small terms in FP32)
// (Knuth's TwoSum and the FMA product split, as in the compensated dot
// product of Ogita, Rump and Oishi, "Accurate sum and dot product", 2005).
// The result S + C carries about 2^-46 of sum |a b|.  The rn intrinsics keep
// the compiler from fusing the rounded product p into a later add.
struct __align__(16) QFF { float4 h, l; };

__device__ __forceinline__ QFF ff_split(const Q64& v) {
  QFF r;
  r.h = make_float4(__double2float_rn(v.x), __double2float_rn(v.y), __double2float_rn(v.z),
                    __double2float_rn(v.w));
  r.l = make_float4(__double2float_rn(v.x - (double)r.h.x), __double2float_rn(v.y - (double)r.h.y),
                    __double2float_rn(v.z - (double)r.h.z), __double2float_rn(v.w - (double)r.h.w));
  return r;
}

// (S, C) += sg (ah + al)(bh + bl), sg = +1 or -1 (applied to a)
template <int SG>
__device__ __forceinline__ void ff_mac(float& S, float& C, float ah, float al, float bh, float bl) {
  const float a = SG > 0 ? ah : -ah, a2 = SG > 0 ? al : -al;
  const float p = __fmul_rn(a, bh);
  const float e = __fmaf_rn(a, bh, -p);
  const float sn = __fadd_rn(S, p);
  const float bp = __fsub_rn(sn, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(sn, bp)), __fsub_rn(p, bp));
  S = sn;
  C = __fadd_rn(C, __fadd_rn(err, e));
  C = __fmaf_rn(a, bl, C);
  C = __fmaf_rn(a2, bh, C);
}

// acc += x y, Hamilton product (Sec. 2.2), in float-float
__device__ __forceinline__ void ff_qmac(float S[4], float C[4], const QFF& x, const QFF& y) {
  const float4 xh = x.h, xl = x.l, yh = y.h, yl = y.l;
  ff_mac<+1>(S[0], C[0], xh.x, xl.x, yh.x, yl.x); ff_mac<-1>(S[0], C[0], xh.y, xl.y, yh.y, yl.y);
  ff_mac<-1>(S[0], C[0], xh.z, xl.z, yh.z, yl.z); ff_mac<-1>(S[0], C[0], xh.w, xl.w, yh.w, yl.w);
  ff_mac<+1>(S[1], C[1], xh.x, xl.x, yh.y, yl.y); ff_mac<+1>(S[1], C[1], xh.y, xl.y, yh.x, yl.x);
  ff_mac<+1>(S[1], C[1], xh.z, xl.z, yh.w, yl.w); ff_mac<-1>(S[1], C[1], xh.w, xl.w, yh.z, yl.z);
  ff_mac<+1>(S[2], C[2], xh.x, xl.x, yh.z, yl.z); ff_mac<-1>(S[2], C[2], xh.y, xl.y, yh.w, yl.w);
  ff_mac<+1>(S[2], C[2], xh.z, xl.z, yh.x, yl.x); ff_mac<+1>(S[2], C[2], xh.w, xl.w, yh.y, yl.y);
  ff_mac<+1>(S[3], C[3], xh.x, xl.x, yh.w, yl.w); ff_mac<+1>(S[3], C[3], xh.y, xl.y, yh.z, yl.z);
  ff_mac<-1>(S[3], C[3], xh.z, xl.z, yh.y, yl.y); ff_mac<+1>(S[3], C[3], xh.w, xl.w, yh.x, yl.x);
}

// Accumulates entry (ty, tx) of tile (tm, tn) over [kb, ke) with one worker,
// in float-float (FF) or in native FP64.  The loads are laid out so that
// consecutive threads read consecutive addresses of the operand's storage.
template <bool FF>
__device__ __noinline__ Q64 rf_tile_acc_t(const RfJob& j, int tm, int tn, int kb, int ke, Q64* sm, int tid,
                             int bar_id) {
  using E = typename std::conditional<FF, QFF, Q64>::type;
  static_assert(sizeof(E) == sizeof(Q64), "one slot layout");
  E (*xs)[kRfBK + 1] = reinterpret_cast<E (*)[kRfBK + 1]>(sm);
  E (*ys)[kRfTS + 1] = reinterpret_cast<E (*)[kRfTS + 1]>(sm + kRfTS * (kRfBK + 1));
  const int tx = tid % kRfTS, ty = tid / kRfTS;
  const int m0 = tm * kRfTS, n0 = tn * kRfTS;
  Q64 acc = q64_zero();
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
  const int xa = tid / kRfBK, xb = tid % kRfBK;          // xh = 0: contiguous along l
  const int xr = j.xh ? xb : xa, xl = j.xh ? xa : xb;    // xh = 1: contiguous along rows
  const int yl = j.yh ? tid % kRfBK : tid / kRfTS;       // yh = 1: contiguous along l
  const int yc = j.yh ? tid / kRfBK : tid % kRfTS;       // yh = 0: contiguous along columns
  for (int k0 = kb; k0 < ke; k0 += kRfBK) {
    const Q64 xv = ld_opx(j.X, j.xh, j.M, ke, m0 + xr, k0 + xl);
    const Q64 yv = ld_opy(j.Y, j.yh, ke, j.N, k0 + yl, n0 + yc);
    worker_bar(bar_id);   // the previous slice is no longer read
    if constexpr (FF) {
      xs[xr][xl] = ff_split(xv);
      ys[yl][yc] = ff_split(yv);
    } else {
      xs[xr][xl] = xv;
      ys[yl][yc] = yv;
    }
    worker_bar(bar_id);
    const int lend = ke - k0 < kRfBK ? ke - k0 : kRfBK;
    if constexpr (FF) {
      if (lend == kRfBK) {
#pragma unroll 4
        for (int l = 0; l < kRfBK; ++l) ff_qmac(S, C, xs[ty][l], ys[l][tx]);
      } else {
        for (int l = 0; l < lend; ++l) ff_qmac(S, C, xs[ty][l], ys[l][tx]);
      }
    } else {
      for (int l = 0; l < lend; ++l) q64_fma(acc, xs[ty][l], ys[l][tx]);
    }
  }
  if constexpr (FF) {
    acc.x = (double)S[0] + (double)C[0];
    acc.y = (double)S[1] + (double)C[1];
    acc.z = (double)S[2] + (double)C[2];
    acc.w = (double)S[3] + (double)C[3];
  }
  return acc;
}

__device__ __forceinline__ Q64 rf_tile_acc(const RfJob& j, int tm, int tn, int kb, int ke, Q64* sm,
                                           int tid, int bar_id) {
  return j.fp64 ? rf_tile_acc_t<false>(j, tm, tn, kb, ke, sm, tid, bar_id)
                : rf_tile_acc_t<true>(j, tm, tn, kb, ke, sm, tid, bar_id);
}

__device__ __forceinline__ double rf_sq(const Q64& a) {
  return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
}

// Epilogue of one finished tile entry: store, or the norm partials.
__device__ void rf_epilogue(const RfJob& j, int tm, int tn, int tid, const Q64& acc,
                            double* nd, double* nz) {
  const int i = tm * kRfTS + tid / kRfTS, c = tn * kRfTS + tid % kRfTS;
  if (i >= j.M || c >= j.N) return;
  const int64_t oin = (int64_t)i * j.Zin.ld + c;
  if (j.norm) {
    const Q64 z = ldq64(j.Zin, oin);
    const Q64 d{z.x - acc.x, z.y - acc.y, z.z - acc.z, z.w - acc.w};
    *nd += rf_sq(d);
    *nz += rf_sq(z);
    return;
  }
  Q64 v{j.alpha * acc.x, j.alpha * acc.y, j.alpha * acc.z, j.alpha * acc.w};
  if (j.beta != 0.0) {
    const Q64 z = ldq64(j.Zin, oin);
    v.x += j.beta * z.x; v.y += j.beta * z.y; v.z += j.beta * z.z; v.w += j.beta * z.w;
  }
  if (j.minus_eye && i == c) v.x -= 1.0;
  stq64(j.Zout, (int64_t)i * j.Zout.ld + c, v);
}

// Sum of a worker's 256 values in a fixed order (warp shuffles, then warps).
__device__ double rf_worker_sum(double v, double* sh, int tid, int bar_id) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) sh[tid >> 5] = v;
  worker_bar(bar_id);
  double s = 0.0;
  if (tid == 0)
    for (int w = 0; w < kRfTileThreads / 32; ++w) s += sh[w];
  worker_bar(bar_id);
  return s;
}

// One step of up to three independent products (at most one with `norm`).
__device__ void rf_gemm_step(const RfArgs& a, const RfJob* jobs, int njobs, double* norm_out,
                             int vb, int vg, unsigned char* smem) {
  __shared__ int last_sh[kRfWorkers];
  __shared__ double red_sh[kRfWorkers][kRfTileThreads / 32];
  const int worker = threadIdx.x / kRfTileThreads, wtid = threadIdx.x % kRfTileThreads;
  Q64* wsm = reinterpret_cast<Q64*>(smem) + worker * kRfWorkerQ64;
  const int bar_id = 1 + worker;
  int items[3], ibase[3], tbase[3], pbase[3];
  int total = 0, tiles_total = 0, parts_total = 0;
  for (int q = 0; q < 3; ++q) {
    items[q] = q < njobs ? jobs[q].tiles * jobs[q].splits : 0;
    ibase[q] = total;
    tbase[q] = tiles_total;
    pbase[q] = parts_total;
    total += items[q];
    if (q < njobs && jobs[q].splits > 1) {   // counters and partials: split jobs only
      tiles_total += jobs[q].tiles;
      parts_total += items[q];
    }
  }
  // one item per worker 0 of every CTA first, then worker 1
  for (int t = vb + vg * worker; t < total; t += vg * kRfWorkers) {
    const int q = t < ibase[1] ? 0 : (t < ibase[2] ? 1 : 2);
    const RfJob& j = jobs[q];
    const int tt = t - ibase[q];
    const int tile = tt % j.tiles, sp = tt / j.tiles;
    const int tm = tile / j.tn, tn = tile % j.tn;
    const int kb = sp * j.kchunk;
    const int ke = kb + j.kchunk < j.K ? kb + j.kchunk : j.K;
    Q64 acc = rf_tile_acc(j, tm, tn, kb, ke, wsm, wtid, bar_id);
    if (j.splits > 1) {
      Q64* slot = a.part + ((size_t)pbase[q] + (size_t)tile * j.splits + sp) * kRfTileThreads;
      slot[wtid] = acc;
      __threadfence();
      worker_bar(bar_id);
      if (wtid == 0) last_sh[worker] = atomicAdd(a.cnt + tbase[q] + tile, 1u) == (unsigned)(j.splits - 1);
      worker_bar(bar_id);
      if (!last_sh[worker]) continue;
      __threadfence();
      const Q64* src = a.part + ((size_t)pbase[q] + (size_t)tile * j.splits) * kRfTileThreads + wtid;
      acc = q64_zero();
      for (int s = 0; s < j.splits; ++s) {   // in k order; written by other SMs
        const double* p = reinterpret_cast<const double*>(src + (size_t)s * kRfTileThreads);
        acc.x += __ldcg(p); acc.y += __ldcg(p + 1); acc.z += __ldcg(p + 2); acc.w += __ldcg(p + 3);
      }
      if (wtid == 0) a.cnt[tbase[q] + tile] = 0u;   // ready for the next step
    }
    double nd = 0.0, nz = 0.0;
    rf_epilogue(j, tm, tn, wtid, acc, &nd, &nz);
    if (j.norm) {
      nd = rf_worker_sum(nd, red_sh[worker], wtid, bar_id);
      nz = rf_worker_sum(nz, red_sh[worker], wtid, bar_id);
      if (wtid == 0) {
        a.normpart[2 * tile] = nd;
        a.normpart[2 * tile + 1] = nz;
        __threadfence();
        const unsigned done = atomicAdd(a.cnt + kRfMaxTiles, 1u);
        if (done == (unsigned)(j.tiles - 1)) {   // the last tile folds, in tile order
          __threadfence();
          double sd = 0.0, sz = 0.0;
          for (int u = 0; u < j.tiles; ++u) {
            sd += __ldcg(a.normpart + 2 * u);
            sz += __ldcg(a.normpart + 2 * u + 1);
          }
          norm_out[0] = sd;
          norm_out[1] = sz;
          a.cnt[kRfMaxTiles] = 0u;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Solves.

// One warp: row `row` of Z = Y R^-1 in FP64 with the packed FP32 factor R
// (R_ll taken as 1 / invd[l]); k <= 32 U.
template <int U>
__device__ void rf_trsm_row(const QPtr& Y, const QPtr& Z, int row, int k, const float* rpk) {
  const float4* Rs = reinterpret_cast<const float4*>(rpk);
  const float* invd = rpk + 4 * (k * (k + 1) / 2);
  const int lane = threadIdx.x & 31;
  Q64 t[U];
  const int64_t yo = (int64_t)row * Y.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    t[u] = c < k ? ldq64(Y, yo + c) : q64_zero();
  }
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
    const int lend = k - 32 * uu < 32 ? k - 32 * uu : 32;
    for (int ll = 0; ll < lend; ++ll) {
      const int l = 32 * uu + ll;
      const double s = (double)invd[l];
      const Q64 z{__shfl_sync(0xffffffffu, t[uu].x, ll) * s, __shfl_sync(0xffffffffu, t[uu].y, ll) * s,
                  __shfl_sync(0xffffffffu, t[uu].z, ll) * s, __shfl_sync(0xffffffffu, t[uu].w, ll) * s};
      const float4* Rrow = Rs + (packed_row(l, k) - l);   // R_l,c at Rrow + c, c >= l
#pragma unroll
      for (int u = uu; u < U; ++u) {
        const int c = lane + 32 * u;
        if (c > l && c < k) q64_fms_f(t[u], z, Rrow[c]);
      }
      if (lane == ll) t[uu] = z;
    }
  }
  const int64_t zo = (int64_t)row * Z.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    if (c < k) stq64(Z, zo + c, t[u]);
  }
}

__device__ __noinline__ void rf_trsm_row_any(const QPtr& Y, const QPtr& Z, int row, int k, const float* rpk) {
  if (k <= 32) rf_trsm_row<1>(Y, Z, row, k, rpk);
  else if (k <= 64) rf_trsm_row<2>(Y, Z, row, k, rpk);
  else if (k <= 96) rf_trsm_row<3>(Y, Z, row, k, rpk);
  else rf_trsm_row<4>(Y, Z, row, k, rpk);
}

// Z0 = Y0 R^-1 (rows0 rows) and Z1 = Y1 R^-1 (rows1 rows), R = chol32(G).
// With kap_out, CTA 0 writes (max R_ll / min R_ll)^2 there.
__device__ void rf_solve_step(const RfArgs& a, const QPtr& G, const QPtr& Y0, const QPtr& Z0,
                              int rows0, const QPtr* Y1, const QPtr* Z1, int rows1, double* kap_out,
                              int vb, int vg, unsigned char* smem) {
  const int k = a.k;
  const int rows = rows0 + (Y1 != nullptr ? rows1 : 0);
  if (vb >= rows) return;   // CTA-uniform; CTA 0 always holds a row
  float* rpk = reinterpret_cast<float*>(smem);
  // the factor only preconditions: a lost pivot (G beyond FP32's reach, e.g.
  // from the random start block) is retried with a shifted diagonal, every
  // CTA alike; only a second loss is reported
  __shared__ int32_t bad_sh;
  if (threadIdx.x == 0) bad_sh = 0;
  __syncthreads();
  sm_chol(G, k, rpk, &bad_sh, smem + rf_chol_off(k), nullptr);
  __syncthreads();
  if (bad_sh != 0) {
    __syncthreads();
    if (threadIdx.x == 0) bad_sh = 0;
    __syncthreads();
    sm_chol(G, k, rpk, &bad_sh, smem + rf_chol_off(k), nullptr, kCholShift);
    __syncthreads();
    if (bad_sh != 0 && threadIdx.x == 0 && vb == 0) set_status(a.status, QMCUR_ERR_ILL_CONDITIONED);
  }
  if (kap_out != nullptr && vb == 0 && threadIdx.x == 0) {
    const float* invd = rpk + 4 * (k * (k + 1) / 2);
    float lo = invd[0], hi = invd[0];
    for (int l = 1; l < k; ++l) { lo = fminf(lo, invd[l]); hi = fmaxf(hi, invd[l]); }
    const double q = (double)hi / (double)lo;
    *kap_out = q * q;
  }
  const int warp = threadIdx.x >> 5, nw = kRfThreads / 32;
  for (int i = warp;; i += nw) {
    const int row = vb + vg * i;
    if (row >= rows) break;
    if (row < rows0) rf_trsm_row_any(Y0, Z0, row, k, rpk);
    else rf_trsm_row_any(*Y1, *Z1, row - rows0, k, rpk);
  }
  __syncthreads();   // shared memory is reused by the next step
}

// ---------------------------------------------------------------------------
// The program.

__device__ __forceinline__ RfJob job(const QPtr& X, int xh, const QPtr& Y, int yh, const QPtr& Z,
                                     int M, int N, int K) {
  RfJob j{};
  j.X = X; j.Y = Y; j.Zin = Z; j.Zout = Z;
  j.M = M; j.N = N; j.K = K; j.xh = xh; j.yh = yh;
  j.alpha = 1.0; j.beta = 0.0;
  return j;
}

// k-range splits: enough items to give every worker one, at most kRfMaxSplits,
// and the partials of all split jobs of a step within kRfMaxParts.
__device__ void plan_jobs(RfJob* jobs, int n, int workers) {
  int tiles_all = 0;
  for (int q = 0; q < n; ++q) {
    jobs[q].tn = (jobs[q].N + kRfTS - 1) / kRfTS;
    jobs[q].tiles = ((jobs[q].M + kRfTS - 1) / kRfTS) * jobs[q].tn;
    tiles_all += jobs[q].tiles;
  }
  int parts = 0;
  for (int q = 0; q < n; ++q) {
    const int slices = (jobs[q].K + kRfBK - 1) / kRfBK;
    int sp = workers / (tiles_all > 0 ? tiles_all : 1);
    if (sp > kRfMaxSplits) sp = kRfMaxSplits;
    if (sp > slices) sp = slices;
    if (sp < 1) sp = 1;
    const int per = (slices + sp - 1) / sp;
    jobs[q].kchunk = per * kRfBK;
    jobs[q].splits = (slices + per - 1) / per;
    if (jobs[q].splits > 1) parts += jobs[q].tiles * jobs[q].splits;
  }
  if (parts > kRfMaxParts)
    for (int q = 0; q < n; ++q) {
      jobs[q].splits = 1;
      jobs[q].kchunk = ((jobs[q].K + kRfBK - 1) / kRfBK) * kRfBK;
    }
}

__device__ __forceinline__ bool rf_sync(const RfArgs& a, unsigned& target) {
  return grid_sync(a.bar, a.status, target);
}

__device__ __forceinline__ uint4 rf_philox(uint4 c, uint2 key) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) { key.x += 0x9E3779B9u; key.y += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
  }
  return c;
}

// The stopping rule's state, identical in every CTA.
struct StopState {
  double prev_rho;   // last rho above the rounding floor
  int prev_s;        // its iteration (0: none yet)
  double contr;      // observed contraction per iteration (0: unknown)
  int floor_hits;    // consecutive iterations at the floor without a history
};

// Whether the P about to be formed at iteration s is within kAngleTol of S.
// rho_s (from nd = ||Z - P M'||^2, nz = ||Z||^2) times 4 kappa^2 bounds the
// angle of the current P, and the angle shrinks by a constant factor per
// iteration.  rho has a floor set by the float-float products that form Z
// (about 2^-46 sqrt(k) relative): values above 32 times it are reliable.
// Below it, rho is extrapolated from the last reliable value at the
// contraction seen between two reliable values; with only one reliable value,
// the fall from it onto the floor bounds the contraction.  Iteration 1 starts
// from the random block, whose rho means nothing.
__device__ __forceinline__ bool stop_now(StopState& st, int s, double nd, double nz, double kap2,
                                         int k) {
  if (s < 2 || !(nz > 0.0)) return false;
  const double rho = sqrt(fmax(nd, 0.0) / nz);
  const double reliable = 32.0 * 0x1.0p-46 * sqrt((double)k);
  double est, contr;
  if (rho > reliable) {
    if (st.prev_s > 0) st.contr = fmin(rho / st.prev_rho, 0.999);
    st.prev_rho = rho;
    st.prev_s = s;
    st.floor_hits = 0;
    est = rho;
    contr = st.contr;
  } else if (st.prev_s > 0 && st.contr > 0.0) {
    est = st.prev_rho * pow(st.contr, (double)(s - st.prev_s));
    contr = st.contr;
  } else if (st.prev_s > 0) {
    est = rho;
    contr = fmin(reliable / st.prev_rho, 0.999);   // at most the fall onto the floor
  } else {
    // at the floor with no history: W^H W leaves span(P) invariant to the
    // products' accuracy; twice in a row settles it
    return ++st.floor_hits >= 2 || 4.0 * rho * kap2 <= kAngleTol;
  }
  const double angle = 4.0 * est * kap2;
  if (angle <= kAngleTol) return true;
  return contr > 0.0 && angle * contr <= kAngleTol;
}

__global__ void __launch_bounds__(kRfThreads, 1) k_pinv_refine(const __grid_constant__ RfArgs a) {
  extern __shared__ __align__(16) unsigned char smr[];
  __shared__ int stop_sh;
  const int vb = blockIdx.x, vg = gridDim.x;
  const int r = a.r, c = a.c, k = a.k;
  unsigned target = 0;
  // random start block P0 (entries uniform in [-1/2, 1/2), Philox counters)
  for (int64_t e = (int64_t)vb * blockDim.x + threadIdx.x; e < (int64_t)c * k;
       e += (int64_t)vg * blockDim.x) {
    const uint4 x = rf_philox(make_uint4((unsigned)e, (unsigned)(e >> 32), 0x52u, 0x46u),
                              make_uint2((unsigned)a.seed, (unsigned)(a.seed >> 32)));
    const int64_t off = (e / k) * a.P[0].ld + e % k;
    stq64(a.P[0], off, Q64{(double)x.x * 0x1.0p-32 - 0.5, (double)x.y * 0x1.0p-32 - 0.5,
                           (double)x.z * 0x1.0p-32 - 0.5, (double)x.w * 0x1.0p-32 - 0.5});
  }
  if (!rf_sync(a, target)) return;
  RfJob jb[3];
  jb[0] = job(a.W, 0, a.P[0], 0, a.Y, r, k, c);   // Y = W P0
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  StopState st{0.0, 0, 0.0, 0};
  int cur = 0, s = 1;
  bool converged = false;
  for (; s <= a.max_iter; ++s) {
    const QPtr& P = a.P[cur];
    const QPtr& Pn = a.P[cur ^ 1];
    jb[0] = job(a.W, 1, a.Y, 0, a.Z, c, k, r);   // Z = W^H Y
    plan_jobs(jb, 1, a.workers);
    rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
    if (!rf_sync(a, target)) return;
    jb[0] = job(P, 1, a.Z, 0, a.M, k, k, c);     // M = P^H Z
    jb[1] = job(P, 1, P, 0, a.E, k, k, c);       // E = P^H P - I
    jb[1].minus_eye = 1;
    plan_jobs(jb, 2, a.workers);
    rf_gemm_step(a, jb, 2, nullptr, vb, vg, smr);
    if (!rf_sync(a, target)) return;
    // Z' = Z R_Y^-1 with R_Y = chol32(M); then M' = M - E M on the tile workers
    rf_solve_step(a, a.M, a.Z, a.Zp, c, nullptr, nullptr, 0, a.kap2 + s, vb, vg, smr);
    jb[0] = job(a.E, 0, a.M, 0, a.Mp, k, k, k);
    jb[0].Zin = a.M;
    jb[0].alpha = -1.0;
    jb[0].beta = 1.0;
    jb[0].fp64 = 1;
    plan_jobs(jb, 1, a.workers);
    rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
    if (!rf_sync(a, target)) return;
    jb[0] = job(a.Zp, 1, a.Zp, 0, a.Gp, k, k, c);   // G' = Z'^H Z'
    jb[1] = job(P, 0, a.Mp, 0, a.Z, c, k, k);       // ||Z - P M'||, ||Z||
    jb[1].norm = 1;
    jb[1].fp64 = 1;   // its cancellation sets the floor of rho
    plan_jobs(jb, 2, a.workers);
    rf_gemm_step(a, jb, 2, a.norms + 2 * s, vb, vg, smr);
    if (!rf_sync(a, target)) return;
    if (threadIdx.x == 0)
      stop_sh = stop_now(st, s, __ldcg(a.norms + 2 * s), __ldcg(a.norms + 2 * s + 1),
                         __ldcg(a.kap2 + s), k);
    __syncthreads();
    converged = stop_sh != 0;
    rf_solve_step(a, a.Gp, a.Zp, Pn, c, nullptr, nullptr, 0, nullptr, vb, vg, smr);   // P <- Z' R'^-1
    if (!rf_sync(a, target)) return;
    jb[0] = job(a.W, 0, Pn, 0, a.Y, r, k, c);    // Y = W P
    plan_jobs(jb, 1, a.workers);
    rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
    if (!rf_sync(a, target)) return;
    cur ^= 1;
    if (converged) break;
  }
  const QPtr& P = a.P[cur];
  // U = P (W P)^+ by CholeskyQR2 with FP32 factors and the E2 correction
  jb[0] = job(a.Y, 1, a.Y, 0, a.G1, k, k, r);
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  rf_solve_step(a, a.G1, a.Y, a.Q1, r, &P, &a.T1, c, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  jb[0] = job(a.Q1, 1, a.Q1, 0, a.G2, k, k, r);
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  rf_solve_step(a, a.G2, a.Q1, a.Q2, r, &a.T1, &a.T2, c, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  jb[0] = job(a.Q2, 1, a.Q2, 0, a.E2, k, k, r);
  jb[0].minus_eye = 1;
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  jb[0] = job(a.T2, 0, a.E2, 0, a.V, c, k, k);   // V = T2 - T2 E2
  jb[0].Zin = a.T2;
  jb[0].alpha = -1.0;
  jb[0].beta = 1.0;
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (!rf_sync(a, target)) return;
  jb[0] = job(a.V, 0, a.Q2, 1, a.U, c, r, k);    // U = V Q2^H
  plan_jobs(jb, 1, a.workers);
  rf_gemm_step(a, jb, 1, nullptr, vb, vg, smr);
  if (vb == 0 && threadIdx.x == 0) {
    const int iters = s <= a.max_iter ? s : a.max_iter;
    if (a.rank_out != nullptr) { a.rank_out[0] = k; a.rank_out[1] = iters; }
    if (!converged) set_status(a.status, QMCUR_ERR_NO_CONVERGENCE);
  }
}

QPtr carve64(Carve& cv, int64_t rows, int64_t cols) {
  QPtr q;
  const int64_t ld = (cols + 1) / 2 * 2;
  double* base = cv.take<double>((size_t)(4 * rows * ld));
  for (int t = 0; t < 4; ++t) q.p[t] = base ? base + (size_t)t * rows * ld : nullptr;
  q.ld = ld;
  q.dtype = QMCUR_F64;
  return q;
}

struct RfWs {
  RfArgs a;
  unsigned* zero_base;   // counters and barrier words, zeroed before the launch
  size_t zero_bytes;
};

RfWs carve_refine(Carve& cv, int64_t r, int64_t c, int64_t k) {
  RfWs w{};
  RfArgs& a = w.a;
  a.P[0] = carve64(cv, c, k);
  a.P[1] = carve64(cv, c, k);
  a.Y = carve64(cv, r, k);
  a.Z = carve64(cv, c, k);
  a.Zp = carve64(cv, c, k);
  a.M = carve64(cv, k, k);
  a.E = carve64(cv, k, k);
  a.Mp = carve64(cv, k, k);
  a.Gp = carve64(cv, k, k);
  a.G1 = carve64(cv, k, k);
  a.G2 = carve64(cv, k, k);
  a.E2 = carve64(cv, k, k);
  a.Q1 = carve64(cv, r, k);
  a.Q2 = carve64(cv, r, k);
  a.T1 = carve64(cv, c, k);
  a.T2 = carve64(cv, c, k);
  a.V = carve64(cv, c, k);
  a.part = cv.take<Q64>((size_t)kRfMaxParts * kRfTileThreads);
  a.normpart = cv.take<double>((size_t)2 * kRfMaxTiles);
  a.norms = cv.take<double>((size_t)2 * (kRfMaxIter + 1));
  a.kap2 = cv.take<double>((size_t)(kRfMaxIter + 1));
  w.zero_base = cv.take<unsigned>((size_t)(kRfMaxTiles + 8));
  w.zero_bytes = (size_t)(kRfMaxTiles + 8) * sizeof(unsigned);
  a.cnt = w.zero_base;
  a.bar = w.zero_base + kRfMaxTiles + 4;
  return w;
}

}  // namespace

size_t pinv_refine_ws_bytes(int64_t r, int64_t c, int64_t k) {
  Carve cv(nullptr, 0);
  carve_refine(cv, r, c, k);
  return cv.off;
}

// U = W_k^+ (k = min(rank_cap, r, c)) by the refined subspace method above.
// max_iter <= 0 selects 30 iterations at most.
qmcur_status launch_pinv_refine(const qmcur_qmat* W, double rcond, int32_t rank_cap,
                                int32_t max_iter, qmcur_qmat* U, int32_t* rank_out, uint64_t seed,
                                void* ws, size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!valid_qmat(W) || !valid_qmat(U)) return QMCUR_ERR_INVALID_ARG;
  const int64_t r = W->rows, c = W->cols;
  if (r < 1 || c < 1 || U->rows != c || U->cols != r) return QMCUR_ERR_INVALID_ARG;
  if (!(rcond >= 0.0)) return QMCUR_ERR_INVALID_ARG;
  // the method keeps exactly k singular values; it certifies sigma_k / sigma_1
  // only down to ~1e-4 (its FP32 factors), so a larger rcond could cut below k
  if (rank_cap < 1 || rcond > 1e-6) return QMCUR_ERR_UNSUPPORTED;
  const int64_t nmin = r < c ? r : c;
  const int k = (int)(rank_cap < nmin ? rank_cap : nmin);
  if (k > kSmallCholMax || r > kRfMaxDim || c > kRfMaxDim) return QMCUR_ERR_UNSUPPORTED;
  if (max_iter <= 0) max_iter = 30;
  if (max_iter > kRfMaxIter) max_iter = kRfMaxIter;
  Carve cv(ws, ws_bytes);
  RfWs w = carve_refine(cv, r, c, k);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      dev < 0 || dev >= 64)
    return QMCUR_ERR_CUDA;
  static bool attr_set[64] = {};
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_pinv_refine, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rf_smem(kSmallCholMax)) != cudaSuccess)
      return QMCUR_ERR_CUDA;
    attr_set[dev] = true;
  }
  const size_t smem = rf_smem(k);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pinv_refine, kRfThreads, smem) !=
      cudaSuccess)
    return QMCUR_ERR_CUDA;
  if (per_sm < 1) return QMCUR_ERR_CUDA;
  const int grid = cta_cap(sms);
  RfArgs& a = w.a;
  for (int t = 0; t < 4; ++t) a.W.p[t] = W->plane[t];
  a.W.ld = W->ld;
  a.W.dtype = W->dtype;
  for (int t = 0; t < 4; ++t) a.U.p[t] = U->plane[t];
  a.U.ld = U->ld;
  a.U.dtype = U->dtype;
  a.r = (int)r;
  a.c = (int)c;
  a.k = k;
  a.max_iter = max_iter;
  a.seed = seed;
  a.status = dev_status;
  a.rank_out = rank_out;
  a.workers = grid * kRfWorkers;
  if (cudaMemsetAsync(w.zero_base, 0, w.zero_bytes, st) != cudaSuccess) return QMCUR_ERR_CUDA;
  void* args[] = {(void*)&a};
  return cuda_ok(cudaLaunchCooperativeKernel((const void*)k_pinv_refine, dim3(grid),
                                             dim3(kRfThreads), args, smem, st));
}

}  // namespace qmcur
