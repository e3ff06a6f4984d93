// Rank-capped pseudo-inverse U = W_k^+ to FP64-level accuracy on GB300, whose
// FP64 units run at 1/64 of its FP32 rate (about 2 FP64 FMA per clock per SM).
//
// The truncated inverse of Sec. 2.2 / Algorithm 1 keeps the k = rank_cap
// largest singular triplets of W (r x c): U = V_k Sigma_k^-1 P_k^H.  It only
// depends on the top-k right singular subspace S = span(V_k): for ANY basis
// P of S (full column rank, not necessarily orthonormal),
//   U = P (W P)^+,
// because W P = P_k Sigma_k (V_k^H P) and (V_k^H P) is invertible.  So the
// method finds S to working accuracy by subspace iteration and never factors
// anything in high precision: every k x k Cholesky factor is taken in FP32
// (one CTA, shared memory) and used only as a right preconditioner, Z R^-1
// with the FP32 R applied in the working precision.  Such a solve changes the
// basis but not its span, so the FP32 rounding of R never reaches the
// result; it only leaves the bases orthonormal to FP32 accuracy, and the one
// place where orthonormality matters (the final Q^+ = Q^H) is corrected to
// first order with the Gram matrix E = Q^H Q - I.
//
// Working precision: float-float on the FP32 pipe.  Every intermediate matrix
// is stored as an unevaluated pair of FP32 values per entry (h, l), h = fl(h +
// l), about 48 significant bits; products accumulate exactly-rounded FP32
// products and sums with their error terms (TwoProd by FMA and Knuth's
// TwoSum, as in the compensated dot product of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005), so that a
// product carries about 2^-46 of sum |x| |y|.  W is split into pairs once.
//
// Iteration s, from P (c x k, near-orthonormal) and Y = W P:
//   Z = W^H Y;  M = Y^H Y (= P^H Z);  E = P^H P - I
//   R_Y = chol32(M);  Z' = Z R_Y^-1      (= W^H Q with Q = Y R_Y^-1, the left
//                                         basis normalised);  M' = M - E M
//                                        (P (I - E) P^H: the projector on
//                                         span P to first order in E)
//   G' = Z'^H Z';  X = W Z';  rho_s = ||Z - P M'||_F / ||Z||_F
//   R' = chol32(G');  P <- Z' R'^-1;  Y <- X R'^-1 (= W P)
// rho_s measures how far W^H W moves span(P); times kappa^2 (kappa^2 taken
// from the diagonal of R_Y, whose Gram M ~ Sigma_k^2) it bounds the angle of
// span(P) to S, and the angle shrinks by (sigma_{k+1} / sigma_k)^2 per
// iteration.  The iteration stops when the predicted angle of the new P is
// below kAngleTol (extrapolated at the observed contraction once rho_s
// reaches its rounding floor), or after max_iter iterations
// (QMCUR_ERR_NO_CONVERGENCE: the spectrum has no usable gap at k).
//
// Then U = P (W P)^+ by CholeskyQR2 with FP32 factors:
//   G1 = Y^H Y;  R1 = chol32(G1);  Q1 = Y R1^-1, T1 = P R1^-1
//   G2 = Q1^H Q1;  R2 = chol32(G2);  Q2 = Q1 R2^-1, T2 = T1 R2^-1
//                                            (Y = Q2 R2 R1, P = T2 R2 R1)
//   E2 = Q2^H Q2 - I;  V = T2 - T2 E2 ~ T2 (I + E2)^-1;  U = V Q2^H,
// i.e. U = T2 Q2^+ = P (R2 R1)^-1 Q2^+ = P Y^+, with ||E2|| ~ u32 ||E1||, so
// that the first-order correction leaves O(||E2||^2) behind.
//
// Everything runs in ONE cooperative persistent kernel of one 512-thread CTA
// per SM, with a bounded grid barrier between steps (4 per iteration).  A
// product step cuts its products into (8 x 8 output tile, 16-deep k-slice)
// units and deals each of the 8 x SMs tile workers (64 threads, one per tile
// entry, each carrying the quaternion's four components) one contiguous run
// of units, so every worker gets the same work to within one slice; a tile
// split over several runs sums their partials in k order (the last run to
// arrive does it), so results do not depend on timing.  In a solve step
// every CTA that holds rows factors the Gram matrix itself (identical
// arithmetic, identical factors, no barrier) and solves its rows, one warp
// per row.  Every CTA evaluates the stopping rule itself from the same global
// values, so all take the same branch.
#include "small_impl.cuh"

namespace qmcur {
namespace {

constexpr int kRfThreads = kCholThreads;             // 512
constexpr int kRfTileThreads = 64;                   // a worker: one thread per tile entry
constexpr int kRfWorkers = kRfThreads / kRfTileThreads;
constexpr int kRfTS = 8;                             // output tile edge (quaternions)
constexpr int kRfBK = 16;                            // k-slice
constexpr int kRfMaxGrid = 160;                      // CTAs at most (one per SM)
constexpr int kRfMaxWorkers = kRfMaxGrid * kRfWorkers;
constexpr int kRfMaxTiles = 32768;                   // tiles of the norm product
constexpr int kRfMaxDim = 16384;                     // r, c at most
constexpr int kRfMaxIter = 64;
constexpr double kAngleTol = 1e-14;                  // target angle of span(P) to S
constexpr float kCholShift = 1e-5f;                  // relative diagonal shift of a retried factor

static_assert(kRfWorkers * kRfTileThreads == kRfThreads, "whole tile workers");
static_assert(kRfTS * kRfTS == kRfTileThreads, "one thread per tile entry");
static_assert((kRfMaxDim + kRfTS - 1) / kRfTS * ((kSmallCholMax + kRfTS - 1) / kRfTS) <= kRfMaxTiles,
              "norm tiles");

// ---------------------------------------------------------------------------
// Float-float arithmetic.  A pair (h, l) stands for h + l.  The rn
// intrinsics keep the compiler from fusing a rounded product into a later
// add, which would break the error terms.

struct __align__(16) QFF { float4 h, l; };   // one quaternion entry as pairs

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// (h, l) = the pair of s + c, renormalised
__device__ __forceinline__ void ff_norm(float s, float c, float& h, float& l) {
  float e;
  two_sum(s, c, h, e);
  l = e;
}

// r = a + b
__device__ __forceinline__ void ff_add1(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  two_sum(ah, bh, s, e);
  ff_norm(s, __fadd_rn(__fadd_rn(al, bl), e), rh, rl);
}

__device__ __forceinline__ QFF qff_zero() {
  return QFF{make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
}

__device__ __forceinline__ QFF qff_conj(QFF v) {
  v.h.y = -v.h.y; v.h.z = -v.h.z; v.h.w = -v.h.w;
  v.l.y = -v.l.y; v.l.z = -v.l.z; v.l.w = -v.l.w;
  return v;
}

__device__ __forceinline__ QFF qff_add(const QFF& a, const QFF& b) {
  QFF r;
  ff_add1(a.h.x, a.l.x, b.h.x, b.l.x, r.h.x, r.l.x);
  ff_add1(a.h.y, a.l.y, b.h.y, b.l.y, r.h.y, r.l.y);
  ff_add1(a.h.z, a.l.z, b.h.z, b.l.z, r.h.z, r.l.z);
  ff_add1(a.h.w, a.l.w, b.h.w, b.l.w, r.h.w, r.l.w);
  return r;
}

__device__ __forceinline__ QFF qff_neg(QFF a) {
  a.h = make_float4(-a.h.x, -a.h.y, -a.h.z, -a.h.w);
  a.l = make_float4(-a.l.x, -a.l.y, -a.l.z, -a.l.w);
  return a;
}

// Loads and stores: kDtypeFF planes hold float2 (h, l) per entry; F64 and F32
// planes (the caller's W and U, the FP32 factor inverses) are split / rounded
// on the way.
__device__ __forceinline__ QFF ldff(const QPtr& q, int64_t off) {
  QFF v;
  if (q.dtype == kDtypeFF) {
    const float2 a = reinterpret_cast<const float2*>(q.p[0])[off];
    const float2 b = reinterpret_cast<const float2*>(q.p[1])[off];
    const float2 c = reinterpret_cast<const float2*>(q.p[2])[off];
    const float2 d = reinterpret_cast<const float2*>(q.p[3])[off];
    v.h = make_float4(a.x, b.x, c.x, d.x);
    v.l = make_float4(a.y, b.y, c.y, d.y);
  } else if (q.dtype == QMCUR_F64) {
    float hh[4], ll[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const double x = reinterpret_cast<const double*>(q.p[t])[off];
      hh[t] = __double2float_rn(x);
      ll[t] = __double2float_rn(x - (double)hh[t]);
    }
    v.h = make_float4(hh[0], hh[1], hh[2], hh[3]);
    v.l = make_float4(ll[0], ll[1], ll[2], ll[3]);
  } else {
    v.h = make_float4(reinterpret_cast<const float*>(q.p[0])[off],
                      reinterpret_cast<const float*>(q.p[1])[off],
                      reinterpret_cast<const float*>(q.p[2])[off],
                      reinterpret_cast<const float*>(q.p[3])[off]);
    v.l = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  return v;
}

__device__ __forceinline__ void stff(const QPtr& q, int64_t off, const QFF& v) {
  if (q.dtype == kDtypeFF) {
    reinterpret_cast<float2*>(q.p[0])[off] = make_float2(v.h.x, v.l.x);
    reinterpret_cast<float2*>(q.p[1])[off] = make_float2(v.h.y, v.l.y);
    reinterpret_cast<float2*>(q.p[2])[off] = make_float2(v.h.z, v.l.z);
    reinterpret_cast<float2*>(q.p[3])[off] = make_float2(v.h.w, v.l.w);
  } else if (q.dtype == QMCUR_F64) {
    reinterpret_cast<double*>(q.p[0])[off] = (double)v.h.x + (double)v.l.x;
    reinterpret_cast<double*>(q.p[1])[off] = (double)v.h.y + (double)v.l.y;
    reinterpret_cast<double*>(q.p[2])[off] = (double)v.h.z + (double)v.l.z;
    reinterpret_cast<double*>(q.p[3])[off] = (double)v.h.w + (double)v.l.w;
  } else {
    reinterpret_cast<float*>(q.p[0])[off] = __fadd_rn(v.h.x, v.l.x);
    reinterpret_cast<float*>(q.p[1])[off] = __fadd_rn(v.h.y, v.l.y);
    reinterpret_cast<float*>(q.p[2])[off] = __fadd_rn(v.h.z, v.l.z);
    reinterpret_cast<float*>(q.p[3])[off] = __fadd_rn(v.h.w, v.l.w);
  }
}

// One product of a step: Zout = alpha op(X) op(Y) + beta Zin - [minus_eye] I,
// alpha in {1, -1}, beta in {0, 1}; op(X) M x K (X stored K x M when xh:
// op(X) = X^H), op(Y) K x N likewise.  With norm, nothing is stored: the step
// folds ||Zin - op(X) op(Y)||_F^2 and ||Zin||_F^2 into norm_out[0..1] (fixed
// order).  With upper, only the tiles on and above the diagonal are formed
// (a Hermitian result that is read through its upper triangle).
struct RfJob {
  QPtr X, Y, Zin, Zout;
  int M, N, K;
  int xh, yh;
  int neg;              // alpha = -1
  int add_in;           // beta = 1
  int minus_eye;
  int norm;
  int upper;
  int fp32;             // plain FP32 products of the leading parts (stored with l = 0)
  float scale;          // exact power of two applied to the stored result (0: none)
  QPtr Zout2;           // a second copy of the stored result (p[0] null: none)
  // filled by rf_plan
  int tm, tn;           // tile rows, tile columns
  int slices;           // k-slices of a full-depth tile
  int units, ubase;     // units of the job, first unit in the step
};

struct RfArgs {
  QPtr W;              // r x c input (F32 or F64 planes)
  QPtr Wf;             // W as pairs
  int r, c, k;
  int max_iter;
  uint64_t seed;
  // float-float workspaces
  QPtr P[2], Y, Z, Zp, X, M, E, Mp, Gp, G1, G2, E2, Q1, Q2, T1, T2, V;
  QPtr U;              // c x r output
  QPtr U2;             // optional second copy of U (p[0] null: none), e.g. F32 beside F64
  QFF* part;           // 2 x kRfMaxWorkers x kRfTileThreads partials of split tiles
  unsigned* cnt;       // kRfMaxWorkers split-tile arrival counts, then the norm fold's
  double* normpart;    // kRfMaxTiles x 2 tile norm partials
  double* norms;       // (kRfMaxIter + 1) x 2
  double* kap2;        // kRfMaxIter + 1
  unsigned* bar;       // grid barrier words
  unsigned* wmax;      // bits of max |W_ij| over the planes (atomicMax, zeroed)
  int32_t* status;
  int32_t* rank_out;
  int workers;         // tile workers of the (virtual) grid: CTAs x kRfWorkers
};

// Shared memory: the tile workers' double-buffered operand slices, or the
// packed factor and the Cholesky buffers.
constexpr int kRfWorkerQ = 2 * kRfTS * (kRfBK + 1) + 2 * kRfBK * (kRfTS + 1);
constexpr size_t rf_chol_off(int k) { return (sm_trsm_bytes(k) + 15) / 16 * 16; }
constexpr size_t rf_smem(int k) {
  const size_t g = (size_t)kRfWorkers * kRfWorkerQ * sizeof(QFF);
  const size_t f = rf_chol_off(k) + sm_chol_bytes();
  return g > f ? g : f;
}

// ---------------------------------------------------------------------------
// Products.

__device__ __forceinline__ void worker_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kRfTileThreads) : "memory");
}

// The four real products of one quaternion component, added into (S, C):
// p_i = sg_i a_i b_i exactly as (p_i, e_i); the four are summed pairwise with
// their errors before one TwoSum into S, which keeps the dependency chain
// through S one TwoSum long per k step; the cross terms a_h b_l + a_l b_h go
// to C in FP32.
template <int S0, int S1, int S2, int S3>
__device__ __forceinline__ void ff_comp4(float& S, float& C, float a0, float a0l, float b0,
                                         float b0l, float a1, float a1l, float b1, float b1l,
                                         float a2, float a2l, float b2, float b2l, float a3,
                                         float a3l, float b3, float b3l) {
  const float x0 = S0 > 0 ? a0 : -a0, x1 = S1 > 0 ? a1 : -a1;
  const float x2 = S2 > 0 ? a2 : -a2, x3 = S3 > 0 ? a3 : -a3;
  const float y0 = S0 > 0 ? a0l : -a0l, y1 = S1 > 0 ? a1l : -a1l;
  const float y2 = S2 > 0 ? a2l : -a2l, y3 = S3 > 0 ? a3l : -a3l;
  const float p0 = __fmul_rn(x0, b0), p1 = __fmul_rn(x1, b1);
  const float p2 = __fmul_rn(x2, b2), p3 = __fmul_rn(x3, b3);
  float c = __fmaf_rn(x0, b0, -p0);
  c = __fadd_rn(c, __fmaf_rn(x1, b1, -p1));
  c = __fadd_rn(c, __fmaf_rn(x2, b2, -p2));
  c = __fadd_rn(c, __fmaf_rn(x3, b3, -p3));
  float s01, e01, s23, e23, s, e;
  two_sum(p0, p1, s01, e01);
  two_sum(p2, p3, s23, e23);
  two_sum(s01, s23, s, e);
  float sn, en;
  two_sum(S, s, sn, en);
  S = sn;
  c = __fadd_rn(c, __fadd_rn(__fadd_rn(e01, e23), __fadd_rn(e, en)));
  c = __fmaf_rn(x0, b0l, c); c = __fmaf_rn(y0, b0, c);
  c = __fmaf_rn(x1, b1l, c); c = __fmaf_rn(y1, b1, c);
  c = __fmaf_rn(x2, b2l, c); c = __fmaf_rn(y2, b2, c);
  c = __fmaf_rn(x3, b3l, c); c = __fmaf_rn(y3, b3, c);
  C = __fadd_rn(C, c);
}

// The operands of one product as a tile worker reads them.
struct RfOp {
  QPtr X, Y;
  int M, N, xh, yh;
};

// (S, C) += x y, the Hamilton product (Sec. 2.2) in float-float
__device__ __forceinline__ void ff_qmac(float S[4], float C[4], const QFF& x, const QFF& y) {
  const float4 a = x.h, al = x.l, b = y.h, bl = y.l;
  // z0 = x0 y0 - x1 y1 - x2 y2 - x3 y3
  ff_comp4<+1, -1, -1, -1>(S[0], C[0], a.x, al.x, b.x, bl.x, a.y, al.y, b.y, bl.y, a.z, al.z, b.z,
                           bl.z, a.w, al.w, b.w, bl.w);
  // z1 = x0 y1 + x1 y0 + x2 y3 - x3 y2
  ff_comp4<+1, +1, +1, -1>(S[1], C[1], a.x, al.x, b.y, bl.y, a.y, al.y, b.x, bl.x, a.z, al.z, b.w,
                           bl.w, a.w, al.w, b.z, bl.z);
  // z2 = x0 y2 - x1 y3 + x2 y0 + x3 y1
  ff_comp4<+1, -1, +1, +1>(S[2], C[2], a.x, al.x, b.z, bl.z, a.y, al.y, b.w, bl.w, a.z, al.z, b.x,
                           bl.x, a.w, al.w, b.y, bl.y);
  // z3 = x0 y3 + x1 y2 - x2 y1 + x3 y0
  ff_comp4<+1, +1, -1, +1>(S[3], C[3], a.x, al.x, b.w, bl.w, a.y, al.y, b.z, bl.z, a.z, al.z, b.y,
                           bl.y, a.w, al.w, b.x, bl.x);
}

// S += x y in plain FP32 on the leading parts (the Hamilton product, Sec. 2.2)
__device__ __forceinline__ void f32_qmac(float S[4], const QFF& x, const QFF& y) {
  const float4 a = x.h, b = y.h;
  S[0] = __fmaf_rn(a.x, b.x, S[0]); S[0] = __fmaf_rn(-a.y, b.y, S[0]);
  S[0] = __fmaf_rn(-a.z, b.z, S[0]); S[0] = __fmaf_rn(-a.w, b.w, S[0]);
  S[1] = __fmaf_rn(a.x, b.y, S[1]); S[1] = __fmaf_rn(a.y, b.x, S[1]);
  S[1] = __fmaf_rn(a.z, b.w, S[1]); S[1] = __fmaf_rn(-a.w, b.z, S[1]);
  S[2] = __fmaf_rn(a.x, b.z, S[2]); S[2] = __fmaf_rn(-a.y, b.w, S[2]);
  S[2] = __fmaf_rn(a.z, b.x, S[2]); S[2] = __fmaf_rn(a.w, b.y, S[2]);
  S[3] = __fmaf_rn(a.x, b.w, S[3]); S[3] = __fmaf_rn(a.y, b.z, S[3]);
  S[3] = __fmaf_rn(-a.z, b.y, S[3]); S[3] = __fmaf_rn(a.w, b.x, S[3]);
}

// Entry (ty, tx) = (tid / 8, tid % 8) of tile (tm, tn), accumulated over
// [kb, ke) by one worker; the thread carries the four components (four
// independent dependency chains).  Slices are double-buffered (one barrier
// per slice); each thread loads two entries of the X slice and two of the Y
// slice, laid out so that consecutive threads read consecutive addresses of
// the operand's storage.
// With FF false the products are plain FP32 on the leading parts.
template <bool FF>
__device__ __noinline__ QFF rf_tile_acc(const RfOp op, int tm, int tn, int kb, int ke, QFF* sm,
                                        int tid, int bar_id) {
  QFF (*xs)[kRfTS][kRfBK + 1] = reinterpret_cast<QFF (*)[kRfTS][kRfBK + 1]>(sm);
  QFF (*ys)[kRfBK][kRfTS + 1] =
      reinterpret_cast<QFF (*)[kRfBK][kRfTS + 1]>(sm + 2 * kRfTS * (kRfBK + 1));
  const int ty = tid / kRfTS, tx = tid % kRfTS;
  const int xl_along = !op.xh, yl_along = op.yh;   // storage contiguous along l
  int xi[2], xk[2], yj[2], yk[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int e = tid + u * kRfTileThreads;   // 0 .. 127
    xi[u] = xl_along ? (e >> 4) : (e & 7);
    xk[u] = xl_along ? (e & 15) : (e >> 3);
    yj[u] = yl_along ? (e >> 4) : (e & 7);
    yk[u] = yl_along ? (e & 15) : (e >> 3);
  }
  const int m0 = tm * kRfTS, n0 = tn * kRfTS;
  auto ldx = [&](int l0, int u) -> QFF {
    const int i = m0 + xi[u], l = l0 + xk[u];
    if (i >= op.M || l >= ke) return qff_zero();
    if (!op.xh) return ldff(op.X, (int64_t)i * op.X.ld + l);
    return qff_conj(ldff(op.X, (int64_t)l * op.X.ld + i));
  };
  auto ldy = [&](int l0, int u) -> QFF {
    const int j = n0 + yj[u], l = l0 + yk[u];
    if (j >= op.N || l >= ke) return qff_zero();
    if (!op.yh) return ldff(op.Y, (int64_t)l * op.Y.ld + j);
    return qff_conj(ldff(op.Y, (int64_t)j * op.Y.ld + l));
  };
  QFF vx0 = ldx(kb, 0), vx1 = ldx(kb, 1), vy0 = ldy(kb, 0), vy1 = ldy(kb, 1);
  xs[0][xi[0]][xk[0]] = vx0;
  xs[0][xi[1]][xk[1]] = vx1;
  ys[0][yk[0]][yj[0]] = vy0;
  ys[0][yk[1]][yj[1]] = vy1;
  worker_bar(bar_id);
  float S[4] = {0.f, 0.f, 0.f, 0.f}, C[4] = {0.f, 0.f, 0.f, 0.f};
  int b = 0;
  for (int k0 = kb; k0 < ke; k0 += kRfBK, b ^= 1) {
    const bool more = k0 + kRfBK < ke;
    if (more) {
      vx0 = ldx(k0 + kRfBK, 0);
      vx1 = ldx(k0 + kRfBK, 1);
      vy0 = ldy(k0 + kRfBK, 0);
      vy1 = ldy(k0 + kRfBK, 1);
    }
    const QFF* xr = xs[b][ty];
    const QFF (*yr)[kRfTS + 1] = ys[b];
    const int lend = ke - k0 < kRfBK ? ke - k0 : kRfBK;
    if (!FF) {
#pragma unroll 4
      for (int l = 0; l < lend; ++l) f32_qmac(S, xr[l], yr[l][tx]);
    } else if (lend == kRfBK) {
#pragma unroll 2
      for (int l = 0; l < kRfBK; ++l) ff_qmac(S, C, xr[l], yr[l][tx]);
    } else {
      for (int l = 0; l < lend; ++l) ff_qmac(S, C, xr[l], yr[l][tx]);
    }
    if (more) {
      xs[b ^ 1][xi[0]][xk[0]] = vx0;
      xs[b ^ 1][xi[1]][xk[1]] = vx1;
      ys[b ^ 1][yk[0]][yj[0]] = vy0;
      ys[b ^ 1][yk[1]][yj[1]] = vy1;
    }
    worker_bar(bar_id);   // the next slice is stored; this one is no longer read
  }
  QFF acc;
  ff_norm(S[0], C[0], acc.h.x, acc.l.x);
  ff_norm(S[1], C[1], acc.h.y, acc.l.y);
  ff_norm(S[2], C[2], acc.h.z, acc.l.z);
  ff_norm(S[3], C[3], acc.h.w, acc.l.w);
  return acc;
}

// Epilogue of one finished tile entry: store, or the norm partials (of the
// leading parts: only the size of rho matters).
__device__ void rf_epilogue(const RfJob& j, int tm, int tn, int tid, const QFF& acc, double* nd,
                            double* nz) {
  const int i = tm * kRfTS + tid / kRfTS, c = tn * kRfTS + tid % kRfTS;
  if (i >= j.M || c >= j.N) return;
  const int64_t oin = (int64_t)i * j.Zin.ld + c;
  if (j.norm) {
    const QFF z = ldff(j.Zin, oin);
    const QFF d = qff_add(z, qff_neg(acc));
    const double dx = d.h.x, dy = d.h.y, dz = d.h.z, dw = d.h.w;
    const double zx = z.h.x, zy = z.h.y, zz = z.h.z, zw = z.h.w;
    *nd += dx * dx + dy * dy + dz * dz + dw * dw;
    *nz += zx * zx + zy * zy + zz * zz + zw * zw;
    return;
  }
  QFF v = j.neg ? qff_neg(acc) : acc;
  if (j.add_in) v = qff_add(v, ldff(j.Zin, oin));
  if (j.minus_eye && i == c) ff_add1(v.h.x, v.l.x, -1.f, 0.f, v.h.x, v.l.x);
  if (j.scale != 0.f) {   // a power of two: exact
    v.h = make_float4(v.h.x * j.scale, v.h.y * j.scale, v.h.z * j.scale, v.h.w * j.scale);
    v.l = make_float4(v.l.x * j.scale, v.l.y * j.scale, v.l.z * j.scale, v.l.w * j.scale);
  }
  stff(j.Zout, (int64_t)i * j.Zout.ld + c, v);
  if (j.Zout2.p[0] != nullptr) stff(j.Zout2, (int64_t)i * j.Zout2.ld + c, v);
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

// Units of every job and their place in the step; returns the step's total.
__device__ int rf_plan(RfJob* jobs, int n) {
  int total = 0;
  for (int q = 0; q < n; ++q) {
    RfJob& j = jobs[q];
    j.tm = (j.M + kRfTS - 1) / kRfTS;
    j.tn = (j.N + kRfTS - 1) / kRfTS;
    j.slices = (j.K + kRfBK - 1) / kRfBK;
    if (j.upper) {
      j.units = 0;
      for (int t = 0; t < j.tm; ++t) j.units += (j.tn > t ? j.tn - t : 0) * j.slices;
    } else {
      j.units = j.tm * j.tn * j.slices;
    }
    j.ubase = total;
    total += j.units;
  }
  return total;
}

// Tile (tm, tn) and slice s of unit ul of a job.
__device__ __forceinline__ void rf_locate(const RfJob& j, int ul, int& tm, int& tn, int& s) {
  if (j.upper) {
    tm = 0;
    for (int ru = j.tn * j.slices; ul >= ru && tm + 1 < j.tm; ru = (j.tn - tm) * j.slices) {
      ul -= ru;
      ++tm;
    }
    tn = tm + ul / j.slices;
    s = ul % j.slices;
  } else {
    const int t = ul / j.slices;
    s = ul - t * j.slices;
    tm = t / j.tn;
    tn = t - tm * j.tn;
  }
}

// Worker w of nw takes units [rf_start(w), rf_start(w + 1)).
__device__ __forceinline__ int rf_start(int w, int nw, int total) {
  return (int)(((int64_t)w * total) / nw);
}

// The worker whose run holds unit x.
__device__ __forceinline__ int rf_owner(int x, int nw, int total) {
  return (int)((((int64_t)x + 1) * nw - 1) / total);
}

// One step of up to three independent products (at most one with `norm`).
// The workers of CTA vb of the virtual grid are workers kRfWorkers vb ..
// kRfWorkers (vb + 1) - 1, so that small steps spread over the SMs.  A run that covers a tile only in part leaves its
// partial in the slot of its first tile (2w) or of its last (2w + 1); the
// tile's counter is that of the worker holding its first unit (no other
// split tile starts in that worker's run), and the last run to arrive sums
// the partials in run order.
__device__ __noinline__ void rf_gemm_step(const RfArgs& a, RfJob* jobs, int njobs, double* norm_out,
                                          unsigned char* smem, int vb) {
  __shared__ int last_sh[kRfWorkers];
  __shared__ double red_sh[kRfWorkers][kRfTileThreads / 32];
  const int worker = threadIdx.x / kRfTileThreads, wtid = threadIdx.x % kRfTileThreads;
  QFF* wsm = reinterpret_cast<QFF*>(smem) + worker * kRfWorkerQ;
  const int bar_id = 1 + worker;
  const int total = rf_plan(jobs, njobs);
  const int nw = a.workers;
  const int w = kRfWorkers * vb + worker;
  const int u_begin = rf_start(w, nw, total), u_end = rf_start(w + 1, nw, total);
  for (int u = u_begin; u < u_end;) {
    int q = 0;
    while (q + 1 < njobs && u >= jobs[q + 1].ubase) ++q;
    const RfJob& j = jobs[q];
    int tm, tn, s;
    rf_locate(j, u - j.ubase, tm, tn, s);
    const int ns = j.slices;
    const int tile_u0 = u - s;
    const int s_end = ns < s + (u_end - u) ? ns : s + (u_end - u);
    const int ke = s_end * kRfBK < j.K ? s_end * kRfBK : j.K;
    const RfOp op{j.X, j.Y, j.M, j.N, j.xh, j.yh};
    QFF acc = j.fp32 ? rf_tile_acc<false>(op, tm, tn, s * kRfBK, ke, wsm, wtid, bar_id)
                     : rf_tile_acc<true>(op, tm, tn, s * kRfBK, ke, wsm, wtid, bar_id);
    u += s_end - s;
    if (s > 0 || s_end < ns) {   // a tile split over several runs
      // the runs holding the tile's units, in k order: from the owner of a
      // unit, the next run starts where that owner's ends (runs may be empty)
      const int wa = rf_owner(tile_u0, nw, total);
      int nseg = 0;
      for (int x = tile_u0; x < tile_u0 + ns; x = rf_start(rf_owner(x, nw, total) + 1, nw, total))
        ++nseg;
      const int slot = rf_start(w, nw, total) >= tile_u0 ? 2 * w : 2 * w + 1;
      a.part[(size_t)slot * kRfTileThreads + wtid] = acc;
      __threadfence();
      worker_bar(bar_id);
      if (wtid == 0) last_sh[worker] = atomicAdd(a.cnt + wa, 1u) == (unsigned)(nseg - 1);
      worker_bar(bar_id);
      if (!last_sh[worker]) continue;
      __threadfence();
      acc = qff_zero();
      for (int x = tile_u0; x < tile_u0 + ns;) {   // in k order; written by other SMs
        const int v = rf_owner(x, nw, total);
        const int sv = rf_start(v, nw, total) >= tile_u0 ? 2 * v : 2 * v + 1;
        const float4* p = reinterpret_cast<const float4*>(a.part + (size_t)sv * kRfTileThreads + wtid);
        acc = qff_add(acc, QFF{__ldcg(p), __ldcg(p + 1)});
        x = rf_start(v + 1, nw, total);
      }
      if (wtid == 0) a.cnt[wa] = 0u;   // ready for the next step
    }
    double nd = 0.0, nz = 0.0;
    rf_epilogue(j, tm, tn, wtid, acc, &nd, &nz);
    if (j.norm) {
      const int tile = tm * j.tn + tn;
      const double sd = rf_worker_sum(nd, red_sh[worker], wtid, bar_id);
      const double sz = rf_worker_sum(nz, red_sh[worker], wtid, bar_id);
      if (wtid == 0) {
        a.normpart[2 * tile] = sd;
        a.normpart[2 * tile + 1] = sz;
        __threadfence();
        last_sh[worker] = atomicAdd(a.cnt + nw, 1u) == (unsigned)(j.tm * j.tn - 1);
      }
      worker_bar(bar_id);
      if (last_sh[worker]) {   // the last tile folds them all: strided, then in thread order
        __threadfence();
        double fd = 0.0, fz = 0.0;
        for (int t = wtid; t < j.tm * j.tn; t += kRfTileThreads) {
          fd += __ldcg(a.normpart + 2 * t);
          fz += __ldcg(a.normpart + 2 * t + 1);
        }
        fd = rf_worker_sum(fd, red_sh[worker], wtid, bar_id);
        fz = rf_worker_sum(fz, red_sh[worker], wtid, bar_id);
        if (wtid == 0) {
          norm_out[0] = fd;
          norm_out[1] = fz;
          a.cnt[nw] = 0u;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Factors.

// ---------------------------------------------------------------------------
// Solves.

// (S, C) += sg (ah + al) b for an exact FP32 b (a factor entry)
template <int SG>
__device__ __forceinline__ void ff_mac1(float& S, float& C, float ah, float al, float b) {
  const float a = SG > 0 ? ah : -ah, a2 = SG > 0 ? al : -al;
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  float sn, err;
  two_sum(S, p, sn, err);
  S = sn;
  C = __fadd_rn(C, __fadd_rn(err, e));
  C = __fmaf_rn(a2, b, C);
}

// t -= z r in float-float, r an FP32 quaternion (Hamilton product z r)
__device__ __forceinline__ void ff_qmsub1(float4& th, float4& tl, const float4 zh, const float4 zl,
                                          const float4 r) {
  ff_mac1<-1>(th.x, tl.x, zh.x, zl.x, r.x); ff_mac1<+1>(th.x, tl.x, zh.y, zl.y, r.y);
  ff_mac1<+1>(th.x, tl.x, zh.z, zl.z, r.z); ff_mac1<+1>(th.x, tl.x, zh.w, zl.w, r.w);
  ff_mac1<-1>(th.y, tl.y, zh.x, zl.x, r.y); ff_mac1<-1>(th.y, tl.y, zh.y, zl.y, r.x);
  ff_mac1<-1>(th.y, tl.y, zh.z, zl.z, r.w); ff_mac1<+1>(th.y, tl.y, zh.w, zl.w, r.z);
  ff_mac1<-1>(th.z, tl.z, zh.x, zl.x, r.z); ff_mac1<+1>(th.z, tl.z, zh.y, zl.y, r.w);
  ff_mac1<-1>(th.z, tl.z, zh.z, zl.z, r.x); ff_mac1<-1>(th.z, tl.z, zh.w, zl.w, r.y);
  ff_mac1<-1>(th.w, tl.w, zh.x, zl.x, r.w); ff_mac1<-1>(th.w, tl.w, zh.y, zl.y, r.z);
  ff_mac1<+1>(th.w, tl.w, zh.z, zl.z, r.y); ff_mac1<-1>(th.w, tl.w, zh.w, zl.w, r.x);
}

// z = t s in float-float, s an exact FP32 scalar
__device__ __forceinline__ void ff_scale1(float& zh, float& zl, float th, float tl, float sc) {
  zh = __fmul_rn(th, sc);
  zl = __fmaf_rn(tl, sc, __fmaf_rn(th, sc, -zh));
}

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// One warp: row `row` of Z = Y R^-1 in float-float with the packed FP32
// factor R (R_ll taken as 1 / invd[l], so that every solve with this factor
// applies the same matrix); k <= 32 U.  Each column l: z_l = t_l / R_ll from
// its owner lane, then t_c -= z_l R_lc for the later columns of every lane.
template <int U>
__device__ void rf_trsm_row(const QPtr& Y, const QPtr& Z, int row, int k, const float* rpk) {
  const float4* Rs = reinterpret_cast<const float4*>(rpk);
  const float* invd = rpk + 4 * (k * (k + 1) / 2);
  const int lane = threadIdx.x & 31;
  float4 th[U], tl[U];
  const int64_t yo = (int64_t)row * Y.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    const QFF v = c < k ? ldff(Y, yo + c) : qff_zero();
    th[u] = v.h;
    tl[u] = v.l;
  }
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
    const int lend = k - 32 * uu < 32 ? k - 32 * uu : 32;
    for (int ll = 0; ll < lend; ++ll) {
      const int l = 32 * uu + ll;
      const float sc = invd[l];
      float4 zh, zl;
      ff_scale1(zh.x, zl.x, shfl_f(th[uu].x, ll), shfl_f(tl[uu].x, ll), sc);
      ff_scale1(zh.y, zl.y, shfl_f(th[uu].y, ll), shfl_f(tl[uu].y, ll), sc);
      ff_scale1(zh.z, zl.z, shfl_f(th[uu].z, ll), shfl_f(tl[uu].z, ll), sc);
      ff_scale1(zh.w, zl.w, shfl_f(th[uu].w, ll), shfl_f(tl[uu].w, ll), sc);
      const float4* Rrow = Rs + (packed_row(l, k) - l);   // R_l,c at Rrow + c, c >= l
#pragma unroll
      for (int u = uu; u < U; ++u) {
        const int c = lane + 32 * u;
        if (c > l && c < k) ff_qmsub1(th[u], tl[u], zh, zl, Rrow[c]);
      }
      if (lane == ll) { th[uu] = zh; tl[uu] = zl; }
    }
  }
  const int64_t zo = (int64_t)row * Z.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    if (c < k) {
      QFF v;
      ff_norm(th[u].x, tl[u].x, v.h.x, v.l.x);
      ff_norm(th[u].y, tl[u].y, v.h.y, v.l.y);
      ff_norm(th[u].z, tl[u].z, v.h.z, v.l.z);
      ff_norm(th[u].w, tl[u].w, v.h.w, v.l.w);
      stff(Z, zo + c, v);
    }
  }
}

__device__ __noinline__ void rf_trsm_row_any(const QPtr& Y, const QPtr& Z, int row, int k,
                                             const float* rpk) {
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
  return j;
}

// The barrier between steps: the grid's, or the CTA's own when the virtual
// grid is one CTA (vg == 1: one problem per CTA).
__device__ __forceinline__ bool rf_sync(const RfArgs& a, int vg, unsigned& target) {
  if (vg == 1) {
    __syncthreads();   // the CTA's own global writes, then its reads
    return true;
  }
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
// the fall from it onto the floor bounds the contraction, applied once per
// iteration since that value.  Iteration 1 starts from the random block, whose
// rho means nothing.
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
    // one reliable value, then the floor: the fall onto the floor bounds the
    // contraction, and every further iteration at the floor applies it again
    contr = fmin(reliable / st.prev_rho, 0.999);
    est = fmin(rho, st.prev_rho * pow(contr, (double)(s - st.prev_s)));
  } else {
    // at the floor with no history: W^H W leaves span(P) invariant to the
    // products' accuracy; twice in a row settles it
    return ++st.floor_hits >= 2 || 4.0 * rho * kap2 <= kAngleTol;
  }
  const double angle = 4.0 * est * kap2;
  if (angle <= kAngleTol) return true;
  return contr > 0.0 && angle * contr <= kAngleTol;
}

// The whole program over a virtual grid of vg CTAs, this one vb: the
// single-problem kernel passes (blockIdx.x, gridDim.x) and grid barriers;
// the batched kernel passes (0, 1) and CTA barriers.
__device__ __forceinline__ void rf_program(const RfArgs& a, int vb, int vg, unsigned char* smr) {
  __shared__ int stop_sh;
  const int r = a.r, c = a.c, k = a.k;
  unsigned target = 0;
  if (vg == 1) {   // one CTA owns the counters: clear them itself
    for (int i = threadIdx.x; i <= a.workers; i += blockDim.x) a.cnt[i] = 0u;
    if (threadIdx.x == 0) *a.wmax = 0u;
    __syncthreads();
  }
  // The pairs keep FP32's exponent range and Z = W^H W P scales as |W|^2, so
  // W is scaled by an exact power of two 2^-e to max |W_ij| in [1, 2); U is
  // scaled back by 2^-e in its store ((2^-e W)^+ = 2^e W^+).
  const int64_t nW = (int64_t)r * c, nP = (int64_t)c * k;
  {
    float mx = 0.f;
    for (int64_t e = (int64_t)vb * blockDim.x + threadIdx.x; e < nW; e += (int64_t)vg * blockDim.x) {
      const QFF v = ldff(a.W, (e / c) * a.W.ld + e % c);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.h.x), fabsf(v.h.y)), fmaxf(fabsf(v.h.z), fabsf(v.h.w))));
      if (!isfinite(v.h.x + v.h.y + v.h.z + v.h.w)) mx = INFINITY;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(a.wmax, __float_as_uint(mx));
  }
  if (!rf_sync(a, vg, target)) return;
  const float wm = __uint_as_float(__ldcg(a.wmax));
  if (!isfinite(wm)) {
    if (vb == 0 && threadIdx.x == 0) set_status(a.status, QMCUR_ERR_NONFINITE);
    return;   // every CTA alike
  }
  const int wexp = wm > 0.f ? ilogbf(wm) : 0;
  const float wsc = ldexpf(1.f, -wexp);
  // W split into pairs once; random start block P0 (FP32 entries uniform in
  // [-1/2, 1/2), Philox counters)
  for (int64_t e = (int64_t)vb * blockDim.x + threadIdx.x; e < nW + nP;
       e += (int64_t)vg * blockDim.x) {
    if (e < nW) {
      const int64_t i = e / c, j = e % c;
      QFF v = ldff(a.W, i * a.W.ld + j);
      v.h = make_float4(v.h.x * wsc, v.h.y * wsc, v.h.z * wsc, v.h.w * wsc);
      v.l = make_float4(v.l.x * wsc, v.l.y * wsc, v.l.z * wsc, v.l.w * wsc);
      stff(a.Wf, i * a.Wf.ld + j, v);
    } else {
      const int64_t f = e - nW;
      const uint4 x = rf_philox(make_uint4((unsigned)f, (unsigned)(f >> 32), 0x52u, 0x46u),
                                make_uint2((unsigned)a.seed, (unsigned)(a.seed >> 32)));
      const float s = 0x1.0p-24f;
      QFF v = qff_zero();
      v.h = make_float4((float)(x.x >> 8) * s - 0.5f, (float)(x.y >> 8) * s - 0.5f,
                        (float)(x.z >> 8) * s - 0.5f, (float)(x.w >> 8) * s - 0.5f);
      stff(a.P[0], (f / k) * a.P[0].ld + f % k, v);
    }
  }
  if (!rf_sync(a, vg, target)) return;
  RfJob jb[3];
  jb[0] = job(a.Wf, 0, a.P[0], 0, a.Y, r, k, c);   // Y = W P0
  jb[0].fp32 = 1;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (!rf_sync(a, vg, target)) return;
  StopState st{0.0, 0, 0.0, 0};
  int cur = 0, s = 1;
  bool converged = false;
  for (; s <= a.max_iter; ++s) {
    const QPtr& P = a.P[cur];
    const QPtr& Pn = a.P[cur ^ 1];
    // The Gram products G' (here) and G1, G2 (the ending) only feed FP32
    // Cholesky factors, right preconditioners, so they are plain FP32
    // products.  Iteration 1 starts from the random block: its rho means
    // nothing, so it forms neither E, M' nor the norms, and its Z and M
    // (which only feed the FP32 factors and the next basis, whose span the
    // later iterations correct) are plain FP32 products too; X = W Z' stays
    // float-float, so that the Y it gives is W P to working accuracy.
    const bool first = s == 1;
    jb[0] = job(a.Wf, 1, a.Y, 0, a.Z, c, k, r);   // Z = W^H Y
    jb[1] = job(a.Y, 1, a.Y, 0, a.M, k, k, r);    // M = Y^H Y
    jb[2] = job(P, 1, P, 0, a.E, k, k, c);        // E = P^H P - I
    jb[2].minus_eye = 1;
    jb[0].fp32 = jb[1].fp32 = first;
    rf_gemm_step(a, jb, first ? 2 : 3, nullptr, smr, vb);
    if (!rf_sync(a, vg, target)) return;
    // Z' = Z R_Y^-1 with R_Y = chol32(M); then M' = M - E M on the tile workers
    rf_solve_step(a, a.M, a.Z, a.Zp, c, nullptr, nullptr, 0, a.kap2 + s, vb, vg, smr);
    if (!first) {
      jb[0] = job(a.E, 0, a.M, 0, a.Mp, k, k, k);
      jb[0].Zin = a.M;
      jb[0].neg = 1;
      jb[0].add_in = 1;
      rf_gemm_step(a, jb, 1, nullptr, smr, vb);
    }
    if (!rf_sync(a, vg, target)) return;
    jb[0] = job(a.Zp, 1, a.Zp, 0, a.Gp, k, k, c);   // G' = Z'^H Z' (feeds chol32 only)
    jb[0].upper = 1;
    jb[0].fp32 = 1;
    jb[1] = job(a.Wf, 0, a.Zp, 0, a.X, r, k, c);    // X = W Z'
    jb[2] = job(P, 0, a.Mp, 0, a.Z, c, k, k);       // ||Z - P M'||, ||Z||
    jb[2].norm = 1;
    rf_gemm_step(a, jb, first ? 2 : 3, a.norms + 2 * s, smr, vb);
    if (!rf_sync(a, vg, target)) return;
    if (threadIdx.x == 0)
      stop_sh = !first && stop_now(st, s, __ldcg(a.norms + 2 * s), __ldcg(a.norms + 2 * s + 1),
                                   __ldcg(a.kap2 + s), k);
    __syncthreads();
    converged = stop_sh != 0;
    // R' = chol32(G'):  P <- Z' R'^-1,  Y <- X R'^-1 (= W P)
    rf_solve_step(a, a.Gp, a.Zp, Pn, c, &a.X, &a.Y, r, nullptr, vb, vg, smr);
    if (!rf_sync(a, vg, target)) return;
    cur ^= 1;
    if (converged) break;
  }
  const QPtr& P = a.P[cur];
  // U = P (W P)^+ by CholeskyQR2 with FP32 factors and the E2 correction
  jb[0] = job(a.Y, 1, a.Y, 0, a.G1, k, k, r);   // feeds chol32 only
  jb[0].upper = 1;
  jb[0].fp32 = 1;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (!rf_sync(a, vg, target)) return;
  rf_solve_step(a, a.G1, a.Y, a.Q1, r, &P, &a.T1, c, nullptr, vb, vg, smr);
  if (!rf_sync(a, vg, target)) return;
  jb[0] = job(a.Q1, 1, a.Q1, 0, a.G2, k, k, r);   // feeds chol32 only
  jb[0].upper = 1;
  jb[0].fp32 = 1;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (!rf_sync(a, vg, target)) return;
  rf_solve_step(a, a.G2, a.Q1, a.Q2, r, &a.T1, &a.T2, c, nullptr, vb, vg, smr);
  if (!rf_sync(a, vg, target)) return;
  jb[0] = job(a.Q2, 1, a.Q2, 0, a.E2, k, k, r);
  jb[0].minus_eye = 1;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (!rf_sync(a, vg, target)) return;
  jb[0] = job(a.T2, 0, a.E2, 0, a.V, c, k, k);   // V = T2 - T2 E2
  jb[0].Zin = a.T2;
  jb[0].neg = 1;
  jb[0].add_in = 1;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (!rf_sync(a, vg, target)) return;
  jb[0] = job(a.V, 0, a.Q2, 1, a.U, c, r, k);    // U = V Q2^H, back to W's scale
  jb[0].scale = wsc;
  jb[0].Zout2 = a.U2;
  rf_gemm_step(a, jb, 1, nullptr, smr, vb);
  if (vb == 0 && threadIdx.x == 0) {
    const int iters = s <= a.max_iter ? s : a.max_iter;
    if (a.rank_out != nullptr) { a.rank_out[0] = k; a.rank_out[1] = iters; }
    if (!converged) set_status(a.status, QMCUR_ERR_NO_CONVERGENCE);
  }
}

__global__ void __launch_bounds__(kRfThreads, 1) k_pinv_refine(const __grid_constant__ RfArgs a) {
  extern __shared__ __align__(16) unsigned char smr[];
  rf_program(a, (int)blockIdx.x, (int)gridDim.x, smr);
}

// One problem per CTA: CTA b runs the program args[order[b]] alone, its
// arguments copied to shared memory (the order puts the largest problems
// first, so that the small ones fill in behind them).  Its status goes to
// the problem's own word, cleared here, and from there to the batch's.
__global__ void __launch_bounds__(kRfThreads, 1) k_pinv_refine_each(const RfArgs* __restrict__ args,
                                                                    const int* __restrict__ order,
                                                                    int32_t* batch_status) {
  extern __shared__ __align__(16) unsigned char smr[];
  __shared__ RfArgs sa;
  if (threadIdx.x == 0) {
    sa = args[order[blockIdx.x]];
    *sa.status = 0;
  }
  __syncthreads();
  rf_program(sa, 0, 1, smr);
  __syncthreads();
  if (threadIdx.x == 0 && batch_status != nullptr) {
    const int32_t e = *(volatile int32_t*)sa.status;
    if (e != 0) set_status(batch_status, e);
  }
}

// A rows x cols matrix of pairs: four planes of float2, row stride ld.
QPtr carve_ff(Carve& cv, int64_t rows, int64_t cols) {
  QPtr q;
  const int64_t ld = (cols + 1) / 2 * 2;
  float2* base = cv.take<float2>((size_t)(4 * rows * ld));
  for (int t = 0; t < 4; ++t) q.p[t] = base ? base + (size_t)t * rows * ld : nullptr;
  q.ld = ld;
  q.dtype = kDtypeFF;
  return q;
}

struct RfWs {
  RfArgs a;
  unsigned* zero_base;   // counters and barrier words, zeroed before the launch
  size_t zero_bytes;
};

// Workspace of one program: the float-float matrices, the split-tile
// partials and counters of `workers` tile workers, and the tile partials of
// the norm product (c x k).
RfWs carve_refine(Carve& cv, int64_t r, int64_t c, int64_t k, int workers = kRfMaxWorkers) {
  RfWs w{};
  RfArgs& a = w.a;
  a.Wf = carve_ff(cv, r, c);
  a.P[0] = carve_ff(cv, c, k);
  a.P[1] = carve_ff(cv, c, k);
  a.Y = carve_ff(cv, r, k);
  a.Z = carve_ff(cv, c, k);
  a.Zp = carve_ff(cv, c, k);
  a.X = carve_ff(cv, r, k);
  a.M = carve_ff(cv, k, k);
  a.E = carve_ff(cv, k, k);
  a.Mp = carve_ff(cv, k, k);
  a.Gp = carve_ff(cv, k, k);
  a.G1 = carve_ff(cv, k, k);
  a.G2 = carve_ff(cv, k, k);
  a.E2 = carve_ff(cv, k, k);
  a.Q1 = carve_ff(cv, r, k);
  a.Q2 = carve_ff(cv, r, k);
  a.T1 = carve_ff(cv, c, k);
  a.T2 = carve_ff(cv, c, k);
  a.V = carve_ff(cv, c, k);
  const int64_t norm_tiles = ((c + kRfTS - 1) / kRfTS) * ((k + kRfTS - 1) / kRfTS);
  a.part = cv.take<QFF>((size_t)2 * workers * kRfTileThreads);
  a.normpart = cv.take<double>((size_t)2 * norm_tiles);
  a.norms = cv.take<double>((size_t)2 * (kRfMaxIter + 1));
  a.kap2 = cv.take<double>((size_t)(kRfMaxIter + 1));
  w.zero_base = cv.take<unsigned>((size_t)(workers + 8));
  w.zero_bytes = (size_t)(workers + 8) * sizeof(unsigned);
  a.cnt = w.zero_base;                     // workers + 1 counters
  a.wmax = w.zero_base + workers + 2;
  a.bar = w.zero_base + workers + 4;
  return w;
}

// The caller's W and U as the program reads and writes them.
void rf_bind(RfArgs& a, const qmcur_qmat* W, const qmcur_qmat* U) {
  for (int t = 0; t < 4; ++t) a.W.p[t] = W->plane[t];
  a.W.ld = W->ld;
  a.W.dtype = W->dtype;
  for (int t = 0; t < 4; ++t) a.U.p[t] = U->plane[t];
  a.U.ld = U->ld;
  a.U.dtype = U->dtype;
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
  int grid = cta_cap(sms);
  if (grid > kRfMaxGrid) grid = kRfMaxGrid;
  RfArgs& a = w.a;
  rf_bind(a, W, U);
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

// ---------------------------------------------------------------------------
// One problem per CTA (the batched path): each problem's arguments, built on
// the host over its own carve of the batch's arena with the tile workers of
// one CTA; CTA b runs the problem order[b].

size_t refine_each_ws_bytes(int64_t r, int64_t c, int64_t k) {
  Carve cv(nullptr, 0);
  carve_refine(cv, r, c, k, kRfWorkers);
  return cv.off;
}

size_t refine_each_args_bytes() { return sizeof(RfArgs); }

// W r x c (F32 or F64), U c x r (F64), U2 (c x r F32, or NULL); status is the
// problem's own status word, rank_out its {k, iterations}.
qmcur_status refine_each_build(const qmcur_qmat* W, int32_t rank_cap, int32_t max_iter,
                               qmcur_qmat* U, qmcur_qmat* U2, int32_t* rank_out, int32_t* status,
                               uint64_t seed, void* ws, size_t ws_bytes, void* args_out,
                               int* k_out) {
  if (!valid_qmat(W) || !valid_qmat(U) || (U2 != nullptr && !valid_qmat(U2)) || status == nullptr)
    return QMCUR_ERR_INVALID_ARG;
  const int64_t r = W->rows, c = W->cols;
  if (U->rows != c || U->cols != r || (U2 != nullptr && (U2->rows != c || U2->cols != r)))
    return QMCUR_ERR_INVALID_ARG;
  const int64_t nmin = r < c ? r : c;
  if (rank_cap < 1) return QMCUR_ERR_UNSUPPORTED;
  const int k = (int)(rank_cap < nmin ? rank_cap : nmin);
  if (k > kSmallCholMax || r > kRfMaxDim || c > kRfMaxDim) return QMCUR_ERR_UNSUPPORTED;
  if (max_iter <= 0) max_iter = 30;
  if (max_iter > kRfMaxIter) max_iter = kRfMaxIter;
  Carve cv(ws, ws_bytes);
  RfWs w = carve_refine(cv, r, c, k, kRfWorkers);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  RfArgs& a = w.a;
  rf_bind(a, W, U);
  if (U2 != nullptr) {
    for (int t = 0; t < 4; ++t) a.U2.p[t] = U2->plane[t];
    a.U2.ld = U2->ld;
    a.U2.dtype = U2->dtype;
  }
  a.r = (int)r;
  a.c = (int)c;
  a.k = k;
  a.max_iter = max_iter;
  a.seed = seed;
  a.status = status;
  a.rank_out = rank_out;
  a.workers = kRfWorkers;
  *static_cast<RfArgs*>(args_out) = a;
  *k_out = k;
  return QMCUR_OK;
}

qmcur_status refine_each_launch(const void* dargs, const int* dorder, int count, int kmax,
                                int32_t* batch_status, cudaStream_t st) {
  if (count < 1 || kmax < 1 || kmax > kSmallCholMax) return QMCUR_ERR_INVALID_ARG;
  const size_t smem = rf_smem(kmax);
  if (cudaFuncSetAttribute(k_pinv_refine_each, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  k_pinv_refine_each<<<count, kRfThreads, smem, st>>>(static_cast<const RfArgs*>(dargs), dorder,
                                                       batch_status);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
