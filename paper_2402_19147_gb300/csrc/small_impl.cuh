// Device code of the small dense quaternion kernels, shared by the
// standalone kernels (small.cu) and the fused subspace pseudo-inverse
// (pinv_fast.cu).  A GEMM tile is computed by a worker of 256 threads, a
// Cholesky factor by one CTA of 512, a triangular-solve row by one warp.
#pragma once

#include "small.cuh"

namespace qmcur {

constexpr int kSmTS = 16;    // 16 x 16 quaternion outputs per tile, one per thread
constexpr int kSmBK = 32;    // k-slice per stage; the next is prefetched into registers
constexpr int kSmTileThreads = 256;
// Shared memory of one tile worker, in float4 (one quaternion each): the
// op(X) slice [16][32 + 1] and the op(Y)^T slice [32][16 + 1]; the padding
// keeps the transposed stores free of bank conflicts.
constexpr int kSmGemmQuats = kSmTS * (kSmBK + 1) + kSmBK * (kSmTS + 1);

// Named barrier over the 256 threads of one tile worker.
__device__ __forceinline__ void worker_sync(int bar_id) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(kSmTileThreads) : "memory");
}

// Loads of one k-slice of one operand, viewed as a (rows x k) matrix: 16 x 32
// entries, two per thread.  KMAJOR: entry (r, k) lives at P[r][k] (read
// coalesced along k); otherwise at P[k][r] (coalesced along r).  CONJ
// negates the imaginary planes.  Slots (r, k) are returned for the store.
template <bool KMAJOR, bool CONJ>
__device__ __forceinline__ void sm_load(const QPtr& P, int rows_lim, int k_lim, int r0, int k0,
                                        int tid, float4 v[2], int sr[2], int sk[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * kSmTileThreads;
    int rr, kk;
    if (KMAJOR) { rr = e / kSmBK; kk = e % kSmBK; }
    else { kk = e / kSmTS; rr = e % kSmTS; }
    const int gr = r0 + rr, gk = k0 + kk;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gr < rows_lim && gk < k_lim) {
      const int64_t off = KMAJOR ? (int64_t)gr * P.ld + gk : (int64_t)gk * P.ld + gr;
      a.x = reinterpret_cast<const float*>(P.p[0])[off];
      a.y = reinterpret_cast<const float*>(P.p[1])[off];
      a.z = reinterpret_cast<const float*>(P.p[2])[off];
      a.w = reinterpret_cast<const float*>(P.p[3])[off];
      if (CONJ) { a.y = -a.y; a.z = -a.z; a.w = -a.w; }
    }
    v[h] = a;
    sr[h] = rr;
    sk[h] = kk;
  }
}

// Accumulates one 16 x 16 output tile (tm, tn) of op(X) op(Y) over the
// k-range [kb, ke) with the 256 threads of worker `bar_id` (thread index tid
// in 0..255); thread (ty, tx) = (tid / 16, tid % 16) holds entry (ty, tx).
template <bool XH, bool YH>
__device__ __forceinline__ float4 sm_tile_acc_t(const SmallGemmArgs& a, int tm, int tn, int kb,
                                                int ke, float4* sm, int tid, int bar_id) {
  float4 (*xs)[kSmBK + 1] = reinterpret_cast<float4 (*)[kSmBK + 1]>(sm);
  float4 (*ys)[kSmTS + 1] = reinterpret_cast<float4 (*)[kSmTS + 1]>(sm + kSmTS * (kSmBK + 1));
  const int tx = tid % kSmTS, ty = tid / kSmTS;
  const int m0 = tm * kSmTS, n0 = tn * kSmTS;
  float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
  float4 xv[2], yv[2];
  int xr[2], xk[2], yr[2], yk[2];
  // op(X) as (m x k): identity -> X[m][k]; X^H -> conj(X[k][m]).
  // op(Y)^T as (n x k): identity -> Y[k][n]; Y^H -> conj(Y[n][k]).
  sm_load<!XH, XH>(a.X, a.M, ke, m0, kb, tid, xv, xr, xk);
  sm_load<YH, YH>(a.Y, a.N, ke, n0, kb, tid, yv, yr, yk);
  for (int k0 = kb; k0 < ke; k0 += kSmBK) {
    worker_sync(bar_id);   // the previous tile or slice is no longer read
    xs[xr[0]][xk[0]] = xv[0]; xs[xr[1]][xk[1]] = xv[1];
    ys[yk[0]][yr[0]] = yv[0]; ys[yk[1]][yr[1]] = yv[1];
    worker_sync(bar_id);
    if (k0 + kSmBK < ke) {
      sm_load<!XH, XH>(a.X, a.M, ke, m0, k0 + kSmBK, tid, xv, xr, xk);
      sm_load<YH, YH>(a.Y, a.N, ke, n0, k0 + kSmBK, tid, yv, yr, yk);
    }
#pragma unroll 8
    for (int l = 0; l < kSmBK; ++l) {
      const float4 p = xs[ty][l], q = ys[l][tx];
      z0 = fmaf(p.x, q.x, z0); z0 = fmaf(-p.y, q.y, z0); z0 = fmaf(-p.z, q.z, z0); z0 = fmaf(-p.w, q.w, z0);
      z1 = fmaf(p.x, q.y, z1); z1 = fmaf(p.y, q.x, z1); z1 = fmaf(p.z, q.w, z1); z1 = fmaf(-p.w, q.z, z1);
      z2 = fmaf(p.x, q.z, z2); z2 = fmaf(-p.y, q.w, z2); z2 = fmaf(p.z, q.x, z2); z2 = fmaf(p.w, q.y, z2);
      z3 = fmaf(p.x, q.w, z3); z3 = fmaf(p.y, q.z, z3); z3 = fmaf(-p.z, q.y, z3); z3 = fmaf(p.w, q.x, z3);
    }
  }
  return make_float4(z0, z1, z2, z3);
}

__device__ __forceinline__ float4 sm_tile_acc(const SmallGemmArgs& a, int tm, int tn, int kb, int ke,
                                              float4* sm, int tid, int bar_id) {
  if (!a.xh && !a.yh) return sm_tile_acc_t<false, false>(a, tm, tn, kb, ke, sm, tid, bar_id);
  if (a.xh && !a.yh) return sm_tile_acc_t<true, false>(a, tm, tn, kb, ke, sm, tid, bar_id);
  if (!a.xh && a.yh) return sm_tile_acc_t<false, true>(a, tm, tn, kb, ke, sm, tid, bar_id);
  return sm_tile_acc_t<true, true>(a, tm, tn, kb, ke, sm, tid, bar_id);
}

// Epilogue of entry (ty, tx) of tile (tm, tn): Z = alpha acc + beta Z.
__device__ __forceinline__ void sm_tile_store(const SmallGemmArgs& a, int tm, int tn, int tid,
                                              float4 acc) {
  const int i = tm * kSmTS + tid / kSmTS, j = tn * kSmTS + tid % kSmTS;
  if (i >= a.M || j >= a.N) return;
  const int64_t off = (int64_t)i * a.Z.ld + j;
  const float zz[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (a.Z.dtype == QMCUR_F64) {
      double* p = reinterpret_cast<double*>(a.Z.p[t]) + off;
      double v = (double)(a.alpha * zz[t]);
      if (a.beta != 0.f) v += (double)a.beta * *p;
      *p = v;
    } else {
      float* p = reinterpret_cast<float*>(a.Z.p[t]) + off;
      float v = a.alpha * zz[t];
      if (a.beta != 0.f) v = fmaf(a.beta, *p, v);
      *p = v;
    }
  }
}

// One whole tile: Z(tile) = alpha op(X) op(Y) + beta Z(tile).
__device__ __forceinline__ void sm_gemm_tile(const SmallGemmArgs& a, int tm, int tn, float4* sm,
                                             int tid, int bar_id) {
  sm_tile_store(a, tm, tn, tid, sm_tile_acc(a, tm, tn, 0, a.K, sm, tid, bar_id));
}

// ---------------------------------------------------------------------------
// Quaternion helpers.

// conj(a) b
__device__ __forceinline__ float4 q_conj_mul(const float4 a, const float4 b) {
  return make_float4(a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w,
                     a.x * b.y - a.y * b.x - a.z * b.w + a.w * b.z,
                     a.x * b.z + a.y * b.w - a.z * b.x - a.w * b.y,
                     a.x * b.w - a.y * b.z + a.z * b.y - a.w * b.x);
}

// acc - conj(a) b
__device__ __forceinline__ float4 q_sub_conj_mul(float4 acc, const float4 a, const float4 b) {
  const float4 m = q_conj_mul(a, b);
  acc.x -= m.x; acc.y -= m.y; acc.z -= m.z; acc.w -= m.w;
  return acc;
}

// acc - a b
__device__ __forceinline__ float4 q_sub_mul(float4 acc, const float4 a, const float4 b) {
  acc.x -= a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w;
  acc.y -= a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z;
  acc.z -= a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y;
  acc.w -= a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x;
  return acc;
}

__device__ __forceinline__ float4 q_add(float4 a, const float4 b) {
  a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
  return a;
}

__device__ __forceinline__ float4 q_sub(float4 a, const float4 b) {
  a.x -= b.x; a.y -= b.y; a.z -= b.z; a.w -= b.w;
  return a;
}

__device__ __forceinline__ float4 q_scale(float4 a, float s) {
  a.x *= s; a.y *= s; a.z *= s; a.w *= s;
  return a;
}

__device__ __forceinline__ float q_norm2(const float4 a) {
  return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
}

// Start of row j in the row-major packed upper triangle of a k x k matrix.
__host__ __device__ __forceinline__ int packed_row(int j, int k) { return j * k - j * (j - 1) / 2; }

// ---------------------------------------------------------------------------
// Cholesky factor of a small Hermitian positive definite matrix.
//
// G = R^H R with R upper triangular and a real positive diagonal (Sec. 2.2's
// quaternion matrices: R^H is the conjugate transpose).  Right-looking and
// blocked by kCholNb rows.  For the block of rows b0 .. b0 + nb - 1, whose
// entries already carry every earlier block's update:
//   panel:  R11 = chol(A11) (nb x nb) and R12 = R11^-H A12; each thread takes
//           one column c >= b0 and forms R11 itself (identical arithmetic in
//           every thread, so no barrier is needed between the two);
//   update: A22 -= R12^H R12 on the entries (j, c), c >= j >= b0 + nb.
// Two barriers per block.  The upper triangle, row-major packed, is spread
// over the CTA: entry e = s * kCholThreads + tid lives in register slot s of
// thread tid (S = ceil(k (k + 1) / 2 / kCholThreads) slots, a template
// parameter).  Rows grow with the slot index, so the finished rows occupy a
// prefix of every warp's slots: the update walks the slots downwards and
// leaves at the first one whose 32 entries are all finished (warp-uniform).
// The owners of the next block's rows publish them to shared memory as they
// update them.
//
// Output (the layout the triangular solve stages): the upper triangle of R,
// row-major packed, one float4 (quaternion) per entry, then 1 / R_ll for
// l = 0 .. k - 1 as floats: rpk_floats(k) floats in all.

constexpr int kCholThreads = 512;
constexpr int kCholNb = 4;
constexpr int kCholPacked = kSmallCholMax * (kSmallCholMax + 1) / 2;
constexpr int kCholSlots = (kCholPacked + kCholThreads - 1) / kCholThreads;

// Floats of the packed factor: k (k + 1) / 2 quaternions and k reciprocals.
__host__ __device__ constexpr int rpk_floats(int k) { return 4 * (k * (k + 1) / 2) + k; }

// Shared-memory bytes of sm_chol: raw and factored rows of one block, the pivot floor.
__host__ __device__ constexpr size_t sm_chol_bytes() {
  return (size_t)2 * kCholNb * kSmallCholMax * 16 + 16;
}

// ---------------------------------------------------------------------------
// Row solves that ride along with the factorisation.  Z = Y R^-1 needs, for
// its column l, only rows 0 .. l of R.  Rows b0 .. b0 + nb - 1 are final once
// the panel of block b0 has passed its barrier, so a warp that holds a row of
// Y can take the columns of block b while the panel of block b + 1 runs.  The
// panel only occupies the warps of the first kSolvePanelWarps (its column
// threads); the other warps of the CTA each carry one row.  The arithmetic per
// column is that of the plain row solve below: z_l = t_l / R_ll, taken from
// its owner lane with shuffles, then t_c -= z_l R_lc for every later column.
// The row warps sit on the SM sub-partitions (warp % 4) that hold no panel
// warp, so that they do not take issue slots from the panel.

// One or two solves with one factor: rows [0, rows0) belong to the first.
struct SolveJobs {
  QPtr Y0, Y1, Z0, Z1;
  int rows0, rows;
  int vb, vg;   // this CTA's index and the number of CTAs sharing the rows
};

// One of two plane sets, selected field by field (selecting between the two
// structs would take their addresses and put them on the stack).
__device__ __forceinline__ QPtr qptr_pick(bool second, const QPtr& a, const QPtr& b) {
  QPtr q;
#pragma unroll
  for (int t = 0; t < 4; ++t) q.p[t] = second ? b.p[t] : a.p[t];
  q.ld = second ? b.ld : a.ld;
  q.dtype = second ? b.dtype : a.dtype;
  return q;
}

// Row i of the CTA's rows (row-warp i, or past the row warps: the plain row
// solve takes those once R is complete).
// (vb, vg): the CTA's index among the vg CTAs that share the solve.
__device__ __forceinline__ int solve_row_of(int i, int vb, int vg) { return vb + vg * i; }

// Panel warps of order k (their sub-partitions are 0 .. pw - 1), row warps
// (the warps of the other sub-partitions), and the row-warp index of a warp.
__device__ __forceinline__ int solve_panel_warps(int k) { return (k + 31) / 32; }
__device__ __forceinline__ int solve_row_warps(int k) {
  return (4 - solve_panel_warps(k)) * (kCholThreads / 128);
}
__device__ __forceinline__ int solve_row_index(int warp, int k) {
  const int pw = solve_panel_warps(k);
  return (warp & 3) < pw ? -1 : (warp >> 2) * (4 - pw) + ((warp & 3) - pw);
}

template <int U>   // column slots per lane: k <= 32 U
struct SolveRow {
  float4 t[U];
  int row;   // -1: this warp carries no row
  int job;
  int local;

  __device__ __forceinline__ void load(const SolveJobs& sj, int k) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    row = -1;
#pragma unroll
    for (int u = 0; u < U; ++u) t[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int ri = solve_row_index(warp, k);
    if (ri < 0) return;
    const int rg = solve_row_of(ri, sj.vb, sj.vg);
    if (rg >= sj.rows) return;
    row = rg;
    job = rg < sj.rows0 ? 0 : 1;
    local = job == 0 ? rg : rg - sj.rows0;
    const QPtr Y = qptr_pick(job != 0, sj.Y0, sj.Y1);
    const int64_t yo = (int64_t)local * Y.ld;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = lane + 32 * u;
      if (c < k)
        t[u] = make_float4(reinterpret_cast<const float*>(Y.p[0])[yo + c],
                           reinterpret_cast<const float*>(Y.p[1])[yo + c],
                           reinterpret_cast<const float*>(Y.p[2])[yo + c],
                           reinterpret_cast<const float*>(Y.p[3])[yo + c]);
    }
  }

  // Columns l0 .. l0 + nb - 1 of slot UB (l0 >> 5 == UB) from the packed R.
  template <int UB>
  __device__ __forceinline__ void cols_u(int l0, int nb, int k, const float* rpk) {
    const float4* Rs = reinterpret_cast<const float4*>(rpk);
    const float* invd = rpk + 4 * (k * (k + 1) / 2);
    const int lane = threadIdx.x & 31;
    for (int l = l0; l < l0 + nb; ++l) {
      const int ll = l & 31;
      const float s = invd[l];
      const float4 z = make_float4(__shfl_sync(0xffffffffu, t[UB].x, ll) * s,
                                   __shfl_sync(0xffffffffu, t[UB].y, ll) * s,
                                   __shfl_sync(0xffffffffu, t[UB].z, ll) * s,
                                   __shfl_sync(0xffffffffu, t[UB].w, ll) * s);
      // R_l,c sits at Rrow + c for c >= l; a clamped c below l reads an
      // earlier entry of the packed array, whose product is discarded.
      const float4* Rrow = Rs + (packed_row(l, k) - l);
#pragma unroll
      for (int u = UB; u < U; ++u) {
        if (32 * u < k) {   // warp-uniform: the slot holds columns
          const int c = lane + 32 * u;
          const int cc = c < k ? c : k - 1;
          const float4 nt = q_sub_mul(t[u], z, Rrow[cc > l ? cc : l]);
          t[u] = (c > l && c < k) ? nt : t[u];
        }
      }
      t[UB] = (lane == ll) ? z : t[UB];
    }
  }

  // Columns l0 .. l0 + nb - 1, within one 32-column slot.
  __device__ __forceinline__ void cols(int l0, int nb, int k, const float* rpk) {
    static_assert(U >= 1 && U <= 3, "one case per slot");
    const int ub = l0 >> 5;
    if (ub == 0) cols_u<0>(l0, nb, k, rpk);
    else if (U > 1 && ub == 1) cols_u<(U > 1 ? 1 : 0)>(l0, nb, k, rpk);
    else if (U > 2) cols_u<(U > 2 ? 2 : 0)>(l0, nb, k, rpk);
  }

  __device__ __forceinline__ void store(const SolveJobs& sj, int k) const {
    const int lane = threadIdx.x & 31;
    const QPtr Z = qptr_pick(job != 0, sj.Z0, sj.Z1);
    const int64_t zo = (int64_t)local * Z.ld;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c = lane + 32 * u;
      if (c < k) {
        reinterpret_cast<float*>(Z.p[0])[zo + c] = t[u].x;
        reinterpret_cast<float*>(Z.p[1])[zo + c] = t[u].y;
        reinterpret_cast<float*>(Z.p[2])[zo + c] = t[u].z;
        reinterpret_cast<float*>(Z.p[3])[zo + c] = t[u].w;
      }
    }
  }
};

// Row slots of the ride-along solves for S register slots of the factor (the
// largest k with S slots is at most 32 RU), or 0: no ride-along, the caller
// solves every row.  From S = 5 (k > 63) on, the row state on top of the
// factor's slots would spill registers.
__host__ __device__ constexpr int chol_ride_slots(int S) {
  return S >= 5 ? 0 : S * kCholThreads <= 32 * 33 / 2 ? 1 : 2;
}

template <int S>
__device__ __forceinline__ int sm_chol_s(const QPtr& G, int k, float* rpk, int32_t* status,
                                          unsigned char* smraw, const SolveJobs* sj,
                                          float diag_shift_rel) {
  static_assert(32 % kCholNb == 0, "a block of columns stays in one slot");
  constexpr int RU = chol_ride_slots(S);
  constexpr int RUs = RU > 0 ? RU : 1;
  float4* Pn = reinterpret_cast<float4*>(smraw);            // [kCholNb][kSmallCholMax] raw rows
  float4* Rp = Pn + kCholNb * kSmallCholMax;               // [kCholNb][kSmallCholMax] factored rows
  float* floor_sh = reinterpret_cast<float*>(Rp + kCholNb * kSmallCholMax);
  const int tid = threadIdx.x;
  const int np = k * (k + 1) / 2;
  SolveRow<RUs> rs;
  rs.row = -1;
  if (RU > 0 && sj != nullptr) rs.load(*sj, k);   // the loads overlap those of G
  // optional shift of the diagonal by diag_shift_rel * max_l G_ll (a shifted
  // factor of an ill-conditioned G, for callers that only precondition with it)
  float shift = 0.f;
  if (diag_shift_rel > 0.f) {
    __shared__ float dmax_sh;
    if (tid < 32) {
      float mx = 0.f;
      for (int l = tid; l < k; l += 32) {
        const int64_t off = (int64_t)l * G.ld + l;
        mx = fmaxf(mx, G.dtype == kDtypeFF ? reinterpret_cast<const float2*>(G.p[0])[off].x
                       : G.dtype == QMCUR_F64 ? (float)reinterpret_cast<const double*>(G.p[0])[off]
                                              : reinterpret_cast<const float*>(G.p[0])[off]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (tid == 0) dmax_sh = mx;
    }
    __syncthreads();
    shift = diag_shift_rel * dmax_sh;
  }
  float4 v[S];
  unsigned jc[(S + 1) / 2];   // (j << 8 | c) in 16 bits, two slots per word
#pragma unroll
  for (int s = 0; s < (S + 1) / 2; ++s) jc[s] = 0u;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = s * kCholThreads + tid;
    v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e < np) {
      const float b = 2.0f * (float)k + 1.0f;
      int j = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.f))) * 0.5f);
      if (j < 0) j = 0;
      if (j > k - 1) j = k - 1;
      while (j > 0 && packed_row(j, k) > e) --j;
      while (j + 1 < k && packed_row(j + 1, k) <= e) ++j;
      const int c = j + (e - packed_row(j, k));
      jc[s >> 1] |= (((unsigned)j << 8) | (unsigned)c) << (16 * (s & 1));
      const int64_t off = (int64_t)j * G.ld + c;
      if (G.dtype == kDtypeFF)    // a float-float Gram matrix: its leading parts
        v[s] = make_float4(reinterpret_cast<const float2*>(G.p[0])[off].x,
                           reinterpret_cast<const float2*>(G.p[1])[off].x,
                           reinterpret_cast<const float2*>(G.p[2])[off].x,
                           reinterpret_cast<const float2*>(G.p[3])[off].x);
      else if (G.dtype == QMCUR_F64)   // an FP64 Gram matrix, factored in FP32
        v[s] = make_float4((float)reinterpret_cast<const double*>(G.p[0])[off],
                           (float)reinterpret_cast<const double*>(G.p[1])[off],
                           (float)reinterpret_cast<const double*>(G.p[2])[off],
                           (float)reinterpret_cast<const double*>(G.p[3])[off]);
      else
        v[s] = make_float4(reinterpret_cast<const float*>(G.p[0])[off],
                           reinterpret_cast<const float*>(G.p[1])[off],
                           reinterpret_cast<const float*>(G.p[2])[off],
                           reinterpret_cast<const float*>(G.p[3])[off]);
      if (j == c) v[s].x += shift;
      if (j < kCholNb) Pn[j * kSmallCholMax + c] = v[s];
      if (e == 0) {
        const float g00 = fabsf(v[s].x);
        *floor_sh = (g00 > 0.f && isfinite(g00) ? g00 : 1.f) * 1e-30f;
      }
    }
  }
  __syncthreads();
  const float floor_v = *floor_sh;
  const int wlast = tid | 31;
  float4* Rq = reinterpret_cast<float4*>(rpk);
  float* Rinvd = rpk + 4 * np;
  for (int b0 = 0; b0 < k; b0 += kCholNb) {
    const int nb = k - b0 < kCholNb ? k - b0 : kCholNb;
    // ---- panel: thread tid owns column c = b0 + tid
    if (tid < k - b0) {
      const int c = b0 + tid;
      float4 a[kCholNb][kCholNb];   // A11, upper part used; missing rows act as identity
#pragma unroll
      for (int p = 0; p < kCholNb; ++p)
#pragma unroll
        for (int q = p; q < kCholNb; ++q)
          a[p][q] = (q < nb) ? Pn[p * kSmallCholMax + b0 + q]
                             : make_float4(p == q ? 1.f : 0.f, 0.f, 0.f, 0.f);
      bool bad = false;
      float rd[kCholNb];
#pragma unroll
      for (int p = 0; p < kCholNb; ++p) {
        float d = a[p][p].x;
#pragma unroll
        for (int q = 0; q < p; ++q) d -= q_norm2(a[q][p]);
        if (!(d > 0.f) || !isfinite(d)) { bad = true; d = floor_v; }
        rd[p] = rsqrtf(d);   // 1 / R_pp within 2 ulp, far below CholeskyQR's own u kappa^2
        a[p][p] = make_float4(d * rd[p], 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = p + 1; q < kCholNb; ++q) {   // R_pq = (A_pq - sum_l conj(R_lp) R_lq) / R_pp
          float4 t = a[p][q];
#pragma unroll
          for (int l = 0; l < p; ++l) t = q_sub_conj_mul(t, a[l][p], a[l][q]);
          a[p][q] = q_scale(t, rd[p]);
        }
      }
      if (bad && tid == 0) set_status(status, QMCUR_ERR_ILL_CONDITIONED);
      // the pivot rows of this block are final after the next barrier
      // column c of R12 (or of R11 when c < b0 + nb): y_p = (x_p - sum_l conj(R_lp) y_l) / R_pp
      float4 y[kCholNb];
#pragma unroll
      for (int p = 0; p < kCholNb; ++p) {
        float4 t = (p < nb && c >= b0 + p) ? Pn[p * kSmallCholMax + c] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < p; ++l) t = q_sub_conj_mul(t, a[l][p], y[l]);
        y[p] = (c >= b0 + p) ? q_scale(t, rd[p]) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (c == b0 + p) y[p] = a[p][p];   // the diagonal exactly as the pivot
      }
#pragma unroll
      for (int p = 0; p < kCholNb; ++p) {
        Rp[p * kSmallCholMax + c] = (p < nb) ? y[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (p < nb && c >= b0 + p) Rq[packed_row(b0 + p, k) + c - (b0 + p)] = y[p];
        if (c == b0 + p) Rinvd[c] = rd[p];
      }
    } else if (RU > 0 && rs.row >= 0 && b0 > 0) {
      rs.cols(b0 - kCholNb, kCholNb, k, rpk);   // the previous block's columns
    }
    __syncthreads();
    // ---- update of the trailing entries; the next block's rows are published
    const int nb0 = b0 + nb;
    if (nb0 < k) {
      const int first_live = packed_row(nb0, k);
#pragma unroll
      for (int s = S - 1; s >= 0; --s) {
        if (s * kCholThreads + wlast < first_live) break;   // warp-uniform
        const int e = s * kCholThreads + tid;
        const unsigned w = jc[s >> 1] >> (16 * (s & 1));
        const int j = (int)((w >> 8) & 0xffu), c = (int)(w & 0xffu);
        if (e < np && j >= nb0) {   // many entries per thread: skipping idle ones pays here
          float4 t;
          if constexpr (kCholNb == 4) {   // tree sum of the four products
            const float4 m0 = q_conj_mul(Rp[0 * kSmallCholMax + j], Rp[0 * kSmallCholMax + c]);
            const float4 m1 = q_conj_mul(Rp[1 * kSmallCholMax + j], Rp[1 * kSmallCholMax + c]);
            const float4 m2 = q_conj_mul(Rp[2 * kSmallCholMax + j], Rp[2 * kSmallCholMax + c]);
            const float4 m3 = q_conj_mul(Rp[3 * kSmallCholMax + j], Rp[3 * kSmallCholMax + c]);
            t = q_sub(v[s], q_add(q_add(m0, m1), q_add(m2, m3)));
          } else {
            t = v[s];
#pragma unroll
            for (int p = 0; p < kCholNb; ++p)
              t = q_sub_conj_mul(t, Rp[p * kSmallCholMax + j], Rp[p * kSmallCholMax + c]);
          }
          v[s] = t;
          if (j < nb0 + kCholNb) Pn[(j - nb0) * kSmallCholMax + c] = t;
        }
      }
    }
    __syncthreads();
  }
  if (RU > 0 && rs.row >= 0) {
    const int lb0 = (k - 1) / kCholNb * kCholNb;
    rs.cols(lb0, k - lb0, k, rpk);
    rs.store(*sj, k);
  }
  return RU > 0 && sj != nullptr ? solve_row_warps(k) : 0;
}

template <int S>
__device__ __forceinline__ int sm_chol_from(int need, const QPtr& G, int k, float* rpk,
                                            int32_t* status, unsigned char* smraw,
                                            const SolveJobs* sj, float diag_shift_rel) {
  if (need <= S) return sm_chol_s<S>(G, k, rpk, status, smraw, sj, diag_shift_rel);
  if constexpr (S < kCholSlots)
    return sm_chol_from<S + 1>(need, G, k, rpk, status, smraw, sj, diag_shift_rel);
  return 0;
}

// One CTA of kCholThreads threads: the packed factor R (FP32) with G = R^H R,
// for 1 <= k <= kSmallCholMax (rpk 16-byte aligned, rpk_floats(k) floats).
// Only the upper triangle of G is read; G may be FP32, FP64 or float-float
// pairs (rounded to FP32 as it is read).  diag_shift_rel > 0 factors G + diag_shift_rel *
// max_l G_ll I instead.  A non-positive or non-finite pivot
// sets ILL_CONDITIONED and continues with a tiny pivot.  With sj, rpk must be
// in shared memory.  Returns n, the number of row warps: the rows
// solve_row_of(i, vb, vg), i < n, of the solves Z = Y R^-1 were done along the way;
// the other rows (all of them when n = 0) are left to the caller.
__device__ __forceinline__ int sm_chol(const QPtr& G, int k, float* rpk, int32_t* status,
                                        unsigned char* smraw, const SolveJobs* sj = nullptr,
                                        float diag_shift_rel = 0.f) {
  return sm_chol_from<1>((k * (k + 1) / 2 + kCholThreads - 1) / kCholThreads, G, k, rpk, status,
                         smraw, sj, diag_shift_rel);
}

// ---------------------------------------------------------------------------
// Triangular solve Z = Y R^-1 (R k x k upper triangular, real diagonal): row
// z of Z solves z R = y, i.e. z_l = (y_l - sum_{i<l} z_i R_il) / R_ll.  One
// warp per row, lane owning columns lane + 32 u; column by column, z_l is
// taken from its owner with shuffles and every later column takes its update
// at once.  The slot updates are branch-free (clamped indices, selected
// results): short branchy bodies leave a lone warp waiting on instruction
// fetch.  R (the packed factor above) sits in shared memory.

__host__ __device__ constexpr size_t sm_trsm_bytes(int k) { return (size_t)rpk_floats(k) * 4; }

// One warp: row `row` of Z = Y R^-1 (Z may alias Y), k <= 32 U.
template <int U>
__device__ __forceinline__ void sm_trsm_row(const QPtr& Y, const QPtr& Z, int row, int k,
                                            const unsigned char* smraw) {
  const float4* Rs = reinterpret_cast<const float4*>(smraw);
  const float* invd = reinterpret_cast<const float*>(smraw) + 4 * (k * (k + 1) / 2);
  const int lane = threadIdx.x & 31;
  float4 t[U];
  int cc[U];   // column of each slot, clamped into [0, k) for the loads
  const int64_t yo = (int64_t)row * Y.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    cc[u] = c < k ? c : k - 1;
    t[u] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < k)
      t[u] = make_float4(reinterpret_cast<const float*>(Y.p[0])[yo + c],
                         reinterpret_cast<const float*>(Y.p[1])[yo + c],
                         reinterpret_cast<const float*>(Y.p[2])[yo + c],
                         reinterpret_cast<const float*>(Y.p[3])[yo + c]);
  }
#pragma unroll
  for (int uu = 0; uu < U; ++uu) {
    const int lend = k - 32 * uu < 32 ? k - 32 * uu : 32;   // columns of this slot
    for (int ll = 0; ll < lend; ++ll) {
      const int l = 32 * uu + ll;
      const float s = invd[l];
      const float4 z = make_float4(__shfl_sync(0xffffffffu, t[uu].x, ll) * s,
                                   __shfl_sync(0xffffffffu, t[uu].y, ll) * s,
                                   __shfl_sync(0xffffffffu, t[uu].z, ll) * s,
                                   __shfl_sync(0xffffffffu, t[uu].w, ll) * s);
      // R_l,c sits at Rrow + c for c >= l; a clamped c below l reads an
      // earlier entry of the packed array, whose product is discarded.
      const float4* Rrow = Rs + (packed_row(l, k) - l);
#pragma unroll
      for (int u = uu; u < U; ++u) {
        const int c = lane + 32 * u;
        const float4 nt = q_sub_mul(t[u], z, Rrow[cc[u] > l ? cc[u] : l]);
        t[u] = (c > l && c < k) ? nt : t[u];
      }
      t[uu] = (lane == ll) ? z : t[uu];
    }
  }
  const int64_t zo = (int64_t)row * Z.ld;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = lane + 32 * u;
    if (c < k) {
      reinterpret_cast<float*>(Z.p[0])[zo + c] = t[u].x;
      reinterpret_cast<float*>(Z.p[1])[zo + c] = t[u].y;
      reinterpret_cast<float*>(Z.p[2])[zo + c] = t[u].z;
      reinterpret_cast<float*>(Z.p[3])[zo + c] = t[u].w;
    }
  }
}

__device__ __forceinline__ void sm_trsm_row_any(const QPtr& Y, const QPtr& Z, int row, int k,
                                                const unsigned char* smraw) {
  static_assert(kSmallCholMax <= 128, "four column slots per lane");
  if (k <= 32) sm_trsm_row<1>(Y, Z, row, k, smraw);
  else if (k <= 64) sm_trsm_row<2>(Y, Z, row, k, smraw);
  else if (k <= 96) sm_trsm_row<3>(Y, Z, row, k, smraw);
  else sm_trsm_row<4>(Y, Z, row, k, smraw);
}

}  // namespace qmcur
