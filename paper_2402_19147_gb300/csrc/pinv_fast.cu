// Rank-capped pseudo-inverse U = W_k^+ by subspace iteration in FP32.
//
// The truncated inverse of Sec. 2.2 / Algorithm 1 depends only on the top-k
// singular subspaces of W.  With k = rank_cap:
//   Y0 = W Omega (Omega a Philox Gaussian c x k), Q0 = orth(Y0)
//   P1 = orth(W^H Q0), Q1 = orth(W P1), P = orth(W^H Q1)      (two iterations)
//   W P = Q R  (CholeskyQR2),  U = P R^-1 Q^H.
// Because P has orthonormal columns, P (W P)^+ is the Moore-Penrose inverse of
// W P P^H, i.e. of W restricted to span(P); when span(P) is the top-k right
// singular subspace this is W_k^+.  The subspace error after the two
// iterations is of order (sigma_{k+1}/sigma_k)^4 plus FP32 rounding.
// orth() is CholeskyQR (G = Y^H Y = R^H R, Q = Y R^-1), applied twice
// (CholeskyQR2) where orthonormality to working accuracy matters.
//
// Every step is a small quaternion GEMM (op(X) op(Y), op in {N, H}) or a
// solve: G = R^H R (Cholesky) then Z = Y R^-1 (one warp per row).  The 20
// steps run in ONE persistent kernel of 512-thread CTAs (two GEMM tile
// workers of 256 threads each) over a virtual grid of vg CTAs: the whole GPU
// with a bounded grid barrier between steps (k_pinv_fused, one problem), or
// one CTA with a CTA barrier (k_pinv_fused_each, one problem per CTA, the
// batched path).  A GEMM step is a list of work items (16 x 16 output tile,
// k-range) dealt to the workers one SM at a time.  Steps with fewer tiles
// than workers split their k-range; every split writes its partial tile to
// the workspace and the last of a tile's splits to finish (an atomic count
// per tile) sums the partials in split order and writes the tile, so the
// result does not depend on timing.  A Gram step Y^H Y feeds only the
// Cholesky, which reads the upper triangle, so only tiles on or above the
// diagonal are formed.  In a solve step every CTA that owns rows factors G
// itself (identical arithmetic, so identical factors, without a barrier),
// and the warps that hold rows solve them along with the factorisation.
#include "small_impl.cuh"

namespace qmcur {
namespace {

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
    const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Gaussian quaternion entry e of a matrix with `cols` columns (Box-Muller on
// two Philox words per pair of components); counter (e_lo, e_hi, stream, 7).
__device__ __forceinline__ void randn_entry(const QPtr& out, int64_t e, int cols, uint64_t seed,
                                            uint32_t stream) {
  {
    const uint4 x = philox(make_uint4((unsigned)e, (unsigned)(e >> 32), stream, 7u),
                           make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
    const float u0 = ((float)x.x + 1.0f) * 0x1.0p-32f, v0 = (float)x.y * 0x1.0p-32f;
    const float u1 = ((float)x.z + 1.0f) * 0x1.0p-32f, v1 = (float)x.w * 0x1.0p-32f;
    const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u1));
    float s0, c0, s1, c1;
    sincospif(2.0f * v0, &s0, &c0);
    sincospif(2.0f * v1, &s1, &c1);
    const int64_t i = e / cols, j = e % cols;
    float* p0 = reinterpret_cast<float*>(out.p[0]);
    float* p1 = reinterpret_cast<float*>(out.p[1]);
    float* p2 = reinterpret_cast<float*>(out.p[2]);
    float* p3 = reinterpret_cast<float*>(out.p[3]);
    p0[i * out.ld + j] = r0 * c0;
    p1[i * out.ld + j] = r0 * s0;
    p2[i * out.ld + j] = r1 * c1;
    p3[i * out.ld + j] = r1 * s1;
  }
}

}  // namespace

// Workspace of the subspace method for an r x c intersection with cap k.
struct FastWs {
  QPtr W32, Om, Y, Q, Z, P, G, T;
  int32_t* info;
};

// Split-k partial tiles (256 quaternions each) and per-tile arrival counts.
constexpr int kMaxPartTiles = 1024;

static QPtr carve_q(Carve& cv, int64_t rows, int64_t cols) {
  QPtr q;
  const int64_t ld = (cols + 3) / 4 * 4;
  float* base = cv.take<float>((size_t)(4 * rows * ld));
  for (int t = 0; t < 4; ++t) q.p[t] = base ? base + (size_t)t * rows * ld : nullptr;
  q.ld = ld;
  q.dtype = QMCUR_F32;
  return q;
}

static FastWs carve_fast(Carve& cv, int64_t r, int64_t c, int64_t k) {
  FastWs w;
  const int64_t mx = r > c ? r : c;
  w.W32 = carve_q(cv, r, c);
  w.Om = carve_q(cv, c, k);
  w.Y = carve_q(cv, mx, k);
  w.Q = carve_q(cv, mx, k);
  w.Z = carve_q(cv, mx, k);
  w.P = carve_q(cv, mx, k);
  w.G = carve_q(cv, k, k);
  w.T = carve_q(cv, mx, k);
  w.info = cv.take<int32_t>(4);
  return w;
}

size_t pinv_fast_ws_bytes(int64_t r, int64_t c, int64_t k) {
  Carve cv(nullptr, 0);
  carve_fast(cv, r, c, k);
  cv.take<float4>((size_t)kMaxPartTiles * kSmTileThreads);   // split-k partials
  cv.take<unsigned>(4 + kMaxPartTiles);   // grid barrier, then split-k counts
  return cv.off;
}

enum { PH_PREP = 0, PH_GEMM = 1, PH_SOLVE = 2 };

// One product of a GEMM step (or one solve of a PH_SOLVE step).
struct Job {
  SmallGemmArgs g;   // PH_SOLVE: g.Z = g.X R^-1, g.M rows, g.K = k
  int splits;        // PH_GEMM: k-range splits per tile (1: no partials)
  int kchunk;        // PH_GEMM: k-range of one split (a multiple of kSmBK)
  int upper;         // PH_GEMM: square output, only tiles (tm <= tn) are formed
};

// A step holds one or two independent jobs of the same kind (two products
// of one input, or two solves with one factor), sharing one grid barrier.
// A PH_SOLVE step factors G = R^H R and then solves with R: every CTA that
// owns rows factors G itself, into its own shared memory, so the factor
// needs neither a grid barrier nor a round trip through global memory.
struct Phase {
  int kind;
  int k;        // PH_SOLVE: order of G
  int njobs;
  QPtr G;       // PH_SOLVE: the Gram matrix (upper triangle read)
  Job job[2];
};

constexpr int kMaxPhases = 32;
constexpr int kMaxSplits = 8;   // k-range splits of a GEMM step at most

struct FusedProg {
  int nph;
  Phase ph[kMaxPhases];
  QView Win;
  QPtr W32, Om;
  int r, c, k;
  uint64_t seed;
  unsigned* bar;
  unsigned* cnt;   // kMaxPartTiles split-k arrival counts, zero between steps
  float4* part;    // kMaxPartTiles partial tiles
  int32_t* status;
  int32_t* rank_out;
};

static_assert(sizeof(FusedProg) <= 32000, "kernel parameter space");

// Tile (tm, tn) of work tile t: row-major over the tile grid, or for `upper`
// column-major over the upper triangle (t = tn (tn + 1) / 2 + tm).
__device__ __forceinline__ void tile_of(int t, int tn_count, int upper, int& tm, int& tn) {
  if (!upper) {
    tm = t / tn_count;
    tn = t % tn_count;
    return;
  }
  int c = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (c * (c + 1) / 2 > t) --c;
  while ((c + 1) * (c + 2) / 2 <= t) ++c;
  tn = c;
  tm = t - c * (c + 1) / 2;
}

__device__ __forceinline__ float4 f4add(float4 a, const float4 b) {
  a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
  return a;
}

constexpr int kFusedThreads = kCholThreads;
constexpr int kFusedWorkers = kFusedThreads / kSmTileThreads;
static_assert(kFusedWorkers * kSmTileThreads == kFusedThreads, "whole tile workers");

// Dynamic shared memory of the fused kernel for cap k: the larger of the
// tile workers' slices and a solve step's packed R followed by the Cholesky
// buffers.
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t solve_chol_off(int k) { return (sm_trsm_bytes(k) + 15) / 16 * 16; }
constexpr size_t fused_smem(int k) {
  return cmax((size_t)kFusedWorkers * kSmGemmQuats * 16, solve_chol_off(k) + sm_chol_bytes());
}

// The program's steps, run by vg CTAs of which this is number vb: vg = the
// grid with a grid barrier between steps (one problem on the whole GPU), or
// vg = 1 with a CTA barrier (one problem per CTA, the batched path).
__device__ __forceinline__ void fused_program(const FusedProg& P, int vb, int vg) {
  extern __shared__ __align__(16) unsigned char smf[];
  const int worker = threadIdx.x / kSmTileThreads, wtid = threadIdx.x % kSmTileThreads;
  float4* wsm = reinterpret_cast<float4*>(smf) + worker * kSmGemmQuats;
  unsigned bar_target = 0;
  for (int q = 0; q < P.nph; ++q) {
    const Phase& ph = P.ph[q];
    if (ph.kind == PH_PREP) {
      const int64_t nW = (int64_t)P.r * P.c, nO = (int64_t)P.c * P.k;
      for (int64_t e = (int64_t)vb * blockDim.x + threadIdx.x; e < nW + nO;
           e += (int64_t)vg * blockDim.x) {
        if (e < nW) {
          const int64_t i = e / P.c, j = e % P.c;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            reinterpret_cast<float*>(P.W32.p[t])[i * P.W32.ld + j] = (float)ld_as_double(P.Win, t, i, j);
        } else {
          const int64_t f = e - nW;
          randn_entry(P.Om, f, P.k, P.seed, 0x51u);
        }
      }
    } else if (ph.kind == PH_GEMM) {
      __shared__ int last_sh[kFusedWorkers];
      int tnc[2], ntiles[2], items[2];
      for (int j = 0; j < 2; ++j) {
        const Job& jb = ph.job[j];
        const int tmc = j < ph.njobs ? (jb.g.M + kSmTS - 1) / kSmTS : 0;
        tnc[j] = j < ph.njobs ? (jb.g.N + kSmTS - 1) / kSmTS : 0;
        ntiles[j] = jb.upper ? tnc[j] * (tnc[j] + 1) / 2 : tmc * tnc[j];
        items[j] = ntiles[j] * (j < ph.njobs ? jb.splits : 0);
      }
      // item -> one per SM first (worker 0 of every CTA), then worker 1;
      // job 1's items follow job 0's, with their own partials and counts
      for (int t = vb + vg * worker; t < items[0] + items[1]; t += vg * kFusedWorkers) {
        const int j = t < items[0] ? 0 : 1;
        const Job& jb = ph.job[j];
        const int tt = j == 0 ? t : t - items[0];
        const int tile = tt % ntiles[j], sp = tt / ntiles[j];
        int tm, tn;
        tile_of(tile, tnc[j], jb.upper, tm, tn);
        const int kb = sp * jb.kchunk;
        const int ke = kb + jb.kchunk < jb.g.K ? kb + jb.kchunk : jb.g.K;
        const float4 acc = sm_tile_acc(jb.g, tm, tn, kb, ke, wsm, wtid, 1 + worker);
        if (jb.splits == 1) {
          sm_tile_store(jb.g, tm, tn, wtid, acc);
          continue;
        }
        const size_t pbase = j == 0 ? 0 : (size_t)items[0];
        unsigned* cnt = P.cnt + (j == 0 ? 0 : ntiles[0]) + tile;
        P.part[(pbase + (size_t)tile * jb.splits + sp) * kSmTileThreads + wtid] = acc;
        __threadfence();
        worker_sync(1 + worker);
        if (wtid == 0) last_sh[worker] = atomicAdd(cnt, 1u) == (unsigned)(jb.splits - 1);
        worker_sync(1 + worker);
        if (last_sh[worker]) {
          __threadfence();
          // every partial in flight at once, then the sum in split order
          const float4* src = P.part + (pbase + (size_t)tile * jb.splits) * kSmTileThreads + wtid;
          float4 part[kMaxSplits];
#pragma unroll
          for (int q2 = 0; q2 < kMaxSplits; ++q2)
            part[q2] = q2 < jb.splits ? __ldcg(src + (size_t)q2 * kSmTileThreads) : make_float4(0.f, 0.f, 0.f, 0.f);
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q2 = 0; q2 < kMaxSplits; ++q2) sum = f4add(sum, part[q2]);
          sm_tile_store(jb.g, tm, tn, wtid, sum);
          if (wtid == 0) *cnt = 0u;   // ready for the next step, after the grid barrier
        }
      }
    } else {   // PH_SOLVE
      const int rows0 = ph.job[0].g.M, rows = rows0 + (ph.njobs > 1 ? ph.job[1].g.M : 0);
      if (vb < rows) {   // CTAs without rows skip the factorisation
        SolveJobs sj;
        sj.Y0 = ph.job[0].g.X;
        sj.Z0 = ph.job[0].g.Z;
        sj.Y1 = ph.job[1].g.X;
        sj.Z1 = ph.job[1].g.Z;
        sj.rows0 = rows0;
        sj.rows = rows;
        sj.vb = vb;
        sj.vg = vg;
        // R packed at the start of shared memory, as the row solves read it;
        // the first kSolveRowWarps rows of this CTA are solved along the way
        const int rode = sm_chol(ph.G, ph.k, reinterpret_cast<float*>(smf), P.status,
                                 smf + solve_chol_off(ph.k), &sj);
        const int warp = threadIdx.x >> 5, nw = kFusedThreads / 32;
        for (int i = rode + warp;; i += nw) {
          const int row = solve_row_of(i, vb, vg);
          if (row >= rows) break;
          const Job& jb = ph.job[row < rows0 ? 0 : 1];
          sm_trsm_row_any(jb.g.X, jb.g.Z, row < rows0 ? row : row - rows0, jb.g.K, smf);
        }
      }
    }
    if (q + 1 < P.nph) {
      if (vg == 1) __syncthreads();   // the CTA's own global writes, then its reads
      else if (!grid_sync(P.bar, P.status, bar_target)) return;
    }
  }
  if (vb == 0 && threadIdx.x == 0 && P.rank_out != nullptr) {
    P.rank_out[0] = P.k;
    P.rank_out[1] = 2;
  }
}

__global__ void __launch_bounds__(kFusedThreads, 1) k_pinv_fused(const __grid_constant__ FusedProg P) {
  fused_program(P, (int)blockIdx.x, (int)gridDim.x);
}

// One problem per CTA: CTA b runs the program progs[order[b]] alone (the
// order puts the largest problems first, so that the small ones fill in).
__global__ void __launch_bounds__(kFusedThreads) k_pinv_fused_each(const FusedProg* __restrict__ progs,
                                                                   const int* __restrict__ order) {
  fused_program(progs[order[blockIdx.x]], 0, 1);
}

// Product X (op) Y (op) -> Z of a GEMM step.
struct GemmSpec {
  bool xh, yh;
  int M, N, K;
  QPtr X, Y, Z;
  bool upper;   // Z square and only its upper triangle is needed (a Gram)
};

struct ProgBuilder {
  FusedProg p{};
  bool ok = true;
  int workers = 1;   // tile workers of the launch
  Phase* next(int kind) {
    if (p.nph >= kMaxPhases) { ok = false; return nullptr; }
    Phase* ph = &p.ph[p.nph++];
    ph->kind = kind;
    return ph;
  }
  static int tiles_of(const GemmSpec& s) {
    const int tmc = (s.M + kSmTS - 1) / kSmTS, tnc = (s.N + kSmTS - 1) / kSmTS;
    return (s.upper && s.M == s.N) ? tnc * (tnc + 1) / 2 : tmc * tnc;
  }
  // one or two products in one step; k-range splits fill the workers
  void gemm(const GemmSpec* specs, int n) {
    Phase* ph = next(PH_GEMM);
    if (ph == nullptr) return;
    ph->njobs = n;
    int all_tiles = 0;
    for (int j = 0; j < n; ++j) all_tiles += tiles_of(specs[j]);
    int used = 0, cnts = 0;
    for (int j = 0; j < n; ++j) {
      const GemmSpec& s = specs[j];
      Job& jb = ph->job[j];
      jb.g = SmallGemmArgs{s.X, s.Y, s.Z, s.M, s.N, s.K, 1.0f, 0.0f, s.xh ? 1 : 0, s.yh ? 1 : 0};
      jb.upper = (s.upper && s.M == s.N) ? 1 : 0;
      const int ntiles = tiles_of(s);
      const int slices = (s.K + kSmBK - 1) / kSmBK;
      int splits = workers / all_tiles;
      if (splits > kMaxSplits) splits = kMaxSplits;
      if (splits > slices) splits = slices;
      if (splits < 2) splits = 1;
      const int per = (slices + splits - 1) / splits;
      jb.kchunk = per * kSmBK;
      jb.splits = (slices + per - 1) / per;
      if (jb.splits > 1) {
        used += ntiles * jb.splits;   // partial tiles of the step
        cnts += ntiles;
      }
    }
    if (used > kMaxPartTiles || cnts > kMaxPartTiles) {   // no room: no splits
      for (int j = 0; j < n; ++j) {
        ph->job[j].splits = 1;
        ph->job[j].kchunk = ((specs[j].K + kSmBK - 1) / kSmBK) * kSmBK;
      }
    }
  }
  void gemm(const GemmSpec& s) { gemm(&s, 1); }
  void gemm2(const GemmSpec& a, const GemmSpec& b) {
    const GemmSpec two[2] = {a, b};
    gemm(two, 2);
  }
  // G = R^H R, then Z = Y R^-1 (Y, Z rows x k; Z may be Y), and a second
  // solve with the same R
  void solve(const QPtr& G, const QPtr& Y, const QPtr& Z, int rows, int k, const QPtr* Y2 = nullptr,
             const QPtr* Z2 = nullptr, int rows2 = 0) {
    Phase* ph = next(PH_SOLVE);
    if (ph == nullptr) return;
    ph->k = k;
    ph->G = G;
    ph->njobs = Y2 != nullptr ? 2 : 1;
    ph->job[0].g = SmallGemmArgs{Y, Y, Z, rows, k, k, 1.0f, 0.0f, 0, 0};
    ph->job[0].splits = 1;
    if (Y2 != nullptr) {
      ph->job[1].g = SmallGemmArgs{*Y2, *Y2, *Z2, rows2, k, k, 1.0f, 0.0f, 0, 0};
      ph->job[1].splits = 1;
    }
  }
  GemmSpec gram(const QPtr& Y, int rows, int k, const QPtr& G) {
    return GemmSpec{true, false, k, k, rows, Y, Y, G, true};
  }
};

// The subspace program for the r x c W with cap k into b (its workers set),
// over the carve w; U receives W_k^+.
static void build_program(ProgBuilder& b, const FastWs& w, const qmcur_qmat* U, int ri, int ci,
                          int k) {
  b.p.ph[b.p.nph++].kind = PH_PREP;
  // Intermediate bases only have to span the subspaces (one CholeskyQR
  // pass); each product with W starts from an orthonormal basis, because
  // forming it from the unnormalised one and solving afterwards would scale
  // its rounding by the basis' condition number.  The last P and Q are
  // orthonormal to working accuracy (CholeskyQR2), and W P = Q R2 R1.
  const QPtr Uo = [&] {
    QPtr q;
    for (int t = 0; t < 4; ++t) q.p[t] = U->plane[t];
    q.ld = U->ld;
    q.dtype = U->dtype;
    return q;
  }();
  b.gemm(GemmSpec{false, false, ri, k, ci, w.W32, w.Om, w.Y, false});          // Y = W Omega
  b.gemm(b.gram(w.Y, ri, k, w.G));                                              // Q0 = orth(Y)
  b.solve(w.G, w.Y, w.Q, ri, k);
  b.gemm(GemmSpec{true, false, ci, k, ri, w.W32, w.Q, w.Z, false});            // P1 = orth(W^H Q0)
  b.gemm(b.gram(w.Z, ci, k, w.G));
  b.solve(w.G, w.Z, w.P, ci, k);
  b.gemm(GemmSpec{false, false, ri, k, ci, w.W32, w.P, w.Y, false});           // Q1 = orth(W P1)
  b.gemm(b.gram(w.Y, ri, k, w.G));
  b.solve(w.G, w.Y, w.Q, ri, k);
  b.gemm(GemmSpec{true, false, ci, k, ri, w.W32, w.Q, w.Z, false});            // Z = W^H Q1
  // P = orth2(Z): T = Z R1^-1, P = T R2^-1.  T is orthonormal to working
  // accuracy and R2 close to I, so Y = W P is formed as (W T) R2^-1 beside
  // the second Gram matrix and solved with P.
  b.gemm(b.gram(w.Z, ci, k, w.G));
  b.solve(w.G, w.Z, w.T, ci, k);
  b.gemm2(b.gram(w.T, ci, k, w.G), GemmSpec{false, false, ri, k, ci, w.W32, w.T, w.Y, false});
  b.solve(w.G, w.T, w.P, ci, k, &w.Y, &w.Y, ri);
  // Q = orth2(Y), Y = Q R2 R1, and U = P R1^-1 R2^-1 Q^H: the solves of P
  // ride along with those of the basis, one factor at a time
  b.gemm(b.gram(w.Y, ri, k, w.G));
  b.solve(w.G, w.Y, w.T, ri, k, &w.P, &w.Z, ci);                               // R1
  b.gemm(b.gram(w.T, ri, k, w.G));
  b.solve(w.G, w.T, w.Q, ri, k, &w.Z, &w.Y, ci);                               // R2
  b.gemm(GemmSpec{false, true, ci, ri, k, w.Y, w.Q, Uo, false});
}

qmcur_status launch_pinv_fast(const qmcur_qmat* W, int32_t rank_cap, qmcur_qmat* U,
                              int32_t* rank_out, uint64_t seed, void* ws, size_t ws_bytes,
                              int32_t* dev_status, cudaStream_t st) {
  const int64_t r = W->rows, c = W->cols;
  const int64_t nmin = r < c ? r : c;
  if (rank_cap < 1) return QMCUR_ERR_UNSUPPORTED;   // the method needs the cap
  const int k = (int)(rank_cap < nmin ? rank_cap : nmin);
  if (k > kSmallCholMax || r > 65535 || c > 65535) return QMCUR_ERR_UNSUPPORTED;
  Carve cv(ws, ws_bytes);
  FastWs w = carve_fast(cv, r, c, k);
  float4* part = cv.take<float4>((size_t)kMaxPartTiles * kSmTileThreads);
  unsigned* bar = cv.take<unsigned>(4 + kMaxPartTiles);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      dev < 0 || dev >= 64)
    return QMCUR_ERR_CUDA;
  static bool attr_set[64] = {};
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_pinv_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fused_smem(kSmallCholMax)) != cudaSuccess)
      return QMCUR_ERR_CUDA;
    attr_set[dev] = true;
  }
  const size_t smem = fused_smem(k);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pinv_fused, kFusedThreads, smem) !=
      cudaSuccess)
    return QMCUR_ERR_CUDA;
  if (per_sm < 1) return QMCUR_ERR_CUDA;
  const int ri = (int)r, ci = (int)c;
  // one CTA per SM at most: a GEMM step has at most ~2 x SMs useful items
  const int grid = cta_cap(sms);
  ProgBuilder b;
  b.workers = grid * kFusedWorkers;
  build_program(b, w, U, ri, ci, k);
  if (!b.ok) return QMCUR_ERR_UNSUPPORTED;
  b.p.Win = view(W);
  b.p.W32 = w.W32;
  b.p.Om = w.Om;
  b.p.r = ri;
  b.p.c = ci;
  b.p.k = k;
  b.p.seed = seed;
  b.p.bar = bar;
  b.p.cnt = bar + 4;
  b.p.part = part;
  b.p.status = dev_status;
  b.p.rank_out = rank_out;
  if (cudaMemsetAsync(bar, 0, (4 + kMaxPartTiles) * sizeof(unsigned), st) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  void* args[] = {(void*)&b.p};
  return cuda_ok(cudaLaunchCooperativeKernel((const void*)k_pinv_fused, dim3(grid),
                                             dim3(kFusedThreads), args, smem, st));
}

// ---------------------------------------------------------------------------
// One problem per CTA (the batched path): each problem's program, built with
// a single tile worker (no split-k partials), over its own carve of the
// batch's arena; CTA b runs the program order[b].

size_t pinv_each_ws_bytes(int64_t r, int64_t c, int64_t k) {
  Carve cv(nullptr, 0);
  carve_fast(cv, r, c, k);
  return cv.off;
}

size_t pinv_each_prog_bytes() { return sizeof(FusedProg); }

qmcur_status pinv_each_build(const qmcur_qmat* W, int32_t rank_cap, qmcur_qmat* U,
                             int32_t* rank_out, uint64_t seed, void* ws, size_t ws_bytes,
                             int32_t* dev_status, void* prog_out, int* k_out) {
  const int64_t r = W->rows, c = W->cols;
  const int64_t nmin = r < c ? r : c;
  if (rank_cap < 1) return QMCUR_ERR_UNSUPPORTED;
  const int k = (int)(rank_cap < nmin ? rank_cap : nmin);
  if (k > kSmallCholMax || r > 65535 || c > 65535) return QMCUR_ERR_UNSUPPORTED;
  Carve cv(ws, ws_bytes);
  FastWs w = carve_fast(cv, r, c, k);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  ProgBuilder b;
  b.workers = 1;   // one CTA: never split k (no partial tiles)
  build_program(b, w, U, (int)r, (int)c, k);
  if (!b.ok) return QMCUR_ERR_UNSUPPORTED;
  b.p.Win = view(W);
  b.p.W32 = w.W32;
  b.p.Om = w.Om;
  b.p.r = (int)r;
  b.p.c = (int)c;
  b.p.k = k;
  b.p.seed = seed;
  b.p.bar = nullptr;
  b.p.cnt = nullptr;
  b.p.part = nullptr;
  b.p.status = dev_status;
  b.p.rank_out = rank_out;
  *static_cast<FusedProg*>(prog_out) = b.p;
  *k_out = k;
  return QMCUR_OK;
}

qmcur_status pinv_each_launch(const void* dprogs, const int* dorder, int count, int kmax,
                              cudaStream_t st) {
  const size_t smem = fused_smem(kmax);
  if (cudaFuncSetAttribute(k_pinv_fused_each, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  k_pinv_fused_each<<<count, kFusedThreads, smem, st>>>(static_cast<const FusedProg*>(dprogs), dorder);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
