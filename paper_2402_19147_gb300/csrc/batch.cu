// Batched, grouped QMCUR: many independent problems of uneven shapes
// decomposed with one launch per stage over a device problem table, the
// whole pipeline captured once in a CUDA graph (qmcur_batch_plan) and
// replayed (qmcur_batch_run).
//
// Stages (Algorithm 1 per problem, U = W^+ with the rank cap):
//   k_batch_norm_chunk, k_batch_norm_fold   column and row squared norms (FP32
//                    runs of 4 planes x 8 entries carried in FP64, fixed
//                    order; A read once, in 32-row chunks), ||A||_F^2, the
//                    probabilities (Sec. 3.1);
//   k_batch_sample   one CTA per index set per problem (the Philox sampler of
//                    the single-problem path, stream_id = problem index);
//   k_batch_gather   C, R, W per problem;
//   k_batch_jacobi   one CTA per problem: FP32 one-sided quaternion Jacobi on
//                    the (<= 80 x 80) intersection held in shared memory, the
//                    rcond / rank-cap truncation, U = V Sigma^-2 G^H;
//   or k_pinv_fused_each (opts->pinv_method = QMCUR_PINV_SUBSPACE_FP32):
//                    one CTA per problem runs the FP32 subspace program of
//                    the single-problem path (pinv_fast.cu) on its own
//                    intersection, largest problems first;
//   or k_pinv_refine_each (opts->pinv_method = QMCUR_PINV_REFINED_FP64):
//                    one CTA per problem runs the FP64-accurate refined
//                    program of the single-problem path (pinv_refine.cu),
//                    writing U in FP64 and its FP32 copy for the GEMMs;
//   k_batch_gemm     grouped quaternion GEMMs over a flattened tile list
//                    (T = U R, then Z = C T with the residual fused), tile
//                    shape chosen per GEMM by timing the candidates at plan
//                    time (the autotuner); in a split precision both are
//                    instead one grouped tcgen05 launch each over stacked
//                    operand pieces (k_split_table, then k_qgemm_tc);
//   k_batch_fold     per problem, the tile partials of the residual in order.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "sample_impl.cuh"
#include "small.cuh"
#include "tc_group.cuh"

namespace qmcur {

// The subspace core, one problem per CTA (pinv_fast.cu).
size_t pinv_each_ws_bytes(int64_t r, int64_t c, int64_t k);
size_t pinv_each_prog_bytes();
qmcur_status pinv_each_build(const qmcur_qmat* W, int32_t rank_cap, qmcur_qmat* U,
                             int32_t* rank_out, uint64_t seed, void* ws, size_t ws_bytes,
                             int32_t* dev_status, void* prog_out, int* k_out);
qmcur_status pinv_each_launch(const void* dprogs, const int* dorder, int count, int kmax,
                              cudaStream_t st);
// The FP64-accurate refined core, one problem per CTA (pinv_refine.cu).
size_t refine_each_ws_bytes(int64_t r, int64_t c, int64_t k);
size_t refine_each_args_bytes();
qmcur_status refine_each_build(const qmcur_qmat* W, int32_t rank_cap, int32_t max_iter,
                               qmcur_qmat* U, qmcur_qmat* U2, int32_t* rank_out, int32_t* status,
                               uint64_t seed, void* ws, size_t ws_bytes, void* args_out,
                               int* k_out);
qmcur_status refine_each_launch(const void* dargs, const int* dorder, int count, int kmax,
                                int32_t* batch_status, cudaStream_t st);

constexpr int kBatchMaxCore = 80;      // largest min(r, c) held by k_batch_jacobi
constexpr int64_t kBatchCoreSmem = 200 * 1024;   // bytes of G and V in shared memory

struct BatchProblem {
  QView A;                 // m x n, F32
  int m, n, c, r, rank_cap;
  double* col_p;           // n
  double* row_p;           // m
  int32_t* J;              // c
  int32_t* I;              // r
  QView C, R, W, U, T;     // F32: m x c, r x n, r x c, c x r, c x n
  QView U64;               // F64 c x r (the refined core only; else unset)
  double* out3;            // {rel, num, den}
  int32_t* info;           // {rank, sweeps, status}
  int tile_base2;          // first tile of this problem in the second GEMM's list
  int tiles2;              // its number of tiles
  int64_t colpart_off;     // its column partials in the norms' scratch (doubles)
  int64_t zarow;           // first row of its C pieces in Z's stacked A operand (split plans)
};

// Z = C T's stacked A operand, which the gather fills with C's pieces as it
// gathers C (split plans; base null otherwise): pieces [(q 4 + t)][row][k],
// rows of kpad elements, plane stride `plane` elements.
struct CPieces {
  void* base;
  int64_t kpad, plane;
  int npieces;
  int bf16;
};

struct GTile {
  int prob, m0, n0;
};

namespace {

__device__ __forceinline__ float4 ldf4(const QView& v, int64_t i, int64_t j) {
  const int64_t o = i * v.ld + j;
  return make_float4(reinterpret_cast<const float*>(v.p[0])[o], reinterpret_cast<const float*>(v.p[1])[o],
                     reinterpret_cast<const float*>(v.p[2])[o], reinterpret_cast<const float*>(v.p[3])[o]);
}
__device__ __forceinline__ void stf4(const QView& v, int64_t i, int64_t j, float4 q) {
  const int64_t o = i * v.ld + j;
  reinterpret_cast<float*>(v.p[0])[o] = q.x;
  reinterpret_cast<float*>(v.p[1])[o] = q.y;
  reinterpret_cast<float*>(v.p[2])[o] = q.z;
  reinterpret_cast<float*>(v.p[3])[o] = q.w;
}

// ----------------------------------------------------------------- norms -
// Two passes.  k_batch_norm_chunk: CTA (chunk, b) takes rows 32 chunk ..
// 32 chunk + 31 of problem b, reading each entry once from HBM: the rows'
// squared norms (one warp per row, lanes over columns, FP32 runs of 8
// entries carried in FP64, a warp tree) are complete; the columns' sums over
// the chunk (one thread per column, FP32 runs of 8 rows, in order) go to
// colpart.  k_batch_norm_fold: one CTA per problem adds the chunks' column
// sums in chunk order, forms ||A||_F^2 and the probabilities (Sec. 3.1).
constexpr int kNormChunk = 32;

__global__ void __launch_bounds__(256) k_batch_norm_chunk(const BatchProblem* probs,
                                                          double* colpart_base) {
  const BatchProblem& P = probs[blockIdx.y];
  const int m = P.m, n = P.n;
  const int i0 = blockIdx.x * kNormChunk;
  if (i0 >= m) return;
  const int i1 = i0 + kNormChunk < m ? i0 + kNormChunk : m;
  double* colpart = colpart_base + P.colpart_off + (int64_t)blockIdx.x * n;
  for (int j = threadIdx.x; j < n; j += 256) {
    double s = 0.0;
    for (int r0 = i0; r0 < i1; r0 += 8) {
      float f = 0.f;
      for (int i = r0; i < r0 + 8 && i < i1; ++i) {
        const float4 a = ldf4(P.A, i, j);
        f = fmaf(a.x, a.x, f); f = fmaf(a.y, a.y, f); f = fmaf(a.z, a.z, f); f = fmaf(a.w, a.w, f);
      }
      s += (double)f;
    }
    colpart[j] = s;
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int i = i0 + warp; i < i1; i += 8) {
    double s = 0.0;
    for (int j0 = 0; j0 < n; j0 += 32 * 8) {
      float f = 0.f;
      for (int j = j0 + lane; j < j0 + 32 * 8 && j < n; j += 32) {
        const float4 a = ldf4(P.A, i, j);
        f = fmaf(a.x, a.x, f); f = fmaf(a.y, a.y, f); f = fmaf(a.z, a.z, f); f = fmaf(a.w, a.w, f);
      }
      s += (double)f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) P.row_p[i] = s;
  }
}

__global__ void __launch_bounds__(256) k_batch_norm_fold(const BatchProblem* probs,
                                                         const double* colpart_base, int norm,
                                                         int32_t* status) {
  const BatchProblem& P = probs[blockIdx.x];
  const int m = P.m, n = P.n, chunks = (m + kNormChunk - 1) / kNormChunk;
  const double* colpart = colpart_base + P.colpart_off;
  __shared__ double red[256];
  double tot = 0.0;
  for (int j = threadIdx.x; j < n; j += 256) {
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += colpart[(int64_t)c * n + j];
    P.col_p[j] = s;
    tot += s;
  }
  red[threadIdx.x] = tot;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double F = red[0];
  if (threadIdx.x == 0) {
    P.out3[2] = F;
    int code = 0;
    if (!isfinite(F)) code = QMCUR_ERR_NONFINITE;
    else if (norm && F == 0.0) code = QMCUR_ERR_ZERO_NORM;
    if (code) { P.info[2] = code; set_status(status, code); }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += 256) P.col_p[j] = norm ? P.col_p[j] / F : 1.0 / (double)n;
  for (int i = threadIdx.x; i < m; i += 256) P.row_p[i] = norm ? P.row_p[i] / F : 1.0 / (double)m;
}

// ---------------------------------------------------------------- sample -
__global__ void __launch_bounds__(kSampleThreads)
k_batch_sample(const BatchProblem* probs, SampleArgs base, int32_t* status) {
  extern __shared__ __align__(16) unsigned char dyn[];
  const int b = blockIdx.x / 2, set = blockIdx.x % 2;
  const BatchProblem& P = probs[b];
  SampleArgs a = base;
  a.prob[0] = P.col_p; a.prob[1] = P.row_p;
  a.N[0] = P.n; a.N[1] = P.m;
  a.count[0] = P.c; a.count[1] = P.r;
  a.out[0] = P.J; a.out[1] = P.I;
  a.P[0] = a.P[1] = nullptr;
  a.stream_id = (uint32_t)b;
  a.max_attempts[0] = 64 * (int64_t)P.c + 1024;
  a.max_attempts[1] = 64 * (int64_t)P.r + 1024;
  a.status = status;
  a.attempts_out = nullptr;
  sample_one_set(a, set, 1, dyn);
}

// ---------------------------------------------------------------- gather -
__global__ void k_batch_gather(const BatchProblem* probs, CPieces cp) {
  const BatchProblem& P = probs[blockIdx.y];
  const int64_t nc = (int64_t)P.m * P.c, nr = (int64_t)P.r * P.n, nw = (int64_t)P.r * P.c;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nc + nr + nw;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i, j, si, sj;
    const QView* out;
    if (e < nc) { i = e / P.c; j = e % P.c; si = i; sj = P.J[j]; out = &P.C; }
    else if (e < nc + nr) { const int64_t f = e - nc; i = f / P.n; j = f % P.n; si = P.I[i]; sj = j; out = &P.R; }
    else { const int64_t f = e - nc - nr; i = f / P.c; j = f % P.c; si = P.I[i]; sj = P.J[j]; out = &P.W; }
    const bool in = si >= 0 && si < P.m && sj >= 0 && sj < P.n;
    const float4 v = in ? ldf4(P.A, si, sj) : make_float4(0.f, 0.f, 0.f, 0.f);
    stf4(*out, i, j, v);
    if (e < nc && cp.base != nullptr && P.zarow >= 0) {   // C's pieces: row i, k = j
      const float pl4[4] = {v.x, v.y, v.z, v.w};
      const int64_t rowoff = (P.zarow + i) * cp.kpad + j;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        float pc[3];
        if (cp.bf16) split_value<true, float>(pl4[t], cp.npieces, pc);
        else split_value<false, float>(pl4[t], cp.npieces, pc);
        for (int q = 0; q < cp.npieces; ++q) {
          const int64_t idx = (int64_t)(q * 4 + t) * cp.plane + rowoff;
          if (cp.bf16) reinterpret_cast<__nv_bfloat16*>(cp.base)[idx] = __float2bfloat16_rn(pc[q]);
          else reinterpret_cast<float*>(cp.base)[idx] = pc[q];
        }
      }
    }
  }
}

// ------------------------------------------------- FP32 Jacobi per problem -
__device__ __forceinline__ void circle(int N, int step, int p, int& a, int& b) {
  const int M = N - 1;
  if (p == 0) { a = M; b = step % M; }
  else { a = (step + p) % M; b = (step - p + M) % M; }
}

__global__ void __launch_bounds__(1024) k_batch_jacobi(const BatchProblem* probs, double rcond,
                                                       int max_sweeps) {
  extern __shared__ float4 js[];
  const BatchProblem& P = probs[blockIdx.x];
  const int r = P.r, c = P.c;
  const bool tr = c > r;                 // work on W^H when W is wide
  const int nr = tr ? c : r, nc = tr ? r : c;
  float4* G = js;                        // G[j * nr + i], column j contiguous
  float4* V = js + nr * nc;              // V[j * nc + i]
  float* sig = reinterpret_cast<float*>(V + nc * nc);
  int* pos = reinterpret_cast<int*>(sig + nc);
  __shared__ int rotated, keep_cnt;
  for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
    const int j = e / nr, i = e % nr;
    float4 q = tr ? ldf4(P.W, j, i) : ldf4(P.W, i, j);
    if (tr) { q.y = -q.y; q.z = -q.z; q.w = -q.w; }
    G[e] = q;
  }
  for (int e = threadIdx.x; e < nc * nc; e += blockDim.x)
    V[e] = make_float4((e / nc == e % nc) ? 1.f : 0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  const float tol = sqrtf((float)nr) * 0x1.0p-23f;
  const int N = nc + (nc & 1), npairs = N / 2;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nwarps = blockDim.x / 32;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    __syncthreads();                     // every thread has read the last flag
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int step = 0; step < N - 1; ++step) {
      for (int p = warp; p < npairs; p += nwarps) {
        int a, b;
        circle(N, step, p, a, b);
        if (a >= nc || b >= nc) continue;
        float al = 0.f, be = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
        for (int i = lane; i < nr; i += 32) {
          const float4 x = G[a * nr + i], y = G[b * nr + i];
          al += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
          be += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
          g0 += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
          g1 += x.x * y.y - x.y * y.x - x.z * y.w + x.w * y.z;
          g2 += x.x * y.z + x.y * y.w - x.z * y.x - x.w * y.y;
          g3 += x.x * y.w - x.y * y.z + x.z * y.y - x.w * y.x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          g0 += __shfl_xor_sync(0xffffffffu, g0, o);
          g1 += __shfl_xor_sync(0xffffffffu, g1, o);
          g2 += __shfl_xor_sync(0xffffffffu, g2, o);
          g3 += __shfl_xor_sync(0xffffffffu, g3, o);
        }
        const float gam = sqrtf(g0 * g0 + g1 * g1 + g2 * g2 + g3 * g3);
        if (!(al > 0.f) || !(be > 0.f) || !(gam > tol * sqrtf(al) * sqrtf(be)) ||
            fminf(al, be) < tol * tol * fmaxf(al, be))
          continue;
        if (lane == 0) rotated = 1;
        const float zeta = (be - al) / (2.f * gam);
        const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float cs = 1.f / sqrtf(1.f + t * t), sn = cs * t;
        const float w0 = g0 / gam, w1 = -g1 / gam, w2 = -g2 / gam, w3 = -g3 / gam;
        for (int mat = 0; mat < 2; ++mat) {
          float4* X = mat == 0 ? G : V;
          const int len = mat == 0 ? nr : nc;
          for (int i = lane; i < len; i += 32) {
            const float4 x = X[a * len + i], q = X[b * len + i];
            const float4 y = make_float4(q.x * w0 - q.y * w1 - q.z * w2 - q.w * w3,
                                         q.x * w1 + q.y * w0 + q.z * w3 - q.w * w2,
                                         q.x * w2 - q.y * w3 + q.z * w0 + q.w * w1,
                                         q.x * w3 + q.y * w2 - q.z * w1 + q.w * w0);
            X[a * len + i] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y,
                                         cs * x.z - sn * y.z, cs * x.w - sn * y.w);
            X[b * len + i] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y,
                                         sn * x.z + cs * y.z, sn * x.w + cs * y.w);
          }
        }
      }
      __syncthreads();
    }
    if (!rotated) { ++sweep; break; }
  }
  // singular values, order, truncation
  for (int j = warp; j < nc; j += nwarps) {
    float s = 0.f;
    for (int i = lane; i < nr; i += 32) {
      const float4 q = G[j * nr + i];
      s += q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sig[j] = sqrtf(s);
  }
  if (threadIdx.x == 0) keep_cnt = 0;
  __syncthreads();
  float smax = 0.f;
  for (int j = 0; j < nc; ++j) smax = fmaxf(smax, sig[j]);
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    int ps = 0;
    for (int i = 0; i < nc; ++i) ps += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
    pos[j] = ps;
    if (smax > 0.f && (double)sig[j] > rcond * (double)smax) atomicAdd(&keep_cnt, 1);
  }
  __syncthreads();
  int k = keep_cnt;
  if (P.rank_cap > 0 && k > P.rank_cap) k = P.rank_cap;
  // U[a][b] = sum_{kept j} X[a][j] sigma_j^-2 conj(Y[b][j]); (X, Y) = (V, G) or (G, V)
  for (int e = threadIdx.x; e < c * r; e += blockDim.x) {
    const int ai = e / r, bi = e % r;
    float u0 = 0.f, u1 = 0.f, u2 = 0.f, u3 = 0.f;
    for (int j = 0; j < nc; ++j) {
      if (pos[j] >= k) continue;
      const float w = 1.f / (sig[j] * sig[j]);
      const float4 x = tr ? G[j * nr + ai] : V[j * nc + ai];
      const float4 y = tr ? V[j * nc + bi] : G[j * nr + bi];
      u0 += w * (x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w);
      u1 += w * (-x.x * y.y + x.y * y.x - x.z * y.w + x.w * y.z);
      u2 += w * (-x.x * y.z + x.y * y.w + x.z * y.x - x.w * y.y);
      u3 += w * (-x.x * y.w - x.y * y.z + x.z * y.y + x.w * y.x);
    }
    stf4(P.U, ai, bi, make_float4(u0, u1, u2, u3));
  }
  if (threadIdx.x == 0) { P.info[0] = k; P.info[1] = sweep; }
}

// ------------------------------------------------------- grouped GEMMs ---
// Z = X Y per tile of a problem; which == 0: T = U R (stored), which == 1:
// C T with the residual against A fused (per-tile FP64 partials).
template <int BMQ, int BNQ, int TMQ, int TNQ>
__global__ void __launch_bounds__(256) k_batch_gemm(const BatchProblem* probs, const GTile* tiles,
                                                    int which, double* partial) {
  constexpr int BKQ = 8;
  constexpr int TX = BNQ / TNQ;                 // threads along n
  static_assert((BMQ / TMQ) * (BNQ / TNQ) == 256, "256 threads");
  const GTile tl = tiles[blockIdx.x];
  const BatchProblem& P = probs[tl.prob];
  const QView& X = which == 0 ? P.U : P.C;
  const QView& Y = which == 0 ? P.R : P.T;
  const int M = which == 0 ? P.c : P.m, N = P.n, K = which == 0 ? P.r : P.c;
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  __shared__ float xs[4][BKQ][BMQ];
  __shared__ float ys[4][BKQ][BNQ];
  float acc[TMQ][TNQ][4];
#pragma unroll
  for (int i = 0; i < TMQ; ++i)
#pragma unroll
    for (int j = 0; j < TNQ; ++j)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[i][j][t] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BKQ) {
    for (int e = tid; e < BMQ * BKQ; e += 256) {
      const int mm = e / BKQ, kk = e % BKQ;
      const int gi = tl.m0 + mm, gk = k0 + kk;
      const float4 q = (gi < M && gk < K) ? ldf4(X, gi, gk) : make_float4(0.f, 0.f, 0.f, 0.f);
      xs[0][kk][mm] = q.x; xs[1][kk][mm] = q.y; xs[2][kk][mm] = q.z; xs[3][kk][mm] = q.w;
    }
    for (int e = tid; e < BNQ * BKQ; e += 256) {
      const int kk = e / BNQ, nn = e % BNQ;
      const int gk = k0 + kk, gj = tl.n0 + nn;
      const float4 q = (gk < K && gj < N) ? ldf4(Y, gk, gj) : make_float4(0.f, 0.f, 0.f, 0.f);
      ys[0][kk][nn] = q.x; ys[1][kk][nn] = q.y; ys[2][kk][nn] = q.z; ys[3][kk][nn] = q.w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BKQ; ++kk) {
      float a[TMQ][4], b[TNQ][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
#pragma unroll
        for (int i = 0; i < TMQ; ++i) a[i][t] = xs[t][kk][ty * TMQ + i];
#pragma unroll
        for (int j = 0; j < TNQ; ++j) b[j][t] = ys[t][kk][tx * TNQ + j];
      }
#pragma unroll
      for (int i = 0; i < TMQ; ++i)
#pragma unroll
        for (int j = 0; j < TNQ; ++j) {
          float* z = acc[i][j];
          const float* x = a[i];
          const float* y = b[j];
          z[0] = fmaf(x[0], y[0], z[0]); z[0] = fmaf(-x[1], y[1], z[0]);
          z[0] = fmaf(-x[2], y[2], z[0]); z[0] = fmaf(-x[3], y[3], z[0]);
          z[1] = fmaf(x[0], y[1], z[1]); z[1] = fmaf(x[1], y[0], z[1]);
          z[1] = fmaf(x[2], y[3], z[1]); z[1] = fmaf(-x[3], y[2], z[1]);
          z[2] = fmaf(x[0], y[2], z[2]); z[2] = fmaf(-x[1], y[3], z[2]);
          z[2] = fmaf(x[2], y[0], z[2]); z[2] = fmaf(x[3], y[1], z[2]);
          z[3] = fmaf(x[0], y[3], z[3]); z[3] = fmaf(x[1], y[2], z[3]);
          z[3] = fmaf(-x[2], y[1], z[3]); z[3] = fmaf(x[3], y[0], z[3]);
        }
    }
    __syncthreads();
  }
  if (which == 0) {
#pragma unroll
    for (int i = 0; i < TMQ; ++i)
#pragma unroll
      for (int j = 0; j < TNQ; ++j) {
        const int gi = tl.m0 + ty * TMQ + i, gj = tl.n0 + tx * TNQ + j;
        if (gi < M && gj < N) stf4(P.T, gi, gj, make_float4(acc[i][j][0], acc[i][j][1], acc[i][j][2], acc[i][j][3]));
      }
    return;
  }
  double num = 0.0, den = 0.0;
#pragma unroll
  for (int i = 0; i < TMQ; ++i) {
    float rn = 0.f, rd = 0.f;
#pragma unroll
    for (int j = 0; j < TNQ; ++j) {
      const int gi = tl.m0 + ty * TMQ + i, gj = tl.n0 + tx * TNQ + j;
      if (gi < M && gj < N) {
        const float4 av = ldf4(P.A, gi, gj);
        const float d0 = av.x - acc[i][j][0], d1 = av.y - acc[i][j][1];
        const float d2 = av.z - acc[i][j][2], d3 = av.w - acc[i][j][3];
        rn += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
        rd += av.x * av.x + av.y * av.y + av.z * av.z + av.w * av.w;
      }
    }
    num += (double)rn;
    den += (double)rd;
  }
  __shared__ double red[2][256];
  red[0][tid] = num;
  red[1][tid] = den;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) { red[0][tid] += red[0][tid + w]; red[1][tid] += red[1][tid + w]; }
    __syncthreads();
  }
  if (tid == 0) {
    partial[2 * blockIdx.x] = red[0][0];
    partial[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void k_batch_fold(const BatchProblem* probs, const double* partial) {
  const BatchProblem& P = probs[blockIdx.x];
  if (threadIdx.x != 0) return;
  double num = 0.0, den = 0.0;
  for (int t = 0; t < P.tiles2; ++t) {
    num += partial[2 * (P.tile_base2 + t)];
    den += partial[2 * (P.tile_base2 + t) + 1];
  }
  P.out3[0] = den > 0.0 ? sqrt(num / den) : __longlong_as_double(0x7ff8000000000000ll);
  P.out3[1] = num;
  P.out3[2] = den;
}

struct TileCfg {
  int bm, bn;
};
constexpr TileCfg kCfgs[2] = {{64, 64}, {32, 32}};

void launch_batch_gemm(int cfg, const BatchProblem* probs, const GTile* tiles, int ntiles, int which,
                       double* partial, cudaStream_t st) {
  if (ntiles <= 0) return;
  if (cfg == 0) k_batch_gemm<64, 64, 4, 4><<<ntiles, 256, 0, st>>>(probs, tiles, which, partial);
  else k_batch_gemm<32, 32, 2, 2><<<ntiles, 256, 0, st>>>(probs, tiles, which, partial);
}

std::vector<GTile> make_tiles(const std::vector<BatchProblem>& ps, int which, int cfg,
                              std::vector<int>* base = nullptr, std::vector<int>* count = nullptr) {
  std::vector<GTile> t;
  for (size_t b = 0; b < ps.size(); ++b) {
    const int M = which == 0 ? ps[b].c : ps[b].m, N = ps[b].n;
    if (base) base->push_back((int)t.size());
    int cnt = 0;
    for (int m0 = 0; m0 < M; m0 += kCfgs[cfg].bm)
      for (int n0 = 0; n0 < N; n0 += kCfgs[cfg].bn) { t.push_back(GTile{(int)b, m0, n0}); ++cnt; }
    if (count) count->push_back(cnt);
  }
  return t;
}

}  // namespace

// ----------------------------------------------------------------- plan ----
constexpr int kBatchStages = 7;   // norms, sampler, gathers, core, T = U R, Z = C T, fold

struct BatchPlan {
  int count = 0;
  std::vector<BatchProblem> host;
  BatchProblem* dprobs = nullptr;
  GTile* dtiles1 = nullptr;
  GTile* dtiles2 = nullptr;
  int ntiles1 = 0, ntiles2 = 0, cfg1 = 0, cfg2 = 0;
  double* partial = nullptr;
  void* arena = nullptr;
  int32_t* status = nullptr;
  size_t jac_smem = 0, samp_smem = 0;
  bool subspace = false;      // the core: subspace programs instead of the Jacobi
  bool refined = false;       // the core: FP64-accurate refined programs
  void* progs = nullptr;      // device: one subspace program (or refined arguments) per problem
  int* order = nullptr;       // device: problems, largest first
  void* pinv_arena = nullptr;
  int kmax = 0;
  double* colpart = nullptr;  // the norms' per-chunk column sums
  int max_chunks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  qmcur_opts opts{};
  // Z = C T on the tensor cores (opts.prec a split precision): the stacked
  // operand pieces (C's written by the gather, T's by the T stage), the
  // group tables and the tile width
  bool tc = false;
  void* A_all = nullptr;
  void* B_all = nullptr;
  int64_t rows_a = 0, rows_b = 0, kpad = 0;
  TcGroupProb* dgprobs = nullptr;
  TcGroupTile* dgtiles = nullptr;
  int ngtiles = 0, tc_bn = 128;
  // T = U R on the tensor cores, as T^T = R^T U in the split of T (BF16X6
  // under the mixed split) with its epilogue writing Z = C T's B pieces:
  // every problem's R^T (n x r) as rows of A1_all, its U (c x r) as rows of
  // B1_all, K padded to the largest r
  void* A1_all = nullptr;
  void* B1_all = nullptr;
  int64_t rows_a1 = 0, rows_b1 = 0, kpad1 = 0;
  TcSplitJob* djobs1 = nullptr;
  int njobs1 = 0, split_tiles1 = 0;
  TcGroupProb* dgprobs1 = nullptr;
  TcGroupTile* dgtiles1 = nullptr;
  int ngtiles1 = 0;
  // stage boundaries, recorded by the captured graph (qmcur_batch_stage_ms)
  cudaEvent_t ev[kBatchStages + 1] = {};
};

// With timed, the stage boundaries are recorded into p->ev (inside the
// captured graph: one event-record node per boundary).
static qmcur_status enqueue_batch(BatchPlan* p, cudaStream_t st, bool timed = false) {
  auto mark = [&](int i) {   // an external record: a node of the captured graph
    if (timed) cudaEventRecordWithFlags(p->ev[i], st, cudaEventRecordExternal);
  };
  const int norm = p->opts.sampler == QMCUR_SAMPLER_NORM;
  mark(0);
  k_batch_norm_chunk<<<dim3(p->max_chunks, p->count), 256, 0, st>>>(p->dprobs, p->colpart);
  k_batch_norm_fold<<<p->count, 256, 0, st>>>(p->dprobs, p->colpart, norm, p->status);
  mark(1);
  SampleArgs base{};
  base.seed = p->opts.seed;
  base.norm = norm;
  k_batch_sample<<<2 * p->count, kSampleThreads, p->samp_smem, st>>>(p->dprobs, base, p->status);
  mark(2);
  CPieces cp{};
  if (p->tc) {
    cp.base = p->A_all;
    cp.kpad = p->kpad;
    cp.plane = p->rows_a * p->kpad;
    cp.npieces = tc_group_npieces(p->opts.prec);
    cp.bf16 = tc_group_epr(p->opts.prec) == 32;   // 32 BF16 or 16 TF32 per 64-byte row
  }
  k_batch_gather<<<dim3(64, p->count), 256, 0, st>>>(p->dprobs, cp);
  mark(3);
  if (p->refined) {
    const qmcur_status s =
        refine_each_launch(p->progs, p->order, p->count, p->kmax, p->status, st);
    if (s != QMCUR_OK) return s;
  } else if (p->subspace) {
    const qmcur_status s = pinv_each_launch(p->progs, p->order, p->count, p->kmax, st);
    if (s != QMCUR_OK) return s;
  } else {
    k_batch_jacobi<<<p->count, 1024, p->jac_smem, st>>>(
        p->dprobs, p->opts.rcond, p->opts.max_sweeps > 0 ? p->opts.max_sweeps : 30);
  }
  mark(4);
  if (p->tc) {
    qmcur_status s = tc_group_split(p->opts.prec, p->djobs1, p->njobs1, p->split_tiles1, st, 0);
    if (s != QMCUR_OK) return s;
    s = tc_group_t_pieces(p->opts.prec, p->A1_all, p->rows_a1, p->B1_all, p->rows_b1, p->kpad1,
                          p->dgtiles1, p->ngtiles1, p->dgprobs1, p->B_all, p->kpad, p->rows_b,
                          p->status, st);
    if (s != QMCUR_OK) return s;
  } else {
    launch_batch_gemm(p->cfg1, p->dprobs, p->dtiles1, p->ntiles1, 0, nullptr, st);
  }
  mark(5);
  if (p->tc) {
    // (C's pieces come from the gather, T's from the T stage)
    qmcur_status s = tc_group_residual(p->opts.prec, p->tc_bn, p->A_all, p->rows_a, p->B_all, p->rows_b,
                          p->kpad, p->dgtiles, p->ngtiles, p->dgprobs, p->partial, p->status, st);
    if (s != QMCUR_OK) return s;
  } else {
    launch_batch_gemm(p->cfg2, p->dprobs, p->dtiles2, p->ntiles2, 1, p->partial, st);
  }
  mark(6);
  k_batch_fold<<<p->count, 32, 0, st>>>(p->dprobs, p->partial);
  mark(7);
  return cuda_ok(cudaGetLastError());
}

// The tile list of the grouped tensor-core Z = C T at tile width bn (128
// rows of a problem's output by bn columns), with each problem's first tile
// and tile count for the fold.
static std::vector<TcGroupTile> group_tiles(const std::vector<BatchProblem>& ps, int bn,
                                            std::vector<int>* base, std::vector<int>* count) {
  std::vector<TcGroupTile> t;
  for (size_t b = 0; b < ps.size(); ++b) {
    base->push_back((int)t.size());
    int cnt = 0;
    for (int m0 = 0; m0 < ps[b].m; m0 += 128)
      for (int n0 = 0; n0 < ps[b].n; n0 += bn) { t.push_back(TcGroupTile{(int)b, m0, n0}); ++cnt; }
    count->push_back(cnt);
  }
  return t;
}

// Sets the grouped tiles of width bn (device list, partials, fold ranges).
static qmcur_status set_group_tiles(BatchPlan* p, int bn, cudaStream_t st) {
  std::vector<int> b2, c2;
  std::vector<TcGroupTile> t = group_tiles(p->host, bn, &b2, &c2);
  cudaFree(p->dgtiles);
  cudaFree(p->partial);
  p->dgtiles = nullptr;
  p->partial = nullptr;
  if (cudaMalloc(&p->dgtiles, t.size() * sizeof(TcGroupTile)) != cudaSuccess ||
      cudaMalloc(&p->partial, 2 * t.size() * sizeof(double)) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  if (cudaMemcpyAsync(p->dgtiles, t.data(), t.size() * sizeof(TcGroupTile), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  for (int b = 0; b < p->count; ++b) { p->host[b].tile_base2 = b2[b]; p->host[b].tiles2 = c2[b]; }
  p->ngtiles = (int)t.size();
  p->tc_bn = bn;
  if (cudaMemcpyAsync(p->dprobs, p->host.data(), p->count * sizeof(BatchProblem),
                      cudaMemcpyHostToDevice, st) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  // the host vector must outlive its copy
  return cudaStreamSynchronize(st) == cudaSuccess ? QMCUR_OK : QMCUR_ERR_CUDA;
}

// Time the grouped Z = C T at the candidate tile widths on the real batch
// (after a first pass has filled T); the faster stays.
static qmcur_status autotune_group(BatchPlan* p, cudaStream_t st) {
  float best = 1e30f;
  int best_bn = 128;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int cands[2] = {128, 64};
  for (int bn : cands) {
    qmcur_status s = set_group_tiles(p, bn, st);
    if (s != QMCUR_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
    auto run = [&]() {
      return tc_group_residual(p->opts.prec, bn, p->A_all, p->rows_a, p->B_all, p->rows_b, p->kpad,
                               p->dgtiles, p->ngtiles, p->dgprobs, p->partial, p->status, st);
    };
    if ((s = run()) != QMCUR_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return s; }
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 3; ++rep) run();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_bn = bn; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return set_group_tiles(p, best_bn, st);
}

// Time the candidate tile shapes of one grouped GEMM on the real batch.
static int autotune(BatchPlan* p, int which, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::vector<int>, int> cache;
  std::vector<int> key{which};
  for (auto& b : p->host) { key.push_back(which == 0 ? b.c : b.m); key.push_back(b.n); key.push_back(b.c); }
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  float best = 1e30f;
  int best_cfg = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int cfg = 0; cfg < 2; ++cfg) {
    std::vector<GTile> t = make_tiles(p->host, which, cfg);
    GTile* dt = nullptr;
    if (cudaMalloc(&dt, t.size() * sizeof(GTile)) != cudaSuccess) continue;
    cudaMemcpyAsync(dt, t.data(), t.size() * sizeof(GTile), cudaMemcpyHostToDevice, st);
    double* part = nullptr;
    cudaMalloc(&part, 2 * t.size() * sizeof(double));
    launch_batch_gemm(cfg, p->dprobs, dt, (int)t.size(), which, part, st);   // warm
    cudaEventRecord(e0, st);
    for (int rep = 0; rep < 3; ++rep) launch_batch_gemm(cfg, p->dprobs, dt, (int)t.size(), which, part, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_cfg = cfg; }
    cudaFree(part);
    cudaFree(dt);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = best_cfg;
  return best_cfg;
}

static void free_plan(BatchPlan* p) {
  if (p == nullptr) return;
  for (cudaEvent_t& e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->dprobs);
  cudaFree(p->dtiles1);
  cudaFree(p->dtiles2);
  cudaFree(p->partial);
  cudaFree(p->arena);
  cudaFree(p->progs);
  cudaFree(p->order);
  cudaFree(p->pinv_arena);
  cudaFree(p->colpart);
  cudaFree(p->A_all);
  cudaFree(p->B_all);
  cudaFree(p->dgprobs);
  cudaFree(p->dgtiles);
  cudaFree(p->A1_all);
  cudaFree(p->B1_all);
  cudaFree(p->djobs1);
  cudaFree(p->dgprobs1);
  cudaFree(p->dgtiles1);
  delete p;
}

}  // namespace qmcur

using namespace qmcur;

// T = U R on the tensor cores for a split precision, as T^T = R^T U: the
// stacked pieces of every problem's R^T (A operand, rows n) and U (B
// operand, rows c), the split jobs that cut them, the problem table (K = r;
// zrow = the problem's first row zrow[b] of Z = C T's B operand, which the
// epilogue fills with T's pieces) and the tile list (n in 128-row tiles, c
// in kGroupTBn-wide ones).
static qmcur_status build_t_stage(BatchPlan* p, const std::vector<int64_t>& zrow,
                                  cudaStream_t stream) {
  const int32_t pr = p->opts.prec;
  const int64_t epr = tc_group_epr(pr, 0);
  const int count = p->count;
  std::vector<int64_t> rrow(count), urow(count);
  int64_t rmax = 1;
  for (int b = 0; b < count; ++b) {
    rrow[b] = p->rows_a1;
    urow[b] = p->rows_b1;
    p->rows_a1 += p->host[b].n;
    p->rows_b1 += p->host[b].c;
    rmax = std::max<int64_t>(rmax, p->host[b].r);
  }
  p->kpad1 = (rmax + epr - 1) / epr * epr;
  if (p->rows_a1 > INT32_MAX / 2 || p->rows_b1 > INT32_MAX / 2) return QMCUR_ERR_UNSUPPORTED;
  const size_t ba = tc_group_piece_bytes(pr, p->rows_a1, p->kpad1, 0);
  const size_t bb = tc_group_piece_bytes(pr, p->rows_b1, p->kpad1, 0);
  if (cudaMalloc(&p->A1_all, ba) != cudaSuccess || cudaMalloc(&p->B1_all, bb) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  cudaMemsetAsync(p->A1_all, 0, ba, stream);
  cudaMemsetAsync(p->B1_all, 0, bb, stream);
  std::vector<TcSplitJob> jobs;
  std::vector<TcGroupProb> gp(count);
  std::vector<TcGroupTile> tiles;
  int stiles = 0;
  auto add_job = [&](const QView& S, bool trans, void* dst, int64_t rows, int64_t K, int64_t row0,
                     int64_t rows_total) {
    TcSplitJob j{};
    j.S = S;
    j.dst = dst;
    j.rows = rows;
    j.K = K;
    j.kp_job = (K + epr - 1) / epr * epr;
    j.kpad = p->kpad1;
    j.row0 = row0;
    j.plane_stride = rows_total * p->kpad1;
    j.trans = trans ? 1 : 0;
    j.tiles_k = (int)((j.kp_job + 63) / 64);
    j.first_tile = stiles;
    stiles += j.tiles_k * (int)((rows + 31) / 32);
    jobs.push_back(j);
  };
  for (int b = 0; b < count; ++b) {
    const BatchProblem& P = p->host[b];
    add_job(P.R, true, p->A1_all, P.n, P.r, rrow[b], p->rows_a1);    // A[j][k] = R[k][j]
    add_job(P.U, false, p->B1_all, P.c, P.r, urow[b], p->rows_b1);   // B[i][k] = U[i][k]
    TcGroupProb& g = gp[b];
    g = TcGroupProb{};
    g.m = P.n;
    g.n = P.c;
    g.K = P.r;
    g.kblocks = (int)(((P.r + epr - 1) / epr * epr) / epr);
    g.arow = (int)rrow[b];
    g.brow = (int)urow[b];
    g.zrow = zrow[b];
    for (int m0 = 0; m0 < P.n; m0 += 128)
      for (int n0 = 0; n0 < P.c; n0 += kGroupTBn) tiles.push_back(TcGroupTile{b, m0, n0});
  }
  p->njobs1 = (int)jobs.size();
  p->split_tiles1 = stiles;
  p->ngtiles1 = (int)tiles.size();
  if (cudaMalloc(&p->djobs1, jobs.size() * sizeof(TcSplitJob)) != cudaSuccess ||
      cudaMalloc(&p->dgprobs1, gp.size() * sizeof(TcGroupProb)) != cudaSuccess ||
      cudaMalloc(&p->dgtiles1, tiles.size() * sizeof(TcGroupTile)) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  cudaMemcpyAsync(p->djobs1, jobs.data(), jobs.size() * sizeof(TcSplitJob), cudaMemcpyHostToDevice, stream);
  cudaMemcpyAsync(p->dgprobs1, gp.data(), gp.size() * sizeof(TcGroupProb), cudaMemcpyHostToDevice, stream);
  cudaMemcpyAsync(p->dgtiles1, tiles.data(), tiles.size() * sizeof(TcGroupTile), cudaMemcpyHostToDevice,
                  stream);
  // the host vectors must outlive their copies
  return cudaStreamSynchronize(stream) == cudaSuccess ? QMCUR_OK : QMCUR_ERR_CUDA;
}

extern "C" {

qmcur_status qmcur_batch_plan(int32_t count, const qmcur_qmat* A, const int64_t* c, const int64_t* r,
                              const int32_t* rank_cap, const qmcur_opts* opts, void** plan_out,
                              int32_t* dev_status, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_batch_plan");
  if (count < 1 || A == nullptr || c == nullptr || r == nullptr || opts == nullptr || plan_out == nullptr)
    return QMCUR_ERR_INVALID_ARG;
  if (opts->sampler != QMCUR_SAMPLER_NORM && opts->sampler != QMCUR_SAMPLER_UNIFORM) return QMCUR_ERR_INVALID_ARG;
  const bool refined = opts->pinv_method == QMCUR_PINV_REFINED_FP64;
  const bool subspace = opts->pinv_method == QMCUR_PINV_SUBSPACE_FP32 || refined;
  if (subspace && rank_cap == nullptr) return QMCUR_ERR_UNSUPPORTED;   // the methods need caps
  // the refined core keeps exactly k values and certifies sigma_k / sigma_1
  // only down to ~1e-4 (its FP32 factors): as in qmcur_pinv_core, no larger rcond
  if (refined && !(opts->rcond >= 0.0 && opts->rcond <= 1e-6)) return QMCUR_ERR_UNSUPPORTED;
  for (int b = 0; b < count; ++b) {
    if (!valid_qmat(&A[b], true, false)) return QMCUR_ERR_INVALID_ARG;
    if (c[b] < 1 || c[b] > A[b].cols || r[b] < 1 || r[b] > A[b].rows) return QMCUR_ERR_INVALID_ARG;
    if (subspace) {
      const int64_t nmin = c[b] < r[b] ? c[b] : r[b];
      const int64_t k = rank_cap[b] < nmin ? rank_cap[b] : nmin;
      if (rank_cap[b] < 1 || k > kSmallCholMax) return QMCUR_ERR_UNSUPPORTED;
    } else {
      // the Jacobi core keeps G (n_r x n_c) and V (n_c x n_c) in shared memory
      const int64_t nr = c[b] > r[b] ? c[b] : r[b], nc = c[b] < r[b] ? c[b] : r[b];
      if (nc > kBatchMaxCore || (nr * nc + nc * nc) * 16 > kBatchCoreSmem) return QMCUR_ERR_UNSUPPORTED;
    }
    if (A[b].rows > (1 << 20) || A[b].cols > 48 * 1024) return QMCUR_ERR_UNSUPPORTED;
  }
  const int32_t pr = opts->prec;
  const bool tc = pr == QMCUR_PREC_BF16X3 || pr == QMCUR_PREC_BF16X6 ||
                  pr == QMCUR_PREC_BF16_MIXED || pr == QMCUR_PREC_TF32X3;
  BatchPlan* p = new BatchPlan();
  p->count = count;
  p->opts = *opts;
  p->status = dev_status;
  p->tc = tc;
  // one arena: per problem col_p, row_p, J, I, C, R, W, U, T, out3, info
  std::vector<size_t> off;
  size_t total = 0;
  auto take = [&](size_t bytes) { size_t o = total; total += align_up(bytes, 256); return o; };
  struct Offs { size_t cp, rp, J, I, C, R, W, U, T, o3, info, U64; };
  std::vector<Offs> os(count);
  size_t max_rc = 0, max_nm = 0;
  for (int b = 0; b < count; ++b) {
    const int64_t m = A[b].rows, n = A[b].cols;
    Offs& o = os[b];
    o.cp = take(8 * n); o.rp = take(8 * m); o.J = take(4 * c[b]); o.I = take(4 * r[b]);
    o.C = take(16 * m * c[b]); o.R = take(16 * r[b] * n); o.W = take(16 * r[b] * c[b]);
    o.U = take(16 * c[b] * r[b]); o.T = take(16 * c[b] * n); o.o3 = take(24); o.info = take(12);
    o.U64 = refined ? take(32 * c[b] * r[b]) : 0;
    const int64_t nr = c[b] > r[b] ? c[b] : r[b], nc = c[b] < r[b] ? c[b] : r[b];
    max_rc = std::max(max_rc, (size_t)(nr * nc + nc * nc));
    max_nm = std::max(max_nm, (size_t)(n > m ? n : m));
  }
  if (cudaMalloc(&p->arena, total) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  cudaMemsetAsync(p->arena, 0, total, stream);
  char* base = static_cast<char*>(p->arena);
  auto q = [&](size_t o, int64_t rows, int64_t cols) {
    QView v;
    for (int t = 0; t < 4; ++t) v.p[t] = base + o + (size_t)t * rows * cols * 4;
    v.rows = rows; v.cols = cols; v.ld = cols; v.dtype = QMCUR_F32;
    return v;
  };
  p->host.resize(count);
  for (int b = 0; b < count; ++b) {
    BatchProblem& P = p->host[b];
    const Offs& o = os[b];
    P.A = view(&A[b]);
    P.m = (int)A[b].rows; P.n = (int)A[b].cols; P.c = (int)c[b]; P.r = (int)r[b];
    P.rank_cap = rank_cap ? rank_cap[b] : 0;
    P.col_p = reinterpret_cast<double*>(base + o.cp);
    P.row_p = reinterpret_cast<double*>(base + o.rp);
    P.J = reinterpret_cast<int32_t*>(base + o.J);
    P.I = reinterpret_cast<int32_t*>(base + o.I);
    P.C = q(o.C, P.m, P.c); P.R = q(o.R, P.r, P.n); P.W = q(o.W, P.r, P.c);
    P.U = q(o.U, P.c, P.r); P.T = q(o.T, P.c, P.n);
    if (refined) {
      for (int t = 0; t < 4; ++t) P.U64.p[t] = base + o.U64 + (size_t)t * P.c * P.r * 8;
      P.U64.rows = P.c; P.U64.cols = P.r; P.U64.ld = P.r; P.U64.dtype = QMCUR_F64;
    }
    P.out3 = reinterpret_cast<double*>(base + o.o3);
    P.info = reinterpret_cast<int32_t*>(base + o.info);
  }
  if (subspace) {
    // one subspace program (or refined program's arguments) per problem over
    // its own carve of one arena; CTA order: the most work
    // (r c k + max(r, c) k^2) first
    p->subspace = !refined;
    p->refined = refined;
    std::vector<size_t> woff(count);
    size_t wtotal = 0;
    for (int b = 0; b < count; ++b) {
      const int64_t nmin = c[b] < r[b] ? c[b] : r[b];
      const int64_t k = rank_cap[b] < nmin ? rank_cap[b] : nmin;
      woff[b] = wtotal;
      wtotal += align_up(refined ? refine_each_ws_bytes(r[b], c[b], k)
                                 : pinv_each_ws_bytes(r[b], c[b], k), 256);
    }
    const size_t pb = refined ? refine_each_args_bytes() : pinv_each_prog_bytes();
    std::vector<char> hprogs((size_t)count * pb);
    std::vector<double> work(count);
    if (cudaMalloc(&p->pinv_arena, wtotal) != cudaSuccess ||
        cudaMalloc(&p->progs, hprogs.size()) != cudaSuccess ||
        cudaMalloc(&p->order, count * sizeof(int)) != cudaSuccess) {
      free_plan(p);
      return QMCUR_ERR_CUDA;
    }
    for (int b = 0; b < count; ++b) {
      const BatchProblem& P = p->host[b];
      auto toq = [](const QView& v) {
        qmcur_qmat q;
        for (int t = 0; t < 4; ++t) q.plane[t] = v.p[t];
        q.rows = v.rows; q.cols = v.cols; q.ld = v.ld; q.dtype = v.dtype; q.reserved = 0;
        return q;
      };
      qmcur_qmat Wq = toq(P.W), Uq = toq(P.U);
      int k = 0;
      const uint64_t seed_b = opts->seed ^ (0x9e3779b97f4a7c15ull + (uint64_t)b);
      char* ws_b = static_cast<char*>(p->pinv_arena) + woff[b];
      qmcur_status s;
      if (refined) {
        qmcur_qmat U64q = toq(P.U64);
        s = refine_each_build(&Wq, P.rank_cap, opts->max_sweeps, &U64q, &Uq, P.info, P.info + 2,
                              seed_b, ws_b, wtotal - woff[b], hprogs.data() + (size_t)b * pb, &k);
      } else {
        s = pinv_each_build(&Wq, P.rank_cap, &Uq, P.info, seed_b, ws_b, wtotal - woff[b],
                            dev_status, hprogs.data() + (size_t)b * pb, &k);
      }
      if (s != QMCUR_OK) { free_plan(p); return s; }
      p->kmax = std::max(p->kmax, k);
      const double rr = (double)P.r, cc = (double)P.c;
      work[b] = rr * cc * k + std::max(rr, cc) * k * k;
    }
    std::vector<int> ord(count);
    for (int b = 0; b < count; ++b) ord[b] = b;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work[x] > work[y]; });
    cudaMemcpyAsync(p->progs, hprogs.data(), hprogs.size(), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(p->order, ord.data(), count * sizeof(int), cudaMemcpyHostToDevice, stream);
    // the host copies above must be complete before the vectors go away
    if (cudaStreamSynchronize(stream) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  }
  {
    int64_t coff = 0;
    for (int b = 0; b < count; ++b) {
      const int chunks = (p->host[b].m + kNormChunk - 1) / kNormChunk;
      p->host[b].colpart_off = coff;
      coff += (int64_t)chunks * p->host[b].n;
      p->max_chunks = std::max(p->max_chunks, chunks);
    }
    if (p->max_chunks > 65535 || cudaMalloc(&p->colpart, (size_t)coff * sizeof(double)) != cudaSuccess) {
      free_plan(p);
      return QMCUR_ERR_CUDA;
    }
  }
  if (cudaMalloc(&p->dprobs, count * sizeof(BatchProblem)) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  cudaMemcpyAsync(p->dprobs, p->host.data(), count * sizeof(BatchProblem), cudaMemcpyHostToDevice, stream);
  p->jac_smem = max_rc * sizeof(float4) + (size_t)kBatchMaxCore * 8 + 64;
  p->samp_smem = ((max_nm + 31) / 32 * 4 + 15) / 16 * 16 + max_nm * 8;
  if ((!subspace && cudaFuncSetAttribute(k_batch_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)p->jac_smem) != cudaSuccess) ||
      cudaFuncSetAttribute(k_batch_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->samp_smem) !=
          cudaSuccess) {
    free_plan(p);
    return QMCUR_ERR_CUDA;
  }
  if (tc) {
    // stacked operand pieces of Z = C T: every problem's C (m x c) as rows of
    // A_all and its T^T (n x c) as rows of B_all, K padded to the largest c
    const int64_t epr = tc_group_epr(pr);
    std::vector<int64_t> arow(count), brow(count);
    int64_t cmax = 1;
    for (int b = 0; b < count; ++b) {
      arow[b] = p->rows_a;
      brow[b] = p->rows_b;
      p->rows_a += p->host[b].m;
      p->rows_b += p->host[b].n;
      cmax = std::max<int64_t>(cmax, p->host[b].c);
    }
    p->kpad = (cmax + epr - 1) / epr * epr;
    if (p->rows_a > INT32_MAX / 2 || p->rows_b > INT32_MAX / 2) { free_plan(p); return QMCUR_ERR_UNSUPPORTED; }
    const size_t ba = tc_group_piece_bytes(pr, p->rows_a, p->kpad);
    const size_t bb = tc_group_piece_bytes(pr, p->rows_b, p->kpad);
    std::vector<TcGroupProb> gp(count);
    if (cudaMalloc(&p->A_all, ba) != cudaSuccess || cudaMalloc(&p->B_all, bb) != cudaSuccess) {
      free_plan(p);
      return QMCUR_ERR_CUDA;
    }
    cudaMemsetAsync(p->A_all, 0, ba, stream);
    cudaMemsetAsync(p->B_all, 0, bb, stream);
    for (int b = 0; b < count; ++b) {
      const BatchProblem& P = p->host[b];
      // A[i][k] = C[i][k] is written by the gather, B[j][k] = T[k][j] by the
      // T stage's epilogue
      p->host[b].zarow = arow[b];
      TcGroupProb& g = gp[b];
      bool av = P.A.ld % 4 == 0;
      for (int t = 0; t < 4; ++t) {
        g.a[t] = reinterpret_cast<const float*>(P.A.p[t]);
        av = av && reinterpret_cast<uintptr_t>(P.A.p[t]) % 16 == 0;
      }
      g.lda = P.A.ld;
      g.m = P.m;
      g.n = P.n;
      g.K = P.c;
      g.kblocks = (int)(((P.c + epr - 1) / epr * epr) / epr);
      g.arow = (int)arow[b];
      g.brow = (int)brow[b];
      g.a_vec = av ? 1 : 0;
    }
    if (cudaMalloc(&p->dgprobs, gp.size() * sizeof(TcGroupProb)) != cudaSuccess) {
      free_plan(p);
      return QMCUR_ERR_CUDA;
    }
    cudaMemcpyAsync(p->dgprobs, gp.data(), gp.size() * sizeof(TcGroupProb), cudaMemcpyHostToDevice, stream);
    if (cudaStreamSynchronize(stream) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
    const qmcur_status st1 = build_t_stage(p, brow, stream);
    if (st1 != QMCUR_OK) { free_plan(p); return st1; }
  }
  // first pass (un-captured): fills T and the operands so that the GEMM
  // candidates can be timed on real data
  {
    p->cfg1 = p->cfg2 = 0;
    std::vector<GTile> t1 = make_tiles(p->host, 0, 0), t2 = make_tiles(p->host, 1, 0);
    cudaMalloc(&p->dtiles1, t1.size() * sizeof(GTile));
    cudaMalloc(&p->dtiles2, t2.size() * sizeof(GTile));
    cudaMalloc(&p->partial, 2 * t2.size() * sizeof(double));
    cudaMemcpyAsync(p->dtiles1, t1.data(), t1.size() * sizeof(GTile), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(p->dtiles2, t2.data(), t2.size() * sizeof(GTile), cudaMemcpyHostToDevice, stream);
    p->ntiles1 = (int)t1.size();
    p->ntiles2 = (int)t2.size();
    std::vector<int> b2, c2;
    make_tiles(p->host, 1, 0, &b2, &c2);
    for (int b = 0; b < count; ++b) { p->host[b].tile_base2 = b2[b]; p->host[b].tiles2 = c2[b]; }
    cudaMemcpyAsync(p->dprobs, p->host.data(), count * sizeof(BatchProblem), cudaMemcpyHostToDevice, stream);
    if (tc) {
      const qmcur_status s = set_group_tiles(p, 128, stream);
      if (s != QMCUR_OK) { free_plan(p); return s; }
    }
    qmcur_status s = enqueue_batch(p, stream);
    if (s != QMCUR_OK) { free_plan(p); return s; }
  }
  // autotune the two grouped GEMMs, rebuild their tile lists
  p->cfg1 = tc ? 0 : autotune(p, 0, stream);   // a split plan runs T on the tensor cores
  if (!tc) p->cfg2 = autotune(p, 1, stream);
  {
    cudaFree(p->dtiles1); cudaFree(p->dtiles2);
    p->dtiles1 = p->dtiles2 = nullptr;
    if (!tc) { cudaFree(p->partial); p->partial = nullptr; }
    std::vector<int> b2, c2;
    std::vector<GTile> t1 = make_tiles(p->host, 0, p->cfg1), t2 = make_tiles(p->host, 1, p->cfg2, &b2, &c2);
    if (!tc)
      for (int b = 0; b < count; ++b) { p->host[b].tile_base2 = b2[b]; p->host[b].tiles2 = c2[b]; }
    if (cudaMalloc(&p->dtiles1, t1.size() * sizeof(GTile)) != cudaSuccess ||
        cudaMalloc(&p->dtiles2, t2.size() * sizeof(GTile)) != cudaSuccess ||
        (!tc && cudaMalloc(&p->partial, 2 * t2.size() * sizeof(double)) != cudaSuccess)) {
      free_plan(p);
      return QMCUR_ERR_CUDA;
    }
    cudaMemcpyAsync(p->dtiles1, t1.data(), t1.size() * sizeof(GTile), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(p->dtiles2, t2.data(), t2.size() * sizeof(GTile), cudaMemcpyHostToDevice, stream);
    cudaMemcpyAsync(p->dprobs, p->host.data(), count * sizeof(BatchProblem), cudaMemcpyHostToDevice, stream);
    p->ntiles1 = (int)t1.size();
    p->ntiles2 = (int)t2.size();
    if (cudaStreamSynchronize(stream) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  }
  if (tc) {
    // T of the first pass is current (the SIMT T = U R did not change)
    const qmcur_status s = autotune_group(p, stream);
    if (s != QMCUR_OK) { free_plan(p); return s; }
  }
  // capture the whole pipeline once, on a private stream (the caller's may be
  // the legacy default stream, which cannot be captured)
  if (cudaStreamSynchronize(stream) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  cudaStream_t cap = nullptr;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  for (cudaEvent_t& e : p->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { cudaStreamDestroy(cap); free_plan(p); return QMCUR_ERR_CUDA; }
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaStreamDestroy(cap);
    free_plan(p);
    return QMCUR_ERR_CUDA;
  }
  qmcur_status s = enqueue_batch(p, cap, true);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(cap, &g);
  cudaStreamDestroy(cap);
  if (s != QMCUR_OK || ec != cudaSuccess || g == nullptr) { if (g) cudaGraphDestroy(g); free_plan(p); return s != QMCUR_OK ? s : QMCUR_ERR_CUDA; }
  p->graph = g;
  if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) { free_plan(p); return QMCUR_ERR_CUDA; }
  *plan_out = p;
  return QMCUR_OK;
}

qmcur_status qmcur_batch_run(void* plan, cudaStream_t stream) {
  NvtxRange nvtx_range("qmcur_batch_run");
  if (plan == nullptr) return QMCUR_ERR_INVALID_ARG;
  return cuda_ok(cudaGraphLaunch(static_cast<BatchPlan*>(plan)->exec, stream));
}

qmcur_status qmcur_batch_stage_ms(void* plan, float* ms, int32_t n) {
  BatchPlan* p = static_cast<BatchPlan*>(plan);
  if (p == nullptr || ms == nullptr || n < 0 || n > kBatchStages) return QMCUR_ERR_INVALID_ARG;
  if (p->ev[kBatchStages] == nullptr) return QMCUR_ERR_INVALID_ARG;
  bool ok = cudaEventSynchronize(p->ev[kBatchStages]) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i) ok = cudaEventElapsedTime(ms + i, p->ev[i], p->ev[i + 1]) == cudaSuccess;
  if (!ok) {
    (void)cudaGetLastError();   // leave no error behind for the next call
    return QMCUR_ERR_CUDA;
  }
  return QMCUR_OK;
}

qmcur_status qmcur_batch_view(const void* plan, int32_t index, qmcur_batch_item* out) {
  const BatchPlan* p = static_cast<const BatchPlan*>(plan);
  if (p == nullptr || out == nullptr || index < 0 || index >= p->count) return QMCUR_ERR_INVALID_ARG;
  const BatchProblem& P = p->host[index];
  auto toq = [](const QView& v) {
    qmcur_qmat q;
    for (int t = 0; t < 4; ++t) q.plane[t] = v.p[t];
    q.rows = v.rows; q.cols = v.cols; q.ld = v.ld; q.dtype = v.dtype; q.reserved = 0;
    return q;
  };
  out->col_p = P.col_p; out->row_p = P.row_p; out->J = P.J; out->I = P.I;
  out->C = toq(P.C); out->R = toq(P.R); out->W = toq(P.W); out->U = toq(P.U);
  out->out3 = P.out3; out->info = P.info;
  out->gemm_tiles[0] = p->tc ? kGroupTBn : kCfgs[p->cfg1].bm;
  out->gemm_tiles[1] = p->tc ? p->tc_bn : kCfgs[p->cfg2].bm;
  return QMCUR_OK;
}

qmcur_status qmcur_batch_copy(const void* plan, int32_t index, int32_t what, void* dst,
                              size_t dst_bytes, cudaStream_t stream) {
  const BatchPlan* p = static_cast<const BatchPlan*>(plan);
  if (p == nullptr || dst == nullptr || index < 0 || index >= p->count) return QMCUR_ERR_INVALID_ARG;
  const BatchProblem& P = p->host[index];
  const void* src = nullptr;
  size_t bytes = 0;
  switch (what) {
    case 0: src = P.col_p; bytes = 8 * (size_t)P.n; break;
    case 1: src = P.row_p; bytes = 8 * (size_t)P.m; break;
    case 2: src = P.J; bytes = 4 * (size_t)P.c; break;
    case 3: src = P.I; bytes = 4 * (size_t)P.r; break;
    case 4: src = P.C.p[0]; bytes = 16 * (size_t)P.m * P.c; break;
    case 5: src = P.R.p[0]; bytes = 16 * (size_t)P.r * P.n; break;
    case 6: src = P.W.p[0]; bytes = 16 * (size_t)P.r * P.c; break;
    case 7: src = P.U.p[0]; bytes = 16 * (size_t)P.c * P.r; break;
    case 8: src = P.out3; bytes = 24; break;
    case 9: src = P.info; bytes = 12; break;
    case 10:   // U in FP64: the refined core only
      if (!p->refined) return QMCUR_ERR_INVALID_ARG;
      src = P.U64.p[0]; bytes = 32 * (size_t)P.c * P.r; break;
    default: return QMCUR_ERR_INVALID_ARG;
  }
  if (dst_bytes < bytes) return QMCUR_ERR_INVALID_ARG;
  return cuda_ok(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, stream));
}

void qmcur_batch_destroy(void* plan) { free_plan(static_cast<BatchPlan*>(plan)); }

}  // extern "C"
