// Small dense quaternion kernels (see small.cuh).
#include "small.cuh"

namespace qmcur {
namespace {

constexpr int TS = 16;   // 16 x 16 quaternion outputs per CTA, one per thread
constexpr int BKS = 32;  // k-slice per stage; the next slice is prefetched into registers

struct SmallGemmArgs {
  QPtr X, Y, Z;
  int M, N, K;
  float alpha, beta;
};

// Loads of one k-slice of one operand, viewed as a (rows x k) matrix: 16 x 32
// entries, two per thread.  KMAJOR: entry (r, k) lives at P[r][k] (read
// coalesced along k); otherwise at P[k][r] (coalesced along r).  CONJ
// negates the imaginary planes.  Slots (r, k) are returned for the store.
template <bool KMAJOR, bool CONJ>
__device__ __forceinline__ void small_load(const QPtr& P, int rows_lim, int k_lim, int r0, int k0,
                                           int tid, float v[2][4], int sr[2], int sk[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * 256;
    int rr, kk;
    if (KMAJOR) { rr = e / BKS; kk = e % BKS; }
    else { kk = e / TS; rr = e % TS; }
    const int gr = r0 + rr, gk = k0 + kk;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (gr < rows_lim && gk < k_lim) {
      const int64_t off = KMAJOR ? (int64_t)gr * P.ld + gk : (int64_t)gk * P.ld + gr;
      a0 = reinterpret_cast<const float*>(P.p[0])[off];
      a1 = reinterpret_cast<const float*>(P.p[1])[off];
      a2 = reinterpret_cast<const float*>(P.p[2])[off];
      a3 = reinterpret_cast<const float*>(P.p[3])[off];
      if (CONJ) { a1 = -a1; a2 = -a2; a3 = -a3; }
    }
    v[h][0] = a0; v[h][1] = a1; v[h][2] = a2; v[h][3] = a3;
    sr[h] = rr;
    sk[h] = kk;
  }
}

template <bool XH, bool YH>
__global__ void __launch_bounds__(TS * TS) k_qgemm_small(SmallGemmArgs a) {
  __shared__ float xs[4][TS][BKS + 1];   // xs[t][i][l] = op(X)(m0 + i, k0 + l)
  __shared__ float ys[4][BKS][TS + 1];   // ys[t][l][j] = op(Y)(k0 + l, n0 + j)
  const int tid = threadIdx.x, tx = tid % TS, ty = tid / TS;
  const int m0 = blockIdx.y * TS, n0 = blockIdx.x * TS;
  float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
  float xv[2][4], yv[2][4];
  int xr[2], xk[2], yr[2], yk[2];
  // op(X) as (m x k): identity -> X[m][k]; X^H -> conj(X[k][m]).
  // op(Y)^T as (n x k): identity -> Y[k][n]; Y^H -> conj(Y[n][k]).
  small_load<!XH, XH>(a.X, a.M, a.K, m0, 0, tid, xv, xr, xk);
  small_load<YH, YH>(a.Y, a.N, a.K, n0, 0, tid, yv, yr, yk);
  for (int k0 = 0; k0 < a.K; k0 += BKS) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      xs[t][xr[0]][xk[0]] = xv[0][t]; xs[t][xr[1]][xk[1]] = xv[1][t];
      ys[t][yk[0]][yr[0]] = yv[0][t]; ys[t][yk[1]][yr[1]] = yv[1][t];
    }
    __syncthreads();
    if (k0 + BKS < a.K) {
      small_load<!XH, XH>(a.X, a.M, a.K, m0, k0 + BKS, tid, xv, xr, xk);
      small_load<YH, YH>(a.Y, a.N, a.K, n0, k0 + BKS, tid, yv, yr, yk);
    }
#pragma unroll 8
    for (int l = 0; l < BKS; ++l) {
      const float a0 = xs[0][ty][l], a1 = xs[1][ty][l], a2 = xs[2][ty][l], a3 = xs[3][ty][l];
      const float b0 = ys[0][l][tx], b1 = ys[1][l][tx], b2 = ys[2][l][tx], b3 = ys[3][l][tx];
      z0 = fmaf(a0, b0, z0); z0 = fmaf(-a1, b1, z0); z0 = fmaf(-a2, b2, z0); z0 = fmaf(-a3, b3, z0);
      z1 = fmaf(a0, b1, z1); z1 = fmaf(a1, b0, z1); z1 = fmaf(a2, b3, z1); z1 = fmaf(-a3, b2, z1);
      z2 = fmaf(a0, b2, z2); z2 = fmaf(-a1, b3, z2); z2 = fmaf(a2, b0, z2); z2 = fmaf(a3, b1, z2);
      z3 = fmaf(a0, b3, z3); z3 = fmaf(a1, b2, z3); z3 = fmaf(-a2, b1, z3); z3 = fmaf(a3, b0, z3);
    }
    __syncthreads();
  }
  const int i = m0 + ty, j = n0 + tx;
  if (i < a.M && j < a.N) {
    const int64_t off = (int64_t)i * a.Z.ld + j;
    const float zz[4] = {z0, z1, z2, z3};
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
}

// Packed upper triangle, column-major: (i, j), i <= j.
__device__ __forceinline__ int tri(int i, int j) { return j * (j + 1) / 2 + i; }

// Upper-triangle pair (j, l), j <= l, of flat index e in packed column order.
__device__ __forceinline__ void untri(int e, int& j, int& l) {
  int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (c * (c + 1) / 2 > e) --c;
  while ((c + 1) * (c + 2) / 2 <= e) ++c;
  l = c;
  j = e - c * (c + 1) / 2;
}

// Right-looking factorisation with one barrier per step: step i applies
// the rank-one update of row i to the trailing matrix (scaling on the fly
// by 1/A_ii) while the scaling of row i-1, which no reader of step i
// touches, is written out; the inverse defers the finalisation of each
// column in the same way.
__global__ void __launch_bounds__(512) k_chol_inv(QPtr G, int k, QPtr Rinv, int32_t* status) {
  extern __shared__ float4 sm[];
  float4* A = sm;                       // packed upper G, overwritten by R
  float4* Ri = sm + k * (k + 1) / 2;    // packed upper running sums, then R^-1
  __shared__ float piv[kSmallCholMax];  // R_ii
  const float* G0 = reinterpret_cast<const float*>(G.p[0]);
  const float* G1 = reinterpret_cast<const float*>(G.p[1]);
  const float* G2 = reinterpret_cast<const float*>(G.p[2]);
  const float* G3 = reinterpret_cast<const float*>(G.p[3]);
  const int npk = k * (k + 1) / 2;
  for (int e = threadIdx.x; e < npk; e += blockDim.x) {
    int j, l;
    untri(e, j, l);
    const int64_t off = (int64_t)j * G.ld + l;
    A[e] = make_float4(G0[off], G1[off], G2[off], G3[off]);
    Ri[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  const float g00 = fabsf(A[0].x);
  const float floor_v = (g00 > 0.f ? g00 : 1.f) * 1e-30f;
  // G = R^H R: with d = A_ii, R_il = A_il / sqrt(d), and the trailing update
  // A_jl -= conj(A_ij) A_il / d for i < j <= l.
  for (int i = 0; i < k; ++i) {
    float d = A[tri(i, i)].x;
    const bool bad = !(d > 0.f) || !isfinite(d);
    if (bad) d = floor_v;
    if (threadIdx.x == 0) {
      if (bad) set_status(status, QMCUR_ERR_ILL_CONDITIONED);
      piv[i] = sqrtf(d);
    }
    const float inv_d = 1.0f / d;
    const int n = k - i - 1;
    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {
      int jj, ll;
      untri(e, jj, ll);
      const int j = i + 1 + jj, l = i + 1 + ll;
      const float4 a = A[tri(i, j)], b = A[tri(i, l)];
      float4 z = A[tri(j, l)];
      // z -= conj(a) * b / d
      z.x -= (a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w) * inv_d;
      z.y -= (a.x * b.y - a.y * b.x - a.z * b.w + a.w * b.z) * inv_d;
      z.z -= (a.x * b.z + a.y * b.w - a.z * b.x - a.w * b.y) * inv_d;
      z.w -= (a.x * b.w - a.y * b.z + a.z * b.y - a.w * b.x) * inv_d;
      A[tri(j, l)] = z;
    }
    if (i > 0) {   // finish row i - 1
      const int p = i - 1;
      const float rinv = 1.0f / piv[p];
      for (int l = p + threadIdx.x; l < k; l += blockDim.x) {
        const float4 q = A[tri(p, l)];
        A[tri(p, l)] = (l == p) ? make_float4(piv[p], 0.f, 0.f, 0.f)
                                : make_float4(q.x * rinv, q.y * rinv, q.z * rinv, q.w * rinv);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) A[tri(k - 1, k - 1)] = make_float4(piv[k - 1], 0.f, 0.f, 0.f);
  __syncthreads();
  // Rinv R = I column by column: S_ij = sum_{l<j} Rinv_il R_lj is kept in Ri;
  // Rinv_ij = (delta_ij - S_ij) / R_jj for i <= j (formed on the fly), then
  // S_il += Rinv_ij R_jl for i <= j < l; column j is written back one step
  // later, when nothing reads it.
  for (int j = 0; j < k; ++j) {
    const float inv = 1.0f / piv[j];
    const int w = j + 1, cnt = w * (k - j - 1);
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int i = e % w, l = j + 1 + e / w;
      const float4 sv = Ri[tri(i, j)];
      const float4 a = make_float4(((i == j) ? 1.f - sv.x : -sv.x) * inv, -sv.y * inv,
                                   -sv.z * inv, -sv.w * inv);
      const float4 b = A[tri(j, l)];
      float4 z = Ri[tri(i, l)];
      z.x += a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w;
      z.y += a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z;
      z.z += a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y;
      z.w += a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x;
      Ri[tri(i, l)] = z;
    }
    if (j > 0) {   // finalise column j - 1
      const int c = j - 1;
      const float ic = 1.0f / piv[c];
      for (int i = threadIdx.x; i <= c; i += blockDim.x) {
        const float4 sv = Ri[tri(i, c)];
        Ri[tri(i, c)] = make_float4(((i == c) ? 1.f - sv.x : -sv.x) * ic, -sv.y * ic,
                                    -sv.z * ic, -sv.w * ic);
      }
    }
    __syncthreads();
  }
  {
    const int c = k - 1;
    const float ic = 1.0f / piv[c];
    for (int i = threadIdx.x; i <= c; i += blockDim.x) {
      const float4 sv = Ri[tri(i, c)];
      Ri[tri(i, c)] = make_float4(((i == c) ? 1.f - sv.x : -sv.x) * ic, -sv.y * ic, -sv.z * ic,
                                  -sv.w * ic);
    }
  }
  __syncthreads();
  float* O0 = reinterpret_cast<float*>(Rinv.p[0]);
  float* O1 = reinterpret_cast<float*>(Rinv.p[1]);
  float* O2 = reinterpret_cast<float*>(Rinv.p[2]);
  float* O3 = reinterpret_cast<float*>(Rinv.p[3]);
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    const float4 q = (i <= j) ? Ri[tri(i, j)] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t off = (int64_t)i * Rinv.ld + j;
    O0[off] = q.x; O1[off] = q.y; O2[off] = q.z; O3[off] = q.w;
  }
}

__global__ void k_set_rank(int32_t* rank_out, int k, int iters) {
  rank_out[0] = k;
  rank_out[1] = iters;
}

}  // namespace

qmcur_status small_qgemm(bool xh, bool yh, int M, int N, int K, float alpha, const QPtr& X,
                         const QPtr& Y, float beta, const QPtr& Z, cudaStream_t st) {
  if (M < 1 || N < 1 || K < 1) return QMCUR_ERR_INVALID_ARG;
  SmallGemmArgs a{X, Y, Z, M, N, K, alpha, beta};
  dim3 grid((N + TS - 1) / TS, (M + TS - 1) / TS);
  if (grid.y > 65535) return QMCUR_ERR_UNSUPPORTED;
  if (!xh && !yh) k_qgemm_small<false, false><<<grid, TS * TS, 0, st>>>(a);
  else if (xh && !yh) k_qgemm_small<true, false><<<grid, TS * TS, 0, st>>>(a);
  else if (!xh && yh) k_qgemm_small<false, true><<<grid, TS * TS, 0, st>>>(a);
  else k_qgemm_small<true, true><<<grid, TS * TS, 0, st>>>(a);
  return cuda_ok(cudaGetLastError());
}

qmcur_status small_chol_inv(const QPtr& G, int k, const QPtr& Rinv, int32_t* status,
                            cudaStream_t st) {
  if (k < 1 || k > kSmallCholMax) return QMCUR_ERR_UNSUPPORTED;
  const size_t smem = (size_t)k * (k + 1) * sizeof(float4);
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return QMCUR_ERR_CUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kSmallCholMax * (kSmallCholMax + 1) * sizeof(float4))) !=
        cudaSuccess)
      return QMCUR_ERR_CUDA;
    attr_set[dev] = true;
  }
  k_chol_inv<<<1, 512, smem, st>>>(G, k, Rinv, status);
  return cuda_ok(cudaGetLastError());
}

void small_set_rank(int32_t* rank_out, int k, int iters, cudaStream_t st) {
  k_set_rank<<<1, 1, 0, st>>>(rank_out, k, iters);
}

}  // namespace qmcur
