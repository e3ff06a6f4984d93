// U = W^+ through the QSVD of W (Sec. 2.2), truncated by rcond / rank_cap.
//
// One-sided (Hestenes) Jacobi in FP64 quaternion arithmetic.  With
// n_c = min(r, c) columns G = W (c <= r) or G = W^H (c > r), every step of a
// sweep orthogonalises n_c/2 disjoint column pairs (round-robin "circle"
// ordering), accumulating the same right rotations into V (n_c x n_c).  A pair
// (a, b) with alpha = |g_a|^2, beta = |g_b|^2, gamma = g_a^H g_b in H is
// rotated when |gamma| > tol sqrt(alpha beta): with g = |gamma|, u = gamma/g,
// the column b is first right-multiplied by conj(u) (which makes the inner
// product real, g), then a real Jacobi rotation with
//   zeta = (beta - alpha) / (2g), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   cs = 1/sqrt(1 + t^2), sn = cs t
// gives g_a' = cs g_a - sn g_b conj(u), g_b' = sn g_a + cs g_b conj(u).
// At convergence G V-rotated has orthogonal columns g_j = sigma_j p_j, so
//   W^+ = sum_{kept j} v_j sigma_j^-2 g_j^H            (c <= r)
//   W^+ = sum_{kept j} g_j sigma_j^-2 v_j^H            (c > r).
//
// One CTA (128 threads) handles one pair at a time; the steps of a sweep are
// separated by a grid-wide barrier (cooperative launch, bounded spin).
#include "common.cuh"

namespace qmcur {
namespace {

constexpr int kPinvThreads = 128;

struct Q4 { double x, y, z, w; };

__device__ __forceinline__ Q4 ldq(const double* base, int64_t idx) {
  const double2* p = reinterpret_cast<const double2*>(base + idx * 4);
  double2 a = p[0], b = p[1];
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void stq(double* base, int64_t idx, Q4 q) {
  double2* p = reinterpret_cast<double2*>(base + idx * 4);
  p[0] = make_double2(q.x, q.y);
  p[1] = make_double2(q.z, q.w);
}

struct PinvArgs {
  QView W;           // r x c input
  double* G;         // n_r x n_c, column-major, 4 doubles per entry
  double* V;         // n_c x n_c
  int64_t nr, nc;    // rows / columns of G
  int transposed;    // 1 if G = W^H
  double tol;
  int max_sweeps;
  unsigned* bar;     // [0] arrive count, [1] generation, [2] abort flag
  unsigned* rot;     // per-sweep rotation counters [max_sweeps]
  const double* colnorm2;   // |g_j|^2 of the initial columns (k_pinv_colnorm)
  int* sweeps_done;
  int32_t* status;
};

__global__ void k_pinv_init(PinvArgs a) {
  const int64_t total_g = a.nr * a.nc;
  const int64_t total_v = a.nc * a.nc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total_g + total_v;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < total_g) {
      const int64_t j = e / a.nr, i = e % a.nr;   // G[i][j]
      Q4 q;
      if (!a.transposed) {
        q = {ld_as_double(a.W, 0, i, j), ld_as_double(a.W, 1, i, j), ld_as_double(a.W, 2, i, j),
             ld_as_double(a.W, 3, i, j)};
      } else {  // G = W^H: G[i][j] = conj(W[j][i])
        q = {ld_as_double(a.W, 0, j, i), -ld_as_double(a.W, 1, j, i), -ld_as_double(a.W, 2, j, i),
             -ld_as_double(a.W, 3, j, i)};
      }
      stq(a.G, j * a.nr + i, q);
    } else {
      const int64_t f = e - total_g;
      const int64_t j = f / a.nc, i = f % a.nc;
      stq(a.V, j * a.nc + i, Q4{i == j ? 1.0 : 0.0, 0.0, 0.0, 0.0});
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.bar[0] = 0; a.bar[1] = 0; a.bar[2] = 0;
    *a.sweeps_done = 0;
  }
  if (blockIdx.x == 0)
    for (int s = threadIdx.x; s < a.max_sweeps; s += blockDim.x) a.rot[s] = 0u;
}

// Grid-wide barrier for a cooperative launch.  Returns false if the wait ran
// out (then the abort flag is raised and every CTA leaves at its next barrier).
__device__ bool grid_barrier(unsigned* bar, int32_t* status) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* vabort = bar + 2;
    int ok = (*vabort == 0u);
    if (ok) {
      const unsigned gen = *vgen;
      __threadfence();
      const unsigned arrived = atomicAdd(bar, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        unsigned long long spins = 0;
        while (*vgen == gen) {
          if (*vabort != 0u) { ok = 0; break; }
          if (++spins > kSpinLimit) {
            atomicExch(bar + 2, 1u);
            set_status(status, QMCUR_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

__device__ __forceinline__ void circle_pair(int64_t N, int64_t step, int64_t p, int64_t& a, int64_t& b) {
  // players 0..N-1 (N even); player N-1 fixed, the others rotate.
  const int64_t M = N - 1;
  if (p == 0) { a = M; b = step % M; }
  else { a = (step + p) % M; b = (step - p + M) % M; }
}

__device__ __forceinline__ double block_sum128(double v, double* sh, int slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[slot * 4 + warp] = v;
  return 0.0;
}

// |g_j|^2 of every initial column, one CTA per column, in a fixed order.
__global__ void __launch_bounds__(kPinvThreads) k_pinv_colnorm(const double* G, int64_t nr,
                                                               double* colnorm2) {
  __shared__ double red[4];
  const double* g = G + (int64_t)blockIdx.x * nr * 4;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nr * 4; i += kPinvThreads) s += g[i] * g[i];
  block_sum128(s, red, 0);
  __syncthreads();
  if (threadIdx.x == 0) colnorm2[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

constexpr int kJacRegRows = 4;

// |x|^2, |y|^2 and conj(x) * y, accumulated
__device__ __forceinline__ void pair_dots(const Q4 x, const Q4 y, double& al, double& be, double& g0,
                                          double& g1, double& g2, double& g3) {
  al += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
  be += y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w;
  g0 += x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
  g1 += x.x * y.y - x.y * y.x - x.z * y.w + x.w * y.z;
  g2 += x.x * y.z + x.y * y.w - x.z * y.x - x.w * y.y;
  g3 += x.x * y.w - x.y * y.z + x.z * y.y - x.w * y.x;
}

// row i of the pair (x, q) -> (cs x - sn q w, sn x + cs q w)
__device__ __forceinline__ void rotate_rows(double* xa, double* xb, int64_t i, const Q4 x, const Q4 q,
                                            double cs, double sn, const Q4 w) {
  const Q4 y = {q.x * w.x - q.y * w.y - q.z * w.z - q.w * w.w,
                q.x * w.y + q.y * w.x + q.z * w.w - q.w * w.z,
                q.x * w.z - q.y * w.w + q.z * w.x + q.w * w.y,
                q.x * w.w + q.y * w.z - q.z * w.y + q.w * w.x};
  stq(xa, i, Q4{cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z, cs * x.w - sn * y.w});
  stq(xb, i, Q4{sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z, sn * x.w + cs * y.w});
}

__global__ void __launch_bounds__(kPinvThreads) k_pinv_jacobi(PinvArgs a) {
  __shared__ double red[6 * 4];
  __shared__ double rot_sh[6];
  __shared__ int rotated_sh;
  __shared__ double floor_sh;
  const int64_t nc = a.nc, nr = a.nr;
  // Pairs of columns that are both below (n_c tol)^2 of the largest column
  // norm^2 are numerically zero (an exactly low-rank input leaves many, at
  // about (sqrt(n_r) u |X|)^2): rotating them only stirs rounding noise and
  // never converges.  The floor sits at singular values ~1e-13 sigma_1 and
  // below, far under any truncation.
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int64_t j = 0; j < nc; ++j) mx = fmax(mx, a.colnorm2[j]);
    floor_sh = (double)nc * (double)nc * a.tol * a.tol * mx;
  }
  __syncthreads();
  const double zero_floor = floor_sh;
  const int64_t N = (nc % 2 == 0) ? nc : nc + 1;
  const int64_t npairs = N / 2;
  const int64_t steps = N - 1;
  const bool in_regs = nr <= (int64_t)kJacRegRows * kPinvThreads;   // nc <= nr
  int sweep = 0;
  for (; sweep < a.max_sweeps; ++sweep) {
    if (threadIdx.x == 0) rotated_sh = 0;
    for (int64_t step = 0; step < steps; ++step) {
      for (int64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
        int64_t ca, cb;
        circle_pair(N, step, p, ca, cb);
        if (ca >= nc || cb >= nc) continue;   // the dummy player of an odd count
        double* ga = a.G + ca * nr * 4;
        double* gb = a.G + cb * nr * 4;
        double* va = a.V + ca * nc * 4;
        double* vb = a.V + cb * nc * 4;
        double al = 0, be = 0, g0 = 0, g1 = 0, g2 = 0, g3 = 0;
        // Up to kJacRegRows rows per thread: both columns of G and of V are
        // loaded into registers before the reduction (the loads of V overlap
        // it) and rotated there; longer columns stream through the loops.
        Q4 xg[kJacRegRows], yg[kJacRegRows], xv[kJacRegRows], yv[kJacRegRows];
        if (in_regs) {
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            const int64_t i = threadIdx.x + (int64_t)u * kPinvThreads;
            xg[u] = i < nr ? ldq(ga, i) : Q4{0.0, 0.0, 0.0, 0.0};
            yg[u] = i < nr ? ldq(gb, i) : Q4{0.0, 0.0, 0.0, 0.0};
          }
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            const int64_t i = threadIdx.x + (int64_t)u * kPinvThreads;
            xv[u] = i < nc ? ldq(va, i) : Q4{0.0, 0.0, 0.0, 0.0};
            yv[u] = i < nc ? ldq(vb, i) : Q4{0.0, 0.0, 0.0, 0.0};
          }
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u)
            pair_dots(xg[u], yg[u], al, be, g0, g1, g2, g3);
        } else {
          for (int64_t i = threadIdx.x; i < nr; i += kPinvThreads)
            pair_dots(ldq(ga, i), ldq(gb, i), al, be, g0, g1, g2, g3);
        }
        block_sum128(al, red, 0);
        block_sum128(be, red, 1);
        block_sum128(g0, red, 2);
        block_sum128(g1, red, 3);
        block_sum128(g2, red, 4);
        block_sum128(g3, red, 5);
        __syncthreads();
        // the rotation, once per pair: FP64 square roots and divisions are
        // long sequences on GB300's FP64 pipe, so thread 0 forms it and the
        // others read it (rot_sh[0] < 0: skip the pair)
        if (threadIdx.x == 0) {
          double s6[6];
#pragma unroll
          for (int q = 0; q < 6; ++q)
            s6[q] = (red[q * 4 + 0] + red[q * 4 + 1]) + (red[q * 4 + 2] + red[q * 4 + 3]);
          const double a2 = s6[0], b2 = s6[1];
          const double gam = sqrt(s6[2] * s6[2] + s6[3] * s6[3] + s6[4] * s6[4] + s6[5] * s6[5]);
          // Skip pairs already orthogonal to working accuracy, and pairs whose
          // smaller column is below tol relative to the larger one (numerically
          // zero next to it: rotating it only stirs rounding noise).
          if (!(a2 > 0.0) || !(b2 > 0.0) || !(gam > a.tol * sqrt(a2) * sqrt(b2)) ||
              fmin(a2, b2) < a.tol * a.tol * fmax(a2, b2) || fmax(a2, b2) < zero_floor) {
            rot_sh[0] = -1.0;
          } else {
            rotated_sh = 1;
            const double zeta = (b2 - a2) / (2.0 * gam);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cs = 1.0 / sqrt(1.0 + t * t);
            const double ig = 1.0 / gam;
            rot_sh[0] = cs;
            rot_sh[1] = cs * t;
            // w = conj(u), u = gamma / g
            rot_sh[2] = s6[2] * ig;
            rot_sh[3] = -s6[3] * ig;
            rot_sh[4] = -s6[4] * ig;
            rot_sh[5] = -s6[5] * ig;
          }
        }
        __syncthreads();
        const double cs = rot_sh[0], sn = rot_sh[1];
        const double w0 = rot_sh[2], w1 = rot_sh[3], w2 = rot_sh[4], w3 = rot_sh[5];
        __syncthreads();   // rot_sh and red are rewritten by the next pair
        if (cs < 0.0) continue;
        const Q4 w = {w0, w1, w2, w3};
        if (in_regs) {
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            const int64_t i = threadIdx.x + (int64_t)u * kPinvThreads;
            if (i < nr) rotate_rows(ga, gb, i, xg[u], yg[u], cs, sn, w);
            if (i < nc) rotate_rows(va, vb, i, xv[u], yv[u], cs, sn, w);
          }
        } else {
          for (int64_t i = threadIdx.x; i < nr; i += kPinvThreads)
            rotate_rows(ga, gb, i, ldq(ga, i), ldq(gb, i), cs, sn, w);
          for (int64_t i = threadIdx.x; i < nc; i += kPinvThreads)
            rotate_rows(va, vb, i, ldq(va, i), ldq(vb, i), cs, sn, w);
        }
      }
      if (!grid_barrier(a.bar, a.status)) return;
    }
    __syncthreads();
    if (threadIdx.x == 0 && rotated_sh) atomicAdd(a.rot + sweep, 1u);
    if (!grid_barrier(a.bar, a.status)) return;
    const unsigned total = *reinterpret_cast<volatile unsigned*>(a.rot + sweep);
    if (total == 0u) { ++sweep; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.sweeps_done = sweep;
    if (sweep >= a.max_sweeps && *reinterpret_cast<volatile unsigned*>(a.rot + a.max_sweeps - 1) != 0u)
      set_status(a.status, QMCUR_ERR_NO_CONVERGENCE);
  }
}

// sigma_j = |g_j|, order, truncation, and the compacted list of kept columns.
__global__ void __launch_bounds__(1024)
k_pinv_select(const double* G, int64_t nr, int64_t nc, double rcond, int rank_cap,
              double* sig, int* order_pos, int* kidx, double* kw, int* k_out, int32_t* rank_out,
              double* sigma_out, const int* sweeps, int32_t* status) {
  __shared__ double smax_sh;
  __shared__ int nonfinite_sh;
  __shared__ int keep_sh;
  if (threadIdx.x == 0) { smax_sh = 0.0; nonfinite_sh = 0; keep_sh = 0; }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
    double s = 0.0;
    const double* g = G + j * nr * 4;
    for (int64_t i = 0; i < nr * 4; ++i) s += g[i] * g[i];
    s = sqrt(s);
    sig[j] = s;
    if (!isfinite(s)) atomicExch(&nonfinite_sh, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int64_t j = 0; j < nc; ++j) mx = fmax(mx, sig[j]);
    smax_sh = mx;
    if (nonfinite_sh) set_status(status, QMCUR_ERR_NONFINITE);
  }
  __syncthreads();
  const double smax = smax_sh;
  // position of column j in descending order (ties: lower index first)
  for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
    const double s = sig[j];
    int pos = 0;
    for (int64_t i = 0; i < nc; ++i) {
      const double t = sig[i];
      pos += (t > s) || (t == s && i < j);
    }
    order_pos[j] = pos;
    if (smax > 0.0 && s > rcond * smax) atomicAdd(&keep_sh, 1);
  }
  __syncthreads();
  int k = keep_sh;
  if (rank_cap > 0 && k > rank_cap) k = rank_cap;
  for (int64_t j = threadIdx.x; j < nc; j += blockDim.x) {
    const int pos = order_pos[j];
    if (sigma_out != nullptr) sigma_out[pos] = sig[j];
    if (pos < k) {
      kidx[pos] = (int)j;
      kw[pos] = 1.0 / (sig[j] * sig[j]);
    }
  }
  if (threadIdx.x == 0) {
    *k_out = k;
    if (rank_out != nullptr) { rank_out[0] = k; rank_out[1] = *sweeps; }
  }
}

// U[a][b] = sum_pos X[a][j] w_pos conj(Y[b][j]), j = kidx[pos]; U is c x r.
// With unit_w the weights are 1: the truncated QSVD approximation itself.
__global__ void k_pinv_form(const double* X, int64_t ldx, const double* Y, int64_t ldy,
                            const int* kidx, const double* kw, const int* k_in, QView U,
                            int unit_w) {
  const int64_t c = U.rows, r = U.cols;
  const int k = *k_in;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < c * r;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ai = e / r, bi = e % r;
    double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    for (int pos = 0; pos < k; ++pos) {
      const int64_t j = kidx[pos];
      const double w = unit_w ? 1.0 : kw[pos];
      const Q4 x = ldq(X, j * ldx + ai), y = ldq(Y, j * ldy + bi);
      // x * conj(y), scaled by w
      r0 += w * (x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w);
      r1 += w * (-x.x * y.y + x.y * y.x - x.z * y.w + x.w * y.z);
      r2 += w * (-x.x * y.z + x.y * y.w + x.z * y.x - x.w * y.y);
      r3 += w * (-x.x * y.w - x.y * y.z + x.z * y.y + x.w * y.x);
    }
    st_from_double(U, 0, ai, bi, r0);
    st_from_double(U, 1, ai, bi, r1);
    st_from_double(U, 2, ai, bi, r2);
    st_from_double(U, 3, ai, bi, r3);
  }
}

struct PinvWs {
  double* G; double* V; unsigned* bar; unsigned* rot; int* sweeps; double* sig; int* pos;
  int* kidx; double* kw; int* k;
};

PinvWs carve_pinv(Carve& cv, int64_t r, int64_t c, int max_sweeps) {
  const int64_t nc = r < c ? r : c, nr = r < c ? c : r;
  PinvWs w;
  w.G = cv.take<double>((size_t)(nr * nc * 4));
  w.V = cv.take<double>((size_t)(nc * nc * 4));
  w.bar = cv.take<unsigned>(4);
  w.rot = cv.take<unsigned>((size_t)max_sweeps);
  w.sweeps = cv.take<int>(1);
  w.sig = cv.take<double>((size_t)nc);
  w.pos = cv.take<int>((size_t)nc);
  w.kidx = cv.take<int>((size_t)nc);
  w.kw = cv.take<double>((size_t)nc);
  w.k = cv.take<int>(1);
  return w;
}

constexpr int kDefaultSweeps = 40;
constexpr int kMaxSweeps = 256;

}  // namespace

size_t pinv_ws_bytes(int64_t r, int64_t c) {
  Carve cv(nullptr, 0);
  carve_pinv(cv, r, c, kMaxSweeps);
  return cv.off;
}

namespace {

// The one-sided Jacobi sweeps on W (r x c) into the workspace carve w:
// G (orthogonal columns) and V, sweeps counted in w.sweeps.
qmcur_status run_jacobi(const qmcur_qmat* W, const PinvWs& w, int max_sweeps, int32_t* dev_status,
                        cudaStream_t st) {
  const int64_t r = W->rows, c = W->cols;
  PinvArgs a;
  a.W = view(W);
  a.G = w.G;
  a.V = w.V;
  a.transposed = c > r;
  a.nc = a.transposed ? r : c;
  a.nr = a.transposed ? c : r;
  a.tol = sqrt((double)a.nr) * 0x1.0p-52;
  a.max_sweeps = max_sweeps;
  a.bar = w.bar;
  a.rot = w.rot;
  a.sweeps_done = w.sweeps;
  a.status = dev_status;
  a.colnorm2 = w.sig;   // the singular values overwrite it after the sweeps
  {
    const int64_t total = a.nr * a.nc + a.nc * a.nc;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    k_pinv_init<<<blocks, 256, 0, st>>>(a);
  }
  if (a.nc > 2147483647) return QMCUR_ERR_UNSUPPORTED;
  k_pinv_colnorm<<<(unsigned)a.nc, kPinvThreads, 0, st>>>(a.G, a.nr, w.sig);
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QMCUR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return QMCUR_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pinv_jacobi, kPinvThreads, 0) != cudaSuccess)
    return QMCUR_ERR_CUDA;
  const int64_t N = (a.nc % 2 == 0) ? a.nc : a.nc + 1;
  int64_t grid = N / 2;
  const int64_t cap = (int64_t)cta_cap(sms) * (per_sm > 0 ? per_sm : 1);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pinv_jacobi, dim3((unsigned)grid),
                                              dim3(kPinvThreads), args, 0, st);
  return e == cudaSuccess ? QMCUR_OK : QMCUR_ERR_CUDA;
}

}  // namespace

qmcur_status launch_pinv(const qmcur_qmat* W, double rcond, int32_t rank_cap, int32_t max_sweeps,
                         qmcur_qmat* U, int32_t* rank_out, double* sigma_out, void* ws,
                         size_t ws_bytes, int32_t* dev_status, cudaStream_t st) {
  if (!valid_qmat(W) || !valid_qmat(U)) return QMCUR_ERR_INVALID_ARG;
  const int64_t r = W->rows, c = W->cols;
  if (r < 1 || c < 1 || U->rows != c || U->cols != r) return QMCUR_ERR_INVALID_ARG;
  if (!(rcond >= 0.0)) return QMCUR_ERR_INVALID_ARG;
  if (max_sweeps <= 0) max_sweeps = kDefaultSweeps;
  if (max_sweeps > kMaxSweeps) max_sweeps = kMaxSweeps;
  Carve cv(ws, ws_bytes);
  PinvWs w = carve_pinv(cv, r, c, kMaxSweeps);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  qmcur_status s = run_jacobi(W, w, max_sweeps, dev_status, st);
  if (s != QMCUR_OK) return s;
  const bool transposed = c > r;
  const int64_t nc = transposed ? r : c, nr = transposed ? c : r;
  k_pinv_select<<<1, 1024, 0, st>>>(w.G, nr, nc, rcond, rank_cap, w.sig, w.pos, w.kidx, w.kw,
                                     w.k, rank_out, sigma_out, w.sweeps, dev_status);
  {
    const double* X = transposed ? w.G : w.V;
    const int64_t ldx = transposed ? nr : nc;
    const double* Y = transposed ? w.V : w.G;
    const int64_t ldy = transposed ? nc : nr;
    int blocks = (int)((c * r + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_pinv_form<<<blocks, 256, 0, st>>>(X, ldx, Y, ldy, w.kidx, w.kw, w.k, view(U), 0);
  }
  return cuda_ok(cudaGetLastError());
}

// The rank-k truncated QSVD approximation B = X_k of the r x c matrix W: the
// same Jacobi sweeps, then B = sum over kept j of g_j v_j^H (c <= r, G = W V)
// or v_j g_j^H (c > r, G = W^H V).
qmcur_status launch_qsvd_truncated(const qmcur_qmat* W, double rcond, int32_t rank,
                                   int32_t max_sweeps, qmcur_qmat* B, int32_t* rank_out,
                                   double* sigma_out, void* ws, size_t ws_bytes,
                                   int32_t* dev_status, cudaStream_t st) {
  if (!valid_qmat(W) || !valid_qmat(B) || rank < 1) return QMCUR_ERR_INVALID_ARG;
  const int64_t r = W->rows, c = W->cols;
  if (r < 1 || c < 1 || B->rows != r || B->cols != c) return QMCUR_ERR_INVALID_ARG;
  if (!(rcond >= 0.0)) return QMCUR_ERR_INVALID_ARG;
  if (max_sweeps <= 0) max_sweeps = kDefaultSweeps;
  if (max_sweeps > kMaxSweeps) max_sweeps = kMaxSweeps;
  Carve cv(ws, ws_bytes);
  PinvWs w = carve_pinv(cv, r, c, kMaxSweeps);
  if (!cv.ok) return QMCUR_ERR_INVALID_ARG;
  qmcur_status s = run_jacobi(W, w, max_sweeps, dev_status, st);
  if (s != QMCUR_OK) return s;
  const bool transposed = c > r;
  const int64_t nc = transposed ? r : c, nr = transposed ? c : r;
  k_pinv_select<<<1, 1024, 0, st>>>(w.G, nr, nc, rcond, rank, w.sig, w.pos, w.kidx, w.kw, w.k,
                                     rank_out, sigma_out, w.sweeps, dev_status);
  const double* X = transposed ? w.V : w.G;
  const int64_t ldx = transposed ? nc : nr;
  const double* Y = transposed ? w.G : w.V;
  const int64_t ldy = transposed ? nr : nc;
  int blocks = (int)((r * c + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_pinv_form<<<blocks, 256, 0, st>>>(X, ldx, Y, ldy, w.kidx, w.kw, w.k, view(B), 1);
  return cuda_ok(cudaGetLastError());
}

}  // namespace qmcur
