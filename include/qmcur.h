/*
 * qmcur.h - C ABI of libqmcur.so, the GB300 (sm_103a) hot path of quaternion
 * CUR low-rank approximation (QMCUR, arXiv 2402.19147).
 *
 * The calls follow the paper's statement of the problem (Algorithm 1,
 * Sec. 3.1): given a quaternion matrix X in H^{m x n}, column and row counts
 * |J| = c, |I| = r and sampling probabilities {p_j}, {q_i}, produce
 * C = X(:,J), R = X(I,:) and a core U such that X ~ C U R.  The core is the
 * Moore-Penrose inverse of the intersection W = X(I,J); it equals the paper's
 * C^+ X R^+ whenever rank(W) = rank(X) (Lemma 1 and the Penrose conditions).
 *
 * Conventions shared by every call
 * --------------------------------
 * Storage.  A quaternion matrix A = A0 + A1 i + A2 j + A3 k (Sec. 2.2) is held
 *   *split*: four real planes of the same shape, each row-major with the same
 *   row stride `ld` (elements).  All plane pointers are DEVICE pointers owned
 *   by the caller; the library never allocates or frees them.
 * Streams.  Every call enqueues its kernels on the caller's stream and returns
 *   without synchronising.  No call copies between host and device, and no
 *   call allocates device memory: scratch space comes from the caller through
 *   (workspace, ws_bytes), sized by qmcur_workspace_size().  The workspace of
 *   one call may be reused by the next call on the same stream.  So the
 *   single-matrix calls (qmcur_decompose and the per-step calls, the
 *   cooperative pseudo-inverse kernels included) may be captured into a CUDA
 *   graph on the caller's stream; a replay reads the buffers' contents at
 *   replay time.  Launch parameters (shapes, seed, CTA budget) are fixed at
 *   capture.  The batched path captures its own graph (qmcur_batch_plan).
 * Errors.  Argument and shape errors are returned synchronously (nothing is
 *   enqueued).  Errors that depend on the data (non-finite input, zero norm,
 *   too few columns with positive probability, sampling attempt limit, Jacobi
 *   sweep limit, a device-side wait that ran out) are written by the kernels
 *   to the caller's device word *dev_status (first error wins, 0 = OK); the
 *   caller reads it after synchronising.  Kernels never trap or abort.
 *   dev_status may be NULL, in which case such errors are not reported.
 * Indices are 0-based int32; index sets are returned sorted ascending.
 */
#ifndef QMCUR_H
#define QMCUR_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { QMCUR_F32 = 0, QMCUR_F64 = 1 } qmcur_dtype;

/* A device quaternion matrix: plane[t] points to the rows x cols real plane t
 * (t = 0 real, 1 i, 2 j, 3 k), row-major, row stride ld >= cols elements. */
typedef struct {
  void*   plane[4];
  int64_t rows;
  int64_t cols;
  int64_t ld;
  int32_t dtype; /* qmcur_dtype */
  int32_t reserved;
} qmcur_qmat;

/* Sampling strategy of Sec. 3.1: QMCUR_uniform (p_j = 1/n, q_i = 1/m) or
 * QMCUR_length (p_j = ||X(:,j)||^2 / ||X||_F^2, q_i = ||X(i,:)||^2 / ||X||_F^2). */
typedef enum { QMCUR_SAMPLER_UNIFORM = 0, QMCUR_SAMPLER_NORM = 1 } qmcur_sampler;

/* Arithmetic of the reconstruction GEMMs C (U R). */
typedef enum {
  QMCUR_PREC_FP64   = 0, /* FP64 CUDA-core FMA; all operands FP64             */
  QMCUR_PREC_FP32   = 1, /* plain FP32 CUDA-core FMA                           */
  QMCUR_PREC_TF32X3 = 2, /* tensor cores (tcgen05 kind::tf32): each operand
                            split into big + small TF32 parts, products
                            big*big + big*small + small*big, FP32 accumulate  */
  QMCUR_PREC_BF16X3 = 3, /* tensor cores (tcgen05 kind::f16, BF16): hi + lo
                            parts, products hi*hi + hi*lo + lo*hi              */
  QMCUR_PREC_BF16X6 = 4, /* tensor cores, BF16 hi + mid + lo parts, the six
                            products of order <= 2, FP32 accumulate            */
  QMCUR_PREC_BF16_MIXED = 5 /* tensor cores: T = U R with the BF16X6 split and
                            Z = C T with the BF16X3 split.  U = W^+ can be
                            ill-conditioned, so cancellation in U R amplifies
                            operand rounding; C T is the well-conditioned
                            product and holds ~90% of the flops.            */
} qmcur_prec;

typedef enum {
  QMCUR_OK = 0,
  QMCUR_ERR_INVALID_ARG = 1,          /* bad pointer, shape, stride, dtype, size */
  QMCUR_ERR_NONFINITE = 2,            /* NaN or Inf in the input                  */
  QMCUR_ERR_ZERO_NORM = 3,            /* ||X||_F = 0 with the norm sampler        */
  QMCUR_ERR_INSUFFICIENT_SUPPORT = 4, /* fewer positive probabilities than c or r */
  QMCUR_ERR_SAMPLE_LIMIT = 5,         /* max_attempts draws did not give c (r)
                                         distinct indices                         */
  QMCUR_ERR_NO_CONVERGENCE = 6,       /* Jacobi sweep limit reached               */
  QMCUR_ERR_UNSUPPORTED = 7,          /* valid request this build cannot serve    */
  QMCUR_ERR_CUDA = 8,                 /* a CUDA runtime call failed               */
  QMCUR_ERR_TIMEOUT = 9,              /* a bounded device-side wait ran out       */
  QMCUR_ERR_ILL_CONDITIONED = 10      /* FP32 subspace pseudo-inverse met a
                                         non-positive Cholesky pivot            */
} qmcur_status;

/* How qmcur_pinv_core computes the truncated inverse. */
typedef enum {
  QMCUR_PINV_JACOBI_FP64 = 0,  /* full QSVD by FP64 one-sided Jacobi: any rank
                                  rule, FP64 accuracy, slow on GB300's FP64 rate */
  QMCUR_PINV_SUBSPACE_FP32 = 1, /* rank_cap >= 1 required (k = min(rank_cap, r, c)
                                  <= 100): top-k subspaces by two FP32 subspace
                                  iterations with CholeskyQR2, U = P R^-1 Q^H;
                                  assumes sigma_k > sigma_{k+1} clearly, ignores
                                  rcond, does not write sigma_out             */
  QMCUR_PINV_REFINED_FP64 = 2  /* rank_cap >= 1 required (k = min(rank_cap, r, c)
                                  <= 100, r, c <= 16384, rcond <= 1e-6): the top-k
                                  right singular subspace to FP64 accuracy by
                                  subspace iteration with FP64 products and FP32
                                  Cholesky preconditioners, iterated until the
                                  predicted subspace angle is below 1e-14, then
                                  U = P (W P)^+ by CholeskyQR2 with an FP64
                                  orthogonality correction.  Keeps exactly k
                                  singular values (so sigma_k must exceed
                                  rcond sigma_1); the iteration count grows as
                                  1 / log(sigma_k / sigma_{k+1}); does not write
                                  sigma_out                                   */
} qmcur_pinv_method;

/* Human-readable name of a status code (static string). */
const char* qmcur_status_str(int32_t status);

/*
 * qmcur_set_max_ctas - CTA budget of the persistent kernels (the
 * pseudo-inverse's cooperative launches and the tensor-core GEMMs) that the
 * calling host thread launches from now on: 0 (the default) = one CTA per
 * SM; n > 0 = at most n.  The pseudo-inverse is latency-bound and the GEMMs
 * are throughput-bound, so two decompositions on two streams, each held to
 * half of the SMs, overlap one's pseudo-inverse with the other's GEMMs.
 * Keep the budgets of concurrently running streams at or below the SM count
 * in sum: the pseudo-inverse is a cooperative launch that needs all its CTAs
 * resident (its grid barriers give up after ~2 s with QMCUR_ERR_TIMEOUT).
 * qmcur_decompose's opts->max_ctas overrides it for the call.
 * Host errors: INVALID_ARG (n < 0).
 */
qmcur_status qmcur_set_max_ctas(int32_t max_ctas);

/* Bytes of workspace that suffice for every call below on an m x n input with
 * c sampled columns and r sampled rows at precision `prec`. */
size_t qmcur_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec);

/*
 * qmcur_probs - sampling probabilities (Sec. 3.1).
 *   A        m x n input (F32 or F64).
 *   sampler  QMCUR_SAMPLER_NORM: col_p[j] = ||A(:,j)||^2 / ||A||_F^2,
 *            row_p[i] = ||A(i,:)||^2 / ||A||_F^2; the sums run over the four
 *            planes in FP32 (F32 input) or FP64 (F64 input) in short runs that
 *            are accumulated in FP64 in a fixed order (bit-reproducible).
 *            QMCUR_SAMPLER_UNIFORM: col_p[j] = 1/n, row_p[i] = 1/m; A is read
 *            only when fro2 != NULL.
 *   col_p    device double[n]; row_p device double[m] (outputs).
 *   fro2     device double scalar ||A||_F^2 or NULL.
 *   Device errors: NONFINITE, ZERO_NORM (norm sampler only).
 */
qmcur_status qmcur_probs(const qmcur_qmat* A, int32_t sampler, double* col_p, double* row_p,
                         double* fro2, void* workspace, size_t ws_bytes, int32_t* dev_status,
                         cudaStream_t stream);

/*
 * qmcur_probs_noalloc - the same computation and outputs as qmcur_probs, for
 * callers that cannot allocate device memory or pass a workspace (a host
 * framework that owns every device allocation, or a latency-bound loop where
 * cudaMalloc, which may synchronise the device, is not allowed).  The paper
 * has no counterpart: this is a memory-management variant of the call above.
 *   Allocates nothing.  Its scratch is a static 8 MiB device array inside the
 *   library, held on every GPU that loads the library until the process
 *   exits.  Inputs needing more (ceil(m/32) n + ceil(n/256) m + n + m +
 *   ceil(n/32) + 4 doubles, each part padded to 256 bytes, above 8 MiB;
 *   about m n <= 3e7) are rejected with QMCUR_ERR_UNSUPPORTED before
 *   anything is enqueued.  The uniform sampler with fro2 == NULL reads no
 *   input and needs no scratch, so it takes any size.
 *   The first call on a device looks up the array's device address (a CUDA
 *   runtime query, no allocation); make that first call before any stream
 *   capture on that device.  All calls on a device share the array and it
 *   keeps the last call's contents (every entry read is rewritten first, so
 *   results do not depend on it); calls that overlap on the GPU race on it.
 */
qmcur_status qmcur_probs_noalloc(const qmcur_qmat* A, int32_t sampler, double* col_p,
                                 double* row_p, double* fro2, int32_t* dev_status,
                                 cudaStream_t stream);

/*
 * qmcur_sample - Algorithm 1 steps 1-2: draw J subset [n] (|J| = c) from col_p
 * and I subset [m] (|I| = r) from row_p, then gather C = A(:,J) (m x c),
 * R = A(I,:) (r x n) and the intersection W = A(I,J) (r x c).
 *   Draws are without replacement: a draw repeating an accepted index is
 *   rejected.  Draw t uses Philox4x32-10 (Salmon et al., SC'11) with key
 *   (seed_lo, seed_hi) and counter (t_lo, t_hi, stream_id, which), which = 0
 *   for J, 1 for I.  Norm sampler, in exact integers: with M = max p_k =
 *   f 2^e (f in [1, 2)) and B = 63 - ceil(log2 N), q_k = floor(p_k 2^(B-1-e)),
 *   P the prefix sums of the q_k, S = P[N-1] < 2^63; w = (x0<<32|x1)>>11,
 *   target = (w S) >> 53, index = first k with P[k] > target.  Probabilities
 *   must be finite and >= 0; an entry below M 2^-B is never drawn.
 *   Uniform sampler: index = (x0 * n) >> 32, col_p / row_p may be NULL.
 *   max_attempts <= 0 selects 64*count + 1024 draws per set.
 *   J (device int32[c]) and I (device int32[r]) are written sorted ascending.
 *   C, R, W may each be NULL; C and R take A's dtype or the other one (F32/F64
 *   conversion on the fly); W may be F32 or F64.
 *   Requires 1 <= c <= n, 1 <= r <= m.
 *   Device errors: INSUFFICIENT_SUPPORT, SAMPLE_LIMIT, NONFINITE (a
 *   non-finite probability).
 */
qmcur_status qmcur_sample(const qmcur_qmat* A, int32_t sampler, const double* col_p,
                          const double* row_p, int64_t c, int64_t r, uint64_t seed,
                          uint32_t stream_id, int32_t max_attempts, int32_t* J, int32_t* I,
                          qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, void* workspace,
                          size_t ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_pinv_core - U = W^+ (Sec. 2.2 Moore-Penrose inverse through the QSVD;
 * Algorithm 1's core), truncated: singular values sigma_i > rcond * sigma_1
 * are kept, at most rank_cap of them when rank_cap > 0.
 *   W        r x c, F64 (F32 is widened).
 *   U        c x r output, F64 or F32.
 *   rank_out device int32[2] or NULL: {number of kept singular values,
 *            Jacobi sweeps executed}.
 *   sigma_out device double[min(r,c)] quaternion singular values, descending,
 *            or NULL.
 *   method   qmcur_pinv_method.  QMCUR_PINV_JACOBI_FP64: the QSVD is computed
 *            in FP64 by one-sided (Hestenes) Jacobi rotations in quaternion
 *            arithmetic; max_sweeps <= 0 selects 40; rank_out[1] = sweeps.
 *            QMCUR_PINV_SUBSPACE_FP32: see the enum; rank_out = {k, 2}.
 *            QMCUR_PINV_REFINED_FP64: see the enum; max_sweeps is the
 *            iteration limit (<= 0 selects 30, at most 64); rank_out =
 *            {k, iterations}.
 *   Device errors: NO_CONVERGENCE, NONFINITE, TIMEOUT (Jacobi);
 *   ILL_CONDITIONED (subspace, refined: a non-positive FP32 Cholesky pivot,
 *   i.e. sigma_1 / sigma_k beyond ~1e3); NO_CONVERGENCE, TIMEOUT (refined:
 *   no usable gap at k within the iteration limit; U is still written).
 *   UNSUPPORTED (synchronous) when the subspace or refined method is asked
 *   for without a rank cap, with k > 100, or (refined) with rcond > 1e-6 or
 *   r, c > 16384.
 */
qmcur_status qmcur_pinv_core(const qmcur_qmat* W, int32_t method, double rcond, int32_t rank_cap,
                             int32_t max_sweeps, qmcur_qmat* U, int32_t* rank_out,
                             double* sigma_out, void* workspace, size_t ws_bytes,
                             int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_reconstruct - Z = C (U R) (Eq. 1 / Algorithm 1 output), computed as
 * T = U R (c x n) then Z = C T (m x n) with the Hamilton product (Sec. 2.2).
 *   C m x c, U c x r, R r x n, Z m x n.  prec selects the arithmetic
 *   (qmcur_prec); QMCUR_PREC_FP64 needs F64 operands and output, the other
 *   precisions take F32 (U may be F64) and write F32.
 *   Device errors: TIMEOUT.
 */
qmcur_status qmcur_reconstruct(const qmcur_qmat* C, const qmcur_qmat* U, const qmcur_qmat* R,
                               int32_t prec, qmcur_qmat* Z, void* workspace, size_t ws_bytes,
                               int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_residual - relative Frobenius residual ||A - Z||_F / ||A||_F
 * (Example 4.2's error measure).
 *   If Z != NULL it is read (standalone pass over A and Z).  If Z == NULL the
 *   reconstruction C (U R) is formed at precision prec inside the GEMM and
 *   never written (C, U, R required).
 *   mask     NULL or device uint8 m x n (row stride n): only entries with a
 *            nonzero byte (the observed set Omega, Example 4.4) enter both
 *            norms.
 *   out3     device double[3]: {rel, sum |a - z|^2, sum |a|^2}.  Sums are
 *            reduced in a fixed order (bit-reproducible).
 *   Device errors: TIMEOUT.
 */
qmcur_status qmcur_residual(const qmcur_qmat* A, const qmcur_qmat* C, const qmcur_qmat* U,
                            const qmcur_qmat* R, int32_t prec, const uint8_t* mask,
                            const qmcur_qmat* Z, double* out3, void* workspace,
                            size_t ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_gather - C = A(:,J) (m x c), R = A(I,:) (r x n), W = A(I,J) (r x c)
 * for given index sets (Sec. 3.1).  J[c], I[r] device int32 in [0, n), [0, m);
 * out-of-range entries produce zeros.  C, R, W may each be NULL.
 */
qmcur_status qmcur_gather(const qmcur_qmat* A, const int32_t* J, const int32_t* I, int64_t c,
                          int64_t r, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W,
                          cudaStream_t stream);

/*
 * qmcur_reconstruct_backward - gradient of the masked reconstruction loss
 *   L(A) = || P_Omega(A - C U R) ||_F^2,  C = A(:,J), R = A(I,:), U = W^+,
 *   W = A(I,J)
 * (Eq. 1 with the observed set Omega of Example 4.4), through the
 * reconstruction GEMMs and the Moore-Penrose inverse:
 *   dA = scale * dL/dA = scale * (2E + G_C at the columns J + G_R at the rows
 *   I + G_W at (I, J)),  E = P_Omega(A - Z),  G_C = -2 E (UR)^H,
 *   G_R = -2 U^H C^H E,  G_U = -2 C^H E R^H,
 *   G_W = -U^H G_U U^H + (I - W U) G_U^H U U^H + U^H U G_U^H (I - U W)
 * (the fixed-rank derivative of W^+ of Golub and Pereyra; exact where W has
 * the rank of U).  FP32-level arithmetic: the six large products (T = U R,
 * Z = C T, G_C, G_T = -2 C^H E, G_U = G_T R^H and U^H G_T) run on the tensor
 * cores (tcgen05) in the six-product BF16 split of QMCUR_PREC_BF16X6, the
 * small products of G_W in FP32 on the CUDA cores.
 *   A, dA m x n (dA F32 or F64, fully overwritten); C m x c and R r x n F32;
 *   U c x r and W r x c F32 or F64; mask NULL or m x n bytes (row stride n);
 *   J[c], I[r] the index sets used to form C, R, W (device int32).
 *   loss_out: device double scalar L or NULL.  Workspace:
 *   qmcur_backward_workspace_size(m, n, c, r).
 */
size_t qmcur_backward_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r);
qmcur_status qmcur_reconstruct_backward(const qmcur_qmat* A, const uint8_t* mask, const int32_t* J,
                                        const int32_t* I, const qmcur_qmat* C, const qmcur_qmat* U,
                                        const qmcur_qmat* R, const qmcur_qmat* W, double scale,
                                        qmcur_qmat* dA, double* loss_out, void* workspace,
                                        size_t ws_bytes, int32_t* dev_status, cudaStream_t stream);

/* Options of qmcur_decompose and qmcur_batch_plan. */
typedef struct {
  int32_t  sampler;      /* qmcur_sampler */
  int32_t  prec;         /* qmcur_prec of the reconstruction GEMMs */
  uint64_t seed;         /* Philox key */
  uint32_t stream_id;    /* Philox counter word 2 */
  int32_t  max_attempts; /* <= 0: default */
  double   rcond;        /* relative singular value cut of W^+ */
  int32_t  rank_cap;     /* <= 0: no cap */
  int32_t  max_sweeps;   /* <= 0: default */
  int32_t  pinv_method;  /* qmcur_pinv_method */
  int32_t  max_ctas;     /* n > 0: at most n CTAs for the persistent kernels
                            (pseudo-inverse, tensor-core GEMMs) of this call, as
                            qmcur_set_max_ctas(n) would give; 0: the calling
                            thread's budget (qmcur_decompose only) */
} qmcur_opts;

/*
 * qmcur_decompose - one whole QMCUR decomposition (Algorithm 1 with U = W^+)
 * on the stream: qmcur_probs, qmcur_sample, qmcur_pinv_core, then
 * qmcur_residual with the reconstruction fused (Z never written).
 *   Outputs (device, caller-owned): J[c], I[r], C (m x c), R (r x n),
 *   W (r x c, F64), U (c x r, F64), rank_out[2], sigma_out[min(r,c)] (may be
 *   NULL), out3[3] as in qmcur_residual.  col_p[n], row_p[m] (device) receive
 *   the probabilities.
 *   opts->max_ctas > 0 holds the persistent kernels of this call to that many
 *   CTAs (see qmcur_set_max_ctas); several decompositions on several streams
 *   then share the SMs.
 *   Host errors: INVALID_ARG (a NULL argument, opts->max_ctas < 0, or any
 *   error of the four calls).  Device errors: those of the four calls.
 */
qmcur_status qmcur_decompose(const qmcur_qmat* A, int64_t c, int64_t r, const qmcur_opts* opts,
                             double* col_p, double* row_p, int32_t* J, int32_t* I,
                             qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W, qmcur_qmat* U,
                             int32_t* rank_out, double* sigma_out, double* out3,
                             void* workspace, size_t ws_bytes, int32_t* dev_status,
                             cudaStream_t stream);

/*
 * qmcur_qsvd_truncated - the rank-k truncated QSVD approximation
 * B = X_k = P_k Sigma_k V_k^H of Sec. 2.2, the comparator of Example 4.2
 * (QSVD against QMCUR).  The QSVD is computed as in qmcur_pinv_core's
 * QMCUR_PINV_JACOBI_FP64 (one-sided quaternion Jacobi in FP64); the k = rank
 * largest singular values above rcond * sigma_1 are kept.
 *   X        m x n input (F32 or F64).
 *   B        m x n output (F32 or F64), fully overwritten.
 *   rank_out device int32[2] or NULL: {k kept, sweeps}; sigma_out device
 *            double[min(m, n)] or NULL: all singular values, descending.
 *   max_sweeps <= 0 selects 40.  Workspace: qmcur_qsvd_workspace_size(m, n).
 *   Device errors: NO_CONVERGENCE, NONFINITE, TIMEOUT.
 */
size_t qmcur_qsvd_workspace_size(int64_t m, int64_t n);
qmcur_status qmcur_qsvd_truncated(const qmcur_qmat* X, int32_t rank, double rcond,
                                  int32_t max_sweeps, qmcur_qmat* B, int32_t* rank_out,
                                  double* sigma_out, void* workspace, size_t ws_bytes,
                                  int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_core_paper - the paper's own core U = C^+ X R^+ (Algorithm 1 step 3),
 * the least-squares core: no U gives a smaller ||X - C U R||_F.  It equals
 * W^+ of the intersection when rank(W) = rank(X) (Lemma 1), and is the
 * steadier choice on noisy data.
 *   C^+ and R^+ are truncated like W^+ in qmcur_pinv_core (method, rcond,
 *   rank_cap; the subspace method needs rank_cap >= 1 and k <= 100), then
 *   U = C^+ (X R^+) is formed at precision prec as in qmcur_reconstruct.
 *   X  m x n input; C m x c, R r x n (F32, e.g. from qmcur_sample).
 *   Cp c x m and Rp n x r: caller-owned buffers that receive C^+ and R^+
 *   (F32; F64 allowed with QMCUR_PREC_FP64).
 *   U  c x r output (F32; F64 with QMCUR_PREC_FP64).
 *   Workspace: qmcur_core_paper_workspace_size(m, n, c, r, prec).
 *   Device errors: those of qmcur_pinv_core; TIMEOUT.
 */
size_t qmcur_core_paper_workspace_size(int64_t m, int64_t n, int64_t c, int64_t r, int32_t prec);
qmcur_status qmcur_core_paper(const qmcur_qmat* X, const qmcur_qmat* C, const qmcur_qmat* R,
                              int32_t method, double rcond, int32_t rank_cap, int32_t prec,
                              qmcur_qmat* Cp, qmcur_qmat* Rp, qmcur_qmat* U, void* workspace,
                              size_t ws_bytes, int32_t* dev_status, cudaStream_t stream);

/*
 * qmcur_complete_step - one iteration of Algorithm 2 (Example 4.4, quaternion
 * matrix completion from the observed entries Omega).  Iteration t runs
 * Algorithm 1 in full on the current iterate X^t and then re-imposes the
 * observed entries:
 *   col_p, row_p = the probabilities of X^t (opts->sampler, as qmcur_probs);
 *   J, I drawn as qmcur_sample with key opts->seed and opts->stream_id (pass
 *   stream_id = t: every iteration draws new index sets);
 *   C = X^t(:,J), R = X^t(I,:), W = X^t(I,J); U = W^+ truncated by
 *   opts->rcond / opts->rank_cap through opts->pinv_method;
 *   M = C (U R), and in place X^{t+1} = P_{Omega^c}(M) + P_Omega(X^t).
 * The observed entries of X are never written, so from X^0 = P_Omega(Y)
 * every iterate keeps Y's observed values.  M is never stored: the update
 * happens in the epilogue of the product C (U R).
 *   X        m x n, updated in place (F32 for the tensor-core precisions and
 *            QMCUR_PREC_FP32, F64 for QMCUR_PREC_FP64).
 *   mask     device uint8 m x n (row stride n), nonzero = observed; NULL
 *            means every entry is observed (X does not change).
 *   col_p[n], row_p[m], J[c], I[r], C (m x c), R (r x n), W (r x c, F64),
 *            U (c x r, F64): caller-owned device buffers that receive the
 *            iteration's probabilities, index sets and factors, as in
 *            qmcur_decompose; C and R must not alias X.
 *   rank_out device int32[2] or NULL, as in qmcur_pinv_core.
 *   out3     device double[3]: {delta, ||X^{t+1} - X^t||_F^2, ||X^t||_F^2},
 *            delta = Algorithm 2's relative change; stop when delta <= 1e-4
 *            or t >= t_max.  Sums are reduced in a fixed order.
 *   Requires 1 <= c <= n, 1 <= r <= m.
 *   Device errors: those of qmcur_probs, qmcur_sample, qmcur_pinv_core;
 *   TIMEOUT.
 */
qmcur_status qmcur_complete_step(qmcur_qmat* X, const uint8_t* mask, int64_t c, int64_t r,
                                 const qmcur_opts* opts, double* col_p, double* row_p, int32_t* J,
                                 int32_t* I, qmcur_qmat* C, qmcur_qmat* R, qmcur_qmat* W,
                                 qmcur_qmat* U, int32_t* rank_out, double* out3, void* workspace,
                                 size_t ws_bytes, int32_t* dev_status, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Batched QMCUR: many independent problems of uneven shapes.
 *
 * qmcur_batch_plan builds a plan for `count` problems A[b] (host array of
 * descriptors of F32 device matrices, m_b x n_b), with c[b] sampled columns,
 * r[b] sampled rows and rank_cap[b] (NULL: no cap).  It allocates the
 * outputs and scratch of all problems (the only allocating calls of the
 * library are the plan and its destroy), runs the pipeline once, times the
 * candidate tile shapes of the two grouped GEMMs on it and keeps the faster
 * (the autotuner; choices are cached per problem-shape list), then captures
 * the whole pipeline in a CUDA graph.  Limits: min(c,r) <= 80 and
 * (max(c,r) + min(c,r)) * min(c,r) * 16 bytes <= 200 KiB (the pseudo-inverse
 * of each intersection runs in one CTA's shared memory).
 * Per problem b (Algorithm 1 with U = W^+): probabilities of opts->sampler,
 * Philox draws with key opts->seed and stream_id = b, gathers, the core,
 * T = U R and the relative residual of C T (never written), all in FP32.
 * The core follows opts->pinv_method: QMCUR_PINV_JACOBI_FP64 (the default
 * value 0) selects an FP32 one-sided quaternion Jacobi QSVD of W per CTA,
 * truncated at opts->rcond and rank_cap[b] (limits above);
 * QMCUR_PINV_SUBSPACE_FP32 runs the FP32 subspace method of qmcur_pinv_core
 * with one CTA per problem (rank_cap required, k <= 100, no shared-memory
 * limit on the intersection; largest problems first);
 * QMCUR_PINV_REFINED_FP64 runs the FP64-accurate refined method of
 * qmcur_pinv_core with one CTA per problem (same requirements, and
 * opts->rcond <= 1e-6 as for that method, else UNSUPPORTED; max_sweeps is
 * its iteration limit, info[1] the iterations taken, NO_CONVERGENCE in
 * info[2] when the spectrum has no usable gap at the cap) and keeps U in
 * FP64 as well (qmcur_batch_copy what = 10).  opts->prec selects the
 * arithmetic of Z = C T with the fused residual: QMCUR_PREC_FP32 (or FP64) a
 * grouped FP32 CUDA-core GEMM; QMCUR_PREC_BF16X3, BF16X6, TF32X3 or
 * BF16_MIXED (= BF16X3 for this product) one grouped tcgen05 launch over the
 * split operands of all problems, stacked along rows (the plan allocates
 * them), with its tile width (128 or 64 columns) chosen by timing both.
 * T = U R runs in FP32 on the CUDA cores under QMCUR_PREC_FP32 (or FP64);
 * under a split precision it is one grouped tcgen05 launch too, as
 * T^T = R^T U in the split of T (BF16X6 under BF16_MIXED), whose epilogue
 * writes Z's operand pieces directly (T itself is not stored).  dev_status
 * (device int32, may be NULL) receives the first error; per-problem errors
 * also land in info[2] of the problem.  The plan keeps the pointers it was
 * given: A[b] and dev_status must stay valid until qmcur_batch_destroy.
 * qmcur_batch_run replays the graph on `stream` (stream-ordered, no host
 * synchronisation).  qmcur_batch_view returns the device buffers of one
 * problem.  The paper decomposes one matrix at a time; batching is this
 * library's addition.
 */
typedef struct {
  double* col_p;          /* n_b probabilities of the columns */
  double* row_p;          /* m_b probabilities of the rows    */
  int32_t* J;             /* c_b sampled columns, ascending   */
  int32_t* I;             /* r_b sampled rows, ascending      */
  qmcur_qmat C, R, W, U;  /* F32: m x c, r x n, r x c, c x r  */
  double* out3;           /* {rel, sum |a - z|^2, sum |a|^2}  */
  int32_t* info;          /* {rank kept, Jacobi sweeps, status} */
  int32_t gemm_tiles[2];  /* autotuned tile edge of the two grouped GEMMs */
} qmcur_batch_item;

qmcur_status qmcur_batch_plan(int32_t count, const qmcur_qmat* A, const int64_t* c,
                              const int64_t* r, const int32_t* rank_cap, const qmcur_opts* opts,
                              void** plan, int32_t* dev_status, cudaStream_t stream);
qmcur_status qmcur_batch_run(void* plan, cudaStream_t stream);
/* Durations of the stages of the last replay (milliseconds, from events the
 * graph records at the stage boundaries): ms[0] norms, [1] index draws,
 * [2] gathers, [3] core, [4] T = U R, [5] Z = C T with the residual (the
 * operand splits included), [6] the residual fold; n <= 7 of them.  Waits
 * on the host for the last replay to finish; INVALID_ARG for a bad plan,
 * ms or n. */
qmcur_status qmcur_batch_stage_ms(void* plan, float* ms, int32_t n);
qmcur_status qmcur_batch_view(const void* plan, int32_t index, qmcur_batch_item* out);
/* Copy one output of problem `index` into dst (device or host memory, at
 * least the output's size, stream-ordered): what = 0 col_p (n doubles),
 * 1 row_p (m doubles), 2 J (c int32), 3 I (r int32), 4 C, 5 R, 6 W, 7 U
 * (four contiguous F32 planes each), 8 out3 (3 doubles), 9 info (3 int32),
 * 10 U in FP64 (four contiguous F64 planes; plans with the refined core
 * only, INVALID_ARG otherwise). */
qmcur_status qmcur_batch_copy(const void* plan, int32_t index, int32_t what, void* dst,
                              size_t dst_bytes, cudaStream_t stream);
void qmcur_batch_destroy(void* plan);

#ifdef __cplusplus
}
#endif

#endif /* QMCUR_H */
