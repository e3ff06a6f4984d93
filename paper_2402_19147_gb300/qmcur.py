"""Thin ctypes binding of libqmcur.so (C ABI in include/qmcur.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  If the library has
not been built, ``lib()`` raises (there is no CPU fallback).

A quaternion matrix is a torch tensor of shape (4, rows, cols) (planes real,
i, j, k), float32 or float64, on a CUDA device, with unit stride along the
last axis; ``qmat()`` turns it into the C descriptor.
"""
import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqmcur.so")

F32, F64 = 0, 1
SAMPLER_UNIFORM, SAMPLER_NORM = 0, 1
PREC_FP64, PREC_FP32, PREC_TF32X3, PREC_BF16X3, PREC_BF16X6 = 0, 1, 2, 3, 4
PREC_BF16_MIXED = 5
PREC_NAMES = {"fp64": PREC_FP64, "fp32": PREC_FP32, "tf32x3": PREC_TF32X3,
              "bf16x3": PREC_BF16X3, "bf16x6": PREC_BF16X6, "bf16mixed": PREC_BF16_MIXED}
STATUS = {0: "QMCUR_OK", 1: "QMCUR_ERR_INVALID_ARG", 2: "QMCUR_ERR_NONFINITE",
          3: "QMCUR_ERR_ZERO_NORM", 4: "QMCUR_ERR_INSUFFICIENT_SUPPORT",
          5: "QMCUR_ERR_SAMPLE_LIMIT", 6: "QMCUR_ERR_NO_CONVERGENCE",
          7: "QMCUR_ERR_UNSUPPORTED", 8: "QMCUR_ERR_CUDA", 9: "QMCUR_ERR_TIMEOUT",
          10: "QMCUR_ERR_ILL_CONDITIONED"}
PINV_JACOBI_FP64, PINV_SUBSPACE_FP32, PINV_REFINED_FP64 = 0, 1, 2
# pseudo-inverse methods that need rank_cap >= 1 (QMCUR_ERR_UNSUPPORTED otherwise)
_CAPPED_METHODS = (PINV_SUBSPACE_FP32, PINV_REFINED_FP64)


class QmcurError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s" % (where, STATUS.get(code, code)))


class QMat(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p * 4), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("sampler", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
                ("max_attempts", ctypes.c_int32), ("rcond", ctypes.c_double),
                ("rank_cap", ctypes.c_int32), ("max_sweeps", ctypes.c_int32),
                ("pinv_method", ctypes.c_int32), ("max_ctas", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_QP = ctypes.POINTER(QMat)
_I64, _I32, _U32, _U64, _D, _SZ = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t)

# name -> (restype, argtypes); the exported symbols of include/qmcur.h
SIGNATURES = {
    "qmcur_status_str": (ctypes.c_char_p, [_I32]),
    "qmcur_set_max_ctas": (_I32, [_I32]),
    "qmcur_workspace_size": (_SZ, [_I64, _I64, _I64, _I64, _I32]),
    "qmcur_probs": (_I32, [_QP, _I32, _P, _P, _P, _P, _SZ, _P, _P]),
    "qmcur_probs_noalloc": (_I32, [_QP, _I32, _P, _P, _P, _P, _P]),
    "qmcur_sample": (_I32, [_QP, _I32, _P, _P, _I64, _I64, _U64, _U32, _I32, _P, _P,
                            _QP, _QP, _QP, _P, _SZ, _P, _P]),
    "qmcur_pinv_core": (_I32, [_QP, _I32, _D, _I32, _I32, _QP, _P, _P, _P, _SZ, _P, _P]),
    "qmcur_reconstruct": (_I32, [_QP, _QP, _QP, _I32, _QP, _P, _SZ, _P, _P]),
    "qmcur_residual": (_I32, [_QP, _QP, _QP, _QP, _I32, _P, _QP, _P, _P, _SZ, _P, _P]),
    "qmcur_gather": (_I32, [_QP, _P, _P, _I64, _I64, _QP, _QP, _QP, _P]),
    "qmcur_backward_workspace_size": (_SZ, [_I64, _I64, _I64, _I64]),
    "qmcur_reconstruct_backward": (_I32, [_QP, _P, _P, _P, _QP, _QP, _QP, _QP, _D, _QP, _P, _P,
                                          _SZ, _P, _P]),
    "qmcur_batch_plan": (_I32, [_I32, _QP, _P, _P, _P, ctypes.POINTER(Opts), _P, _P, _P]),
    "qmcur_batch_run": (_I32, [_P, _P]),
    "qmcur_batch_stage_ms": (_I32, [_P, _P, _I32]),
    "qmcur_batch_view": (_I32, [_P, _I32, _P]),
    "qmcur_batch_copy": (_I32, [_P, _I32, _I32, _P, _SZ, _P]),
    "qmcur_batch_destroy": (None, [_P]),
    "qmcur_decompose": (_I32, [_QP, _I64, _I64, ctypes.POINTER(Opts), _P, _P, _P, _P,
                               _QP, _QP, _QP, _QP, _P, _P, _P, _P, _SZ, _P, _P]),
    "qmcur_qsvd_workspace_size": (_SZ, [_I64, _I64]),
    "qmcur_qsvd_truncated": (_I32, [_QP, _I32, _D, _I32, _QP, _P, _P, _P, _SZ, _P, _P]),
    "qmcur_core_paper_workspace_size": (_SZ, [_I64, _I64, _I64, _I64, _I32]),
    "qmcur_core_paper": (_I32, [_QP, _QP, _QP, _I32, _D, _I32, _I32, _QP, _QP, _QP, _P, _SZ, _P,
                                _P]),
    "qmcur_complete_step": (_I32, [_QP, _P, _I64, _I64, ctypes.POINTER(Opts), _P, _P, _P, _P,
                                   _QP, _QP, _QP, _QP, _P, _P, _P, _SZ, _P, _P]),
}


def lib():
    """Load libqmcur.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libqmcur.so is not built (run __graft_entry__.build()); "
                               "the library has no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def qmat(t):
    """C descriptor of a (4, rows, cols) CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if t.dim() != 3 or t.shape[0] != 4 or t.stride(2) != 1:
        raise ValueError("quaternion matrix must be (4, rows, cols) with unit column stride")
    if t.dtype not in (torch.float32, torch.float64):
        raise ValueError("quaternion planes must be float32 or float64")
    es = t.element_size()
    q = QMat()
    base = t.data_ptr()
    for k in range(4):
        q.plane[k] = base + k * t.stride(0) * es
    q.rows, q.cols = t.shape[1], t.shape[2]
    q.ld = max(t.stride(1), t.shape[2], 1)
    q.dtype = F64 if t.dtype == torch.float64 else F32
    return q


def _ref(q):
    return None if q is None else ctypes.byref(q)


def _check(code, where):
    if code != 0:
        raise QmcurError(code, where)


def workspace_size(m, n, c, r, prec):
    return int(lib().qmcur_workspace_size(m, n, c, r, prec))


def workspace(m, n, c, r, prec, device="cuda"):
    return torch.empty(workspace_size(m, n, c, r, prec), dtype=torch.uint8, device=device)


def status_tensor(device="cuda"):
    return torch.zeros(1, dtype=torch.int32, device=device)


def probs(A, sampler, col_p, row_p, fro2=None, ws=None, status=None, stream=None):
    _check(lib().qmcur_probs(_ref(qmat(A)), sampler, _ptr(col_p), _ptr(row_p), _ptr(fro2),
                             _ptr(ws), 0 if ws is None else ws.numel(), _ptr(status),
                             _stream(stream)), "qmcur_probs")


def probs_noalloc(A, sampler, col_p, row_p, fro2=None, status=None, stream=None):
    """qmcur_probs without a workspace: scratch is the library's static array."""
    _check(lib().qmcur_probs_noalloc(_ref(qmat(A)), sampler, _ptr(col_p), _ptr(row_p),
                                     _ptr(fro2), _ptr(status), _stream(stream)),
           "qmcur_probs_noalloc")


def sample(A, sampler, col_p, row_p, c, r, seed, stream_id, J, I, C=None, R=None, W=None,
           max_attempts=0, ws=None, status=None, stream=None):
    qC, qR, qW = qmat(C), qmat(R), qmat(W)
    _check(lib().qmcur_sample(_ref(qmat(A)), sampler, _ptr(col_p), _ptr(row_p), c, r,
                              seed, stream_id, max_attempts, _ptr(J), _ptr(I), _ref(qC),
                              _ref(qR), _ref(qW), _ptr(ws), 0 if ws is None else ws.numel(),
                              _ptr(status), _stream(stream)), "qmcur_sample")


def pinv_core(W, U, rcond=1e-10, rank_cap=0, max_sweeps=0, rank_out=None, sigma_out=None,
              ws=None, status=None, stream=None, method=PINV_JACOBI_FP64):
    _check(lib().qmcur_pinv_core(_ref(qmat(W)), method, rcond, rank_cap, max_sweeps,
                                 _ref(qmat(U)),
                                 _ptr(rank_out), _ptr(sigma_out), _ptr(ws),
                                 0 if ws is None else ws.numel(), _ptr(status),
                                 _stream(stream)), "qmcur_pinv_core")


def reconstruct(C, U, R, prec, Z, ws=None, status=None, stream=None):
    _check(lib().qmcur_reconstruct(_ref(qmat(C)), _ref(qmat(U)), _ref(qmat(R)), prec,
                                   _ref(qmat(Z)), _ptr(ws), 0 if ws is None else ws.numel(),
                                   _ptr(status), _stream(stream)), "qmcur_reconstruct")


def residual(A, out3, C=None, U=None, R=None, prec=PREC_FP32, mask=None, Z=None, ws=None,
             status=None, stream=None):
    _check(lib().qmcur_residual(_ref(qmat(A)), _ref(qmat(C)), _ref(qmat(U)), _ref(qmat(R)),
                                prec, _ptr(mask), _ref(qmat(Z)), _ptr(out3), _ptr(ws),
                                0 if ws is None else ws.numel(), _ptr(status),
                                _stream(stream)), "qmcur_residual")


def gather(A, J, I, C=None, R=None, W=None, stream=None):
    _check(lib().qmcur_gather(_ref(qmat(A)), _ptr(J), _ptr(I), J.numel(), I.numel(),
                              _ref(qmat(C)), _ref(qmat(R)), _ref(qmat(W)), _stream(stream)),
           "qmcur_gather")


def reconstruct_backward(A, mask, J, I, C, U, R, W, scale, dA, loss_out=None, ws=None,
                         status=None, stream=None):
    m, n = A.shape[1], A.shape[2]
    if ws is None:
        ws = torch.empty(int(lib().qmcur_backward_workspace_size(m, n, J.numel(), I.numel())),
                         dtype=torch.uint8, device=A.device)
    _check(lib().qmcur_reconstruct_backward(_ref(qmat(A)), _ptr(mask), _ptr(J), _ptr(I),
                                            _ref(qmat(C)), _ref(qmat(U)), _ref(qmat(R)),
                                            _ref(qmat(W)), float(scale), _ref(qmat(dA)),
                                            _ptr(loss_out), _ptr(ws), ws.numel(), _ptr(status),
                                            _stream(stream)), "qmcur_reconstruct_backward")


class MaskedCURLoss(torch.autograd.Function):
    """L(A) = || P_Omega(A - C U R) ||_F^2 for fixed index sets J, I, with
    C = A(:,J), R = A(I,:), U = W^+ (rank cap), W = A(I,J).  Forward and
    backward run in libqmcur (FP32 GEMMs, FP32 subspace or FP64 Jacobi
    pseudo-inverse); the sampling itself is not differentiated."""

    @staticmethod
    def forward(ctx, A, J, I, mask, rank_cap, rcond=1e-10, pinv_method=PINV_SUBSPACE_FP32):
        m, n = A.shape[1], A.shape[2]
        c, r = J.numel(), I.numel()
        dev = A.device
        C = torch.empty(4, m, c, dtype=torch.float32, device=dev)
        R = torch.empty(4, r, n, dtype=torch.float32, device=dev)
        W = torch.empty(4, r, c, dtype=torch.float64, device=dev)
        U = torch.empty(4, c, r, dtype=torch.float64, device=dev)
        st = status_tensor(dev)
        gather(A, J, I, C, R, W)
        ws = workspace(m, n, c, r, PREC_FP32, dev)
        pinv_core(W, U, rcond, rank_cap, 0, None, None, ws, st, method=pinv_method)
        out3 = torch.empty(3, dtype=torch.float64, device=dev)
        residual(A, out3, C, U, R, PREC_FP32, mask, None, ws, st)
        check_status(st, "MaskedCURLoss.forward")
        ctx.save_for_backward(A, J, I, C, U, R, W)
        ctx.mask = mask
        return out3[1].to(A.dtype)

    @staticmethod
    def backward(ctx, g):
        A, J, I, C, U, R, W = ctx.saved_tensors
        dA = torch.empty_like(A)
        st = status_tensor(A.device)
        reconstruct_backward(A, ctx.mask, J, I, C, U, R, W, float(g), dA, status=st)
        return dA, None, None, None, None, None, None


class Batch:
    """A batched QMCUR plan (qmcur_batch_plan): problems As[b] ((4, m_b, n_b)
    float32 CUDA tensors), cs[b] columns, rs[b] rows, rank_caps[b]; one graph
    replay per run().  prec selects the arithmetic of the grouped Z = C T
    (PREC_FP32: CUDA cores; a split precision: one grouped tcgen05 launch).
    get(b, what) copies one output into a new tensor."""

    WHAT = {"col_p": (0, torch.float64), "row_p": (1, torch.float64), "J": (2, torch.int32),
            "I": (3, torch.int32), "C": (4, torch.float32), "R": (5, torch.float32),
            "W": (6, torch.float32), "U": (7, torch.float32), "out3": (8, torch.float64),
            "info": (9, torch.int32), "U64": (10, torch.float64)}

    def __init__(self, As, cs, rs, rank_caps=None, sampler=SAMPLER_NORM, seed=0, rcond=1e-10,
                 max_sweeps=0, stream=None, pinv_method=PINV_JACOBI_FP64, prec=PREC_FP32):
        self.As = list(As)
        n = len(self.As)
        self.shapes = [(a.shape[1], a.shape[2], int(c), int(r)) for a, c, r in zip(self.As, cs, rs)]
        descs = (QMat * n)(*[qmat(a) for a in self.As])
        carr = (ctypes.c_int64 * n)(*[int(x) for x in cs])
        rarr = (ctypes.c_int64 * n)(*[int(x) for x in rs])
        kap = None if rank_caps is None else (ctypes.c_int32 * n)(*[int(x) for x in rank_caps])
        o = Opts(sampler, prec, seed, 0, 0, rcond, 0, max_sweeps, pinv_method, 0)
        self.status = status_tensor(self.As[0].device)
        self.handle = ctypes.c_void_p()
        _check(lib().qmcur_batch_plan(n, descs, carr, rarr, kap, ctypes.byref(o),
                                      ctypes.byref(self.handle), _ptr(self.status),
                                      _stream(stream)), "qmcur_batch_plan")

    def run(self, stream=None):
        _check(lib().qmcur_batch_run(self.handle, _stream(stream)), "qmcur_batch_run")

    STAGES = ("norms", "sample", "gather", "core", "t_gemm", "z_gemm_residual", "fold")

    def stage_ms(self):
        """Durations (ms) of the stages of the last replay, by name; waits for it."""
        out = (ctypes.c_float * len(self.STAGES))()
        _check(lib().qmcur_batch_stage_ms(self.handle, out, len(self.STAGES)),
               "qmcur_batch_stage_ms")
        return dict(zip(self.STAGES, [float(x) for x in out]))

    def get(self, b, what, stream=None):
        code, dt = self.WHAT[what]
        m, n, c, r = self.shapes[b]
        shape = {"col_p": (n,), "row_p": (m,), "J": (c,), "I": (r,), "C": (4, m, c),
                 "R": (4, r, n), "W": (4, r, c), "U": (4, c, r), "out3": (3,), "info": (3,),
                 "U64": (4, c, r)}[what]
        out = torch.empty(shape, dtype=dt, device=self.As[0].device)
        _check(lib().qmcur_batch_copy(self.handle, b, code, _ptr(out),
                                      out.numel() * out.element_size(), _stream(stream)),
               "qmcur_batch_copy")
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value is not None:
            lib().qmcur_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Decomposition:
    """Device buffers of one QMCUR decomposition of an m x n input."""

    def __init__(self, m, n, c, r, prec, dtype=torch.float32, device="cuda"):
        self.m, self.n, self.c, self.r, self.prec = m, n, c, r, prec
        f = dict(device=device)
        self.col_p = torch.empty(n, dtype=torch.float64, **f)
        self.row_p = torch.empty(m, dtype=torch.float64, **f)
        self.J = torch.empty(c, dtype=torch.int32, **f)
        self.I = torch.empty(r, dtype=torch.int32, **f)
        self.C = torch.empty(4, m, c, dtype=dtype, **f)
        self.R = torch.empty(4, r, n, dtype=dtype, **f)
        self.W = torch.empty(4, r, c, dtype=torch.float64, **f)
        self.U = torch.empty(4, c, r, dtype=torch.float64, **f)
        self.rank = torch.zeros(2, dtype=torch.int32, **f)   # {rank, sweeps}
        self.sigma = torch.empty(min(r, c), dtype=torch.float64, **f)
        self.out3 = torch.empty(3, dtype=torch.float64, **f)
        self.status = torch.zeros(1, dtype=torch.int32, **f)
        self.ws = workspace(m, n, c, r, prec, device)


def set_max_ctas(max_ctas):
    """CTA budget of the persistent kernels this thread launches (qmcur_set_max_ctas);
    0 = one CTA per SM."""
    _check(lib().qmcur_set_max_ctas(int(max_ctas)), "qmcur_set_max_ctas")


def decompose(A, D, sampler=SAMPLER_NORM, seed=0, stream_id=0, rcond=1e-10, rank_cap=0,
              max_sweeps=0, max_attempts=0, stream=None, pinv_method=PINV_JACOBI_FP64,
              max_ctas=0):
    """One whole QMCUR decomposition of A into the buffers of D (qmcur_decompose).
    max_ctas > 0 caps the CTAs of its persistent kernels (pseudo-inverse and
    tensor-core GEMMs), so that decompositions on two streams share the GPU."""
    o = Opts(sampler, D.prec, seed, stream_id, max_attempts, rcond, rank_cap, max_sweeps,
             pinv_method, max_ctas)
    qs = [qmat(D.C), qmat(D.R), qmat(D.W), qmat(D.U)]
    _check(lib().qmcur_decompose(_ref(qmat(A)), D.c, D.r, ctypes.byref(o), _ptr(D.col_p),
                                 _ptr(D.row_p), _ptr(D.J), _ptr(D.I), *[_ref(q) for q in qs],
                                 _ptr(D.rank), _ptr(D.sigma), _ptr(D.out3), _ptr(D.ws),
                                 D.ws.numel(), _ptr(D.status), _stream(stream)),
           "qmcur_decompose")


def decompose_many(As, Ds, seeds, nstreams=8, sampler=SAMPLER_NORM, stream_id=0, rcond=1e-10,
                   rank_cap=0, max_sweeps=0, max_attempts=0, pinv_method=PINV_JACOBI_FP64,
                   stream=None):
    """Decompose As[i] into the buffers of Ds[i] with seed seeds[i] (qmcur_decompose),
    nstreams of them in flight.  Each of the nstreams streams holds its
    persistent kernels to SMs // nstreams CTAs, so the budgets never exceed
    the SM count and the cooperative pseudo-inverses can always be resident
    together; the latency-bound pseudo-inverses of some decompositions then
    run beside the GEMMs of others.  The work is ordered after what `stream`
    (default: the current stream) has queued, and `stream` waits for all of
    it, also when a call raises part way (the decompositions already queued
    stay ordered before `stream`'s later work); As and Ds must stay alive
    until `stream` gets past that point.  The pseudo-inverse method is
    checked before anything is queued: the methods that need a rank cap
    raise ValueError when rank_cap < 1."""
    if not (len(As) == len(Ds) == len(seeds)):
        raise ValueError("As, Ds and seeds differ in length")
    if pinv_method in _CAPPED_METHODS and int(rank_cap) < 1:
        raise ValueError("pinv_method %d needs rank_cap >= 1" % pinv_method)
    if not As:
        return
    cur = stream if stream is not None else torch.cuda.current_stream()
    dev = As[0].device
    ns = max(1, min(int(nstreams), len(As)))
    budget = max(1, torch.cuda.get_device_properties(dev).multi_processor_count // ns)
    streams = [torch.cuda.Stream(device=dev) for _ in range(ns)]
    start = torch.cuda.Event()
    start.record(cur)
    for st in streams:
        st.wait_event(start)
    try:
        for i, (A, D, sd) in enumerate(zip(As, Ds, seeds)):
            decompose(A, D, sampler=sampler, seed=sd, stream_id=stream_id, rcond=rcond,
                      rank_cap=rank_cap, max_sweeps=max_sweeps, max_attempts=max_attempts,
                      stream=streams[i % ns], pinv_method=pinv_method, max_ctas=budget)
    finally:
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            cur.wait_event(done)


def qsvd_truncated(X, B, rank, rcond=0.0, max_sweeps=0, rank_out=None, sigma_out=None, ws=None,
                   status=None, stream=None):
    """B = the rank-k truncated QSVD approximation of X (qmcur_qsvd_truncated)."""
    if ws is None:
        ws = torch.empty(int(lib().qmcur_qsvd_workspace_size(X.shape[1], X.shape[2])),
                         dtype=torch.uint8, device=X.device)
    _check(lib().qmcur_qsvd_truncated(_ref(qmat(X)), rank, rcond, max_sweeps, _ref(qmat(B)),
                                      _ptr(rank_out), _ptr(sigma_out), _ptr(ws), ws.numel(),
                                      _ptr(status), _stream(stream)), "qmcur_qsvd_truncated")


def core_paper(X, C, R, Cp, Rp, U, prec=PREC_BF16_MIXED, rcond=1e-10, rank_cap=0,
               method=PINV_SUBSPACE_FP32, ws=None, status=None, stream=None):
    """The paper's core U = C^+ X R^+ (qmcur_core_paper); Cp (c x m) and Rp
    (n x r) receive C^+ and R^+."""
    if ws is None:
        m, n, c, r = X.shape[1], X.shape[2], C.shape[2], R.shape[1]
        ws = torch.empty(int(lib().qmcur_core_paper_workspace_size(m, n, c, r, prec)),
                         dtype=torch.uint8, device=X.device)
    _check(lib().qmcur_core_paper(_ref(qmat(X)), _ref(qmat(C)), _ref(qmat(R)), method, rcond,
                                  rank_cap, prec, _ref(qmat(Cp)), _ref(qmat(Rp)), _ref(qmat(U)),
                                  _ptr(ws), ws.numel(), _ptr(status), _stream(stream)),
           "qmcur_core_paper")


class Completion:
    """Device buffers of Algorithm 2 (quaternion matrix completion) on an
    m x n iterate with c columns and r rows per iteration: the probabilities,
    index sets and factors of the last iteration, and out3 = {delta, ||dX||^2,
    ||X||^2}."""

    def __init__(self, m, n, c, r, prec, dtype=torch.float32, device="cuda"):
        self.m, self.n, self.c, self.r, self.prec = m, n, c, r, prec
        f = dict(device=device)
        self.col_p = torch.empty(n, dtype=torch.float64, **f)
        self.row_p = torch.empty(m, dtype=torch.float64, **f)
        self.J = torch.empty(c, dtype=torch.int32, **f)
        self.I = torch.empty(r, dtype=torch.int32, **f)
        self.C = torch.empty(4, m, c, dtype=dtype, **f)
        self.R = torch.empty(4, r, n, dtype=dtype, **f)
        self.W = torch.empty(4, r, c, dtype=torch.float64, **f)
        self.U = torch.empty(4, c, r, dtype=torch.float64, **f)
        self.rank = torch.zeros(2, dtype=torch.int32, **f)
        self.out3 = torch.empty(3, dtype=torch.float64, **f)
        self.status = torch.zeros(1, dtype=torch.int32, **f)
        self.ws = workspace(m, n, c, r, prec, device)


def complete_step(X, mask, S, t, sampler=SAMPLER_UNIFORM, seed=0, rcond=1e-10, rank_cap=0,
                  max_sweeps=0, pinv_method=PINV_SUBSPACE_FP32, stream=None):
    """Iteration t of Algorithm 2 on X in place (qmcur_complete_step) with the
    buffers of the Completion S; S.out3[0] is the stopping test's relative
    change."""
    o = Opts(sampler, S.prec, seed, t, 0, rcond, rank_cap, max_sweeps, pinv_method, 0)
    _check(lib().qmcur_complete_step(_ref(qmat(X)), _ptr(mask), S.c, S.r, ctypes.byref(o),
                                     _ptr(S.col_p), _ptr(S.row_p), _ptr(S.J), _ptr(S.I),
                                     _ref(qmat(S.C)), _ref(qmat(S.R)), _ref(qmat(S.W)),
                                     _ref(qmat(S.U)), _ptr(S.rank), _ptr(S.out3), _ptr(S.ws),
                                     S.ws.numel(), _ptr(S.status), _stream(stream)),
           "qmcur_complete_step")


def complete(Y, mask, c, r, rank_cap, prec=PREC_BF16_MIXED, sampler=SAMPLER_UNIFORM, seed=0,
             rcond=1e-10, tol=1e-4, t_max=200, pinv_method=PINV_SUBSPACE_FP32, stream=None):
    """Algorithm 2 from X^0 = P_Omega(Y): complete_step for t = 0, 1, ... until
    delta <= tol or t >= t_max.  The loop reads delta back after each
    iteration (one 8-byte device-to-host copy).  Returns (X, S, history)."""
    m, n = Y.shape[1], Y.shape[2]
    S = Completion(m, n, c, r, prec, Y.dtype, Y.device)
    X = torch.where(mask.bool().unsqueeze(0), Y, torch.zeros((), dtype=Y.dtype, device=Y.device))
    history = []
    t = 0
    while True:
        complete_step(X, mask, S, t, sampler, seed, rcond, rank_cap, 0, pinv_method, stream)
        delta = float(S.out3[0].item())
        check_status(S.status, "complete")
        history.append(delta)
        if delta <= tol or t >= t_max:
            break
        t += 1
    return X, S, history


def check_status(status, where="device"):
    code = int(status.item())
    if code != 0:
        raise QmcurError(code, where)
