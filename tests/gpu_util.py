"""Helpers of the GPU parity tests (device transfer, tolerances)."""
import numpy as np
import torch

from paper_2402_19147_gb300 import qmcur as Q

U32 = 2.0 ** -24      # unit roundoff of FP32
U64 = 2.0 ** -53      # unit roundoff of FP64


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def run_status(status):
    torch.cuda.synchronize()
    return int(status.item())


def probs(A_t, sampler):
    m, n = A_t.shape[1], A_t.shape[2]
    col_p = torch.empty(n, dtype=torch.float64, device="cuda")
    row_p = torch.empty(m, dtype=torch.float64, device="cuda")
    fro2 = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = Q.workspace(m, n, 1, 1, Q.PREC_FP32)
    st = Q.status_tensor()
    Q.probs(A_t, sampler, col_p, row_p, fro2, ws, st)
    return col_p, row_p, fro2, run_status(st)
