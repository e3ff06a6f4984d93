"""FP64 gradient of the masked CUR reconstruction loss (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/quat.py).

Loss, with J, I fixed index sets, Omega a mask (Example 4.4's observed set),
C = A(:,J), R = A(I,:), W = A(I,J), U = W_k^+ (Sec. 2.2, truncated):
    L(A) = || P_Omega(A - C U R) ||_F^2.
With the real inner product <X, Y> = Re tr(X^H Y) = sum_t <X_t, Y_t> (Re tr is
cyclic over quaternion matrices) and E = P_Omega(A - Z), Z = C T, T = U R:
    G_C = -2 E T^H,   G_T = -2 C^H E,   G_U = G_T R^H,   G_R = U^H G_T,
and, through the Moore-Penrose inverse (Golub and Pereyra 1973, quaternion form,
valid for a fixed rank),
    dU  = -U dW U + U U^H dW^H (I - W U) + (I - U W) dW^H U^H U
    G_W = -U^H G_U U^H + (I - W U) G_U^H U U^H + U^H U G_U^H (I - U W).
dL/dA = 2 E + G_C scattered to the columns J + G_R to the rows I + G_W to (I, J).
Parity: pinned by central finite differences in FP64 (tests/test_oracle_grad.py).
"""
import numpy as np

from .quat import as_q, qmatmul, conj_transpose, identity, fro2
from .qmcur import gather, pinv_truncated, reconstruct


def masked_loss(A, I, J, mask, rcond=1e-10, rank_cap=0):
    A = as_q(A)
    C, R, W = gather(A, I, J)
    U = pinv_truncated(W, rcond, rank_cap)[0]
    Z = reconstruct(C, U, R)
    w = 1.0 if mask is None else (np.asarray(mask) != 0).astype(np.float64)
    return fro2((A - Z) * w)


def masked_loss_grad(A, I, J, mask, rcond=1e-10, rank_cap=0):
    """Returns (loss, dL/dA) in FP64."""
    A = as_q(A)
    I = np.asarray(I)
    J = np.asarray(J)
    C, R, W = gather(A, I, J)
    U = pinv_truncated(W, rcond, rank_cap)[0]
    T = qmatmul(U, R)
    Z = qmatmul(C, T)
    w = 1.0 if mask is None else (np.asarray(mask) != 0).astype(np.float64)
    E = (A - Z) * w
    H = conj_transpose
    G_C = -2.0 * qmatmul(E, H(T))
    G_T = -2.0 * qmatmul(H(C), E)
    G_U = qmatmul(G_T, H(R))
    G_R = qmatmul(H(U), G_T)
    r, c = W.shape[1], W.shape[2]
    WU = qmatmul(W, U)
    UW = qmatmul(U, W)
    term1 = -qmatmul(qmatmul(H(U), G_U), H(U))
    term2 = qmatmul(qmatmul(identity(r) - WU, H(G_U)), qmatmul(U, H(U)))
    term3 = qmatmul(qmatmul(qmatmul(H(U), U), H(G_U)), identity(c) - UW)
    G_W = term1 + term2 + term3
    G = 2.0 * E
    G[:, :, J] += G_C
    G[:, I, :] += G_R
    G[:, I[:, None], J[None, :]] += G_W
    return fro2(E), G
