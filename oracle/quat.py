"""FP64 quaternion algebra for the QMCUR oracle.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA path and never calls it.

Every function here follows Sec. 2.2 of the paper (arXiv 2402.19147,
"Quaternion and quaternion matrices"):

* a quaternion is a = a0 + a1 i + a2 j + a3 k with i^2 = j^2 = k^2 = ijk = -1,
  ij = -ji = k, jk = -kj = i, ki = -ik = j;
* a quaternion matrix is stored *split*: four real planes A0, A1, A2, A3 of the
  same shape, held as one array of shape (4, m, n);
* conjugate a* = a0 - a1 i - a2 j - a3 k, modulus |a| = sqrt(sum a_t^2);
* A^H is the conjugate transpose, ||A||_F^2 = Tr(A^H A) = sum |a_st|^2.

The matrix product is the bilinear expansion of the Hamilton table, one real
matmul per pair of basis planes.  Parity: pinned (see tests/test_oracle_quat.py:
brute-force scalar products from the table, the complex-adjoint homomorphism,
associativity and the trace identity).
"""
import numpy as np

# Hamilton multiplication table of the basis (1, i, j, k), Sec. 2.2.
# MUL[a][b] = (sign, c) means e_a * e_b = sign * e_c.
MUL = (
    ((+1, 0), (+1, 1), (+1, 2), (+1, 3)),   # 1*1=1, 1*i=i, 1*j=j, 1*k=k
    ((+1, 1), (-1, 0), (+1, 3), (-1, 2)),   # i*1=i, i*i=-1, i*j=k, i*k=-j
    ((+1, 2), (-1, 3), (-1, 0), (+1, 1)),   # j*1=j, j*i=-k, j*j=-1, j*k=i
    ((+1, 3), (+1, 2), (-1, 1), (-1, 0)),   # k*1=k, k*i=j, k*j=-i, k*k=-1
)


def qmul(a, b):
    """Product of two scalar quaternions given as length-4 sequences (Sec. 2.2)."""
    out = [0.0, 0.0, 0.0, 0.0]
    for ia in range(4):
        for ib in range(4):
            s, c = MUL[ia][ib]
            out[c] += s * float(a[ia]) * float(b[ib])
    return np.array(out, dtype=np.float64)


def qconj(a):
    """Conjugate of a scalar quaternion (Sec. 2.2)."""
    a = np.asarray(a, dtype=np.float64)
    return np.array([a[0], -a[1], -a[2], -a[3]])


def as_q(X):
    """Return X as an FP64 array of shape (4, m, n) (split planes)."""
    X = np.asarray(X, dtype=np.float64)
    if X.ndim != 3 or X.shape[0] != 4:
        raise ValueError("quaternion matrix must have shape (4, m, n)")
    return X


def qmatmul(X, Y):
    """Quaternion matrix product Z = X Y for split planes (Sec. 2.2).

    Z_c = sum over (a, b) with e_a e_b = s e_c of s * X_a @ Y_b: sixteen real
    FP64 matmuls, one per pair of planes, signs from the Hamilton table.
    """
    X = as_q(X)
    Y = as_q(Y)
    if X.shape[2] != Y.shape[1]:
        raise ValueError("inner dimensions differ")
    Z = np.zeros((4, X.shape[1], Y.shape[2]), dtype=np.float64)
    for a in range(4):
        for b in range(4):
            s, c = MUL[a][b]
            if s > 0:
                Z[c] += X[a] @ Y[b]
            else:
                Z[c] -= X[a] @ Y[b]
    return Z


def qmatmul_loops(X, Y):
    """Entry-by-entry product with scalar quaternion arithmetic (brute force)."""
    X = as_q(X)
    Y = as_q(Y)
    m, k = X.shape[1], X.shape[2]
    n = Y.shape[2]
    Z = np.zeros((4, m, n))
    for i in range(m):
        for j in range(n):
            acc = np.zeros(4)
            for t in range(k):
                acc += qmul(X[:, i, t], Y[:, t, j])
            Z[:, i, j] = acc
    return Z


def conj_transpose(X):
    """A^H = (a*_ts) (Sec. 2.2): transpose every plane, negate the imaginary ones."""
    X = as_q(X)
    out = np.empty((4, X.shape[2], X.shape[1]))
    out[0] = X[0].T
    out[1] = -X[1].T
    out[2] = -X[2].T
    out[3] = -X[3].T
    return out


def fro2(X):
    """||X||_F^2 = sum over entries of |x|^2 (Sec. 2.2)."""
    X = as_q(X)
    return float(np.sum(X * X))


def trace_real(X):
    """Real part of Tr(X) for a square quaternion matrix."""
    X = as_q(X)
    return float(np.trace(X[0]))


def identity(n):
    out = np.zeros((4, n, n))
    out[0] = np.eye(n)
    return out


def complex_adjoint(X):
    """Complex adjoint chi(X) = [[A, B], [-conj(B), conj(A)]] (2m x 2n complex).

    With X = A + B j, A = X0 + X1 i, B = X2 + X3 i (so X = X0 + X1 i + X2 j +
    X3 k because i j = k).  chi is an injective ring homomorphism that maps
    X^H to chi(X)^H; it is the standard vehicle for the QSVD of Sec. 2.2.
    """
    X = as_q(X)
    A = X[0] + 1j * X[1]
    B = X[2] + 1j * X[3]
    return np.block([[A, B], [-B.conj(), A.conj()]])


def from_complex_adjoint(M):
    """Inverse of complex_adjoint for a matrix of adjoint form.

    The two copies of each block are averaged, which is exact for a matrix of
    adjoint form and symmetrises rounding otherwise.
    """
    M = np.asarray(M)
    m2, n2 = M.shape
    m, n = m2 // 2, n2 // 2
    A = 0.5 * (M[:m, :n] + M[m:, n:].conj())
    B = 0.5 * (M[:m, n:] - M[m:, :n].conj())
    out = np.empty((4, m, n))
    out[0] = A.real
    out[1] = A.imag
    out[2] = B.real
    out[3] = B.imag
    return out
