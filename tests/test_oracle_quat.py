"""Pins of the oracle's quaternion algebra against what Sec. 2.2 fixes."""
import numpy as np
import pytest

from oracle import quat as Q

ONE, I, J, K = (np.eye(4)[t] for t in range(4))


def test_hamilton_rules_from_the_paper():
    # i^2 = j^2 = k^2 = ijk = -1, ij = -ji = k, jk = -kj = i, ki = -ik = j (Sec. 2.2)
    for u in (I, J, K):
        assert np.array_equal(Q.qmul(u, u), -ONE)
    assert np.array_equal(Q.qmul(Q.qmul(I, J), K), -ONE)
    assert np.array_equal(Q.qmul(I, J), K) and np.array_equal(Q.qmul(J, I), -K)
    assert np.array_equal(Q.qmul(J, K), I) and np.array_equal(Q.qmul(K, J), -I)
    assert np.array_equal(Q.qmul(K, I), J) and np.array_equal(Q.qmul(I, K), -J)
    for u in (ONE, I, J, K):
        assert np.array_equal(Q.qmul(ONE, u), u) and np.array_equal(Q.qmul(u, ONE), u)


def test_conjugate_and_modulus():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(4)
    # a a* = |a|^2 (real), with |a| = sqrt(sum a_t^2) (Sec. 2.2)
    p = Q.qmul(a, Q.qconj(a))
    assert np.allclose(p, [np.sum(a * a), 0, 0, 0], atol=1e-15)
    b = rng.standard_normal(4)
    # (ab)* = b* a*, |ab| = |a||b|
    assert np.allclose(Q.qconj(Q.qmul(a, b)), Q.qmul(Q.qconj(b), Q.qconj(a)))
    assert np.isclose(np.linalg.norm(Q.qmul(a, b)), np.linalg.norm(a) * np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 2), (1, 7, 3)])
def test_matmul_equals_brute_force(shape):
    m, k, n = shape
    rng = np.random.default_rng(m * 100 + k * 10 + n)
    X = rng.standard_normal((4, m, k))
    Y = rng.standard_normal((4, k, n))
    assert np.allclose(Q.qmatmul(X, Y), Q.qmatmul_loops(X, Y), rtol=1e-13, atol=1e-13)


def test_complex_adjoint_is_a_homomorphism():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 5, 3))
    Y = rng.standard_normal((4, 3, 6))
    lhs = Q.complex_adjoint(Q.qmatmul(X, Y))
    rhs = Q.complex_adjoint(X) @ Q.complex_adjoint(Y)
    assert np.allclose(lhs, rhs, atol=1e-12)
    assert np.allclose(Q.complex_adjoint(Q.conj_transpose(X)), Q.complex_adjoint(X).conj().T)
    assert np.allclose(Q.from_complex_adjoint(Q.complex_adjoint(X)), X)


def test_real_representation_plane_formulas():
    # the four real-plane formulas the GEMM kernels implement
    rng = np.random.default_rng(2)
    X = rng.standard_normal((4, 4, 4))
    Y = rng.standard_normal((4, 4, 4))
    X0, X1, X2, X3 = X
    Y0, Y1, Y2, Y3 = Y
    Z = Q.qmatmul(X, Y)
    assert np.allclose(Z[0], X0 @ Y0 - X1 @ Y1 - X2 @ Y2 - X3 @ Y3)
    assert np.allclose(Z[1], X0 @ Y1 + X1 @ Y0 + X2 @ Y3 - X3 @ Y2)
    assert np.allclose(Z[2], X0 @ Y2 - X1 @ Y3 + X2 @ Y0 + X3 @ Y1)
    assert np.allclose(Z[3], X0 @ Y3 + X1 @ Y2 - X2 @ Y1 + X3 @ Y0)


def test_associative_not_commutative():
    rng = np.random.default_rng(3)
    X, Y, Z = (rng.standard_normal((4, 4, 4)) for _ in range(3))
    assert np.allclose(Q.qmatmul(Q.qmatmul(X, Y), Z), Q.qmatmul(X, Q.qmatmul(Y, Z)))
    assert not np.allclose(Q.qmatmul(X, Y), Q.qmatmul(Y, X))


def test_conjugate_transpose_reverses_products():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((4, 3, 5))
    Y = rng.standard_normal((4, 5, 2))
    lhs = Q.conj_transpose(Q.qmatmul(X, Y))
    rhs = Q.qmatmul(Q.conj_transpose(Y), Q.conj_transpose(X))
    assert np.allclose(lhs, rhs)


def test_frobenius_is_trace_of_gram():
    # ||A||_F = sqrt(Tr(A^H A)) = sqrt(sum |a_st|^2) (Sec. 2.2)
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 6, 4))
    G = Q.qmatmul(Q.conj_transpose(A), A)
    assert np.isclose(Q.trace_real(G), Q.fro2(A))
    assert np.allclose(G[1:].diagonal(axis1=1, axis2=2), 0.0, atol=1e-13)


def test_reduces_to_real_and_complex_products():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    B = rng.standard_normal((4, 2)) + 1j * rng.standard_normal((4, 2))
    Xq = np.zeros((4, 3, 4)); Xq[0], Xq[1] = A.real, A.imag
    Yq = np.zeros((4, 4, 2)); Yq[0], Yq[1] = B.real, B.imag
    Z = Q.qmatmul(Xq, Yq)
    assert np.allclose(Z[0] + 1j * Z[1], A @ B)
    assert np.allclose(Z[2:], 0.0)
