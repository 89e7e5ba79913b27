"""Pins for the 1D basis and reference matrices of the oracle (Sec. 2, Eq. (matrix1d))."""
import numpy as np
import pytest

from oracle import basis, kron


def test_gll_points_closed_forms():
    assert np.allclose(basis.gll_points(2), [0.0, 0.5, 1.0], atol=1e-15)
    s = 1.0 / np.sqrt(5.0)
    assert np.allclose(basis.gll_points(3), [0.0, (1 - s) / 2, (1 + s) / 2, 1.0], atol=1e-15)
    s = np.sqrt(3.0 / 7.0)
    assert np.allclose(basis.gll_points(4), [0.0, (1 - s) / 2, 0.5, (1 + s) / 2, 1.0], atol=1e-15)


@pytest.mark.parametrize("k", range(2, 8))
def test_lagrange_property_and_partition_of_unity(k):
    z = basis.gll_points(k)
    assert np.allclose(basis.basis_table(k, z), np.eye(k + 1), atol=1e-12)
    x = np.linspace(0, 1, 17)
    assert np.allclose(basis.basis_table(k, x).sum(0), 1.0, atol=1e-12)
    assert np.allclose(basis.basis_table(k, x, 1).sum(0), 0.0, atol=1e-9)
    assert np.allclose(basis.basis_table(k, x, 2).sum(0), 0.0, atol=1e-7)


@pytest.mark.parametrize("q", range(1, 9))
def test_gauss_exactness(q):
    x, w = basis.gauss(q, 0.0, 1.0)
    for p in range(2 * q):
        assert abs(np.dot(w, x ** p) - 1.0 / (p + 1)) < 1e-14


def test_reference_matrices_q2_closed_form():
    # quadratic Lagrange basis on nodes 0, 1/2, 1
    M, L, B = kron.reference_cell_matrices(2)
    assert np.allclose(M, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0, atol=1e-15)
    assert np.allclose(L, np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0, atol=1e-14)
    # phi'' = (4, -8, 4) is constant on the cell
    assert np.allclose(B, np.outer([4, -8, 4], [4, -8, 4]), atol=1e-12)


@pytest.mark.parametrize("k", range(2, 8))
def test_reference_matrix_invariants(k):
    M, L, B = kron.reference_cell_matrices(k)
    z = basis.gll_points(k)
    one = np.ones(k + 1)
    # row sums of M integrate the basis functions; total mass 1
    assert abs(one @ M @ one - 1.0) < 1e-13
    # constants and linears have zero second derivative; constants zero first derivative
    assert np.allclose(L @ one, 0.0, atol=1e-10)
    assert np.allclose(B @ one, 0.0, atol=1e-8)
    assert np.allclose(B @ z, 0.0, atol=1e-8)
    # int (x')^2 = 1, int (x^2)'' ^2 = 4
    assert abs(z @ L @ z - 1.0) < 1e-12
    assert abs((z ** 2) @ B @ (z ** 2) - 4.0) < 1e-8
    assert np.all(np.linalg.eigvalsh(M) > 0)
