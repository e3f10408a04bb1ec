"""Pins of the oracle's quadrature rules and bases against closed forms."""
import numpy as np
import pytest

from oracle import quadrature as qr
from oracle.fem import Mesh


def test_gauss_legendre_closed_forms():
    t, w = qr.gauss_legendre(2)
    assert np.allclose(t, [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], atol=1e-15)
    t, w = qr.gauss_legendre(3)
    s = 0.5 * np.sqrt(3.0 / 5.0)
    assert np.allclose(t, [0.5 - s, 0.5, 0.5 + s], atol=1e-15)
    assert np.allclose(w, [5 / 18, 4 / 9, 5 / 18], atol=1e-15)


def test_gauss_lobatto_closed_forms():
    assert np.allclose(qr.gauss_lobatto_points(2), [0, 1], atol=1e-15)
    assert np.allclose(qr.gauss_lobatto_points(3), [0, 0.5, 1], atol=1e-15)
    s = 0.5 / np.sqrt(5.0)
    assert np.allclose(qr.gauss_lobatto_points(4), [0, 0.5 - s, 0.5 + s, 1], atol=1e-15)
    s = 0.5 * np.sqrt(3.0 / 7.0)
    assert np.allclose(qr.gauss_lobatto_points(5), [0, 0.5 - s, 0.5, 0.5 + s, 1], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8])
def test_gauss_exactness(n):
    t, w = qr.gauss_legendre(n)
    for p in range(2 * n):
        assert abs(np.sum(w * t ** p) - 1.0 / (p + 1)) < 5e-14
    # one degree beyond exactness must fail (guards against a rule with too few points)
    assert abs(np.sum(w * t ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_properties(k):
    z = qr.h1_nodes(k)
    assert np.allclose(qr.lagrange(z, z), np.eye(k + 1), atol=1e-14)
    t = np.linspace(0, 1, 17)
    assert np.allclose(qr.lagrange(z, t).sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(qr.lagrange_deriv(z, t).sum(axis=1), 0.0, atol=1e-12)
    # derivative against a central difference of the values
    eps = 1e-6
    fd = (qr.lagrange(z, t + eps) - qr.lagrange(z, t - eps)) / (2 * eps)
    assert np.allclose(qr.lagrange_deriv(z, t), fd, atol=1e-7)
    # reproduces x^k exactly
    for p in range(k + 1):
        assert np.allclose(qr.lagrange(z, t) @ z ** p, t ** p, atol=1e-13)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2)])
def test_dense_element_matrices(dim, k):
    m = Mesh((2,) * dim, (0.0,) * dim, (1.0,) * dim, k)
    assert abs(m.alpha.sum() - 1.0) < 1e-14
    # gradient of a linear function of the reference coordinates is exact
    a = np.arange(1, dim + 1) * 0.7
    f = m.href @ a + 0.3
    for r in range(dim):
        assert np.allclose(m.Gh[:, r, :] @ f, a[r], atol=1e-13)
    # degree-k polynomial in every direction is reproduced at the quadrature points
    g = np.prod(m.href ** k, axis=1)
    assert np.allclose(m.Bh @ g, np.prod(m.qref ** k, axis=1), atol=1e-13)
    # L2 basis reproduces degree k-1 and sums to one
    assert np.allclose(m.Bl.sum(axis=1), 1.0, atol=1e-14)
    gl = np.prod(m.lref ** (k - 1), axis=1)
    assert np.allclose(m.Bl @ gl, np.prod(m.qref ** (k - 1), axis=1), atol=1e-13)


def test_mesh_numbering_and_nodes():
    m = Mesh((3, 2), (0.0, 0.0), (3.0, 1.0), 2)
    assert m.NV == 7 * 5 and m.NE == 6 and m.n_unknowns == 2 * 2 * 35 + 6 * 4
    x0 = m.initial_nodes()
    # lattice node (i0, i1) at (i0 * 0.5, i1 * 0.25)
    i = np.arange(m.NV)
    assert np.allclose(x0[0], (i % 7) * 0.5) and np.allclose(x0[1], (i // 7) * 0.25)
    # element 4 = (ex=1, ey=1): local node 0 is lattice (2, 2)
    assert m.conn[4, 0] == 2 + 7 * 2
    fixed = m.boundary_mask(0b1111)
    assert fixed[0].sum() == 2 * 5 and fixed[1].sum() == 2 * 7
