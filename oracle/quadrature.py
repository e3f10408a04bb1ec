"""1D quadrature rules and Lagrange bases on the reference interval [0, 1].

The paper defers the finite element spaces to its Sec. 2.1 (H1 space Q_k for x and v,
discontinuous L2 space Q_{k-1} for e) without naming the nodal bases or the rule.
Readings used here (and by the CUDA path, independently implemented there):

* H1 basis: Lagrange polynomials of degree k at the k+1 Gauss-Lobatto points;
* L2 basis: Lagrange polynomials of degree k-1 at the k Gauss-Legendre points;
* quadrature: tensor Gauss-Legendre with 2k points per direction.

Pinned by tests/test_oracle_basis.py (closed-form nodes and weights, polynomial
exactness, Kronecker-delta and partition-of-unity properties).
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def gauss_legendre(n):
    """n-point Gauss-Legendre points and weights mapped from [-1, 1] to [0, 1]."""
    t, w = _leg.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gauss_lobatto_points(n):
    """n >= 2 Gauss-Lobatto points on [0, 1]: the end points and the roots of P'_{n-1}."""
    if n < 2:
        raise ValueError("Gauss-Lobatto needs at least two points")
    inner = _leg.Legendre.basis(n - 1).deriv().roots() if n > 2 else np.zeros(0)
    t = np.concatenate(([-1.0], np.sort(np.real(inner)), [1.0]))
    return 0.5 * (t + 1.0)


def lagrange(nodes, t):
    """Values phi[i, j] = l_j(t_i) of the Lagrange polynomials through ``nodes``."""
    nodes = np.asarray(nodes, dtype=float)
    t = np.asarray(t, dtype=float)
    m = len(nodes)
    phi = np.ones((len(t), m))
    for j in range(m):
        for l in range(m):
            if l != j:
                phi[:, j] *= (t - nodes[l]) / (nodes[j] - nodes[l])
    return phi


def lagrange_deriv(nodes, t):
    """Derivatives dphi[i, j] = l_j'(t_i), by the product rule over the factors."""
    nodes = np.asarray(nodes, dtype=float)
    t = np.asarray(t, dtype=float)
    m = len(nodes)
    d = np.zeros((len(t), m))
    for j in range(m):
        for l in range(m):
            if l == j:
                continue
            term = np.full(len(t), 1.0 / (nodes[j] - nodes[l]))
            for i in range(m):
                if i != j and i != l:
                    term = term * (t - nodes[i]) / (nodes[j] - nodes[i])
            d[:, j] += term
    return d


def h1_nodes(k):
    """Nodes of the degree-k H1 basis (k+1 Gauss-Lobatto points)."""
    return gauss_lobatto_points(k + 1)


def l2_nodes(k):
    """Nodes of the degree-(k-1) L2 basis (k Gauss-Legendre points)."""
    return gauss_legendre(k)[0]
