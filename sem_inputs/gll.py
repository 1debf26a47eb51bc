"""Gauss-Lobatto-Legendre (GLL) nodes, quadrature weights and the 1D
collocation differentiation matrix D, in float64.

These are *inputs* of the spectral-element operator: the library call takes D
as an argument, exactly as a Fortran PDE kernel takes its coefficient arrays
(the paper's Fortran front-end, Section 3, ingests such subroutines).  The
definitions are the textbook ones (Deville, Fischer & Mund, "High-Order Methods
for Incompressible Fluid Flow", 2002, Sec. 2.4 and App. B):

* nodes xi_0 = -1 < ... < xi_N = 1 are the roots of (1 - x^2) P_N'(x);
* weights w_j = 2 / (N (N+1) P_N(xi_j)^2);
* D[i][l] = l_l'(xi_i) where l_l is the Lagrange basis on the nodes; off the
  diagonal D[i][l] = P_N(xi_i) / (P_N(xi_l) (xi_i - xi_l)).

Nothing in this module applies the operator itself.
"""
from __future__ import annotations

import numpy as np


def legendre(N: int, x: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Return (P_N(x), P_{N-1}(x)) by the three-term recurrence
    (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}, P_0 = 1, P_1 = x."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, N):
        p_next = ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
        p_prev, p = p, p_next
    return p, p_prev


def gll_nodes(N: int) -> np.ndarray:
    """GLL nodes for polynomial order N >= 1 (n = N+1 nodes), ascending.

    (1 - x^2) P_N'(x) = N (P_{N-1}(x) - x P_N(x)), so the nodes are the zeros
    of g(x) = x P_N(x) - P_{N-1}(x).  With the identity
    x P_N' - P_{N-1}' = N P_N one gets g'(x) = (N+1) P_N(x), so Newton's step is
    x <- x - (x P_N - P_{N-1}) / ((N+1) P_N).  The start is the
    Chebyshev-Gauss-Lobatto set -cos(pi j / N); the end points are fixed points.
    The result is made exactly antisymmetric (xi_{N-j} = -xi_j) so that the
    matrix D built on it is exactly centro-antisymmetric.
    """
    if N < 1:
        raise ValueError("GLL needs N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(100):
        pN, pNm1 = legendre(N, x)
        dx = (x * pN - pNm1) / ((N + 1) * pN)
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    x = 0.5 * (x - x[::-1])
    x[0], x[-1] = -1.0, 1.0
    return x


def gll_weights(N: int, x: np.ndarray | None = None) -> np.ndarray:
    """GLL quadrature weights w_j = 2 / (N (N+1) P_N(xi_j)^2)."""
    if x is None:
        x = gll_nodes(N)
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN * pN)
    return 0.5 * (w + w[::-1])


def gll_diff_matrix(N: int, x: np.ndarray | None = None) -> np.ndarray:
    """Collocation derivative D[i][l] = l_l'(xi_i), shape (n, n), row-major.

    Off-diagonal entries use the closed form P_N(xi_i) / (P_N(xi_l)(xi_i - xi_l));
    each diagonal entry is minus the sum of the rest of its row, so D maps
    constants to zero to rounding.  The matrix is then symmetrised to be exactly
    centro-antisymmetric, D[N-i][N-l] = -D[i][l] bit for bit, which the GLL
    derivative satisfies in exact arithmetic (symmetric node set).
    """
    if x is None:
        x = gll_nodes(N)
    n = N + 1
    pN, _ = legendre(N, x)
    D = np.zeros((n, n), dtype=np.float64)
    for i in range(n):
        for l in range(n):
            if i != l:
                D[i, l] = pN[i] / (pN[l] * (x[i] - x[l]))
    for i in range(n):
        D[i, i] = -np.sum(np.delete(D[i], i))
    D = 0.5 * (D - D[::-1, ::-1])
    return np.ascontiguousarray(D)
